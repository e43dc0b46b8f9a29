"""The cross-entropy search (Section 3.3, batch_search with CEM, warm-started from the parent's best input) on
the GPU: in FP32 bit-exact against the oracle (the same samples, objectives, rankings and refits), in the 3-term
BF16 split by the properties that hold for any precision; and the carrying of each row's best input through
branching (the children's warm start)."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cem(g, lo, hi, ids, M, iters, E, jitter, seed, precision, warm=None, incumbent=False, d_n=None):
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    n = lo.shape[0]
    ub = torch.full((n,), -7.0, device=DEV)
    bu = torch.full((n, g.d), -7.0, device=DEV)
    inc_val = torch.full((1,), np.inf, dtype=torch.float64, device=DEV) if incumbent else None
    inc_u = torch.zeros(g.d, device=DEV) if incumbent else None
    B.bab_rollout_cem(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), n, M, iters, E, jitter, seed,
                      precision, ub, bu, warm_u=None if warm is None else T(warm), inc_val=inc_val, inc_u=inc_u,
                      d_n=None if d_n is None else torch.tensor([d_n], dtype=torch.int32, device=DEV))
    torch.cuda.synchronize()
    out = {"ub": ub.cpu().numpy(), "best_u": bu.cpu().numpy()}
    if incumbent:
        out["inc_val"], out["inc_u"] = float(inc_val.item()), inc_u.cpu().numpy()
    return out


@pytest.mark.parametrize("name,n,M,iters,E,warm", [("tiny", 7, 130, 3, 8, False), ("tiny", 5, 64, 4, 1, True),
                                                   ("tiny", 3, 1, 2, 1, True), ("pushing", 3, 64, 2, 6, True)])
def test_cem_fp32_bit_exact(oracle, gp, name, n, M, iters, E, warm):
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 41)
    d = p["k"] * p["H"]
    lo, hi, ids = W.random_boxes(d, n, seed=42, min_width=0.1, max_width=1.5)
    w = (np.random.default_rng(3).uniform(-1.2, 1.2, size=lo.shape).astype(np.float32) if warm else None)
    g = gp(p)
    r = _cem(g, lo, hi, ids, M, iters, E, 1e-3, 17, B.PREC_FP32, warm=w)
    ub_o, bu_o = oracle.cem(p, lo, hi, ids, M, iters, E, 1e-3, 17, warm_u=w)
    assert np.array_equal(r["ub"].view(np.uint32), ub_o.view(np.uint32))
    assert np.array_equal(r["best_u"].view(np.uint32), bu_o.view(np.uint32))


def test_cem_bf16x3_properties(oracle, gp):
    """Tensor-core objectives: the result is a point of the box whose objective is ub, a warm start inside the box
    is never beaten, and more iterations never do worse."""
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 43)
    lo, hi, ids = W.random_boxes(40, 12, seed=44, min_width=0.2, max_width=1.5)
    g = gp(p)
    warm = (lo + np.random.default_rng(5).uniform(size=lo.shape).astype(np.float32) * (hi - lo)).astype(np.float32)
    r = _cem(g, lo, hi, ids, 256, 3, 16, 1e-3, 9, B.PREC_BF16X3, warm=warm)
    assert np.all(r["best_u"] >= lo) and np.all(r["best_u"] <= hi)
    for i in range(12):
        assert r["ub"][i] == pytest.approx(oracle.objective(p, r["best_u"][i].astype(np.float64)), rel=2e-6)
        assert r["ub"][i] <= oracle.objective(p, warm[i].astype(np.float64)) * (1 + 2e-6)
    r1 = _cem(g, lo, hi, ids, 256, 1, 16, 1e-3, 9, B.PREC_BF16X3, warm=warm)
    assert np.all(r["ub"] <= r1["ub"])


def test_cem_incumbent_and_live_count(oracle, gp):
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("tiny", 45)
    lo, hi, ids = W.random_boxes(10, 9, seed=46, min_width=0.2, max_width=1.0)
    g = gp(p)
    r = _cem(g, lo, hi, ids, 64, 2, 4, 1e-3, 5, B.PREC_FP32, incumbent=True, d_n=6)
    ub_o, bu_o = oracle.cem(p, lo[:6], hi[:6], ids[:6], 64, 2, 4, 1e-3, 5)
    assert np.array_equal(r["ub"][:6].view(np.uint32), ub_o.view(np.uint32))
    assert np.all(r["ub"][6:] == -7.0) and np.all(r["best_u"][6:] == -7.0)   # rows beyond the live count untouched
    best = int(np.argmin(ub_o))
    assert r["inc_val"] == pytest.approx(oracle.objective(p, bu_o[best].astype(np.float64)), rel=1e-12)
    np.testing.assert_array_equal(r["inc_u"], bu_o[best])


def test_cem_argument_errors(gp):
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("tiny", 47)
    lo, hi, ids = W.random_boxes(10, 2, seed=48)
    g = gp(p)
    ub, bu = torch.empty(2, device=DEV), torch.empty(2, 10, device=DEV)
    args = (g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), 2)
    for M, iters, E, prec in ((16, 1, 17, B.PREC_FP32), (16, 0, 4, B.PREC_FP32), (16, 1, 4, B.PREC_BF16),
                              (B.CEM_MAX_SAMPLES + 1, 1, 4, B.PREC_FP32)):
        with pytest.raises(B.BabError):
            B.bab_rollout_cem(*args, M, iters, E, 1e-3, 1, prec, ub, bu)


def test_branch_carries_row_vectors(gp):
    """Children inherit their parent's row vector (the warm start of their search); unpicked rows keep theirs."""
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    lo, hi, ids = W.dyadic_boxes(10, 120, seed=7, max_depth=4)
    lb, ub = W.pool_values(120, seed=8)
    rowu = np.random.default_rng(9).normal(size=lo.shape).astype(np.float32)
    g = gp(W.config_problem("tiny", 0))
    n, d, n_pick = 120, 10, 30
    cap = n + n_pick + 1
    out = [torch.empty(cap, d, device=DEV), torch.empty(cap, d, device=DEV), torch.empty(cap, device=DEV),
           torch.empty(cap, device=DEV), torch.zeros(cap, dtype=torch.int64, device=DEV)]
    orow = torch.full((cap, d), np.nan, device=DEV)
    keep = torch.empty(n, dtype=torch.uint8, device=DEV)
    counts = torch.zeros(3, dtype=torch.int32, device=DEV)
    B.bab_prune_branch_heuristic(g.ctx, d, T(lo), T(hi), T(lb), T(ub), ids_t(ids), n,
                                 torch.tensor([12.0], dtype=torch.float64, device=DEV), n_pick, 0.75, B.PICK_LB, 1.0,
                                 0, cap, *out, keep, counts, row_u=T(rowu), out_row_u=orow)
    torch.cuda.synchronize()
    nc, nr, tot = (int(x) for x in counts.cpu().numpy())
    oid = out[4][:tot].cpu().numpy().astype(np.uint64)
    orow = orow[:tot].cpu().numpy()
    pos = {int(i): k for k, i in enumerate(ids)}
    for q in range(tot):
        src = pos[int(oid[q]) // 2] if q < nc else pos[int(oid[q])]
        np.testing.assert_array_equal(orow[q], rowu[src])
