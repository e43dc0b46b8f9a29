"""The paper's branching heuristics (Section 3.1) on the GPU: the softmax pick-out (a reproducible race) and the
sample-imbalance split dimension, bit-exact against the FP64/FP32 oracle on the same inputs."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _branch(gp, lo, hi, lb, ub, ids, inc, n_pick, rule, T, seed, split_dim=None):
    """Runs bab_prune_branch_heuristic; with split_dim given the output pool also carries the split dimensions."""
    from gpu_util import DEV, T as TT, ids_t
    from paper_2412_09584_gb300 import binding as B
    p, _, _, _ = (W.config_problem("tiny", 0), None, None, None)
    g = gp(p)
    n, d = lo.shape
    cap = n + n_pick + 1
    out = [torch.full((cap, d), np.nan, device=DEV), torch.full((cap, d), np.nan, device=DEV),
           torch.empty(cap, device=DEV), torch.empty(cap, device=DEV), torch.zeros(cap, dtype=torch.int64, device=DEV)]
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device=DEV)
    counts = torch.zeros(3, dtype=torch.int32, device=DEV)
    osd = None if split_dim is None else torch.full((cap,), 7777, dtype=torch.int32, device=DEV)
    B.bab_prune_branch_heuristic(g.ctx, d, TT(lo), TT(hi), TT(lb), TT(ub), ids_t(ids), n,
                                 torch.tensor([inc], dtype=torch.float64, device=DEV), n_pick, 0.75, rule, T, seed,
                                 cap, *out, keep, counts,
                                 split_dim=None if split_dim is None else TT(split_dim, torch.int32),
                                 out_split_dim=osd)
    torch.cuda.synchronize()
    nc, nr, tot = (int(x) for x in counts.cpu().numpy())
    return {"split_dim": None if osd is None else osd[:tot].cpu().numpy(),"keep": keep.cpu().numpy()[:n], "n_children": nc, "n_rest": nr, "lo": out[0][:tot].cpu().numpy(),
            "hi": out[1][:tot].cpu().numpy(), "lb": out[2][:tot].cpu().numpy(), "ub": out[3][:tot].cpu().numpy(),
            "id": out[4][:tot].cpu().numpy().astype(np.uint64)}


def _same(r, o):
    assert np.array_equal(r["keep"], o["keep"])
    assert (r["n_children"], r["n_rest"]) == (o["n_children"], o["n_rest"])
    for key in ("lo", "hi", "lb", "ub"):
        assert np.array_equal(r[key].view(np.uint32), o[key].view(np.uint32)), key
    assert np.array_equal(r["id"], o["id"])


@pytest.mark.parametrize("n,n_pick,T,seed,ties,nans", [(300, 64, 0.05, 1, 0.0, 0.0), (1000, 200, 1.0, 2, 0.2, 0.02),
                                                       (5000, 1024, 0.3, 3, 0.05, 0.0), (40, 8, 1e-3, 4, 0.5, 0.1)])
def test_softmax_pick_out_bit_exact(oracle, gp, n, n_pick, T, seed, ties, nans):
    lo, hi, ids = W.dyadic_boxes(10, n, seed=n + seed, max_depth=5)
    lb, ub = W.pool_values(n, seed=n + 7, nan_frac=nans, tie_frac=ties)
    inc = float(np.nanmedian(lb) + 2.0)
    r = _branch(gp, lo, hi, lb, ub, ids, inc, n_pick, 1, T, seed)
    o = oracle.prune_branch_heuristic(lo, hi, lb, ub, ids, inc, n_pick, pick_rule=1, temperature=T, pick_seed=seed)
    _same(r, o)


@pytest.mark.parametrize("n,M,k", [(37, 64, 5), (300, 1024, 11), (16, 17, 17)])
def test_split_dims_bit_exact(oracle, gp, n, M, k):
    from gpu_util import DEV, T as TT, ids_t
    from paper_2412_09584_gb300 import binding as B
    d = 12
    lo, hi, ids = W.random_boxes(d, n, seed=M, min_width=0.1, max_width=1.5)
    rng = np.random.default_rng(M)
    costs = rng.normal(size=(n, M)).astype(np.float32)
    costs[:, ::7] = costs[:, :1]                     # ties between samples: broken by the sample index
    costs[0, :] = 3.0                                # all equal
    g = gp(W.config_problem("tiny", 0))
    out = torch.empty(n, dtype=torch.int32, device=DEV)
    B.bab_split_dims(g.ctx, d, TT(lo), TT(hi), ids_t(ids), n, 99, TT(costs), M, k, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.split_dims(lo, hi, ids, 99, costs, k))


def test_branch_with_given_split_dims(oracle, gp):
    lo, hi, ids = W.dyadic_boxes(10, 200, seed=5, max_depth=4)
    lb, ub = W.pool_values(200, seed=6)
    sd = np.random.default_rng(1).integers(0, 12, size=200).astype(np.int32)  # some out of range: widest
    r = _branch(gp, lo, hi, lb, ub, ids, 12.0, 50, 0, 1.0, 0, split_dim=sd)
    o = oracle.prune_branch_heuristic(lo, hi, lb, ub, ids, 12.0, 50, pick_rule=0, split_dim=sd)
    _same(r, o)
    # the split dimensions travel with the pool: unpicked rows keep theirs (found by id), children get -1
    pos = {int(i): k for k, i in enumerate(ids)}
    nc = r["n_children"]
    assert np.all(r["split_dim"][:nc] == -1)
    assert np.array_equal(r["split_dim"][nc:], sd[[pos[int(i)] for i in r["id"][nc:]]])


def test_rollout_split_costs_and_choice(oracle, gp):
    """The rollout's per-sample costs are the objective of each sample (FP32 to 1e-5), and the chosen dimension
    maximises the imbalance score of the top samples of those costs (recounted here with numpy)."""
    from gpu_util import DEV, T as TT, ids_t
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 31)
    lo, hi, ids = W.random_boxes(40, 6, seed=32, min_width=0.2, max_width=1.5)
    g = gp(p)
    n, M = 6, 200
    ub = torch.empty(n, device=DEV)
    costs = torch.empty(n, M, device=DEV)
    sd = torch.empty(n, dtype=torch.int32, device=DEV)
    B.bab_rollout_split(g.ctx, g.x0, g.goal, g.H, g.rho, TT(lo), TT(hi), ids_t(ids), n, M, 17, B.PREC_FP32, 5.0, ub, sd,
                        costs=costs)
    torch.cuda.synchronize()
    c, sd = costs.cpu().numpy(), sd.cpu().numpy()
    for i in range(n):
        for m in (0, 57, 199):
            u = np.array([oracle.lib().oracle_sample(17, int(ids[i]), m, j, float(lo[i, j]), float(hi[i, j]))
                          for j in range(40)])
            assert c[i, m] == pytest.approx(oracle.objective(p, u), rel=1e-5)
        k = 10  # ceil(5% of 200)
        top = sorted(range(M), key=lambda m: (c[i, m], m))[:k]
        scores = []
        for j in range(40):
            mid = np.float32(0.5) * np.float32(lo[i, j] + hi[i, j])
            u = np.array([oracle.lib().oracle_sample(17, int(ids[i]), m, j, float(lo[i, j]), float(hi[i, j]))
                          for m in top], dtype=np.float32)
            scores.append(np.float32(hi[i, j] - lo[i, j]) * abs(int((u <= mid).sum()) - int((u >= mid).sum())))
        scores = np.array(scores)
        want = int(np.argmax(scores)) if scores.max() > 0 else int(np.argmax(hi[i] - lo[i]))
        assert sd[i] == want
    assert np.array_equal(ub.cpu().numpy().view(np.uint32), c.min(axis=1).view(np.uint32))


def test_deep_identifiers_bit_exact(oracle, gp):
    """Boxes deeper than 62 splits: the children's identifiers continue as a hash of the path, as in the oracle."""
    lo, hi, _ = W.dyadic_boxes(10, 60, seed=11, max_depth=4)
    rng = np.random.default_rng(12)
    ids = np.concatenate([rng.integers(1 << 62, (1 << 63) - 1, size=30, dtype=np.int64).astype(np.uint64),
                          np.arange(1, 31, dtype=np.uint64) + np.uint64((1 << 62) - 31)])
    lb, ub = W.pool_values(60, seed=13)
    r = _branch(gp, lo, hi, lb, ub, ids, 12.0, 40, 0, 1.0, 0)
    o = oracle.prune_branch_heuristic(lo, hi, lb, ub, ids, 12.0, 40, pick_rule=0)
    _same(r, o)
    assert np.any(r["id"] >= np.uint64(1 << 62))
