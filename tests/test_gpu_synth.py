"""The paper's synthetic objective (Section 4, f(u) = sum 5 u_i^2 + cos(50 u_i)) on the GPU: the sampled search
against the oracle's (the same samples; FP32 against FP64 values), the bound sound against the oracle's exact
per-term minima and close to them, the cross-entropy mode, and Algorithm 2 reaching d g* with the GPU's prune /
pick-out / bisect on a context without a network."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu

G_STAR = -0.9803391  # per-coordinate minimum (oracle pins: -0.980339)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture
def sctx():
    from paper_2412_09584_gb300 import binding as B
    c = B.bab_context_create()
    yield c
    B.bab_destroy(c)


def _search(c, lo, hi, ids, M, seed, iters=0, warm=None, incumbent=False):
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    n, d = lo.shape
    ub = torch.empty(n, device=DEV)
    bu = torch.empty(n, d, device=DEV)
    iv = torch.full((1,), np.inf, dtype=torch.float64, device=DEV) if incumbent else None
    iu = torch.zeros(d, device=DEV) if incumbent else None
    B.bab_synth_search(c, d, T(lo), T(hi), ids_t(ids), n, M, seed, ub, bu, iters=iters, elites=10, jitter=1e-3,
                       warm_u=None if warm is None else T(warm), inc_val=iv, inc_u=iu)
    torch.cuda.synchronize()
    out = {"ub": ub.cpu().numpy(), "best_u": bu.cpu().numpy()}
    if incumbent:
        out["inc_val"], out["inc_u"] = float(iv.item()), iu.cpu().numpy()
    return out


def test_synth_search_matches_oracle(oracle, sctx):
    lo, hi, ids = W.random_boxes(12, 20, seed=51, min_width=0.05, max_width=2.0)
    r = _search(sctx, lo, hi, ids, 300, 7, incumbent=True)
    ub_o, _ = oracle.synth_search(lo, hi, ids, 300, 7)
    assert np.all(np.abs(r["ub"] - ub_o) <= 2e-6 * 12)
    assert np.all(r["best_u"] >= lo) and np.all(r["best_u"] <= hi)
    for i in range(20):
        assert oracle.synth_f(r["best_u"][i].astype(np.float64)) == pytest.approx(float(r["ub"][i]), abs=2e-6 * 12)
    best = int(np.argmin(r["ub"]))
    assert r["inc_val"] == pytest.approx(oracle.synth_f(r["best_u"][best].astype(np.float64)), rel=1e-12)


@pytest.mark.parametrize("n,d,wmax", [(200, 5, 2.0), (300, 33, 0.1), (64, 100, 0.01)])
def test_synth_bound_sound_and_close(oracle, sctx, n, d, wmax):
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    lo, hi, _ = W.random_boxes(d, n, seed=d, min_width=0.0, max_width=wmax)
    lb = torch.empty(n, device=DEV)
    B.bab_synth_bound(sctx, d, T(lo), T(hi), n, lb)
    torch.cuda.synchronize()
    lb = lb.cpu().numpy().astype(np.float64)
    lb_o = oracle.synth_bound(lo, hi)
    assert np.all(lb <= lb_o)
    assert np.all(lb >= lb_o - d * 1e-6 - 1e-6 * np.abs(lb_o))


def test_synth_bound_below_grid_minimum(oracle, sctx):
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    lo, hi, _ = W.random_boxes(2, 30, seed=52, min_width=0.01, max_width=0.6)
    lb = torch.empty(30, device=DEV)
    B.bab_synth_bound(sctx, 2, T(lo), T(hi), 30, lb)
    torch.cuda.synchronize()
    for i in range(30):
        g = np.stack(np.meshgrid(np.linspace(lo[i, 0], hi[i, 0], 201), np.linspace(lo[i, 1], hi[i, 1], 201)), -1)
        assert lb[i].item() <= (5 * g ** 2 + np.cos(50 * g)).sum(-1).min()


def test_synth_cem_warm_start_and_monotone(oracle, sctx):
    lo, hi, ids = W.random_boxes(16, 10, seed=53, min_width=0.1, max_width=1.0)
    warm = (lo + np.random.default_rng(4).uniform(size=lo.shape).astype(np.float32) * (hi - lo)).astype(np.float32)
    r1 = _search(sctx, lo, hi, ids, 128, 3, iters=1, warm=warm)
    r4 = _search(sctx, lo, hi, ids, 128, 3, iters=4, warm=warm)
    assert np.all(r4["ub"] <= r1["ub"])
    for i in range(10):
        assert r1["ub"][i] <= oracle.synth_f(warm[i].astype(np.float64)) + 2e-6 * 16
        assert oracle.synth_f(r4["best_u"][i].astype(np.float64)) == pytest.approx(float(r4["ub"][i]), abs=2e-6 * 16)


def test_synth_bab_reaches_the_optimum(sctx):
    """Algorithm 2 on the GPU (d = 8): search, bound, prune / pick-out / bisect; the incumbent approaches d g* and
    the smallest lower bound of the pool stays below it."""
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    d, n_pick, M = 8, 256, 64
    lo, hi, ids = W.grid_boxes(d, 4)
    n = lo.shape[0]
    cap = n + 400 * n_pick
    f = dict(device=DEV, dtype=torch.float32)
    pools = [{"lo": torch.zeros(cap, d, **f), "hi": torch.zeros(cap, d, **f), "lb": torch.zeros(cap, **f),
              "ub": torch.zeros(cap, **f), "id": torch.zeros(cap, dtype=torch.int64, device=DEV)} for _ in range(2)]
    P = pools[0]
    P["lo"][:n], P["hi"][:n], P["id"][:n] = T(lo), T(hi), ids_t(ids)
    bu = torch.empty(cap, d, **f)
    iv = torch.full((1,), np.inf, dtype=torch.float64, device=DEV)
    iu = torch.zeros(d, **f)
    B.bab_synth_search(sctx, d, P["lo"], P["hi"], P["id"], n, M, 1, P["ub"], bu, inc_val=iv, inc_u=iu)
    B.bab_synth_bound(sctx, d, P["lo"], P["hi"], n, P["lb"])
    keep = torch.empty(cap, dtype=torch.uint8, device=DEV)
    counts = torch.zeros(3, dtype=torch.int32, device=DEV)
    live = torch.tensor([n], dtype=torch.int32, device=DEV)
    cur, nmax = 0, n
    for it in range(300):
        src, dst = pools[cur], pools[cur ^ 1]
        B.bab_prune_branch(sctx, d, src["lo"], src["hi"], src["lb"], src["ub"], src["id"], nmax, iv, n_pick, 0.75,
                           cap, dst["lo"], dst["hi"], dst["lb"], dst["ub"], dst["id"], keep, counts, d_n=live)
        nmax = min(nmax + n_pick, cap - n_pick)
        B.bab_synth_search(sctx, d, dst["lo"], dst["hi"], dst["id"], 2 * n_pick, M, 2 + it, dst["ub"], bu,
                           inc_val=iv, inc_u=iu, d_n=counts[0:1])
        B.bab_synth_bound(sctx, d, dst["lo"], dst["hi"], 2 * n_pick, dst["lb"], d_n=counts[0:1])
        live.copy_(counts[2:3])
        cur ^= 1
    torch.cuda.synchronize()
    nl = int(counts[2].item())
    lbmin = float(pools[cur]["lb"][:nl].min().item())
    inc = float(iv.item())
    print("synthetic BaB: incumbent", inc, "target", d * G_STAR, "min lb", lbmin)
    assert inc == pytest.approx(d * G_STAR, abs=5e-3)
    assert lbmin <= d * G_STAR + 1e-6
    assert B.bab_status(sctx) == 0


def test_synth_argument_errors_and_empty(sctx):
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    lo, hi, ids = W.random_boxes(4, 2, seed=54)
    ub, bu = torch.empty(2, device=DEV), torch.empty(2, 4, device=DEV)
    for M, iters, E in ((B.CEM_MAX_SAMPLES + 1, 0, 1), (16, 2, 17), (16, -1, 4)):
        with pytest.raises(B.BabError):
            B.bab_synth_search(sctx, 4, T(lo), T(hi), ids_t(ids), 2, M, 1, ub, bu, iters=iters, elites=E)
    e = torch.empty(0, 4, device=DEV)
    B.bab_synth_search(sctx, 4, e, e, torch.empty(0, dtype=torch.int64, device=DEV), 0, 16, 1,
                       torch.empty(0, device=DEV), e)
    B.bab_synth_bound(sctx, 4, e, e, 0, torch.empty(0, device=DEV))
    # a context without a network refuses the network calls
    lb = torch.empty(2, device=DEV)
    with pytest.raises(B.BabError):
        B.bab_bound_crown(sctx, T(np.zeros(4)), T(np.zeros(4)), 2, 0.0, T(lo), T(hi), 2, lb)
    torch.cuda.synchronize()
    assert B.bab_status(sctx) == 0
