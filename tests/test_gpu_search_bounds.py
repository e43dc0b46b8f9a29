"""The paper's own bounding (Section 3.2): search-integrated intermediate bounds recorded by the FP32 rollout, and
CROWN with given bounds and propagation early-stop (Algorithm 3), against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _search(g, lo, hi, ids, M, seed):
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    n = lo.shape[0]
    ub = torch.empty(n, device=DEV)
    bu = torch.empty(n, g.d, device=DEV)
    pl = torch.empty(n, g.H, g.sumh, device=DEV)
    pu = torch.empty_like(pl)
    xl = torch.empty(n, g.H + 1, g.p["s"], device=DEV)
    xu = torch.empty_like(xl)
    B.bab_rollout_search_bounds(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), n, M, seed, ub, pl, pu,
                                xl, xu, best_u=bu)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in dict(ub=ub, best_u=bu, pl=pl, pu=pu, xl=xl, xu=xu).items()}


@pytest.mark.parametrize("name,n,M", [("tiny", 9, 130), ("pushing", 4, 70)])
def test_search_bounds_match_oracle(oracle, gp, name, n, M):
    p = W.config_problem(name, 21)
    d = p["k"] * p["H"]
    lo, hi, ids = W.random_boxes(d, n, seed=22, min_width=0.1, max_width=1.0)
    g = gp(p)
    r = _search(g, lo, hi, ids, M, 5)
    # the same search as bab_rollout (the extremes are recorded on the side)
    plain = g.rollout(lo, hi, ids, M=M, seed=5)
    assert np.array_equal(r["ub"].view(np.uint32), plain["ub"].view(np.uint32))
    assert np.array_equal(r["best_u"].view(np.uint32), plain["best_u"].view(np.uint32))
    opl, opu, oxl, oxu = oracle.search_bounds(p, lo, hi, ids, M, 5)
    for got, want in ((r["pl"], opl), (r["pu"], opu), (r["xl"], oxl), (r["xu"], oxu)):
        scale = np.maximum(np.abs(want).max(axis=tuple(range(1, want.ndim)), keepdims=True), 1.0)
        assert np.all(np.abs(got - want) <= REL * scale)
    np.testing.assert_array_equal(r["xl"][:, 0], np.broadcast_to(p["x0"], r["xl"][:, 0].shape))


@pytest.mark.parametrize("t_stop", [0, 2, 5])
def test_crown_given_matches_oracle(oracle, gp, t_stop):
    """Given the oracle's search-integrated bounds (rounded to FP32, the same inputs on both sides), the GPU's
    early-stop CROWN equals the oracle's."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("tiny", 23)
    lo, hi, ids = W.random_boxes(10, 33, seed=24, min_width=0.1, max_width=1.0)
    pl, pu, xl, xu = (a.astype(np.float32) for a in oracle.search_bounds(p, lo, hi, ids, 64, 7))
    g = gp(p)
    lb = torch.empty(33, device=DEV)
    B.bab_bound_crown_given(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 33, T(pl), T(pu), T(xl), T(xu), t_stop,
                            lb)
    torch.cuda.synchronize()
    lb_o = oracle.crown_given(p, lo, hi, pl.astype(np.float64), pu.astype(np.float64), xl.astype(np.float64),
                              xu.astype(np.float64), t_stop)
    scale = np.maximum(oracle.crown(p, lo, hi)["scale"], 1.0)
    assert np.all(np.abs(lb.cpu().numpy() - lb_o) <= 1e-4 * scale)


def test_crown_given_with_interval_bounds_is_crown(gp):
    """Fed the interval bounds of bab_bound_ibp and no early stop, it is bab_bound_crown's bound before the
    rounding margin."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 25)
    lo, hi, ids = W.random_boxes(40, 19, seed=26, min_width=0.05, max_width=0.5)
    g = gp(p)
    _, pl, pu, xl, xu = g.ibp(lo, hi)
    c = g.crown(lo, hi)
    lb = torch.empty(19, device=DEV)
    B.bab_bound_crown_given(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 19, T(pl), T(pu), T(xl), T(xu), 0, lb)
    torch.cuda.synchronize()
    np.testing.assert_allclose(lb.cpu().numpy(), c["lb"] + c["margin"], rtol=1e-6, atol=1e-6)
    with pytest.raises(B.BabError):
        B.bab_bound_crown_given(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 19, T(pl), T(pu), T(xl), T(xu),
                                g.H + 1, lb)
