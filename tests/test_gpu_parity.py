"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle, on the same seeded inputs.

Tolerances: FP32 results must lie within 1e-5 relative of the oracle; for bounds "relative" means relative to
the oracle's sum of |every term added into the bound| (the magnitude FP32 rounding scales with, at least 1),
for other values relative to the value.  Bounds from the 3-term BF16 split products on tensor cores have a
stated band of 5e-5 of that scale.  Every returned lower bound must not exceed the oracle's (the outward
margin covers the rounding); integer, index and box outputs are bit-exact.
"""
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
    assert torch.cuda.is_available()




def bound_scale(o):
    """Tolerance scale of a bound: the oracle's sum of |every term added into it| (at least 1), the magnitude
    that FP32 rounding in any evaluation order scales with."""
    return np.maximum(o["scale"], 1.0)


def tiny():
    p = W.config_problem("tiny", 0)
    lo, hi, ids = W.grid_boxes(10, 6)
    return p, lo, hi, ids


# ----------------------------------------------------------------------------------------------------------------
# rollout (Section 3.3)
# ----------------------------------------------------------------------------------------------------------------

def test_samples_bit_identical_single_draw(oracle, gp):
    """With one sample per box the GPU's best_u is that sample: it must equal the oracle's draw bit for bit."""
    p, lo, hi, ids = tiny()
    g = gp(p)
    r = g.rollout(lo, hi, ids, M=1, seed=77)
    _, bu_o, _ = oracle.rollout(p, lo, hi, ids, 1, 77)
    assert np.array_equal(r["best_u"].view(np.uint32), bu_o.view(np.uint32))


@pytest.mark.parametrize("M", [256, 100, 1])
def test_rollout_tiny_matches_oracle(oracle, gp, M):
    p, lo, hi, ids = tiny()
    g = gp(p)
    r = g.rollout(lo, hi, ids, M=M, seed=5, incumbent=True)
    ub_o, bu_o, _ = oracle.rollout(p, lo, hi, ids, M, 5)
    np.testing.assert_allclose(r["ub"], ub_o, rtol=REL, atol=0)
    same = np.all(r["best_u"] == bu_o, axis=1)
    assert same.mean() > 0.9
    for i in np.flatnonzero(~same):  # a different argmin must be a near-tie
        assert oracle.objective(p, r["best_u"][i].astype(np.float64)) <= ub_o[i] * (1 + 2 * REL)
    f_inc = oracle.objective(p, r["inc_u"].astype(np.float64))
    assert r["inc_val"] == pytest.approx(f_inc, rel=1e-10)  # FP64 on both sides, different summation order
    assert r["inc_val"] <= ub_o.min() * (1 + 2 * REL)


def test_rollout_pushing_ragged_tiles(oracle, gp):
    """H=20, 128-wide network; 130 samples = two full 64-row tiles and a ragged one."""
    p = W.config_problem("pushing", 1)
    lo, hi, ids = W.dyadic_boxes(40, 12, seed=3, max_depth=3)
    g = gp(p)
    r = g.rollout(lo, hi, ids, M=130, seed=9, incumbent=True)
    ub_o, bu_o, _ = oracle.rollout(p, lo, hi, ids, 130, 9)
    np.testing.assert_allclose(r["ub"], ub_o, rtol=REL, atol=0)
    f_inc = oracle.objective(p, r["inc_u"].astype(np.float64))
    assert r["inc_val"] == pytest.approx(f_inc, rel=1e-10)  # FP64 on both sides, different summation order


def test_rollout_zero_boxes_and_device_count(oracle, gp):
    p, lo, hi, ids = tiny()
    g = gp(p)
    from gpu_util import T, ids_t, DEV
    from paper_2412_09584_gb300 import binding as B
    ub = torch.full((64,), -7.0, device=DEV)
    B.bab_rollout(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), 0, 16, 1, B.PREC_FP32, ub)
    dn = torch.tensor([10], dtype=torch.int32, device=DEV)
    B.bab_rollout(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), 64, 16, 1, B.PREC_FP32, ub, d_n=dn)
    torch.cuda.synchronize()
    u = ub.cpu().numpy()
    ub_o, _, _ = oracle.rollout(p, lo[:10], hi[:10], ids[:10], 16, 1)
    np.testing.assert_allclose(u[:10], ub_o, rtol=REL)
    assert (u[10:] == -7.0).all()
    with pytest.raises(B.BabError):
        B.bab_rollout(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), 64, 0, 1, B.PREC_FP32, ub)


# ----------------------------------------------------------------------------------------------------------------
# interval bounds
# ----------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,n", [("tiny", 64), ("pushing", 19)])
def test_ibp_matches_oracle_and_contains_it(oracle, gp, name, n):
    p = W.config_problem(name, 2)
    d = p["k"] * p["H"]
    lo, hi, _ = W.random_boxes(d, n, seed=4, min_width=0.0, max_width=0.5)
    g = gp(p)
    lb, pl, pu, xl, xu = g.ibp(lo, hi)
    lb_o, pl_o, pu_o, xl_o, xu_o = oracle.ibp(p, lo, hi)
    for gv, ov in ((pl, pl_o), (pu, pu_o), (xl, xl_o), (xu, xu_o)):
        scale = np.maximum(np.abs(ov), 1.0)
        assert np.all(np.abs(gv - ov) <= REL * scale)
    # outward rounding: the FP32 intervals contain the exact ones
    assert np.all(pl <= pl_o + 1e-12 * np.abs(pl_o)) and np.all(pu >= pu_o - 1e-12 * np.abs(pu_o))
    assert np.all(xl <= xl_o + 1e-12 * np.abs(xl_o)) and np.all(xu >= xu_o - 1e-12 * np.abs(xu_o))
    assert np.all(lb <= lb_o + 1e-12 * np.abs(lb_o))
    np.testing.assert_allclose(lb, lb_o, rtol=REL, atol=REL)


# ----------------------------------------------------------------------------------------------------------------
# CROWN bound
# ----------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,n,maxw", [("tiny", 64, 2.0), ("tiny", 37, 0.3), ("pushing", 21, 0.2),
                                         ("pushing", 5, 2.0), ("pushing", 200, 2.0)])
def test_crown_matches_oracle(oracle, gp, name, n, maxw):
    p = W.config_problem(name, 3)
    d = p["k"] * p["H"]
    if maxw >= 2.0 and name == "tiny":
        lo, hi, _ = W.grid_boxes(d, 6)
        lo, hi = lo[:n], hi[:n]
    else:
        lo, hi, _ = W.random_boxes(d, n, seed=5, min_width=0.0, max_width=maxw)
    g = gp(p)
    r = g.crown(lo, hi)
    o = oracle.crown(p, lo, hi)
    scale = bound_scale(o)
    raw = r["lb"].astype(np.float64) + r["margin"]
    assert np.all(r["margin"] >= 0)
    assert np.all(np.abs(raw - o["lb"]) <= REL * scale), np.max(np.abs(raw - o["lb"]) / scale)
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"])), "returned bound above the exact CROWN bound"
    assert np.all(r["margin"] <= REL * scale)
    mu_scale = np.maximum(np.abs(o["lin_coef"]).max(axis=1, keepdims=True), 1.0)
    assert np.all(np.abs(r["lin_coef"] - o["lin_coef"]) <= REL * mu_scale)


def test_crown_zero_width_box_equals_objective(oracle, gp):
    p = W.config_problem("pushing", 4)
    lo, hi, _ = W.random_boxes(40, 6, seed=6, min_width=0.0, max_width=0.0)
    g = gp(p)
    r = g.crown(lo, hi)
    f = np.array([oracle.objective(p, lo[i].astype(np.float64)) for i in range(6)])
    assert np.all(r["lb"] <= f)
    np.testing.assert_allclose(r["lb"] + r["margin"], f, rtol=REL)


def test_crown_sound_at_sampled_points(oracle, gp):
    p = W.make_problem(4, 2, [32, 32], 5, 0.01, seed=8, weight_scale=1.0)
    lo, hi, _ = W.random_boxes(10, 16, seed=9, min_width=0.05, max_width=0.4)
    g = gp(p)
    r = g.crown(lo, hi)
    rng = np.random.default_rng(0)
    for i in range(16):
        for _ in range(200):
            u = lo[i] + rng.uniform(size=10) * (hi[i] - lo[i])
            assert r["lb"][i] <= oracle.objective(p, u.astype(np.float64))


def test_crown_given_alpha_matches_oracle(oracle, gp):
    p = W.make_problem(4, 2, [32, 32], 5, 0.01, seed=10, weight_scale=0.3)
    lo, hi, _ = W.random_boxes(10, 40, seed=11, min_width=0.3, max_width=1.0)
    alpha = np.random.default_rng(1).uniform(0, 1, size=(40, 5, 64)).astype(np.float32)
    g = gp(p)
    r = g.crown(lo, hi, alpha=alpha)
    o = oracle.crown(p, lo, hi, alpha=alpha.astype(np.float64))
    scale = bound_scale(o)
    assert np.all(np.abs(r["lb"] + r["margin"] - o["lb"]) <= REL * scale)
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))


# ----------------------------------------------------------------------------------------------------------------
# alpha-CROWN: gradient and projected Adam
# ----------------------------------------------------------------------------------------------------------------

def test_alpha_gradient_and_step_match_oracle(oracle, gp):
    p = W.make_problem(4, 2, [32, 32], 5, 0.01, seed=12, weight_scale=0.3)
    lo, hi, _ = W.random_boxes(10, 24, seed=13, min_width=0.3, max_width=1.0)
    g = gp(p)
    best, alpha, hist = g.alpha_steps(lo, hi, steps=1, lr=0.1)
    a0 = oracle.adaptive_alpha(p, lo, hi)
    lb_o, grad_o, _ = oracle.alpha_grad(p, lo, hi, a0)
    gs = np.maximum(np.abs(grad_o).max(axis=(1, 2), keepdims=True), 1e-30)
    assert np.all(np.abs(hist[0]["grad"] - grad_o) <= 1e-4 * gs)
    o = oracle.crown(p, lo, hi, a0)
    scale = bound_scale(o)
    assert np.all(np.abs(hist[0]["lb"] - lb_o) <= REL * scale)
    a = a0.copy()
    m, v = np.zeros_like(a), np.zeros_like(a)
    oracle.adam_ascent(a, m, v, grad_o, 1, 0.1)
    # Adam's first step moves by lr * sign(g) wherever g is clearly nonzero
    clear = np.abs(grad_o) > 1e-3 * gs
    np.testing.assert_allclose(alpha[clear], a[clear], atol=1e-5)


def test_alpha_optimisation_twenty_steps(oracle, gp):
    p = W.make_problem(4, 2, [32, 32], 5, 0.0, seed=14, weight_scale=0.3)
    lo, hi, _ = W.random_boxes(10, 16, seed=15, min_width=0.3, max_width=1.0)
    g = gp(p)
    best, alpha, hist = g.alpha_steps(lo, hi, steps=20, lr=0.1)
    best_o, alpha_o, _, _ = oracle.alpha_optimize(p, lo, hi, 20, 0.1)
    lb0 = oracle.crown(p, lo, hi)["lb"]
    assert np.all(best >= lb0 - 1e-4 * np.maximum(np.abs(lb0), 1))   # never worse than the adaptive slopes
    # every returned bound is sound: below the objective at samples
    rng = np.random.default_rng(2)
    for i in range(16):
        u = lo[i] + rng.uniform(size=(50, 10)) * (hi[i] - lo[i])
        fmin = min(oracle.objective(p, x.astype(np.float64)) for x in u)
        assert best[i] <= fmin
    np.testing.assert_allclose(best, best_o, rtol=1e-3, atol=1e-3)


# ----------------------------------------------------------------------------------------------------------------
# prune / pick out / split: bit-exact
# ----------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,n_pick,inc,ties,nans", [(300, 64, 11.0, 0.0, 0.0), (300, 500, 12.0, 0.1, 0.05),
                                                    (1000, 200, 9.5, 0.3, 0.02), (5000, 1024, 13.0, 0.05, 0.0),
                                                    (77, 0, 10.0, 0.0, 0.0), (64, 32, -1e9, 0.0, 0.0)])
def test_prune_branch_bit_exact(oracle, gp, n, n_pick, inc, ties, nans):
    from paper_2412_09584_gb300 import binding as B
    p, _, _, _ = tiny()
    g = gp(p)
    d = 10
    lo, hi, ids = W.dyadic_boxes(d, n, seed=n + n_pick, max_depth=5)
    lb, ub = W.pool_values(n, seed=n, nan_frac=nans, tie_frac=ties)
    B.bab_status(g.ctx)  # clear
    r = g.prune_branch(lo, hi, lb, ub, ids, inc, n_pick)
    o = oracle.prune_branch(lo, hi, lb, ub, ids, inc, n_pick)
    # a NaN bound is kept and reported through the device status, without failing the call
    assert B.bab_status(g.ctx) == (-6 if np.isnan(lb).any() else 0)
    assert np.array_equal(r["keep"], o["keep"])
    assert (r["n_children"], r["n_rest"]) == (o["n_children"], o["n_rest"])
    for key in ("lo", "hi", "lb", "ub"):
        assert np.array_equal(r[key].view(np.uint32), o[key].view(np.uint32)), key
    assert np.array_equal(r["id"], o["id"])


def test_prune_branch_empty_pool(gp):
    p, _, _, _ = tiny()
    g = gp(p)
    z = np.zeros((0, 10), np.float32)
    r = g.prune_branch(z, z, np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.uint64), 1.0, 8)
    assert r["n_children"] == 0 and r["n_rest"] == 0


# ----------------------------------------------------------------------------------------------------------------
# full-size workload (4096 boxes x 1024 samples x H=20), launch configuration of bench.py, sampled outputs
# ----------------------------------------------------------------------------------------------------------------

def test_pushing_full_size_sampled(oracle, gp):
    p = W.config_problem("pushing", 0)
    lo, hi, ids = W.grid_boxes(40, 12)
    g = gp(p)
    r = g.rollout(lo, hi, ids, M=1024, seed=2024, incumbent=True)
    c = g.crown(lo, hi)
    rows = [0, 1, 777, 2048, 4095]
    ub_o, _, _ = oracle.rollout(p, lo[rows], hi[rows], ids[rows], 1024, 2024)
    np.testing.assert_allclose(r["ub"][rows], ub_o, rtol=REL)
    o = oracle.crown(p, lo[rows], hi[rows])
    scale = bound_scale(o)
    assert np.all(np.abs(c["lb"][rows] + c["margin"][rows] - o["lb"]) <= REL * scale)
    assert np.all(c["lb"][rows] <= o["lb"])
    # properties at every box: bounds below the sampled objective, finite margins
    assert np.all(c["lb"] <= r["ub"]) and np.all(np.isfinite(c["margin"]))
    assert r["inc_val"] == pytest.approx(oracle.objective(p, r["inc_u"].astype(np.float64)), rel=1e-10)


# ----------------------------------------------------------------------------------------------------------------
# tensor-core rollouts (tcgen05): 3-term BF16 split and plain BF16 with an FP32 re-score
# ----------------------------------------------------------------------------------------------------------------

REL_BF16X3 = 1e-5   # three BF16 partial products per FP32 product: about 2^-16 relative each, FP32 accumulation


def test_tc_samples_bit_identical(oracle, gp):
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 7)
    lo, hi, ids = W.dyadic_boxes(40, 9, seed=7, max_depth=3)
    g = gp(p)
    for prec in (B.PREC_BF16X3, B.PREC_BF16):
        r = g.rollout(lo, hi, ids, M=1, seed=31, precision=prec)
        _, bu_o, _ = oracle.rollout(p, lo, hi, ids, 1, 31)
        assert np.array_equal(r["best_u"].view(np.uint32), bu_o.view(np.uint32))


@pytest.mark.parametrize("name,M,n", [("pushing", 256, 10), ("pushing", 300, 10), ("tiny", 256, 10), ("tiny", 77, 10),
                                      ("pushing", 4, 130), ("tiny", 48, 37), ("pushing", 33, 9)])
def test_tc_bf16x3_rollout_matches_oracle(oracle, gp, name, M, n):
    """Sample tiles of 128 rows: M >= 128 spans several tiles per box; smaller M packs 128 // M boxes per tile
    (idle rows when M does not divide 128, a ragged last tile)."""
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 8)
    d = p["k"] * p["H"]
    lo, hi, ids = W.dyadic_boxes(d, n, seed=8, max_depth=3)
    g = gp(p)
    r = g.rollout(lo, hi, ids, M=M, seed=12, precision=B.PREC_BF16X3, incumbent=True)
    ub_o, _, _ = oracle.rollout(p, lo, hi, ids, M, 12)
    np.testing.assert_allclose(r["ub"], ub_o, rtol=REL_BF16X3, atol=0)
    f_best = np.array([oracle.objective(p, u.astype(np.float64)) for u in r["best_u"]])
    assert np.all(f_best <= ub_o * (1 + 2 * REL_BF16X3))
    assert r["inc_val"] == pytest.approx(oracle.objective(p, r["inc_u"].astype(np.float64)), rel=1e-10)


def test_tc_bf16_rollout_topk_rescore(oracle, gp):
    """With a top-k re-score, the k boxes of smallest BF16 ub get the FP32 objective of their best sample, the
    others keep their BF16 value (close to it); the incumbent stays the FP64 objective of its plan."""
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 10)
    lo, hi, ids = W.dyadic_boxes(40, 40, seed=10, max_depth=4)
    g = gp(p)
    r_all = g.rollout(lo, hi, ids, M=64, seed=17, precision=B.PREC_BF16)
    B.bab_set_rescore_topk(g.ctx, 8)
    r = g.rollout(lo, hi, ids, M=64, seed=17, precision=B.PREC_BF16, incumbent=True)
    np.testing.assert_array_equal(r["best_u"], r_all["best_u"])  # the same samples are chosen
    f_best = np.array([oracle.objective(p, u.astype(np.float64)) for u in r["best_u"]])
    rescored = np.isclose(r["ub"], r_all["ub"], rtol=0, atol=0)
    assert rescored.sum() >= 8
    np.testing.assert_allclose(r["ub"][rescored], f_best[rescored], rtol=REL)
    np.testing.assert_allclose(r["ub"], f_best, rtol=5e-2)
    assert r["inc_val"] == pytest.approx(oracle.objective(p, r["inc_u"].astype(np.float64)), rel=1e-10)
    with pytest.raises(B.BabError):
        B.bab_set_rescore_topk(g.ctx, -1)


def test_tc_bf16_rollout_rescored(oracle, gp):
    """BF16 operands pick each box's best sample; its value is then re-scored in FP32, so ub equals the objective
    of the returned plan to FP32 accuracy and is close to the best sampled value."""
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 9)
    lo, hi, ids = W.dyadic_boxes(40, 10, seed=9, max_depth=3)
    g = gp(p)
    r = g.rollout(lo, hi, ids, M=256, seed=13, precision=B.PREC_BF16, incumbent=True)
    ub_o, _, _ = oracle.rollout(p, lo, hi, ids, 256, 13)
    f_best = np.array([oracle.objective(p, u.astype(np.float64)) for u in r["best_u"]])
    np.testing.assert_allclose(r["ub"], f_best, rtol=REL)
    assert np.all(f_best >= ub_o * (1 - 1e-12))
    np.testing.assert_allclose(r["ub"], ub_o, rtol=1e-2)


# ----------------------------------------------------------------------------------------------------------------
# tensor-core CROWN (3-term BF16 split products, margin covers the split)
# ----------------------------------------------------------------------------------------------------------------

REL_TC = 5e-5      # band of the 3-term BF16 split products, relative to the bound's scale
MARGIN_TC = 2e-4   # worst-case split margin: (3.1 * 2^-16 + gamma_K) per product term, relative to the bound's scale


@pytest.mark.parametrize("name,n,maxw", [("tiny", 64, 2.0), ("tiny", 130, 0.3), ("pushing", 21, 0.2),
                                         ("pushing", 200, 2.0)])
def test_crown_tc_matches_oracle(oracle, gp, name, n, maxw):
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 3)
    d = p["k"] * p["H"]
    lo, hi, _ = W.random_boxes(d, n, seed=n, min_width=0.0, max_width=maxw)
    g = gp(p)
    r = g.crown(lo, hi, precision=B.PREC_BF16X3)
    o = oracle.crown(p, lo, hi)
    scale = bound_scale(o)
    raw = r["lb"].astype(np.float64) + r["margin"]
    assert np.all(r["margin"] >= 0)
    assert np.all(np.abs(raw - o["lb"]) <= REL_TC * scale), np.max(np.abs(raw - o["lb"]) / scale)
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"])), "returned bound above the exact CROWN bound"
    assert np.all(r["margin"] <= MARGIN_TC * scale)
    # the coefficients of early steps pass through up to H*L chained split products and lose more relative
    # accuracy than the bound (which is checked above): a sanity band of 1e-3 of the row's L1 norm
    mu_scale = np.maximum(np.abs(o["lin_coef"]).sum(axis=1, keepdims=True), 1.0)
    err = np.abs(r["lin_coef"] - o["lin_coef"]) / mu_scale
    assert np.all(err <= 1e-3), err.max()


def test_crown_tc_given_alpha_and_zero_width(oracle, gp):
    from paper_2412_09584_gb300 import binding as B
    p = W.make_problem(4, 2, [32, 32], 5, 0.01, seed=10, weight_scale=0.3)
    lo, hi, _ = W.random_boxes(10, 40, seed=11, min_width=0.3, max_width=1.0)
    alpha = np.random.default_rng(1).uniform(0, 1, size=(40, 5, 64)).astype(np.float32)
    g = gp(p)
    r = g.crown(lo, hi, alpha=alpha, precision=B.PREC_BF16X3)
    o = oracle.crown(p, lo, hi, alpha=alpha.astype(np.float64))
    scale = bound_scale(o)
    assert np.all(np.abs(r["lb"] + r["margin"] - o["lb"]) <= REL_TC * scale)
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))
    q = W.config_problem("pushing", 4)
    z, _, _ = W.random_boxes(40, 6, seed=6, min_width=0.0, max_width=0.0)
    g2 = gp(q)
    rz = g2.crown(z, z, precision=B.PREC_BF16X3)
    f = np.array([oracle.objective(q, z[i].astype(np.float64)) for i in range(6)])
    assert np.all(rz["lb"] <= f)
    np.testing.assert_allclose(rz["lb"] + rz["margin"], f, rtol=REL_TC)


def test_update_incumbent_matches_rollout_incumbent(gp):
    """The incumbent step as its own call (on another stream) equals the one bab_rollout performs."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 12)
    lo, hi, ids = W.dyadic_boxes(40, 33, seed=12, max_depth=4)
    g = gp(p)
    r = g.rollout(lo, hi, ids, M=128, seed=21, precision=B.PREC_BF16X3, incumbent=True)
    r2 = g.rollout(lo, hi, ids, M=128, seed=21, precision=B.PREC_BF16X3)
    inc_val = torch.full((1,), np.inf, dtype=torch.float64, device=DEV)
    inc_u = torch.zeros(g.d, device=DEV)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        B.bab_update_incumbent(g.ctx, g.x0, g.goal, g.H, g.rho, T(r2["ub"]), T(r2["best_u"]), 33, inc_val, inc_u)
    torch.cuda.synchronize()
    assert float(inc_val.item()) == r["inc_val"]
    np.testing.assert_array_equal(inc_u.cpu().numpy(), r["inc_u"])
