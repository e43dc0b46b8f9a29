"""CROWN with 3-term TF32 split products on the tensor cores (BAB_PREC_TF32X3): Appendix B.1, Theorems 1-2, with
every backward product A' W_l evaluated as A'_hi W_hi + A'_hi W_lo + A'_lo W_hi from TF32 halves (11 significant
bits each) and FP32 accumulation, the backward image streamed through shared memory.

* Against the FP64 oracle: the raw bound (lb + margin) within 1e-5 of the bound's scale, the FP32 tolerance (the
  TF32 halves leave about 2^-22 per product, against 2^-16 for BF16 halves), the returned bound never above the
  oracle's, the margin within 1e-3 of the oracle's FP64 evaluation of the TF32-split margin formula.
* Tighter than the BF16 split: a smaller margin on every box.
* alpha-CROWN through it: each Adam step's bound and gradient against the oracle's at the GPU's own slopes.
* Networks wider than 128 (two 128-row feature blocks per product): against the oracle on a small wide network,
  and at the object-manipulation scale against the oracle's CROWN on the GPU's own interval bounds.
* Refusals: the obstacle cost and hidden widths that are not multiples of 32 (BAB_ERR_UNSUPPORTED).
"""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5
MARGIN_REL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("name,n,maxw,rho", [("tiny", 64, 2.0, None), ("tiny", 130, 0.3, 0.02),
                                             ("pushing", 21, 0.2, None), ("pushing", 200, 2.0, None),
                                             ("pushing", 333, 0.05, 0.01)])
def test_tf32x3_matches_oracle(oracle, gp, name, n, maxw, rho):
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 3)
    if rho is not None:
        p["rho"] = rho
    d = p["k"] * p["H"]
    lo, hi, _ = W.random_boxes(d, n, seed=n + 7, min_width=0.0, max_width=maxw)
    g = gp(p)
    r = g.crown(lo, hi, precision=B.PREC_TF32X3)
    o = oracle.crown_margin(p, lo, hi, prec=2)
    scale = np.maximum(o["scale"], 1.0)
    np.testing.assert_allclose(r["margin"], o["margin"], rtol=MARGIN_REL, atol=0)
    err = np.abs(r["lb"].astype(np.float64) + r["margin"] - o["lb"]) / scale
    assert np.all(err <= REL), err.max()
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"])), "returned bound above the exact CROWN bound"
    # the coefficients of early steps pass through up to H L chained split products: a band of 1e-4 of the row's
    # L1 norm (the BF16 split needs 1e-3)
    oc = oracle.crown(p, lo, hi)
    mu_scale = np.maximum(np.abs(oc["lin_coef"]).sum(axis=1, keepdims=True), 1.0)
    e_mu = np.abs(r["lin_coef"] - oc["lin_coef"]) / mu_scale
    assert np.all(e_mu <= 1e-4), e_mu.max()


def test_tf32x3_tighter_than_bf16x3(oracle, gp):
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 5)
    lo, hi, _ = W.random_boxes(p["k"] * p["H"], 96, seed=5, min_width=0.01, max_width=1.0)
    g = gp(p)
    rt = g.crown(lo, hi, precision=B.PREC_TF32X3)
    rb = g.crown(lo, hi, precision=B.PREC_BF16X3)
    o = oracle.crown(p, lo, hi)
    assert np.all(rt["margin"] < rb["margin"])
    et = np.abs(rt["lb"].astype(np.float64) + rt["margin"] - o["lb"])
    eb = np.abs(rb["lb"].astype(np.float64) + rb["margin"] - o["lb"])
    assert et.mean() < eb.mean()
    assert np.all(rt["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))


def test_tf32x3_zero_width_box_equals_objective(oracle, gp):
    from paper_2412_09584_gb300 import binding as B
    q = W.config_problem("pushing", 4)
    z, _, _ = W.random_boxes(q["k"] * q["H"], 6, seed=6, min_width=0.0, max_width=0.0)
    g = gp(q)
    r = g.crown(z, z, precision=B.PREC_TF32X3)
    f = np.array([oracle.objective(q, z[i].astype(np.float64)) for i in range(6)])
    assert np.all(r["lb"] <= f)
    np.testing.assert_allclose(r["lb"] + r["margin"], f, rtol=REL)


def test_tf32x3_alpha_steps_match_oracle(oracle, gp):
    """Ten projected Adam steps through the TF32-split CROWN; at each step the gradient the GPU computed at its own
    slopes equals the oracle's at those slopes (1e-5 of the row's largest), and the bound is at most the oracle's
    and within the split margin of it."""
    from paper_2412_09584_gb300 import binding as B
    p = W.make_problem(4, 2, [32, 32], 5, 0.01, seed=14, weight_scale=0.3)
    lo, hi, _ = W.random_boxes(10, 16, seed=15, min_width=0.3, max_width=1.0)
    g = gp(p)
    a0 = g.alpha_init(lo, hi).cpu().numpy()
    _, _, hist = g.alpha_steps(lo, hi, steps=10, lr=0.1, precision=B.PREC_TF32X3)
    for k, h in enumerate(hist):
        a_before = (a0 if k == 0 else hist[k - 1]["alpha"]).astype(np.float64)
        lb_o, g_o, _ = oracle.alpha_grad(p, lo, hi, a_before)
        om = oracle.crown_margin(p, lo, hi, alpha=a_before, prec=2)
        scale = np.maximum(om["scale"], 1.0)
        assert np.all(h["lb"] <= lb_o + 1e-12 * np.abs(lb_o))
        assert np.all(np.abs(h["lb"] - lb_o) <= REL * scale + 1.001 * om["margin"]), k
        gs = np.maximum(np.abs(g_o).max(axis=(1, 2)), 1e-30)
        e_g = np.abs(h["grad"] - g_o).max(axis=(1, 2)) / gs
        assert np.all(e_g <= REL), (k, e_g.max())


def test_tf32x3_alpha_optimize_matches_steps(gp):
    """bab_alpha_optimize in TF32x3 (interval bounds once, then bound, adjoint and Adam launches) gives the best
    bound of the same number of separate steps, bit for bit."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 8)
    lo, hi, _ = W.random_boxes(p["k"] * p["H"], 70, seed=8, min_width=0.05, max_width=0.6)
    g = gp(p)
    best_steps, _, _ = g.alpha_steps(lo, hi, steps=4, lr=0.05, precision=B.PREC_TF32X3)
    lb_best = torch.empty(70, device=DEV)
    B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 70, 4, 0.05, lb_best,
                         precision=B.PREC_TF32X3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lb_best.cpu().numpy(), best_steps)


def test_tf32x3_refusals(gp):
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    # hidden widths that are not multiples of 32
    q = W.make_problem(8, 2, [48, 48], 3, 0.01, seed=2)
    g = gp(q)
    lo, hi, _ = W.random_boxes(q["k"] * q["H"], 4, seed=1, min_width=0.01, max_width=0.1)
    lb = torch.empty(4, device=DEV)
    with pytest.raises(B.BabError) as e:
        B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 4, lb, precision=B.PREC_TF32X3)
    assert e.value.code == -7
    # the obstacle cost (a planar pusher: the pushing network)
    p = W.config_problem("pushing", 2)
    g2 = gp(p)
    B.bab_set_cost(g2.ctx, B.COST_PUSHING_OBSTACLES, np.ones(p["H"]), 1.0, [(0.0, 0.0, 0.5)], (0.0, 0.0))
    lo, hi, _ = W.random_boxes(p["k"] * p["H"], 4, seed=2, min_width=0.01, max_width=0.1)
    with pytest.raises(B.BabError) as e:
        B.bab_bound_crown(g2.ctx, g2.x0, g2.goal, g2.H, g2.rho, T(lo), T(hi), 4, lb, precision=B.PREC_TF32X3)
    assert e.value.code == -7
    B.bab_set_cost(g2.ctx, B.COST_SQUARED)   # back to the default: the same call now runs
    B.bab_bound_crown(g2.ctx, g2.x0, g2.goal, g2.H, g2.rho, T(lo), T(hi), 4, lb, precision=B.PREC_TF32X3)
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec_name,oprec,tol", [("bf16x3", 1, 5e-5), ("tf32x3", 2, 1e-5)])
def test_wide_feature_major_matches_oracle(oracle, gp, prec_name, oprec, tol):
    """Hidden widths 160 and 192 (two feature blocks, 16-box tiles, the image streamed).  The GPU's outward-rounded
    interval bounds drift from the oracle's FP64 ones on this network (about 4e-5 of the bound's scale in every
    precision, the FP32 CROWN included), so CROWN is checked on the GPU's own intervals: the raw bound within the
    split's band of the oracle's CROWN (Theorems 1-2) on them, the margin equal to the oracle's formula, never above
    the oracle's bound; with given slopes too.  The bound on the oracle's own intervals stays at least the GPU's."""
    from paper_2412_09584_gb300 import binding as B
    prec = {"bf16x3": B.PREC_BF16X3, "tf32x3": B.PREC_TF32X3}[prec_name]
    p = W.make_problem(8, 2, [160, 192], 4, 0.01, seed=21, weight_scale=0.5)
    d = p["k"] * p["H"]
    g = gp(p)

    def check(lo, hi, alpha=None):
        _, pl, pu, xl, xu = g.ibp(lo, hi)
        r = g.crown(lo, hi, alpha=alpha, precision=prec)
        a64 = None if alpha is None else alpha.astype(np.float64)
        o = oracle.crown_margin(p, lo, hi, intervals=(pl, pu, xl, xu), alpha=a64, prec=oprec)
        scale = np.maximum(o["scale"], 1.0)
        np.testing.assert_allclose(r["margin"], o["margin"], rtol=MARGIN_REL, atol=0)
        err = np.abs(r["lb"].astype(np.float64) + r["margin"] - o["lb"]) / scale
        assert np.all(err <= tol), err.max()
        assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))
        own = oracle.crown_margin(p, lo, hi, alpha=a64, prec=oprec)
        assert np.all(r["lb"] <= own["lb"] + 1e-12 * np.abs(own["lb"]))

    for n, maxw, seed in ((53, 1.0, 3), (16, 0.05, 4)):
        lo, hi, _ = W.random_boxes(d, n, seed=seed, min_width=0.0, max_width=maxw)
        check(lo, hi)
    check(lo, hi, np.random.default_rng(5).uniform(0, 1, size=(16, p["H"], 352)).astype(np.float32))


def test_wide_feature_major_against_box_major(gp):
    """The two-block feature-major kernel (the default at widths up to 256) and the box-major one (variant 1) agree
    within the BF16 split's rounding: the feature-major constant is summed per feature first."""
    from paper_2412_09584_gb300 import binding as B
    p = W.make_problem(8, 2, [160, 192], 4, 0.01, seed=22, weight_scale=0.5)
    g = gp(p)
    lo, hi, _ = W.random_boxes(p["k"] * p["H"], 70, seed=6, min_width=0.0, max_width=1.0)
    rf = g.crown(lo, hi, precision=B.PREC_BF16X3)
    B.bab_set_variant(g.ctx, B.KERNEL_CROWN_TC, 1)
    rb = g.crown(lo, hi, precision=B.PREC_BF16X3)
    B.bab_set_variant(g.ctx, B.KERNEL_CROWN_TC, -1)
    band = 2e-5 * np.maximum(np.abs(rb["lb"]), 1.0) + rb["margin"] + rf["margin"]
    assert np.all(np.abs(rf["lb"] - rb["lb"]) <= band)


@pytest.fixture(scope="module")
def manip():
    from gpu_util import GpuProblem
    p = W.config_problem("manip", 0)
    g = GpuProblem(p)
    yield p, g
    g.close()


def test_tf32x3_manip_on_gpu_intervals(oracle, manip):
    """The object-manipulation scale (MLP 36-256x4-32, H = 40) in TF32x3: the oracle's CROWN on the GPU's own
    interval bounds against the GPU's raw bound, within max(1e-5 x scale, the GPU's margin), the margin equal to the
    oracle's TF32-split formula, never above the oracle's bound."""
    p, g = manip
    lo, hi, _ = W.random_boxes(160, 6, seed=21, min_width=0.002, max_width=0.02)
    _, pl, pu, xl, xu = g.ibp(lo, hi)
    from paper_2412_09584_gb300 import binding as B
    r = g.crown(lo, hi, precision=B.PREC_TF32X3)
    o = oracle.crown_margin(p, lo, hi, intervals=(pl, pu, xl, xu), prec=2)
    scale = np.maximum(o["scale"], 1.0)
    err = np.abs(r["lb"] + r["margin"] - o["lb"]) / scale
    band = np.maximum(REL, r["margin"] / scale)
    assert np.all(err <= band), (err / band).max()
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))
    np.testing.assert_allclose(r["margin"], o["margin"], rtol=MARGIN_REL, atol=0)
