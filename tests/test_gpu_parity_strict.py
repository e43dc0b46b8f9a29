"""Parity of the CROWN bound, its outward margin and the alpha steps with the FP64 oracle at the stated tolerances,
with the interval-bound drift separated out.

* The margin (the rounding-error correction the GPU subtracts, Appendix B.1 products evaluated in FP32 or as
  3-term BF16 splits) against the oracle's FP64 evaluation of the same formula: 1e-3 relative.
* At the object-manipulation scale (MLP 36-256x4-32, H = 40) the GPU's outward-rounded interval bounds widen
  through the 200 unrolled layers, so the GPU bound and the oracle's own bound differ by that drift.  Given the
  GPU's interval bounds, the oracle's CROWN (Theorems 1-2 with those intermediate bounds) must match the GPU's
  raw bound (lb + margin) to 1e-5 of the bound's scale in FP32 and 5e-5 with 3-term BF16 split products, or to
  the GPU's own outward margin where that is larger, and the returned bound must not exceed the oracle's.  The
  margin is larger at this depth: the intervals grow about tenfold every five steps of this random network (to
  widths near 3e5 at step 40), the bound (about -1e10) is a sum of terms of that size that nearly cancel, and the
  rounding of the 200 chained products is charged against those magnitudes (about 1e-4 of the bound's scale in
  FP32, 1.3e-3 with the 3-term split).
* alpha-CROWN: every one of 20 Adam steps, bound and gradient at the GPU's own slopes of that step against the
  oracle's at the same slopes: 1e-5 of the bound's scale and 1e-5 of the row's largest gradient.
"""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5
REL_TC = 5e-5
MARGIN_REL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _prec(name):
    from paper_2412_09584_gb300 import binding as B
    return {"fp32": (B.PREC_FP32, 0), "bf16x3": (B.PREC_BF16X3, 1)}[name]


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("name,n,maxw,rho", [("tiny", 64, 2.0, None), ("tiny", 37, 0.3, 0.02),
                                             ("pushing", 21, 0.2, None), ("pushing", 40, 2.0, None)])
def test_margin_matches_oracle_formula(oracle, gp, prec, name, n, maxw, rho):
    p = W.config_problem(name, 3)
    if rho is not None:
        p["rho"] = rho
    d = p["k"] * p["H"]
    lo, hi, _ = W.random_boxes(d, n, seed=n + 1, min_width=0.0, max_width=maxw)
    g = gp(p)
    gprec, oprec = _prec(prec)
    r = g.crown(lo, hi, precision=gprec)
    o = oracle.crown_margin(p, lo, hi, prec=oprec)
    np.testing.assert_allclose(r["margin"], o["margin"], rtol=MARGIN_REL, atol=0)
    tol = REL if prec == "fp32" else REL_TC
    scale = np.maximum(o["scale"], 1.0)
    assert np.all(np.abs(r["lb"] + r["margin"] - o["lb"]) <= tol * scale)
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))


@pytest.fixture(scope="module")
def manip():
    from gpu_util import GpuProblem
    p = W.config_problem("manip", 0)
    g = GpuProblem(p)
    yield p, g
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("maxw", [0.02, 0.2])
def test_manip_crown_on_gpu_intervals(oracle, manip, prec, maxw):
    """The object-manipulation scale, CROWN separated from the interval bounds: the oracle's Theorem 1-2 bound
    on the GPU's own interval bounds equals the GPU's raw bound within FP32 (or split) rounding; the drift of the
    GPU's outward-rounded intervals from the oracle's FP64 ones is asserted separately, as the wider band it is."""
    p, g = manip
    lo, hi, _ = W.random_boxes(160, 6, seed=21, min_width=maxw / 10, max_width=maxw)
    gprec, oprec = _prec(prec)
    _, pl, pu, xl, xu = g.ibp(lo, hi)
    r = g.crown(lo, hi, precision=gprec)
    o = oracle.crown_margin(p, lo, hi, intervals=(pl, pu, xl, xu), prec=oprec)
    scale = np.maximum(o["scale"], 1.0)
    tol = REL if prec == "fp32" else REL_TC
    err = np.abs(r["lb"] + r["margin"] - o["lb"]) / scale
    band = np.maximum(tol, r["margin"] / scale)
    assert np.all(err <= band), (err / band).max()
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))
    np.testing.assert_allclose(r["margin"], o["margin"], rtol=MARGIN_REL, atol=0)
    # the interval drift on its own: the oracle's bound on its own FP64 intervals is at least the bound on the
    # GPU's wider ones (Lemma 1 relaxations and tangents on wider intervals are looser) and within L H K 2^-23
    own = oracle.crown(p, lo, hi)
    L = len(p["dims"]) - 1
    drift = L * p["H"] * max(p["dims"]) * 2.0 ** -23
    assert np.all(np.abs(own["lb"] - o["lb"]) <= drift * np.maximum(own["scale"], 1.0))


def test_alpha_every_step_matches_oracle(oracle, gp):
    """Twenty projected Adam steps on the GPU; at each step the bound and the gradient the GPU computed at its own
    slopes (read back before the step) equal the oracle's at those slopes."""
    p = W.make_problem(4, 2, [32, 32], 5, 0.01, seed=14, weight_scale=0.3)
    lo, hi, _ = W.random_boxes(10, 16, seed=15, min_width=0.3, max_width=1.0)
    g = gp(p)
    a0 = g.alpha_init(lo, hi).cpu().numpy()
    _, _, hist = g.alpha_steps(lo, hi, steps=20, lr=0.1)
    worst_lb = worst_g = 0.0
    for k, h in enumerate(hist):
        a_before = a0 if k == 0 else hist[k - 1]["alpha"]
        lb_o, g_o, _ = oracle.alpha_grad(p, lo, hi, a_before.astype(np.float64))
        scale = np.maximum(oracle.crown(p, lo, hi, a_before.astype(np.float64))["scale"], 1.0)
        e_lb = np.abs(h["lb"] - lb_o) / scale
        gs = np.maximum(np.abs(g_o).max(axis=(1, 2)), 1e-30)
        e_g = np.abs(h["grad"] - g_o).max(axis=(1, 2)) / gs
        worst_lb, worst_g = max(worst_lb, e_lb.max()), max(worst_g, e_g.max())
        assert np.all(e_lb <= REL), (k, e_lb.max())
        assert np.all(e_g <= REL), (k, e_g.max())
        assert np.all(h["lb"] <= lb_o + 1e-12 * np.abs(lb_o))
    # the trajectory itself (FP32 against FP64 Adam) is compared loosely in test_gpu_parity.py
    assert worst_lb >= 0 and worst_g >= 0
