"""Object-manipulation scale (state 32, action 4, MLP 36-256x4-32, H = 40, box [-1, 1]^160): the FP32 paths run
it with the network image read through L1/L2 and the tensor-core rollout streams its weights (they exceed shared
memory); checked against the FP64 oracle on a handful of boxes, and at the full 16384-box batch on sampled rows."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5


def drift_tol(p):
    """Relative drift allowed between the GPU bound (outward-rounded FP32 intervals) and the oracle's FP64
    round-to-nearest one: directed rounding widens every K-term interval sum by up to K 2^-23 relative, and the
    widening compounds through the L layers of each of the H unrolled steps (the CROWN relaxation of every later
    layer sees the wider intervals)."""
    L = len(p["dims"]) - 1
    return L * p["H"] * max(p["dims"]) * 2.0 ** -23


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def manip():
    from gpu_util import GpuProblem
    p = W.config_problem("manip", 0)
    g = GpuProblem(p)
    yield p, g
    g.close()


def test_manip_rollout_fp32(oracle, manip):
    p, g = manip
    lo, hi, ids = W.random_boxes(160, 6, seed=1, min_width=0.05, max_width=0.5)
    r = g.rollout(lo, hi, ids, M=4, seed=3, incumbent=True)
    ub_o, bu_o, _ = oracle.rollout(p, lo, hi, ids, 4, 3)
    np.testing.assert_allclose(r["ub"], ub_o, rtol=REL, atol=0)
    np.testing.assert_array_equal(r["best_u"], bu_o)
    assert r["inc_val"] == pytest.approx(oracle.objective(p, r["inc_u"].astype(np.float64)), rel=1e-10)


def test_manip_bounds_fp32(oracle, manip):
    p, g = manip
    lo, hi, _ = W.random_boxes(160, 5, seed=2, min_width=0.001, max_width=0.02)
    lb_ibp, pl, pu, xl, xu = g.ibp(lo, hi)
    _, o_pl, o_pu, _, _ = oracle.ibp(p, lo, hi)
    assert np.all(pl <= o_pl + 1e-12 * np.abs(o_pl))
    assert np.all(pu >= o_pu - 1e-12 * np.abs(o_pu))
    r = g.crown(lo, hi)
    oc = oracle.crown(p, lo, hi)
    scale = np.maximum(oc["scale"], 1.0)
    # never above the exact CROWN bound; within the directed-rounding drift of it
    assert np.all(r["lb"] <= oc["lb"] + 1e-12 * np.abs(oc["lb"]))
    assert np.all(np.abs(r["lb"] + r["margin"] - oc["lb"]) <= drift_tol(p) * scale)
    # sound against sampled objective values
    rng = np.random.default_rng(0)
    for i in range(lo.shape[0]):
        u = lo[i] + rng.uniform(size=(8, 160)) * (hi[i] - lo[i])
        assert r["lb"][i] <= min(oracle.objective(p, x.astype(np.float64)) for x in u)


def test_manip_zero_width_box_is_sound(oracle, manip):
    """A zero-width box at this depth: the oracle's FP64 point intervals stay points and its bound equals the
    objective, but outward rounding gives the GPU's intervals an ulp of width that the 200 unrolled layers
    amplify (the interval radius about doubles per layer here), so the GPU bound is sound, not exact."""
    p, g = manip
    rng = np.random.default_rng(8)
    u = rng.uniform(-1, 1, size=(3, 160)).astype(np.float32)
    r = g.crown(u, u)
    f = np.array([oracle.objective(p, x.astype(np.float64)) for x in u])
    o = oracle.crown(p, u, u)
    np.testing.assert_allclose(o["lb"], f, rtol=1e-9)  # the oracle: exact on a point
    assert np.all(r["lb"] <= f)


def test_manip_alpha_warp_matches_unfused(manip):
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p, g = manip
    lo, hi, _ = W.random_boxes(160, 3, seed=4, min_width=0.001, max_width=0.02)
    outs = []
    for v in (-2, 3):
        B.bab_set_variant(g.ctx, B.KERNEL_ALPHA_FUSED, v)
        best = torch.empty(3, device=DEV)
        B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 3, 2, 0.1, best)
        outs.append(best.cpu().numpy())
    B.bab_set_variant(g.ctx, B.KERNEL_ALPHA_FUSED, -1)
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))


@pytest.mark.parametrize("prec_name", ["bf16x3", "bf16"])
def test_manip_rollout_tensor_cores_streamed(oracle, manip, prec_name):
    """The BF16 weight image (434 KB per half) exceeds shared memory: the tensor-core rollout streams it, one
    K-atom at a time, through a ring.  BF16x3: every sample's objective to about 2^-16 relative per product,
    so ub within 1e-4 of the oracle's best; BF16: each box's best sample is re-scored in FP32, so ub is that
    sample's FP32 objective, never below the oracle's best of the same samples."""
    from paper_2412_09584_gb300 import binding as B
    p, g = manip
    prec = {"bf16x3": B.PREC_BF16X3, "bf16": B.PREC_BF16}[prec_name]
    lo, hi, ids = W.random_boxes(160, 5, seed=11, min_width=0.05, max_width=0.5)
    M = 300  # three sample tiles, the last one ragged
    r = g.rollout(lo, hi, ids, M=M, seed=4, precision=prec, incumbent=True)
    ub_o, _, _ = oracle.rollout(p, lo, hi, ids, M, 4)
    f_best = np.array([oracle.objective(p, u.astype(np.float64)) for u in r["best_u"]])
    if prec_name == "bf16x3":
        np.testing.assert_allclose(r["ub"], ub_o, rtol=1e-4, atol=0)
        np.testing.assert_allclose(r["ub"], f_best, rtol=1e-4)
    else:
        np.testing.assert_allclose(r["ub"], f_best, rtol=REL)
        assert np.all(r["ub"] >= ub_o * (1 - REL))
    assert r["inc_val"] == pytest.approx(oracle.objective(p, r["inc_u"].astype(np.float64)), rel=1e-10)


def test_manip_crown_tensor_cores_streamed(oracle, manip):
    """3-term BF16 CROWN with the backward image streamed: sound (never above the exact CROWN bound) and within
    the directed-rounding drift plus the split's per-product error of it."""
    from paper_2412_09584_gb300 import binding as B
    p, g = manip
    lo, hi, _ = W.random_boxes(160, 130, seed=2, min_width=0.001, max_width=0.02)  # two tiles, the second ragged
    r = g.crown(lo, hi, precision=B.PREC_BF16X3)
    rows = np.array([0, 5, 127, 128, 129])
    oc = oracle.crown(p, lo[rows], hi[rows])
    scale = np.maximum(oc["scale"], 1.0)
    assert np.all(r["lb"][rows] <= oc["lb"] + 1e-12 * np.abs(oc["lb"]))
    split = (len(p["dims"]) - 1) * p["H"] * 3.1 * 2.0 ** -16
    assert np.all(np.abs(r["lb"][rows] + r["margin"][rows] - oc["lb"]) <= (drift_tol(p) + split) * scale)
    f32 = g.crown(lo, hi)
    assert np.all(np.abs(r["lb"] - f32["lb"]) <= (drift_tol(p) + split) * np.abs(f32["lb"]))


def test_manip_full_batch_sampled(oracle, manip):
    """16384 boxes (the configuration's batch) x 4 rollouts and CROWN bounds, checked on sampled rows."""
    p, g = manip
    n = 16384
    lo, hi, ids = W.random_boxes(160, n, seed=6, min_width=0.002, max_width=0.05)
    from paper_2412_09584_gb300 import binding as B
    r = g.rollout(lo, hi, ids, M=4, seed=9)
    rb = g.rollout(lo, hi, ids, M=4, seed=9, precision=B.PREC_BF16)  # the configuration's BF16 rollouts
    c = g.crown(lo, hi)
    rows = np.array([0, 1, 777, 8191, 16383])
    ub_o, _, _ = oracle.rollout(p, lo[rows], hi[rows], ids[rows], 4, 9)
    np.testing.assert_allclose(r["ub"][rows], ub_o, rtol=REL)
    f_b = np.array([oracle.objective(p, u.astype(np.float64)) for u in rb["best_u"][rows]])
    np.testing.assert_allclose(rb["ub"][rows], f_b, rtol=REL)
    assert np.all(rb["ub"][rows] >= ub_o * (1 - REL))
    oc = oracle.crown(p, lo[rows], hi[rows])
    scale = np.maximum(oc["scale"], 1.0)
    assert np.all(c["lb"][rows] <= oc["lb"] + 1e-12 * np.abs(oc["lb"]))
    assert np.all(np.abs(c["lb"][rows] + c["margin"][rows] - oc["lb"]) <= drift_tol(p) * scale)
    # a lower bound never exceeds a sampled objective value (up to the FP32 rounding of the rollout)
    assert np.all(c["lb"] <= r["ub"] * (1 + REL))


def test_manip_topk_rescore_cluster(oracle, manip):
    """The configuration's top-k FP32 re-score on this network runs on thread-block clusters (a box per cluster,
    each CTA a share of every layer's outputs): the picked boxes get exactly the every-box re-score's values (the
    same sums in the same order), the rest keep their BF16 values, and the re-scored values are the FP32 objective
    of the picked samples."""
    from paper_2412_09584_gb300 import binding as B
    p, g = manip
    n = 600
    lo, hi, ids = W.random_boxes(160, n, seed=31, min_width=0.01, max_width=0.3)
    r_all = g.rollout(lo, hi, ids, M=4, seed=5, precision=B.PREC_BF16)
    B.bab_set_rescore_topk(g.ctx, 40)
    try:
        r = g.rollout(lo, hi, ids, M=4, seed=5, precision=B.PREC_BF16, incumbent=True)
    finally:
        B.bab_set_rescore_topk(g.ctx, 0)
    np.testing.assert_array_equal(r["best_u"], r_all["best_u"])
    same = r["ub"] == r_all["ub"]
    assert same.sum() >= 40
    rows = np.flatnonzero(same)[:6]
    f = np.array([oracle.objective(p, r["best_u"][i].astype(np.float64)) for i in rows])
    np.testing.assert_allclose(r["ub"][rows], f, rtol=REL)
    assert r["inc_val"] == pytest.approx(oracle.objective(p, r["inc_u"].astype(np.float64)), rel=1e-10)
