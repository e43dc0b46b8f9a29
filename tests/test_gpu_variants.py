"""Launch variants (tile shapes), the fused alpha-CROWN loop and the autotuner: every variant must give the
same results as the others (bit-identical where the arithmetic is the same), and the oracle still agrees."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _problem(name, n, seed=5):
    from gpu_util import GpuProblem
    p = W.config_problem(name, seed)
    d = p["k"] * p["H"]
    lo, hi, ids = W.random_boxes(d, n, seed=seed + 1, min_width=0.2, max_width=2.0)
    return p, lo, hi, ids, GpuProblem(p)


@pytest.mark.parametrize("name,n,M", [("tiny", 37, 256), ("pushing", 9, 200)])
def test_rollout_fp32_variants_bit_identical(oracle, name, n, M):
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, g = _problem(name, n)
    try:
        outs = []
        for v in range(3):
            B.bab_set_variant(g.ctx, B.KERNEL_ROLLOUT_FP32, v)
            outs.append(g.rollout(lo, hi, ids, M=M, seed=77))
        for o in outs[1:]:
            assert np.array_equal(o["ub"].view(np.uint32), outs[0]["ub"].view(np.uint32))
            assert np.array_equal(o["best_u"].view(np.uint32), outs[0]["best_u"].view(np.uint32))
        ub_o, _, _ = oracle.rollout(p, lo, hi, ids, M, 77)
        np.testing.assert_allclose(outs[0]["ub"], ub_o, rtol=1e-5, atol=0)
    finally:
        g.close()


def test_rollout_tc_slots_bit_identical():
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, g = _problem("pushing", 5)
    try:
        outs = []
        for v in (1, 2):
            B.bab_set_variant(g.ctx, B.KERNEL_ROLLOUT_TC, v)
            outs.append(g.rollout(lo, hi, ids, M=300, seed=3, precision=B.PREC_BF16X3))
        assert np.array_equal(outs[0]["ub"].view(np.uint32), outs[1]["ub"].view(np.uint32))
        assert np.array_equal(outs[0]["best_u"].view(np.uint32), outs[1]["best_u"].view(np.uint32))
    finally:
        g.close()


@pytest.mark.parametrize("name,M", [("pushing", 256), ("tiny", 256), ("pushing", 40)])
def test_rollout_fused_step_bf16(oracle, name, M):
    """BF16 rollouts with the output layer of each step and the first layer of the next as one product (the
    default where it applies) against the layer-by-layer kernel: one and two tiles per CTA bit-identical in each;
    every sample's BF16 cost within 1e-4 of its FP64 objective and of the layer-by-layer cost (both measured
    below 1e-5), and each box's pick re-scored to its FP32 objective."""
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, g = _problem(name, 6)
    n, d, seed = lo.shape[0], g.d, 9
    try:
        out = {}
        for v in (1, 2, 3, 4):
            B.bab_set_variant(g.ctx, B.KERNEL_ROLLOUT_TC, v)
            ub = torch.empty(n, device=DEV)
            bu = torch.empty(n, d, device=DEV)
            sd = torch.empty(n, dtype=torch.int32, device=DEV)
            costs = torch.empty(n, M, device=DEV)
            B.bab_rollout_split(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), n, M, seed, B.PREC_BF16,
                                1.0, ub, sd, best_u=bu, costs=costs)
            torch.cuda.synchronize()
            out[v] = (costs.cpu().numpy(), ub.cpu().numpy(), bu.cpu().numpy())
        assert B.bab_status(g.ctx) == 0
        for a_, b_ in ((1, 2), (3, 4)):
            for x, y in zip(out[a_], out[b_]):
                assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
        cf, ubf, buf = out[2]
        cl = out[4][0]
        np.testing.assert_allclose(cf, cl, rtol=1e-4, atol=0)
        for i in range(n):
            for m in range(0, M, max(1, M // 8)):
                u = np.array([oracle.sample(seed, int(ids[i]), m, j, float(lo[i, j]), float(hi[i, j])) for j in range(d)])
                assert cf[i, m] == pytest.approx(oracle.objective(p, u), rel=1e-4)
            assert ubf[i] == pytest.approx(oracle.objective(p, buf[i].astype(np.float64)), rel=1e-5)
    finally:
        g.close()


@pytest.mark.parametrize("name,n,with_alpha", [("tiny", 300, False), ("pushing", 300, False), ("pushing", 211, True),
                                                ("pushing", 5000, False)])
def test_crown_tc_variants_bit_identical(name, n, with_alpha):
    """Staged (each thread's next-layer interval bounds copied to shared memory ahead of use, up to 32 boxes a
    tile; 5000 boxes give each CTA several tiles), one and two unstaged tiles per CTA: the same arithmetic in the
    same order, so every output agrees bit for bit, with and without given slopes."""
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, g = _problem(name, n)
    try:
        alpha = None
        if with_alpha:
            rng = np.random.default_rng(3)
            alpha = rng.uniform(0.0, 1.0, size=(n, g.H, g.sumh)).astype(np.float32)
        outs = []
        for v in (0, 1, 2):
            B.bab_set_variant(g.ctx, B.KERNEL_CROWN_TC, v)
            outs.append(g.crown(lo, hi, alpha=alpha, precision=B.PREC_BF16X3))
        for o in outs[1:]:
            for key in ("lb", "margin", "lin_coef", "lin_const"):
                assert np.array_equal(outs[0][key].view(np.uint32), o[key].view(np.uint32)), key
        assert B.bab_status(g.ctx) == 0
    finally:
        g.close()


@pytest.mark.parametrize("name,n,with_alpha", [("tiny", 300, False), ("pushing", 211, True), ("pushing", 5000, False)])
def test_crown_tc_feature_major_matches_box_major(oracle, name, n, with_alpha):
    """The feature-major kernel (features on the MMA's rows, 32 boxes on its columns) against the staged
    box-major one (16 and 8 epilogue warps bit-identical): the same products, a branch-free relaxation whose
    unstable upper slope is a quotient bounded upward, and the constant summed per feature and then across
    features instead of in one running sum per box, so the downward roundings differ (the tree loses less: the
    feature-major bound is the tighter one, by about 4e-6 relative here); bounds agree to 2e-5 of the bound's
    scale, margins to 1e-3, coefficients to 1e-5 of the row's L1 norm, and both stay below the oracle's bound."""
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, g = _problem(name, n)
    try:
        alpha = None
        if with_alpha:
            alpha = np.random.default_rng(4).uniform(0.0, 1.0, size=(n, g.H, g.sumh)).astype(np.float32)
        outs = []
        for v in (4, 3, 0):
            B.bab_set_variant(g.ctx, B.KERNEL_CROWN_TC, v)
            outs.append(g.crown(lo, hi, alpha=alpha, precision=B.PREC_BF16X3))
        assert B.bab_status(g.ctx) == 0
        f, f8, b = outs
        for key in ("lb", "margin", "lin_coef", "lin_const"):  # 16 and 8 epilogue warps: the same sums
            assert np.array_equal(f[key].view(np.uint32), f8[key].view(np.uint32)), key
        scale = np.maximum(np.abs(b["lin_const"]) + np.abs(b["lb"]), 1.0)
        assert np.all(np.abs(f["lb"].astype(np.float64) - b["lb"]) <= 2e-5 * scale)
        np.testing.assert_allclose(f["margin"], b["margin"], rtol=1e-3, atol=1e-12)
        mu_scale = np.maximum(np.abs(b["lin_coef"]).sum(axis=1, keepdims=True), 1.0)
        assert np.all(np.abs(f["lin_coef"] - b["lin_coef"]) <= 1e-5 * mu_scale)
        rows = np.arange(0, n, max(1, n // 12))
        o = oracle.crown(p, lo[rows], hi[rows], alpha=None if alpha is None else alpha[rows].astype(np.float64))
        assert np.all(f["lb"][rows] <= o["lb"] + 1e-12 * np.abs(o["lb"]))
    finally:
        g.close()


def test_set_variant_rejects_bad_values():
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, g = _problem("tiny", 4)
    try:
        for kernel, bad in ((B.KERNEL_ROLLOUT_FP32, 3), (B.KERNEL_ALPHA_FUSED, -3), (B.KERNEL_ALPHA_FUSED, 4),
                            (B.KERNEL_ROLLOUT_TC, 0),
                            (B.KERNEL_CROWN_TC, 5), (9, 0)):
            with pytest.raises(B.BabError) as e:
                B.bab_set_variant(g.ctx, kernel, bad)
            assert e.value.code == -1
        B.bab_set_variant(g.ctx, B.KERNEL_ALPHA_FUSED, -2)
        assert B.bab_get_variant(g.ctx, B.KERNEL_ALPHA_FUSED) == -2
    finally:
        g.close()


def _optimize(g, lo, hi, steps, variant):
    from gpu_util import T
    from paper_2412_09584_gb300 import binding as B
    n = lo.shape[0]
    B.bab_set_variant(g.ctx, B.KERNEL_ALPHA_FUSED, variant)
    best = torch.empty(n, device="cuda")
    alpha = torch.empty(n, g.H, g.sumh, device="cuda")
    B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, steps, 0.1, best, alpha=alpha,
                         precision=B.PREC_FP32)
    torch.cuda.synchronize()
    return best.cpu().numpy(), alpha.cpu().numpy()


@pytest.mark.parametrize("name,n", [("alpha", 300), ("tiny", 67)])
def test_alpha_fused_matches_unfused_loop(oracle, name, n):
    """One launch for the whole Adam loop gives the separate launches' bounds and slopes."""
    p, lo, hi, ids, g = _problem(name, n, seed=9)
    try:
        b_ref, a_ref = _optimize(g, lo, hi, 20, -2)
        fused = [_optimize(g, lo, hi, 20, v) for v in (3, 0, 1, 2, -1)]
        for b, a in fused[1:]:
            assert np.array_equal(b.view(np.uint32), fused[0][0].view(np.uint32))
            assert np.array_equal(a.view(np.uint32), fused[0][1].view(np.uint32))
        scale = np.maximum(oracle.crown(p, lo, hi)["scale"], 1.0)
        b, a = fused[0]
        # the same arithmetic in the same order, step for step
        assert np.array_equal(b.view(np.uint32), b_ref.view(np.uint32))
        assert np.array_equal(a.view(np.uint32), a_ref.view(np.uint32))
        best_o, _, _, _ = oracle.alpha_optimize(p, lo[:24], hi[:24], 20, 0.1)
        assert np.all(np.abs(b[:24] - best_o) <= 1e-3 * scale[:24])
    finally:
        g.close()


def test_alpha_warp_pushing_matches_unfused_loop():
    """The warp-per-box loop on a network whose weights stay in global memory (4 neurons per lane)."""
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, g = _problem("pushing", 11, seed=2)
    try:
        b_ref, a_ref = _optimize(g, lo, hi, 4, -2)
        b, a = _optimize(g, lo, hi, 4, 3)
        assert np.array_equal(b.view(np.uint32), b_ref.view(np.uint32))
        assert np.array_equal(a.view(np.uint32), a_ref.view(np.uint32))
        # the shared-memory tile does not fit this network
        with pytest.raises(B.BabError) as e:
            _optimize(g, lo, hi, 4, 0)
        assert e.value.code == -7
    finally:
        g.close()


def test_autotune_keeps_results(oracle):
    from gpu_util import T, ids_t
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, g = _problem("tiny", 200, seed=11)
    try:
        before = g.rollout(lo, hi, ids, M=256, seed=5)
        B.bab_autotune(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), lo.shape[0], 256, alpha_steps=4)
        assert B.bab_get_variant(g.ctx, B.KERNEL_ROLLOUT_FP32) in (0, 1, 2)
        assert B.bab_get_variant(g.ctx, B.KERNEL_ROLLOUT_TC) in (1, 2)  # the autotuner keeps the fused step
        assert B.bab_get_variant(g.ctx, B.KERNEL_CROWN_TC) in (0, 1, 2, 3, 4)
        assert B.bab_get_variant(g.ctx, B.KERNEL_ALPHA_FUSED) in (-2, 0, 1, 2, 3)
        after = g.rollout(lo, hi, ids, M=256, seed=5)
        assert np.array_equal(after["ub"].view(np.uint32), before["ub"].view(np.uint32))
        assert B.bab_status(g.ctx) == 0
    finally:
        g.close()
