"""The pushing-with-obstacles cost (Appendix D.4, Eq. pushing_cost) on the GPU against the oracle: the FP32
cross-entropy search bit-exact (its decisions are taken on the FP32 objective), rollouts by value, the interval and
CROWN bounds close to the oracle's and never above them beyond rounding, the FP64 incumbent, and the refusals of
the paths that do not carry this cost."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture
def obst(oracle, gp):
    """A pushing-scale problem with the obstacle cost set on both sides."""
    from paper_2412_09584_gb300 import binding as B

    def make(name="pushing", seed=71, H=None, lam=10.0, n_obs=3):
        p = W.config_problem(name, seed)
        if H is not None:
            p = dict(p, H=H)
        c = W.obstacle_cost(p["H"], seed, n_obs=n_obs, lam=lam)
        # the oracle takes the parameters the GPU holds (FP32)
        f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
        oracle.set_cost(1, f32(c["w"]), float(f32(c["lam"])), f32(c["obstacles"]), f32(c["p0"]))
        g = gp(p)
        B.bab_set_cost(g.ctx, B.COST_PUSHING_OBSTACLES, c["w"], c["lam"], c["obstacles"], c["p0"])
        return p, g
    yield make
    oracle.set_cost(0)


def test_obstacle_cem_fp32_bit_exact(oracle, obst):
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    p, g = obst()
    lo, hi, ids = W.random_boxes(40, 4, seed=72, min_width=0.3, max_width=2.0)
    ub = torch.empty(4, device=DEV)
    bu = torch.empty(4, 40, device=DEV)
    B.bab_rollout_cem(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), 4, 48, 3, 6, 1e-3, 5, B.PREC_FP32,
                      ub, bu)
    torch.cuda.synchronize()
    ub_o, bu_o = oracle.cem(p, lo, hi, ids, 48, 3, 6, 1e-3, 5)
    assert np.array_equal(ub.cpu().numpy().view(np.uint32), ub_o.view(np.uint32))
    assert np.array_equal(bu.cpu().numpy().view(np.uint32), bu_o.view(np.uint32))


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "bf16"])
def test_obstacle_rollout_values_and_incumbent(oracle, obst, precision):
    """ub is the objective of the returned plan (BF16: the pick re-scored in FP32 under the obstacle cost) and the
    minimum over the same samples (BF16 ranks in its own arithmetic, so within its rounding of it)."""
    from paper_2412_09584_gb300 import binding as B
    p, g = obst()
    lo, hi, ids = W.random_boxes(40, 8, seed=73, min_width=0.5, max_width=2.0)
    prec = {"fp32": B.PREC_FP32, "bf16x3": B.PREC_BF16X3, "bf16": B.PREC_BF16}[precision]
    r = g.rollout(lo, hi, ids, M=128, seed=9, precision=prec, incumbent=True)
    ub_o, _, _ = oracle.rollout(p, lo, hi, ids, 128, 9)
    f = np.array([oracle.objective(p, r["best_u"][i].astype(np.float64)) for i in range(8)])
    np.testing.assert_allclose(r["ub"], f, rtol=2e-6)
    if precision == "bf16":
        assert np.all(f >= ub_o * (1 - 1e-12))
        np.testing.assert_allclose(r["ub"], ub_o, rtol=2e-2)
    else:
        np.testing.assert_allclose(r["ub"], ub_o, rtol=2e-6)   # the same samples; the minimum within rounding
    best = int(np.argmin(r["ub"]))
    assert r["inc_val"] == pytest.approx(f[best], rel=1e-10)   # FP64 on both sides, in different orders


def test_obstacle_bf16_topk_rescore(oracle, obst):
    """With a top-k re-score (the per-box kernel), the k boxes of smallest BF16 ub get the FP32 objective of their
    pick under the obstacle cost, equal to the every-box re-score."""
    from paper_2412_09584_gb300 import binding as B
    p, g = obst()
    lo, hi, ids = W.random_boxes(40, 12, seed=74, min_width=0.5, max_width=2.0)
    r_all = g.rollout(lo, hi, ids, M=128, seed=11, precision=B.PREC_BF16)
    B.bab_set_rescore_topk(g.ctx, 4)
    r = g.rollout(lo, hi, ids, M=128, seed=11, precision=B.PREC_BF16)
    np.testing.assert_array_equal(r["best_u"], r_all["best_u"])
    same = r["ub"] == r_all["ub"]
    assert same.sum() >= 4
    f = np.array([oracle.objective(p, u.astype(np.float64)) for u in r["best_u"]])
    np.testing.assert_allclose(r["ub"][same], f[same], rtol=2e-6)


def test_obstacle_bounds_against_oracle(oracle, obst):
    """Interval and CROWN bounds: at most the oracle's exact ones (plus rounding), and close to them."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p, g = obst(H=8, n_obs=4, lam=20.0)
    lo, hi, _ = W.random_boxes(16, 24, seed=74, min_width=0.02, max_width=0.6)
    n = 24
    c_o = oracle.crown(p, lo, hi)
    lb_ibp_o = oracle.ibp(p, lo, hi)[0]
    scale = np.maximum(c_o["scale"], 1.0)
    lb_c = torch.empty(n, device=DEV)
    margin = torch.empty(n, device=DEV)
    B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, lb_c, margin=margin)
    lb_i = torch.empty(n, device=DEV)
    B.bab_bound_ibp(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, lb_i)
    torch.cuda.synchronize()
    lb_c, lb_i = lb_c.cpu().numpy().astype(np.float64), lb_i.cpu().numpy().astype(np.float64)
    assert np.all(lb_c <= c_o["lb"] + 1e-6 * scale)
    assert np.all(lb_c >= c_o["lb"] - 1e-4 * scale)
    ibp_scale = np.maximum(np.abs(lb_ibp_o), 1.0)
    assert np.all(lb_i <= lb_ibp_o + 1e-6 * ibp_scale)
    assert np.all(lb_i >= lb_ibp_o - 1e-4 * ibp_scale)
    # sound against sampled objectives
    rng = np.random.default_rng(5)
    for i in range(0, n, 6):
        us = lo[i] + (hi[i] - lo[i]) * rng.uniform(size=(200, 16))
        fmin = min(oracle.objective(p, u) for u in us)
        assert lb_c[i] <= fmin and lb_i[i] <= fmin


def test_obstacle_crown_tensor_cores(oracle, obst):
    """The tensor-core CROWN (3-term BF16 split products) with the obstacle cost: at most the oracle's exact bound
    (plus rounding), within the split band plus the relaxation's 1e-5 shrink of it, close to the CUDA-core CROWN,
    below sampled objectives; and alpha-CROWN on tensor cores with it, never below the adaptive bound."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p, g = obst(H=8, n_obs=4, lam=20.0)
    n = 150  # two tiles of 128 boxes, the second ragged
    lo, hi, _ = W.random_boxes(16, n, seed=84, min_width=0.02, max_width=0.6)
    c_o = oracle.crown(p, lo, hi)
    scale = np.maximum(c_o["scale"], 1.0)
    lb_t, mg_t, lb_f = (torch.empty(n, device=DEV) for _ in range(3))
    B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, lb_t, precision=B.PREC_BF16X3, margin=mg_t)
    B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, lb_f)
    best = torch.empty(n, device=DEV)
    B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, 5, 0.1, best, precision=B.PREC_BF16X3)
    torch.cuda.synchronize()
    assert B.bab_status(g.ctx) == 0
    lb_t, lb_f, best = (x.cpu().numpy().astype(np.float64) for x in (lb_t, lb_f, best))
    assert np.all(lb_t <= c_o["lb"] + 1e-6 * scale)
    assert np.all(lb_t >= c_o["lb"] - 2e-4 * scale)
    assert np.all(np.abs(lb_t - lb_f) <= 2e-4 * scale)
    assert np.all(best >= lb_t - 1e-5 * scale)
    rng = np.random.default_rng(6)
    for i in range(0, n, 15):
        us = lo[i] + (hi[i] - lo[i]) * rng.uniform(size=(200, 16))
        fmin = min(oracle.objective(p, u) for u in us)
        assert lb_t[i] <= fmin and best[i] <= fmin


def test_obstacle_crown_tc_variants_bit_identical(obst):
    """The obstacle cost on the staged tensor-core CROWN (next-layer interval bounds and state boxes copied to
    shared memory ahead of use) and on one and two unstaged tiles per CTA: bit-identical outputs."""
    from paper_2412_09584_gb300 import binding as B
    p, g = obst(H=8, n_obs=4, lam=20.0)
    n = 150
    lo, hi, _ = W.random_boxes(16, n, seed=85, min_width=0.02, max_width=0.6)
    try:
        outs = []
        for v in (0, 1, 2):
            B.bab_set_variant(g.ctx, B.KERNEL_CROWN_TC, v)
            outs.append(g.crown(lo, hi, precision=B.PREC_BF16X3))
        for o in outs[1:]:
            for key in ("lb", "margin", "lin_coef", "lin_const"):
                assert np.array_equal(outs[0][key].view(np.uint32), o[key].view(np.uint32)), key
        assert B.bab_status(g.ctx) == 0
    finally:
        B.bab_set_variant(g.ctx, B.KERNEL_CROWN_TC, -1)


def test_obstacle_alpha_gradient_and_step(oracle, obst):
    """alpha-CROWN with the obstacle cost: the adjoint gradient at the adaptive slopes and the bound against the
    oracle's, and Adam's first step."""
    p, g = obst(name="tiny", seed=77)
    lo, hi, _ = W.random_boxes(10, 24, seed=78, min_width=0.3, max_width=1.0)
    best, alpha, hist = g.alpha_steps(lo, hi, steps=1, lr=0.1)
    a0 = oracle.adaptive_alpha(p, lo, hi)
    lb_o, grad_o, _ = oracle.alpha_grad(p, lo, hi, a0)
    gs = np.maximum(np.abs(grad_o).max(axis=(1, 2), keepdims=True), 1e-30)
    assert np.all(np.abs(hist[0]["grad"] - grad_o) <= 1e-4 * gs)
    scale = np.maximum(oracle.crown(p, lo, hi, a0)["scale"], 1.0)
    assert np.all(np.abs(hist[0]["lb"] - lb_o) <= 1e-5 * scale)
    assert np.all(hist[0]["lb"] <= lb_o + 1e-12 * np.abs(lb_o))
    a = a0.copy()
    m, v = np.zeros_like(a), np.zeros_like(a)
    oracle.adam_ascent(a, m, v, grad_o, 1, 0.1)
    clear = np.abs(grad_o) > 1e-3 * gs
    assert clear.sum() > 0
    np.testing.assert_allclose(alpha[clear], a[clear], atol=1e-5)


def test_obstacle_alpha_optimize(oracle, obst):
    """bab_alpha_optimize with the obstacle cost: the one-call loop (separate launches, the shared-memory tile, or
    one warp per box) bit-identical to repeated bab_alpha_step; the best bound at least the adaptive CROWN bound (up
    to rounding) and below the objective at sampled points."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p, g = obst(name="tiny", seed=79)
    n = 40
    lo, hi, _ = W.random_boxes(10, n, seed=80, min_width=0.2, max_width=1.5)
    steps = 20
    ref, _, _ = g.alpha_steps(lo, hi, steps=steps, lr=0.1)
    outs = []
    for variant in (-1, -2, 0, 3):
        B.bab_set_variant(g.ctx, B.KERNEL_ALPHA_FUSED, variant)
        lb_best = torch.empty(n, device=DEV)
        B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, steps, 0.1, lb_best)
        torch.cuda.synchronize()
        outs.append(lb_best.cpu().numpy())
    for o in outs:
        assert np.array_equal(o.view(np.uint32), ref.view(np.uint32))
    lb0 = g.crown(lo, hi)["lb"]
    assert np.all(ref >= lb0 - 1e-5 * np.maximum(np.abs(lb0), 1.0))
    assert np.mean(ref > lb0) > 0.5
    rng = np.random.default_rng(81)
    for i in range(n):
        us = lo[i] + (hi[i] - lo[i]) * rng.uniform(size=(100, 10))
        assert ref[i] <= min(oracle.objective(p, u) for u in us)


def test_obstacle_alpha_warp_pushing(obst):
    """The warp-per-box alpha loop with the obstacle cost on the pushing network (H = 20, 3 obstacles): bit-identical
    to the separate bound, adjoint and Adam launches."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p, g = obst()
    n = 24
    lo, hi, _ = W.random_boxes(40, n, seed=83, min_width=0.05, max_width=0.5)
    outs = []
    for variant in (-2, 3):
        B.bab_set_variant(g.ctx, B.KERNEL_ALPHA_FUSED, variant)
        lb_best = torch.empty(n, device=DEV)
        alpha = torch.empty(n, g.H, g.sumh, device=DEV)
        B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, 5, 0.1, lb_best, alpha=alpha)
        torch.cuda.synchronize()
        outs.append((lb_best.cpu().numpy(), alpha.cpu().numpy()))
    assert np.array_equal(outs[0][0].view(np.uint32), outs[1][0].view(np.uint32))
    assert np.array_equal(outs[0][1].view(np.uint32), outs[1][1].view(np.uint32))


def test_obstacle_cost_refusals(obst):
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    p, g = obst(H=5)
    lo, hi, ids = W.random_boxes(10, 3, seed=75)
    lb = torch.empty(3, device=DEV)
    with pytest.raises(B.BabError):
        B.bab_box_grad(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 3, lb, torch.empty(3, 10, device=DEV),
                       torch.empty(3, 10, device=DEV))
    with pytest.raises(B.BabError):   # the tensor-core cross-entropy search
        B.bab_rollout_cem(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), ids_t(ids), 3,
                          16, 2, 4, 1e-3, 1, B.PREC_BF16X3, torch.empty(3, device=DEV), torch.empty(3, 10, device=DEV))
    with pytest.raises(B.BabError):   # horizon beyond the weights
        B.bab_bound_crown(g.ctx, g.x0, g.goal, 6, g.rho, T(np.zeros((3, 12), np.float32)),
                          T(np.ones((3, 12), np.float32)), 3, lb)
    B.bab_set_cost(g.ctx, B.COST_SQUARED)   # back to the default: the same call now runs
    B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 3, lb, precision=B.PREC_BF16X3)


def test_set_cost_argument_errors(gp):
    from paper_2412_09584_gb300 import binding as B
    g = gp(W.config_problem("manip", 76))           # k = 4: not a planar pusher
    with pytest.raises(B.BabError):
        B.bab_set_cost(g.ctx, B.COST_PUSHING_OBSTACLES, np.ones(40), 1.0, [(0, 0, 1)], (0, 0))
    g = gp(W.config_problem("tiny", 76))
    with pytest.raises(B.BabError):
        B.bab_set_cost(g.ctx, 7, np.ones(5), 1.0, [(0, 0, 1)], (0, 0))          # unknown kind
    with pytest.raises(B.BabError):
        B.bab_set_cost(g.ctx, B.COST_PUSHING_OBSTACLES, np.ones(5), 1.0, [(0, 0, 1)] * 9, (0, 0))  # too many
    with pytest.raises(B.BabError):
        B.bab_set_cost(g.ctx, B.COST_PUSHING_OBSTACLES, -np.ones(5), 1.0, [(0, 0, 1)], (0, 0))     # w < 0
    B.bab_set_cost(g.ctx, B.COST_PUSHING_OBSTACLES, np.ones(5), 1.0, [], (0, 0))                 # no obstacles


def test_obstacle_cost_empty_batch(obst):
    """n = 0 is a no-op on every supported path."""
    from gpu_util import DEV, T, ids_t
    from paper_2412_09584_gb300 import binding as B
    p, g = obst(H=5)
    e = torch.empty(0, 10, device=DEV)
    z = torch.empty(0, device=DEV)
    B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, e, e, 0, z)
    B.bab_bound_ibp(g.ctx, g.x0, g.goal, g.H, g.rho, e, e, 0, z)
    B.bab_rollout(g.ctx, g.x0, g.goal, g.H, g.rho, e, e, torch.empty(0, dtype=torch.int64, device=DEV), 0, 64, 1,
                  B.PREC_FP32, z, e)
    torch.cuda.synchronize()
    assert B.bab_status(g.ctx) == 0
