"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
test vectors, hand-worked examples (tests/golden), closed forms, vertex brute
force, dense grids, finite differences, or an independent library routine.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2412_09584_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def hand_problem():
    g = json.load(open(os.path.join(GOLDEN, "hand_crown.json")))
    n = g["network"]
    layers = [(np.array(n["W1"]), np.array(n["b1"])), (np.array(n["W2"]), np.array(n["b2"]))]
    p = dict(dims=n["dims"], params=W.pack_params(layers), x0=np.array(g["x0"], dtype=np.float32),
             goal=np.array(g["goal"], dtype=np.float32), H=g["H"], rho=g["rho"], s=1, k=1)
    return p, g


def scaled_problem(s, k, hidden, H, rho, seed, scale=1.0, bias_shift=None):
    """A random problem; scale multiplies the weights, bias_shift (per hidden layer) is added to biases."""
    p = W.make_problem(s, k, hidden, H, rho, seed, weight_scale=scale)
    layers = W.unpack_params(p)
    if bias_shift is not None:
        layers = [(Wl, bl + (bias_shift[i] if i < len(layers) - 1 else 0.0)) for i, (Wl, bl) in enumerate(layers)]
    p["params"] = W.pack_params([(Wl.astype(np.float64), bl.astype(np.float64)) for Wl, bl in layers])
    return p


# --------------------------------------------------------------------------
# Counter-based sampler: SplitMix64 published reference sequence
# --------------------------------------------------------------------------

def test_splitmix64_reference_sequence(oracle):
    # Reference outputs of SplitMix64 seeded with 1234567 (the test vector
    # published with the generator's reference C implementation).
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
              16408922859458223821]
    gamma = 0x9E3779B97F4A7C15
    x = 1234567
    got = []
    for _ in range(5):
        got.append(oracle.lib().oracle_splitmix64(x))
        x = (x + gamma) % (1 << 64)
    assert got == expect


def test_samples_fp32_formula_and_range(oracle):
    rng = np.random.default_rng(3)
    for _ in range(200):
        lo = np.float32(rng.uniform(-1, 0.5))
        hi = np.float32(lo + rng.uniform(0, 1))
        u = oracle.sample(11, 12345, int(rng.integers(0, 4096)), int(rng.integers(0, 160)), lo, hi)
        assert lo <= u <= hi
    # the draw is r = (top 24 bits) / 2^24 of the chained hash; u = lo + (hi-lo)*r in FP32
    sm = oracle.lib().oracle_splitmix64
    seed, bid, m, j = 5, 77, 3, 9
    h = sm(seed ^ sm(bid))
    h = sm(h ^ ((m << 32) | j))
    r = np.float32(h >> 40) * np.float32(1.0 / 16777216.0)
    lo, hi = np.float32(-0.75), np.float32(0.5)
    assert oracle.sample(seed, bid, m, j, lo, hi) == np.float32(lo + np.float32(np.float32(hi - lo) * r))
    # zero-width interval returns the point
    assert oracle.sample(1, 2, 3, 4, np.float32(0.25), np.float32(0.25)) == np.float32(0.25)


# --------------------------------------------------------------------------
# Objective (Section 3, Eq. trajop)
# --------------------------------------------------------------------------

def test_objective_hand_example(oracle):
    p, g = hand_problem()
    for pt in g["objective_points"]:
        assert oracle.objective(p, np.array(pt["u"])) == pytest.approx(pt["f"], rel=1e-14)


def test_objective_all_active_closed_form(oracle):
    """All ReLUs active: the dynamics are affine, x_{t+1} = (I + Wx) x_t + Wu u_t + c, and f is a quadratic
    evaluated here by plain matrix algebra."""
    s, k, H, rho = 3, 2, 4, 0.05
    rng = np.random.default_rng(9)
    # layer 1 biased far positive; layer 2 has nonnegative weights and bias, so every ReLU is active
    layers = [(rng.normal(size=(8, s + k)), np.full(8, 50.0)),
              (rng.uniform(0, 0.1, size=(8, 8)), np.full(8, 1.0)),
              (0.01 * rng.normal(size=(s, 8)), 0.1 * rng.normal(size=s))]
    p = dict(dims=[s + k, 8, 8, s], params=W.pack_params(layers), x0=rng.normal(size=s).astype(np.float32),
             goal=rng.normal(size=s).astype(np.float32), H=H, rho=rho, s=s, k=k)
    layers = [(Wl.astype(np.float64), bl.astype(np.float64)) for Wl, bl in W.unpack_params(p)]
    Weff = np.eye(s + k)
    beff = np.zeros(s + k)
    for Wl, bl in layers:
        beff = Wl @ beff + bl
        Weff = Wl @ Weff
    rng = np.random.default_rng(0)
    for _ in range(5):
        u = rng.uniform(-1, 1, size=k * H)
        x = p["x0"].astype(np.float64)
        f = 0.0
        for t in range(H):
            ut = u[t * k:(t + 1) * k]
            x = x + Weff[:, :s] @ x + Weff[:, s:] @ ut + beff
            f += np.sum((x - p["goal"]) ** 2) + rho * np.sum(ut ** 2)
        fo, traj, pre = oracle.objective(p, u, with_traj=True)
        assert (pre > 0).all()
        assert fo == pytest.approx(f, rel=1e-12)


# --------------------------------------------------------------------------
# Rollout (Section 3.3)
# --------------------------------------------------------------------------

def test_rollout_is_min_over_its_samples(oracle):
    p = scaled_problem(4, 2, [16, 16], 3, 0.01, seed=2, scale=1.0)
    lo, hi, ids = W.random_boxes(6, 5, seed=4, min_width=0.1, max_width=1.0)
    M, seed = 40, 99
    ub, best_u, best_m = oracle.rollout(p, lo, hi, ids, M, seed)
    for i in range(5):
        vals = []
        for m in range(M):
            u = np.array([oracle.sample(seed, int(ids[i]), m, j, lo[i, j], hi[i, j]) for j in range(6)],
                         dtype=np.float32)
            assert (u >= lo[i]).all() and (u <= hi[i]).all()
            vals.append(oracle.objective(p, u.astype(np.float64)))
        assert ub[i] == min(vals)
        assert best_m[i] == int(np.argmin(vals))
        assert oracle.objective(p, best_u[i].astype(np.float64)) == ub[i]


def test_rollout_zero_width_box(oracle):
    p = W.config_problem("tiny", 1)
    lo, hi, ids = W.random_boxes(10, 3, seed=1, min_width=0.0, max_width=0.0)
    ub, best_u, _ = oracle.rollout(p, lo, hi, ids, 8, 1)
    for i in range(3):
        assert (best_u[i] == lo[i]).all()
        assert ub[i] == oracle.objective(p, lo[i].astype(np.float64))


# --------------------------------------------------------------------------
# IBP intermediate bounds
# --------------------------------------------------------------------------

def test_ibp_contains_sampled_trajectories(oracle):
    p = scaled_problem(4, 2, [16, 16], 4, 0.01, seed=8, scale=1.0)
    lo, hi, ids = W.random_boxes(8, 6, seed=9, min_width=0.05, max_width=1.5)
    lb, pl, pu, xl, xu = oracle.ibp(p, lo, hi)
    rng = np.random.default_rng(1)
    for i in range(6):
        for _ in range(300):
            u = lo[i] + rng.uniform(size=8) * (hi[i] - lo[i])
            f, traj, pre = oracle.objective(p, u, with_traj=True)
            assert (pre >= pl[i] - 1e-12).all() and (pre <= pu[i] + 1e-12).all()
            assert (traj >= xl[i] - 1e-12).all() and (traj <= xu[i] + 1e-12).all()
            assert lb[i] <= f + 1e-12


def test_ibp_zero_width_box_is_forward_pass(oracle):
    p = W.config_problem("tiny", 3)
    lo, hi, _ = W.random_boxes(10, 2, seed=2, min_width=0.0, max_width=0.0)
    lb, pl, pu, xl, xu = oracle.ibp(p, lo, hi)
    for i in range(2):
        f, traj, pre = oracle.objective(p, lo[i].astype(np.float64), with_traj=True)
        np.testing.assert_allclose(pl[i], pre, rtol=0, atol=1e-13)
        np.testing.assert_allclose(pu[i], pre, rtol=0, atol=1e-13)
        np.testing.assert_allclose(xl[i], traj, rtol=0, atol=1e-13)
        np.testing.assert_allclose(xu[i], traj, rtol=0, atol=1e-13)
        assert lb[i] == pytest.approx(f, rel=1e-13)


def test_ibp_single_affine_layer_exact_range(oracle):
    """With no hidden layer and H=1, each coordinate of x_1 is affine in u, so the interval bound is the exact
    range, which vertex enumeration gives."""
    s, k = 3, 6
    p = scaled_problem(s, k, [], 1, 0.0, seed=12, scale=1.0)
    lo, hi, _ = W.random_boxes(k, 4, seed=13, min_width=0.1, max_width=1.2)
    lb, pl, pu, xl, xu = oracle.ibp(p, lo, hi)
    for i in range(4):
        vals = []
        for bits in itertools.product([0, 1], repeat=k):
            u = np.where(np.array(bits) == 1, hi[i], lo[i]).astype(np.float64)
            _, traj, _ = oracle.objective(p, u, with_traj=True)
            vals.append(traj[1])
        vals = np.array(vals)
        np.testing.assert_allclose(xl[i, 1], vals.min(axis=0), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(xu[i, 1], vals.max(axis=0), rtol=1e-12, atol=1e-12)


def test_ibp_hand_example(oracle):
    p, g = hand_problem()
    lo = np.array([g["box"]["lo"]], dtype=np.float32)
    hi = np.array([g["box"]["hi"]], dtype=np.float32)
    lb, pl, pu, xl, xu = oracle.ibp(p, lo, hi)
    e = g["ibp"]
    assert pl[0, 0, 0] == e["pre_lo"] and pu[0, 0, 0] == e["pre_hi"]
    assert xl[0, 1, 0] == e["x1_lo"] and xu[0, 1, 0] == e["x1_hi"]
    assert lb[0] == pytest.approx(e["lb_ibp"], rel=1e-14)


# --------------------------------------------------------------------------
# Relaxations: tangent / chord of s^2, Lemma 1
# --------------------------------------------------------------------------

def test_square_tangent_and_chord(oracle):
    rng = np.random.default_rng(4)
    for _ in range(50):
        L = rng.uniform(-3, 3)
        U = L + rng.uniform(0, 4)
        m = 0.5 * (L + U)
        assert oracle.sq_tangent(m, m) == pytest.approx(m * m, abs=1e-14)
        assert oracle.sq_chord(L, U, L) == pytest.approx(L * L, abs=1e-12)
        assert oracle.sq_chord(L, U, U) == pytest.approx(U * U, abs=1e-12)
        for sv in np.linspace(L, U, 41):
            assert oracle.sq_tangent(m, sv) <= sv * sv + 1e-12
            assert oracle.sq_chord(L, U, sv) >= sv * sv - 1e-12


def test_relu_relaxation_lemma1(oracle):
    cases = [(-2.0, 3.0), (-3.0, 1.0), (0.5, 2.0), (0.0, 1.0), (-2.0, -0.5), (-1.0, 0.0)]
    for l, u in cases:
        zs = np.linspace(l, u, 101)
        for a in (0.0, 0.3, 1.0):
            Dl, cl = oracle.relu_relax(l, u, a, 0)
            Du, cu = oracle.relu_relax(l, u, a, 1)
            relu = np.maximum(zs, 0)
            assert (Dl * zs + cl <= relu + 1e-12).all()
            assert (Du * zs + cu >= relu - 1e-12).all()
        if l < 0 < u:
            Du, cu = oracle.relu_relax(l, u, 0.5, 1)
            assert Du * l + cu == pytest.approx(0.0, abs=1e-12)       # chord touches at l
            assert Du * u + cu == pytest.approx(u, abs=1e-12)         # and at u
            assert oracle.relu_relax(l, u, 0.3, 0) == (0.3, 0.0)
        elif l >= 0:
            assert oracle.relu_relax(l, u, 0.3, 0) == (1.0, 0.0) == oracle.relu_relax(l, u, 0.3, 1)
        else:
            assert oracle.relu_relax(l, u, 0.3, 0) == (0.0, 0.0) == oracle.relu_relax(l, u, 0.3, 1)


# --------------------------------------------------------------------------
# CROWN bound (Appendix B.1)
# --------------------------------------------------------------------------

def test_crown_hand_example(oracle):
    p, g = hand_problem()
    lo = np.array([g["box"]["lo"]], dtype=np.float32)
    hi = np.array([g["box"]["hi"]], dtype=np.float32)
    r = oracle.crown(p, lo, hi)
    e = g["crown_adaptive"]
    assert r["lb"][0] == pytest.approx(e["lb"], rel=1e-14)
    assert r["lin_coef"][0, 0] == pytest.approx(e["lin_coef"][0], rel=1e-14)
    assert r["lin_const"][0] == pytest.approx(e["lin_const"], rel=1e-14)
    assert r["ustar"][0, 0] == e["ustar"][0]
    r0 = oracle.crown(p, lo, hi, alpha=np.zeros((1, 1, 1)))
    assert r0["lb"][0] == pytest.approx(g["crown_alpha0"]["lb"], rel=1e-14)
    lb, grad, _ = oracle.alpha_grad(p, lo, hi, alpha=np.ones((1, 1, 1)))
    assert grad[0, 0, 0] == pytest.approx(g["alpha_grad_at_1"]["grad"], rel=1e-14)


def test_crown_zero_width_box_equals_objective(oracle):
    for name, seed in (("tiny", 4), ("pushing", 5)):
        p = W.config_problem(name, seed)
        d = p["k"] * p["H"]
        lo, hi, _ = W.random_boxes(d, 2, seed=seed, min_width=0.0, max_width=0.0)
        r = oracle.crown(p, lo, hi)
        for i in range(2):
            f = oracle.objective(p, lo[i].astype(np.float64))
            assert r["lb"][i] == pytest.approx(f, rel=1e-11)


def test_crown_sound_on_dense_grid_tiny_boxes(oracle):
    """3^10 grid points inside each of two small boxes of the tiny workload (scaled-up weights so that ReLUs
    are unstable); the bound must not exceed any of them."""
    p = scaled_problem(4, 2, [32, 32], 5, 0.0, seed=21, scale=3.0)
    lo, hi, _ = W.random_boxes(10, 2, seed=22, min_width=0.02, max_width=0.08)
    r = oracle.crown(p, lo, hi)
    _, pl, pu, _, _ = oracle.ibp(p, lo, hi)
    assert ((pl < 0) & (pu > 0)).sum() > 0, "test needs unstable neurons"
    for i in range(2):
        axes = [np.linspace(lo[i, j], hi[i, j], 3) for j in range(10)]
        fmin = np.inf
        for pt in itertools.product(*axes):
            fmin = min(fmin, oracle.objective(p, np.array(pt)))
        assert r["lb"][i] <= fmin + 1e-12


def test_crown_sound_random_points_large_boxes(oracle):
    p = scaled_problem(8, 2, [64, 64, 64], 6, 0.01, seed=23, scale=2.0)
    lo, hi, _ = W.random_boxes(12, 4, seed=24, min_width=0.5, max_width=2.0)
    r = oracle.crown(p, lo, hi)
    assert np.all(r["scale"] >= np.abs(r["lb"]) * (1 - 1e-12))  # the term scale dominates the bound
    lbi = oracle.ibp(p, lo, hi)[0]
    rng = np.random.default_rng(2)
    for i in range(4):
        for _ in range(400):
            u = lo[i] + rng.uniform(size=12) * (hi[i] - lo[i])
            f = oracle.objective(p, u)
            assert r["lb"][i] <= f + 1e-10
            assert lbi[i] <= f + 1e-10
        # the linear function itself is below f at every sample
        for _ in range(50):
            u = lo[i] + rng.uniform(size=12) * (hi[i] - lo[i])
            lin = r["lin_const"][i] + r["lin_coef"][i] @ u + p["rho"] * np.sum(u * u)
            assert lin <= oracle.objective(p, u) + 1e-10
            assert lin >= r["lb"][i] - 1e-10


def _tangent_linear_objective(oracle, p, lo, hi, u):
    """sum_t sum_i [2 m (x_t,i(u) - g_i) - m^2] + rho ||u||^2, the objective with each square replaced by its
    tangent at the midpoint m of its interval bound, evaluated through the true forward pass."""
    _, _, _, xl, xu = oracle.ibp(p, lo[None], hi[None])
    f, traj, _ = oracle.objective(p, u, with_traj=True)
    m = 0.5 * ((xl[0] - p["goal"]) + (xu[0] - p["goal"]))
    val = 0.0
    for t in range(1, p["H"] + 1):
        val += np.sum(2 * m[t] * (traj[t] - p["goal"]) - m[t] ** 2)
    return val + p["rho"] * np.sum(u * u)


def stable_problem(s, k, H, seed, frac_active1, frac_active2):
    """A network whose ReLUs are all stable for |x|, |u| of order 1: layer-1 biases are +-50, layer-2 weights
    are nonnegative with biases +1 (active) or -1000 (inactive), and the output layer is small."""
    rng = np.random.default_rng(seed)
    b1 = np.where(rng.uniform(size=12) < frac_active1, 50.0, -50.0)
    b2 = np.where(rng.uniform(size=12) < frac_active2, 1.0, -1000.0)
    layers = [(rng.normal(size=(12, s + k)), b1), (rng.uniform(0, 0.1, size=(12, 12)), b2),
              (0.05 * rng.normal(size=(s, 12)), 0.1 * rng.normal(size=s))]
    return dict(dims=[s + k, 12, 12, s], params=W.pack_params(layers), x0=rng.normal(size=s).astype(np.float32),
                goal=rng.normal(size=s).astype(np.float32), H=H, rho=0.0, s=s, k=k)


@pytest.mark.parametrize("fracs", [(1.0, 1.0), (0.5, 1.0), (0.6, 0.5)])
def test_crown_stable_network_gives_exact_linear_bound(oracle, fracs):
    """With every ReLU stable on the box the network is affine there, so the bound's linear function must
    equal the tangent-linearised objective at every point, and (rho = 0) its minimum over the box is the
    minimum over the 2^d vertices."""
    s, k, H = 3, 2, 4
    p = stable_problem(s, k, H, 31, *fracs)
    lo, hi, _ = W.random_boxes(k * H, 2, seed=32, min_width=0.2, max_width=1.0)
    _, pl, pu, _, _ = oracle.ibp(p, lo, hi)
    assert not ((pl < 0) & (pu > 0)).any()
    r = oracle.crown(p, lo, hi)
    rng = np.random.default_rng(5)
    for i in range(2):
        for _ in range(20):
            u = lo[i] + rng.uniform(size=k * H) * (hi[i] - lo[i])
            lin = r["lin_const"][i] + r["lin_coef"][i] @ u
            ref = _tangent_linear_objective(oracle, p, lo[i], hi[i], u)
            assert lin == pytest.approx(ref, rel=1e-11, abs=1e-11)
        best = np.inf
        for bits in itertools.product([0, 1], repeat=k * H):
            u = np.where(np.array(bits) == 1, hi[i], lo[i]).astype(np.float64)
            best = min(best, _tangent_linear_objective(oracle, p, lo[i], hi[i], u))
        assert r["lb"][i] == pytest.approx(best, rel=1e-11, abs=1e-11)


def test_crown_any_alpha_is_sound_and_relaxed_identity(oracle):
    p = scaled_problem(4, 2, [32, 32], 5, 0.01, seed=41, scale=3.0)
    lo, hi, _ = W.random_boxes(10, 3, seed=42, min_width=0.1, max_width=0.6)
    rng = np.random.default_rng(6)
    alpha = rng.uniform(0, 1, size=(3, 5, 64))
    lb, g, robj = oracle.alpha_grad(p, lo, hi, alpha)
    np.testing.assert_allclose(robj, lb, rtol=1e-12, atol=1e-12)
    for i in range(3):
        for _ in range(200):
            u = lo[i] + rng.uniform(size=10) * (hi[i] - lo[i])
            assert lb[i] <= oracle.objective(p, u) + 1e-10


# --------------------------------------------------------------------------
# alpha gradient: central finite differences
# --------------------------------------------------------------------------

def test_alpha_gradient_central_fd(oracle):
    # weights and box sized so that the bound is O(1): the stencil difference is then far above FP64 rounding
    p = scaled_problem(4, 2, [32, 32], 5, 0.01, seed=51, scale=0.3)
    lo, hi, _ = W.random_boxes(10, 4, seed=52, min_width=0.5, max_width=1.0)
    _alpha_fd_check(oracle, p, lo, hi, 7)


def test_alpha_gradient_central_fd_obstacle_cost(oracle, obstacle_cost):
    """The same pin with the pushing-with-obstacles cost (Appendix D.4): its relaxation is linear in the states and
    actions and does not depend on the slopes, so dLB/dalpha = A_j z~_j still holds."""
    p = scaled_problem(4, 2, [32, 32], 5, 0.01, seed=53, scale=0.3)
    lo, hi, _ = W.random_boxes(10, 4, seed=54, min_width=0.5, max_width=1.0)
    lb_sq = oracle.crown(p, lo, hi)["lb"]
    obstacle_cost(5, 53, n_obs=3, lam=10.0)
    lb_obs = _alpha_fd_check(oracle, p, lo, hi, 9)
    assert not np.allclose(lb_obs, lb_sq)   # the bound is the obstacle cost's, not the squared distance's


def _alpha_fd_check(oracle, p, lo, hi, seed):
    """The oracle's alpha gradient against central differences of its own bound on 16 coordinates (kinks
    skipped); exact zeros where a slope is unused.  Returns the bound."""
    rng = np.random.default_rng(seed)
    n, H, sumh = lo.shape[0], p["H"], sum(p["dims"][1:-1])
    alpha = rng.uniform(0.05, 0.95, size=(n, H, sumh))
    lb, g, _ = oracle.alpha_grad(p, lo, hi, alpha)
    Ap = oracle.crown(p, lo, hi, alpha)["A_pre"]
    _, pl, pu, _, _ = oracle.ibp(p, lo, hi)
    unstable = (pl < 0) & (pu > 0)
    # zero gradient where the slope is unused: stable neurons, or upper bound selected
    assert (g[~unstable] == 0).all()
    assert (g[unstable & (Ap < 0)] == 0).all()
    cand = np.argwhere(unstable & (Ap > 0))
    assert len(cand) >= 16
    eps = 1e-4
    checked = 0
    for c in cand[rng.permutation(len(cand))]:
        i, t, j = c
        ap, am = alpha.copy(), alpha.copy()
        ap[i, t, j] += eps
        am[i, t, j] -= eps
        rp = oracle.crown(p, lo[i:i + 1], hi[i:i + 1], ap[i:i + 1])
        rm = oracle.crown(p, lo[i:i + 1], hi[i:i + 1], am[i:i + 1])
        if not (np.sign(rp["A_pre"]) == np.sign(rm["A_pre"])).all() or \
                not (np.sign(rp["A_pre"]) == np.sign(Ap[i:i + 1])).all():
            continue  # a relaxation selection flips inside the stencil: kink, skip
        clamp_p = (rp["ustar"] == lo[i:i + 1]) | (rp["ustar"] == hi[i:i + 1])
        clamp_m = (rm["ustar"] == lo[i:i + 1]) | (rm["ustar"] == hi[i:i + 1])
        if not (clamp_p == clamp_m).all():
            continue  # the concretizing point changes face inside the stencil: kink, skip
        fp, fm = rp["lb"][0], rm["lb"][0]
        fd = (fp - fm) / (2 * eps)
        assert g[i, t, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        checked += 1
        if checked == 16:
            break
    assert checked == 16
    return lb


# --------------------------------------------------------------------------
# Adam (independent library implementation)
# --------------------------------------------------------------------------

def test_adam_matches_torch_maximize_with_clamp(oracle):
    import torch
    rng = np.random.default_rng(8)
    x0 = rng.uniform(0, 1, size=50)
    p_t = torch.tensor(x0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p_t], lr=0.1, betas=(0.9, 0.999), eps=1e-8, maximize=True)
    param = x0.copy()
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 21):
        g = rng.normal(size=50)
        p_t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        with torch.no_grad():
            p_t.clamp_(0.0, 1.0)
        oracle.adam_ascent(param, m, v, g, step, 0.1)
        np.testing.assert_allclose(param, p_t.detach().numpy(), rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------
# Prune / pick out / split (Section 3 overview, Section 3.1)
# --------------------------------------------------------------------------

def test_prune_branch_hand_cases(oracle):
    d = 3
    lo = np.array([[-1, -1, -1], [0, -1, -1], [-1, 0, -1], [0, 0, -1], [-0.5, -1, 0]], dtype=np.float32)
    hi = np.array([[0, 1, 1], [1, 1, 1], [1, 1, 0], [1, 1, 0], [0, 0, 1]], dtype=np.float32)
    ids = np.array([8, 9, 10, 11, 12], dtype=np.uint64)
    lb = np.array([1.0, 5.0, np.nan, 3.0, 3.0], dtype=np.float32)
    ub = np.array([2.0, 6.0, 9.0, 4.0, 3.5], dtype=np.float32)
    # inc 3.0: box 1 pruned (5 > 3); NaN kept; lb == inc kept (strict comparison)
    r = oracle.prune_branch(lo, hi, lb, ub, ids, 3.0, n_pick=8)
    assert list(r["keep"]) == [1, 0, 1, 1, 1]
    assert r["n_children"] == 8 and r["n_rest"] == 0
    # box 0 widths (1,2,2): dim 1 (lowest index among the widest); mid 0
    np.testing.assert_array_equal(r["lo"][0], [-1, -1, -1]); np.testing.assert_array_equal(r["hi"][0], [0, 0, 1])
    np.testing.assert_array_equal(r["lo"][1], [-1, 0, -1]); np.testing.assert_array_equal(r["hi"][1], [0, 1, 1])
    assert list(r["id"][:2]) == [16, 17]
    # box 2 widths (2,1,1): dim 0 at 0
    np.testing.assert_array_equal(r["hi"][2], [0, 1, 0]); np.testing.assert_array_equal(r["lo"][3], [0, 0, -1])
    # box 4 widths (0.5,1,1): dim 1 at -0.5
    np.testing.assert_array_equal(r["hi"][6], [0, -0.5, 1]); np.testing.assert_array_equal(r["lo"][7], [-0.5, -0.5, 0])
    assert list(r["id"]) == [16, 17, 20, 21, 22, 23, 24, 25]
    assert list(r["lb"][:2]) == [1.0, 1.0]

    # pick-out over capacity: n_pick=2, eta=0.75 -> ceil(1.5)=2 by (ub, id): boxes 0 (ub 2) and 4 (ub 3.5)
    r = oracle.prune_branch(lo, hi, lb, ub, ids, 3.0, n_pick=2)
    assert r["n_children"] == 4 and r["n_rest"] == 2
    assert list(r["id"]) == [16, 17, 24, 25, 10, 11]
    # n_pick=3, eta=0.5 -> 2 by ub (boxes 0, 4), then 1 by (lb, id) among {2 (NaN), 3 (lb 3)} -> box 3
    r = oracle.prune_branch(lo, hi, lb, ub, ids, 3.0, n_pick=3, eta=0.5)
    assert list(r["id"]) == [16, 17, 22, 23, 24, 25, 10]
    # ub ties are broken by id
    ub2 = np.array([2.0, 6.0, 2.0, 2.0, 2.0], dtype=np.float32)
    r = oracle.prune_branch(lo, hi, lb, ub2, ids, 100.0, n_pick=1, eta=1.0)
    assert list(r["id"]) == [16, 17, 9, 10, 11, 12]


def test_prune_branch_edge_cases(oracle):
    d = 2
    lo = np.zeros((0, d), dtype=np.float32)
    r = oracle.prune_branch(lo, lo, np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.uint64),
                            1.0, n_pick=4)
    assert r["n_children"] == 0 and r["n_rest"] == 0
    lo = np.array([[-1, -1], [0, 0]], dtype=np.float32)
    hi = np.array([[1, 1], [1, 1]], dtype=np.float32)
    r = oracle.prune_branch(lo, hi, np.array([5, 6], np.float32), np.array([7, 8], np.float32),
                            np.array([2, 3], np.uint64), 1.0, n_pick=4)
    assert list(r["keep"]) == [0, 0] and r["n_children"] == 0 and r["n_rest"] == 0
    # deeper than 62 splits the identifier continues as a hash of the path: 2^62 + (splitmix(2 id + c) >> 2)
    for deep in (1 << 62, (1 << 63) - 1, (1 << 63) + 5):
        r = oracle.prune_branch(lo[:1], hi[:1], np.array([0], np.float32), np.array([1], np.float32),
                                np.array([deep], np.uint64), 1.0, n_pick=4)
        assert r["rc"] == 0 and r["n_children"] == 2
        want = [(1 << 62) | (oracle.lib().oracle_splitmix64((2 * deep + c) % (1 << 64)) >> 2) for c in (0, 1)]
        assert [int(v) for v in r["id"]] == want
        assert all((1 << 62) <= v < (1 << 63) for v in want) and want[0] != want[1]
    r = oracle.prune_branch(lo[:1], hi[:1], np.array([0], np.float32), np.array([1], np.float32),
                            np.array([(1 << 62) - 1], np.uint64), 1.0, n_pick=4)
    assert [int(v) for v in r["id"]] == [(1 << 63) - 2, (1 << 63) - 1]


def test_grid_boxes_match_repeated_bisection(oracle):
    """The generator's initial grid equals what repeated widest-dimension bisection of [-1,1]^d produces."""
    d, levels = 10, 6
    lo = np.full((1, d), -1, np.float32)
    hi = np.full((1, d), 1, np.float32)
    ids = np.array([1], np.uint64)
    for _ in range(levels):
        n = len(ids)
        r = oracle.prune_branch(lo, hi, np.zeros(n, np.float32), np.zeros(n, np.float32), ids, np.inf, n_pick=n)
        lo, hi, ids = r["lo"], r["hi"], r["id"]
    glo, ghi, gid = W.grid_boxes(d, levels)
    order = np.argsort(ids)
    gorder = np.argsort(gid)
    np.testing.assert_array_equal(ids[order], gid[gorder])
    np.testing.assert_array_equal(lo[order], glo[gorder])
    np.testing.assert_array_equal(hi[order], ghi[gorder])


# --------------------------------------------------------------------------
# BaB end to end: brute force on a 2-D problem
# --------------------------------------------------------------------------

def test_bab_end_to_end_against_grid(oracle):
    p = scaled_problem(2, 2, [16, 16], 1, 0.0, seed=61, scale=4.0)
    grid = np.linspace(-1, 1, 401)
    fgrid = min(oracle.objective(p, np.array([a, b])) for a in grid for b in grid)
    lo = np.array([[-1, -1]], np.float32)
    hi = np.array([[1, 1]], np.float32)
    inc, inc_u, hist = oracle.bab(p, lo, hi, np.array([1], np.uint64), iters=25, n_pick=8, samples=16, seed=3)
    assert oracle.objective(p, inc_u.astype(np.float64)) == inc
    for h in hist:
        assert h["global_lb"] <= min(fgrid, inc) + 1e-12 or h["pool"] == 0
    # grid resolution 0.005; the objective's slope is O(10): allow 0.05 + 1e-6
    assert inc <= fgrid + 0.05


@pytest.mark.parametrize("adaptive", [False, True])
def test_box_gradient_central_fd(oracle, adaptive):
    """d(bound)/d(box faces) against central differences of the oracle's own bound, at coordinates where no
    relaxation choice, ReLU mask of the interval bounds, adaptive slope or concretization face changes inside the
    stencil (the bound is piecewise smooth in the box)."""
    p = scaled_problem(4, 2, [32, 32], 5, 0.01, seed=61, scale=0.3)
    lo, hi, _ = W.random_boxes(10, 4, seed=62, min_width=0.3, max_width=0.8)
    rng = np.random.default_rng(9)
    alpha = None if adaptive else rng.uniform(0.05, 0.95, size=(4, 5, 64))
    lb, glo, ghi = oracle.box_grad(p, lo, hi, alpha)
    np.testing.assert_allclose(lb, oracle.crown(p, lo, hi, alpha)["lb"], rtol=1e-13)

    def pattern(l_, h_, a_):
        r = oracle.crown(p, l_, h_, a_)
        _, pl, pu, _, _ = oracle.ibp(p, l_, h_)
        face = np.where(r["ustar"] == l_, 1, np.where(r["ustar"] == h_, 2, 0))
        return r["lb"][0], np.concatenate([np.sign(r["A_pre"]).ravel(), (pl > 0).ravel(), (pu > 0).ravel(),
                                           (pu >= -pl).ravel(), face.ravel()])

    eps = 1e-6
    checked = 0
    for _ in range(400):
        i, j, side = rng.integers(4), rng.integers(10), rng.integers(2)
        a_i = None if alpha is None else alpha[i:i + 1]
        lp, hp = lo[i:i + 1].astype(np.float64).copy(), hi[i:i + 1].astype(np.float64).copy()
        lm, hm = lp.copy(), hp.copy()
        (lp if side == 0 else hp)[0, j] += eps
        (lm if side == 0 else hm)[0, j] -= eps
        fp, sp = pattern(lp, hp, a_i)
        fm, sm = pattern(lm, hm, a_i)
        _, s0 = pattern(lo[i:i + 1].astype(np.float64), hi[i:i + 1].astype(np.float64), a_i)
        if not (np.array_equal(sp, sm) and np.array_equal(sp, s0)):
            continue  # a piece boundary inside the stencil: kink, skip
        g = (glo if side == 0 else ghi)[i, j]
        assert g == pytest.approx((fp - fm) / (2 * eps), rel=1e-5, abs=1e-7), (i, j, side)
        checked += 1
        if checked == 24:
            break
    assert checked == 24


def test_box_gradient_stable_one_step_closed_form(oracle):
    """One step of a network whose ReLUs are all stable on the box (an affine map there), rho = 0: the bound is
    f_lin(lo, hi) = sum_i [2 m_i (c_i - g_i) - m_i^2] + sum_j min(mu_j lo_j, mu_j hi_j), with x_1 = c + B u,
    m = c - g + B (lo + hi)/2 (the tangent point: the interval of x_1 - g is exact for an affine map) and
    mu = 2 B^T m.  Its derivative, worked out by hand:
        d/dlo_j = sum_i (c_i - g_i - m_i) B_ij + [mu_j >= 0] mu_j + sum_k (B^T B)_kj u*_k,
    and the same for hi_j with [mu_j < 0]."""
    s_, k = 3, 2
    p = stable_problem(s_, k, 1, 71, 0.6, 0.5)
    lo, hi, _ = W.random_boxes(k, 3, seed=72, min_width=0.2, max_width=0.8)
    _, pl, pu, _, _ = oracle.ibp(p, lo, hi)
    assert not ((pl < 0) & (pu > 0)).any()
    (W1, b1), (W2, b2), (W3, b3) = W.unpack_params(p)
    W1, W2, W3 = W1.astype(np.float64), W2.astype(np.float64), W3.astype(np.float64)
    D1, D2 = np.diag((b1 > 0).astype(float)), np.diag((b2 > 0).astype(float))
    J = W3 @ D2 @ W2 @ D1 @ W1                      # the affine network's Jacobian on the box
    x0, g = p["x0"].astype(np.float64), p["goal"].astype(np.float64)
    a0 = np.concatenate([x0, np.zeros(k)])
    z0 = W3 @ np.maximum(W2 @ np.maximum(W1 @ a0 + b1, 0) + b2, 0) + b3
    c = x0 + z0                                    # x_1 at u = 0
    B = J[:, s_:]
    lb, glo, ghi = oracle.box_grad(p, lo, hi)
    for i in range(3):
        m = c - g + B @ (lo[i] + hi[i]) / 2
        mu = 2 * B.T @ m
        ustar = np.where(mu >= 0, lo[i], hi[i])
        f = np.sum(2 * m * (c - g) - m * m) + np.sum(np.minimum(mu * lo[i], mu * hi[i]))
        assert lb[i] == pytest.approx(f, rel=1e-10, abs=1e-12)
        common = B.T @ (c - g - m) + (B.T @ B) @ ustar
        tol = 1e-10 * max(np.abs(B).sum() * np.abs(m).max(), np.abs(mu).max(), 1.0)  # FP64 cancellation scale
        np.testing.assert_allclose(glo[i], common + np.where(mu >= 0, mu, 0), rtol=1e-9, atol=tol)
        np.testing.assert_allclose(ghi[i], common + np.where(mu < 0, mu, 0), rtol=1e-9, atol=tol)


# --------------------------------------------------------------------------
# The paper's bounding: search-integrated bounds and propagation early-stop
# --------------------------------------------------------------------------

def test_search_bounds_are_sample_extremes(oracle):
    """The empirical bounds are, by definition, the min / max over the search's samples: recomputed here by
    evaluating every sample's trajectory with a direct numpy forward pass."""
    p = W.config_problem("tiny", 3)
    lo, hi, ids = W.random_boxes(10, 3, seed=4, min_width=0.2, max_width=1.0)
    M, seed = 17, 5
    pl, pu, xl, xu = oracle.search_bounds(p, lo, hi, ids, M, seed)
    layers = [(Wl.astype(np.float64), bl.astype(np.float64)) for Wl, bl in W.unpack_params(p)]
    for i in range(3):
        pre_all, x_all = [], []
        for m in range(M):
            u = np.array([oracle.lib().oracle_sample(seed, int(ids[i]), m, j, float(lo[i, j]), float(hi[i, j]))
                          for j in range(10)], dtype=np.float64)
            x = p["x0"].astype(np.float64)
            pres, xs = [], [x.copy()]
            for t in range(p["H"]):
                a = np.concatenate([x, u[t * 2:t * 2 + 2]])
                hs = []
                for l, (Wl, bl) in enumerate(layers):
                    z = Wl @ a + bl
                    if l < len(layers) - 1:
                        hs.append(z)
                        a = np.maximum(z, 0)
                    else:
                        x = x + z
                pres.append(np.concatenate(hs))
                xs.append(x.copy())
            pre_all.append(pres)
            x_all.append(xs)
        pre_all, x_all = np.array(pre_all), np.array(x_all)
        np.testing.assert_allclose(pl[i], pre_all.min(axis=0), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(pu[i], pre_all.max(axis=0), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(xl[i], x_all.min(axis=0), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(xu[i], x_all.max(axis=0), rtol=1e-12, atol=1e-12)


def test_crown_given_reduces_to_crown_and_to_interval_costs(oracle):
    """With the interval bounds and no early stop it is the plain CROWN bound; stopping at the last step leaves
    only the cost terms' interval minima plus the exact minimum of rho ||u||^2 on the box."""
    p = scaled_problem(4, 2, [32, 32], 5, 0.01, seed=81, scale=0.3)
    lo, hi, _ = W.random_boxes(10, 4, seed=82, min_width=0.3, max_width=0.8)
    _, pl, pu, xl, xu = oracle.ibp(p, lo, hi)
    np.testing.assert_allclose(oracle.crown_given(p, lo, hi, pl, pu, xl, xu, 0), oracle.crown(p, lo, hi)["lb"],
                               rtol=1e-13)
    H, g, rho = p["H"], p["goal"].astype(np.float64), p["rho"]
    lb_H = oracle.crown_given(p, lo, hi, pl, pu, xl, xu, H)
    for i in range(4):
        Ls, Us = xl[i, 1:] - g, xu[i, 1:] - g
        cost = np.where((Ls <= 0) & (Us >= 0), 0.0, np.minimum(Ls * Ls, Us * Us)).sum()
        lo_, hi_ = lo[i].astype(np.float64), hi[i].astype(np.float64)
        act = np.where((lo_ <= 0) & (hi_ >= 0), 0.0, np.minimum(lo_ * lo_, hi_ * hi_)).sum()
        assert lb_H[i] == pytest.approx(cost + rho * act, rel=1e-12)


@pytest.mark.parametrize("t_stop", [1, 3])
def test_crown_given_sound_with_sound_bounds(oracle, t_stop):
    """Early stop with sound (interval) bounds is still a sound bound: below the objective at sampled points of
    the box.  The search's empirical ranges lie inside the sound ones (the samples are points of the box)."""
    p = scaled_problem(4, 2, [32, 32], 5, 0.0, seed=83, scale=0.3)
    lo, hi, ids = W.random_boxes(10, 3, seed=84, min_width=0.2, max_width=0.6)
    _, pl, pu, xl, xu = oracle.ibp(p, lo, hi)
    lb = oracle.crown_given(p, lo, hi, pl, pu, xl, xu, t_stop)
    rng = np.random.default_rng(2)
    for i in range(3):
        u = lo[i] + rng.uniform(size=(300, 10)) * (hi[i] - lo[i])
        assert lb[i] <= min(oracle.objective(p, x.astype(np.float64)) for x in u)
    epl, epu, exl, exu = oracle.search_bounds(p, lo, hi, ids, 64, 9)
    assert np.all(epl >= pl - 1e-9) and np.all(epu <= pu + 1e-9)  # the samples lie inside the sound ranges
    assert np.all(exl >= xl - 1e-9) and np.all(exu <= xu + 1e-9)


# --------------------------------------------------------------------------
# The paper's branching heuristics (Section 3.1)
# --------------------------------------------------------------------------

def test_log_det_accuracy(oracle):
    xs = np.geomspace(1e-8, 1e3, 2000).astype(np.float32)
    got = np.array([oracle.log_det(x) for x in xs])
    np.testing.assert_allclose(got, np.log(xs.astype(np.float64)), rtol=4e-7, atol=2e-7)


def test_softmax_pick_race_frequencies(oracle):
    """The smallest race key wins with the softmax probability of Eq. lf_pick: exp(-s_i/T) / sum exp(-s_j/T)."""
    lb = np.array([3.0, 3.5, 4.0, 5.0, 6.0, 3.2], dtype=np.float32)
    T = 0.4
    lmin, lmax = lb.min(), lb.max()
    sc = (lb - lmin) / (lmax - lmin)
    p = np.exp(-sc / T) / np.exp(-sc / T).sum()
    trials = 6000
    wins = np.zeros(len(lb))
    for t in range(trials):
        keys = [oracle.pick_key(float(v), float(lmin), float(lmax), T, 1000 + t, 7 + i) for i, v in enumerate(lb)]
        wins[int(np.argmin(keys))] += 1
    freq = wins / trials
    sigma = np.sqrt(p * (1 - p) / trials)
    assert np.all(np.abs(freq - p) <= 4.5 * sigma + 1e-3), (freq, p)


def test_softmax_pick_cold_limit_and_default_rule(oracle):
    """At a tiny temperature the race picks by smallest lb; with rule 0 and no split dimensions the heuristic
    pass is the plain prune / pick-out / split."""
    lo, hi, ids = W.dyadic_boxes(6, 80, seed=3, max_depth=4)
    lb, ub = W.pool_values(80, seed=4)
    cold = oracle.prune_branch_heuristic(lo, hi, lb, ub, ids, 100.0, 10, eta=0.5, pick_rule=1, temperature=1e-7,
                                         pick_seed=9)
    plain = oracle.prune_branch(lo, hi, lb, ub, ids, 100.0, 10, eta=0.5)
    assert np.array_equal(np.sort(cold["id"][:cold["n_children"]]), np.sort(plain["id"][:plain["n_children"]]))
    same = oracle.prune_branch_heuristic(lo, hi, lb, ub, ids, 100.0, 10, eta=0.5, pick_rule=0)
    for key in ("lo", "hi", "lb", "ub", "id"):
        assert np.array_equal(same[key], plain[key])


def test_split_dims_recount(oracle):
    """The chosen dimension maximises (hi - lo) |n_lo - n_up| over the top_k samples, recounted here with
    numpy from the same counter-based samples; no imbalance anywhere falls back to the widest dimension."""
    rng = np.random.default_rng(5)
    n, d, M, k = 12, 7, 40, 5
    lo, hi, ids = W.random_boxes(d, n, seed=6, min_width=0.2, max_width=1.5)
    costs = rng.normal(size=(n, M)).astype(np.float32)
    costs[3, :] = 1.0                                    # all equal: the top samples are m = 0 .. k-1
    got = oracle.split_dims(lo, hi, ids, 11, costs, k)
    for i in range(n):
        order = sorted(range(M), key=lambda m: (costs[i, m], m))[:k]
        best, jb = 0.0, -1
        for j in range(d):
            mid = np.float32(0.5) * np.float32(lo[i, j] + hi[i, j])
            u = np.array([oracle.lib().oracle_sample(11, int(ids[i]), m, j, float(lo[i, j]), float(hi[i, j]))
                          for m in order], dtype=np.float32)
            sc = np.float32(hi[i, j] - lo[i, j]) * np.float32(abs(int((u <= mid).sum()) - int((u >= mid).sum())))
            if sc > best:
                best, jb = sc, j
        if jb < 0:
            jb = int(np.argmax(hi[i] - lo[i]))
        assert got[i] == jb, i


# --------------------------------------------------------------------------
# Cross-entropy search (Section 3.3)
# --------------------------------------------------------------------------

def test_objective_f32_close_to_fp64(oracle):
    """The FP32 objective the search ranks by is the FP64 objective up to FP32 rounding."""
    for name, seed in (("tiny", 3), ("pushing", 4)):
        p = W.config_problem(name, seed)
        d = p["k"] * p["H"]
        rng = np.random.default_rng(seed)
        for _ in range(5):
            u = rng.uniform(-1, 1, size=d).astype(np.float32)
            f64 = oracle.objective(p, u.astype(np.float64))
            assert oracle.objective_f32(p, u) == pytest.approx(f64, rel=2e-6)


def test_cem_normal_moments_and_support(oracle):
    """Irwin-Hall with four uniforms, centred and scaled: mean 0, variance 1, excess kurtosis -6/(5*4) = -0.3,
    support |z| <= 2 sqrt(3); the first sample of the first iteration is the mean itself."""
    z = np.array([oracle.cem_normal(11, 5, it, m, j) for it in range(1, 3) for m in range(200) for j in range(100)])
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.02
    kurt = np.mean((z - z.mean()) ** 4) / z.var() ** 2 - 3.0
    assert abs(kurt + 0.3) < 0.05
    assert np.abs(z).max() <= 2.0 * np.sqrt(3.0) + 1e-6
    assert all(oracle.cem_normal(11, 5, 0, 0, j) == 0.0 for j in range(10))
    assert oracle.cem_normal(11, 5, 0, 1, 0) != 0.0


def test_cem_single_sample_is_the_start(oracle):
    """One iteration of one sample evaluates the start: the box centre, or the warm start clipped to the box."""
    p = W.config_problem("tiny", 5)
    lo, hi, ids = W.random_boxes(10, 4, seed=6, min_width=0.2, max_width=1.0)
    ub, bu = oracle.cem(p, lo, hi, ids, 1, 1, 1, 1e-3, 9)
    centre = (np.float32(0.5) * (lo + hi)).astype(np.float32)
    np.testing.assert_array_equal(bu, centre)
    np.testing.assert_array_equal(ub, np.array([oracle.objective_f32(p, c) for c in centre], dtype=np.float32))
    warm = np.random.default_rng(1).uniform(-1.5, 1.5, size=lo.shape).astype(np.float32)
    ub, bu = oracle.cem(p, lo, hi, ids, 1, 1, 1, 1e-3, 9, warm_u=warm)
    np.testing.assert_array_equal(bu, np.clip(warm, lo, hi))


def test_cem_first_refit_is_the_elite_mean(oracle):
    """mu after the first iteration is the mean of the E samples of smallest FP32 objective (recounted here)."""
    p = W.config_problem("tiny", 7)
    lo, hi, ids = W.random_boxes(10, 2, seed=8, min_width=0.3, max_width=1.5)
    M, E = 40, 6
    ub, bu, tr = oracle.cem(p, lo, hi, ids, M, 3, E, 1e-3, 13, with_trace=True)
    for i in range(2):
        mu0 = np.float32(0.5) * (lo[i] + hi[i])
        sg0 = np.float32(0.5) * (hi[i] - lo[i])
        S = np.array([[oracle.cem_sample(13, int(ids[i]), 0, m, j, mu0[j], sg0[j], lo[i, j], hi[i, j])
                       for j in range(10)] for m in range(M)], dtype=np.float32)
        f = np.array([oracle.objective_f32(p, S[m]) for m in range(M)])
        elite = sorted(range(M), key=lambda m: (f[m], m))[:E]
        np.testing.assert_allclose(tr[i, 0], S[elite].astype(np.float64).mean(axis=0), rtol=1e-6, atol=1e-7)
        assert np.all(S >= lo[i]) and np.all(S <= hi[i])


def test_cem_monotone_in_iterations_and_warm_start(oracle):
    """More iterations never give a worse best (the first iterations are the same draws), and a warm start
    inside the box is never beaten by the result."""
    p = W.config_problem("tiny", 10)
    lo, hi, ids = W.random_boxes(10, 5, seed=11, min_width=0.3, max_width=1.5)
    prev = None
    for iters in (1, 2, 4):
        ub, _ = oracle.cem(p, lo, hi, ids, 32, iters, 4, 1e-3, 3)
        if prev is not None:
            assert np.all(ub <= prev)
        prev = ub
    warm = (lo + np.random.default_rng(2).uniform(size=lo.shape).astype(np.float32) * (hi - lo)).astype(np.float32)
    ub, bu = oracle.cem(p, lo, hi, ids, 16, 2, 4, 1e-3, 3, warm_u=warm)
    assert np.all(ub <= np.array([oracle.objective_f32(p, w) for w in warm]))
    assert np.all(bu >= lo) and np.all(bu <= hi)
    np.testing.assert_array_equal(ub, np.array([oracle.objective_f32(p, b) for b in bu], dtype=np.float32))


def test_cem_converges_on_convex_problem(oracle):
    """All ReLUs active makes f a convex quadratic in u (closed form by matrix algebra); its box-constrained
    minimum (projected Newton / L-BFGS-B in FP64) is approached by the search from above."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    s, k, H, rho = 3, 2, 4, 0.05
    rng = np.random.default_rng(19)
    layers = [(rng.normal(size=(8, s + k)), np.full(8, 50.0)),
              (rng.uniform(0, 0.1, size=(8, 8)), np.full(8, 1.0)),
              (0.05 * rng.normal(size=(s, 8)), 0.1 * rng.normal(size=s))]
    p = dict(dims=[s + k, 8, 8, s], params=W.pack_params(layers), x0=rng.normal(size=s).astype(np.float32),
             goal=rng.normal(size=s).astype(np.float32), H=H, rho=rho, s=s, k=k)
    lw = [(Wl.astype(np.float64), bl.astype(np.float64)) for Wl, bl in W.unpack_params(p)]
    Weff, beff = np.eye(s + k), np.zeros(s + k)
    for Wl, bl in lw:
        beff = Wl @ beff + bl
        Weff = Wl @ Weff

    def f(u):
        x = p["x0"].astype(np.float64)
        tot = 0.0
        for t in range(H):
            ut = u[t * k:(t + 1) * k]
            x = x + Weff[:, :s] @ x + Weff[:, s:] @ ut + beff
            tot += np.sum((x - p["goal"]) ** 2) + rho * np.sum(ut ** 2)
        return tot

    d = k * H
    best = scipy_opt.minimize(f, np.zeros(d), method="L-BFGS-B", bounds=[(-1, 1)] * d,
                              options=dict(ftol=1e-15, gtol=1e-12, maxiter=10000))
    fstar = best.fun
    lo = np.full((1, d), -1.0, dtype=np.float32)
    hi = np.full((1, d), 1.0, dtype=np.float32)
    ub, bu = oracle.cem(p, lo, hi, np.array([3], dtype=np.uint64), 256, 40, 16, 1e-5, 21)
    assert ub[0] >= fstar * (1 - 1e-5)
    assert ub[0] <= fstar * (1 + 1e-3)
    assert f(bu[0].astype(np.float64)) == pytest.approx(float(ub[0]), rel=1e-5)


# --------------------------------------------------------------------------
# Synthetic objective (Section 4, synthetic example)
# --------------------------------------------------------------------------

def _synth_g_min():
    """The per-coordinate minimum of 5 u^2 + cos(50 u): the root of g' = 10 u - 50 sin(50 u) in the first basin."""
    from scipy.optimize import brentq
    u = brentq(lambda v: 10.0 * v - 50.0 * np.sin(50.0 * v), 0.05, 0.075, xtol=1e-15)
    return u, 5.0 * u * u + np.cos(50.0 * u)


def test_synth_objective_optima(oracle):
    """The paper's description: per coordinate 16 local minima on [-1, 1], two of them global and symmetric; the
    global value is -0.980339 (the printed constant -1.9803 cannot be reached: cos >= -1 and 5 u^2 >= 0)."""
    pytest.importorskip("scipy")
    u = np.linspace(-1.0, 1.0, 400001)
    g = np.array([oracle.synth_f(np.array([v])) for v in u[::50]])
    gv = 5.0 * u * u + np.cos(50.0 * u)
    assert np.allclose(g, gv[::50], rtol=0, atol=1e-14)
    mins = np.where((gv[1:-1] < gv[:-2]) & (gv[1:-1] < gv[2:]))[0] + 1
    assert len(mins) == 16
    ustar, gstar = _synth_g_min()
    assert gstar == pytest.approx(-0.980339, abs=1e-6)
    order = np.argsort(gv[mins])
    assert np.allclose(np.sort(np.abs(u[mins[order[:2]]])), [ustar, ustar], atol=1e-5)
    assert gv[mins[order[2]]] > gstar + 0.01
    assert oracle.synth_f(np.full(7, ustar)) == pytest.approx(7 * gstar, rel=1e-14)


def test_cos_min_brute_force(oracle):
    rng = np.random.default_rng(21)
    for _ in range(300):
        a = rng.uniform(-60, 60)
        b = a + rng.choice([rng.uniform(0, 0.5), rng.uniform(0, 8)])
        grid = np.cos(np.linspace(a, b, 20001))
        m = oracle.cos_min(a, b)
        assert m <= grid.min() + 1e-12
        assert m >= grid.min() - 2e-6   # the grid misses an interior minimum by at most its spacing squared


def test_synth_bound_sound_and_tight_as_boxes_shrink(oracle):
    rng = np.random.default_rng(22)
    for _ in range(20):
        c = rng.uniform(-1, 1, size=2)
        w = rng.uniform(0.001, 0.3, size=2)
        lo = np.float32(np.clip(c - w, -1, 1))[None]
        hi = np.float32(np.clip(c + w, -1, 1))[None]
        lb = oracle.synth_bound(lo, hi)[0]
        g = np.stack(np.meshgrid(np.linspace(lo[0, 0], hi[0, 0], 301), np.linspace(lo[0, 1], hi[0, 1], 301)), -1)
        fg = (5 * g ** 2 + np.cos(50 * g)).sum(-1)
        assert lb <= fg.min() + 1e-12
    # a box of width w around a point: the bound is within O(w) of the value there
    for w in (1e-2, 1e-3, 1e-4):
        x = np.array([0.3, -0.7, 0.05])
        lo, hi = np.float32(x - w)[None], np.float32(x + w)[None]
        gap = oracle.synth_f(x) - oracle.synth_bound(lo, hi)[0]
        assert 0 <= gap <= 3 * 60.0 * w


def test_synth_search_is_min_over_its_samples(oracle):
    lo, hi, ids = W.random_boxes(6, 5, seed=23, min_width=0.2, max_width=1.5)
    ub, bu = oracle.synth_search(lo, hi, ids, 50, 4)
    for i in range(5):
        f = [oracle.synth_f(np.array([oracle.sample(4, int(ids[i]), m, j, float(lo[i, j]), float(hi[i, j]))
                                      for j in range(6)], dtype=np.float64)) for m in range(50)]
        assert ub[i] == min(f)
        assert oracle.synth_f(bu[i].astype(np.float64)) == ub[i]


def test_synth_bab_reaches_the_optimum(oracle):
    """Algorithm 2 on the synthetic objective (d = 2): the incumbent approaches d g* and every lower bound of the
    final pool stays below it; the gap closes."""
    pytest.importorskip("scipy")
    d = 2
    _, gstar = _synth_g_min()
    lo, hi, ids = W.grid_boxes(d, 2)
    lb = oracle.synth_bound(lo, hi)
    ub, bu = oracle.synth_search(lo, hi, ids, 64, 1)
    inc = float(ub.min())
    for it in range(60):
        r = oracle.prune_branch(lo, hi, lb, ub, ids, inc, 16)
        lo, hi, ids = r["lo"], r["hi"], r["id"]
        nc = r["n_children"]
        ub_c, _ = oracle.synth_search(lo[:nc], hi[:nc], ids[:nc], 64, 1 + it)
        lb = r["lb"].astype(np.float64).copy()
        ub = r["ub"].astype(np.float64).copy()
        lb[:nc] = oracle.synth_bound(lo[:nc], hi[:nc])
        ub[:nc] = ub_c
        inc = min(inc, float(ub_c.min()))
    assert inc == pytest.approx(d * gstar, abs=2e-3)
    assert lb.min() <= d * gstar + 1e-9
    assert inc - lb.min() < 0.05


# --------------------------------------------------------------------------
# Pushing-with-obstacles cost (Appendix D.4)
# --------------------------------------------------------------------------

@pytest.fixture
def obstacle_cost(oracle):
    def make(H, seed, **kw):
        c = W.obstacle_cost(H, seed, **kw)
        oracle.set_cost(1, c["w"], c["lam"], c["obstacles"], c["p0"])
        return c
    yield make
    oracle.set_cost(0)


def _push_cost_numpy(p, c, u, traj):
    """The paper's Eq. (pushing_cost) summed over t = 1..H, written out with numpy, plus rho ||u||^2."""
    H, k, s = p["H"], p["k"], p["s"]
    pos = np.array(c["p0"], dtype=np.float64)
    f = 0.0
    for t in range(1, H + 1):
        pos = pos + u[(t - 1) * k:t * k]
        x = traj[t]
        f += c["w"][t - 1] * np.linalg.norm(x - p["goal"])
        for (ox, oy, sz) in c["obstacles"]:
            f += c["lam"] * max(0.0, sz - np.hypot(pos[0] - ox, pos[1] - oy))
            for i in range(s // 2):
                f += c["lam"] * max(0.0, sz - np.hypot(x[2 * i] - ox, x[2 * i + 1] - oy))
    return f + p["rho"] * float(np.sum(u * u))


def test_obstacle_cost_objective_formula(oracle, obstacle_cost):
    p = W.config_problem("pushing", 61)
    c = obstacle_cost(p["H"], 61)
    rng = np.random.default_rng(0)
    hits = 0
    for _ in range(6):
        u = rng.uniform(-1, 1, size=p["k"] * p["H"])
        f, traj, _ = oracle.objective(p, u, with_traj=True)
        assert f == pytest.approx(_push_cost_numpy(p, c, u, traj), rel=1e-12)
        hits += f > _push_cost_numpy(p, dict(c, lam=0.0), u, traj) + 1e-9
    assert hits > 0   # the obstacles are met by some trajectories
    u = rng.uniform(-1, 1, size=p["k"] * p["H"]).astype(np.float32)
    assert oracle.objective_f32(p, u) == pytest.approx(oracle.objective(p, u.astype(np.float64)), rel=2e-6)


def test_obstacle_relaxation_below_penalty(oracle, obstacle_cost):
    """The bound's linear pieces: with all ReLUs of a 0-hidden-step problem stable, CROWN's bound equals the
    cost at a point box, and over boxes it stays below the cost at dense samples."""
    p = W.config_problem("pushing", 62)
    p = dict(p, H=3)
    obstacle_cost(3, 62, n_obs=4)
    d = p["k"] * p["H"]
    rng = np.random.default_rng(1)
    for _ in range(8):
        u = rng.uniform(-1, 1, size=d).astype(np.float32)
        lo, hi = u[None].copy(), u[None].copy()
        c = oracle.crown(p, lo, hi)
        f = oracle.objective(p, u.astype(np.float64))
        assert c["lb"][0] == pytest.approx(f, rel=1e-9, abs=1e-9)
    for _ in range(8):
        ctr = rng.uniform(-1, 1, size=d)
        w = rng.uniform(0.01, 0.3, size=d)
        lo = np.float32(np.clip(ctr - w, -1, 1))[None]
        hi = np.float32(np.clip(ctr + w, -1, 1))[None]
        lb = oracle.crown(p, lo, hi)["lb"][0]
        lb_i = oracle.ibp(p, lo, hi)[0][0]
        us = lo + (hi - lo) * rng.uniform(size=(400, d))
        fs = np.array([oracle.objective(p, v) for v in us])
        assert lb <= fs.min() + 1e-9
        assert lb_i <= fs.min() + 1e-9


def test_obstacle_bab_end_to_end(oracle, obstacle_cost):
    """Algorithm 2 with the obstacle cost on a tiny problem (H = 1, d = 2): the incumbent approaches the dense-grid
    minimum and the lower bounds stay below it."""
    p = W.config_problem("pushing", 63)
    p = dict(p, H=1)
    obstacle_cost(1, 63, n_obs=3, lam=50.0)
    g = np.linspace(-1, 1, 401)
    fg = min(oracle.objective(p, np.array([a, b])) for a in g[::4] for b in g[::4])
    inc, _, hist = oracle.bab(p, *W.grid_boxes(2, 2), iters=40, n_pick=8, samples=64, seed=3)
    assert inc <= fg + 1e-3
    assert hist[-1]["global_lb"] <= fg + 1e-9


def test_obstacle_penalty_relaxation_brute_force(oracle):
    """a . q + b <= ReLU(s - ||q - c||) on every point of the box (dense grid), exact at a point box inside the
    obstacle, and used (nonzero) for boxes straddling or inside the obstacle."""
    rng = np.random.default_rng(64)
    used_n = 0
    for _ in range(200):
        c = rng.normal(size=2)
        sz = rng.uniform(0.2, 1.0)
        ctr = c + rng.normal(size=2) * 0.6 * sz
        w = rng.uniform(0.01, 0.5, size=2) * sz
        l0, u0, l1, u1 = ctr[0] - w[0], ctr[0] + w[0], ctr[1] - w[1], ctr[1] + w[1]
        used, a0, a1, b = oracle.relu_dist_lower(l0, u0, l1, u1, c[0], c[1], sz)
        used_n += used
        g0, g1 = np.meshgrid(np.linspace(l0, u0, 61), np.linspace(l1, u1, 61))
        pen = np.maximum(0.0, sz - np.hypot(g0 - c[0], g1 - c[1]))
        assert np.all(a0 * g0 + a1 * g1 + b <= pen + 1e-12)
        if not used:
            assert a0 == a1 == b == 0.0
    assert used_n > 30
    q = np.array([0.1, -0.2])
    used, a0, a1, b = oracle.relu_dist_lower(q[0], q[0], q[1], q[1], 0.0, 0.0, 1.0)
    assert used and a0 * q[0] + a1 * q[1] + b == pytest.approx(1.0 - np.hypot(*q), abs=1e-15)


# --------------------------------------------------------------------------
# Outward rounding margin of an FP32 / split-BF16 evaluation (oracle_crown_margin)
# --------------------------------------------------------------------------

def _round_half(x, kind):
    """x (float32 array) rounded to the high half of a split: 'bf16' to nearest even with 8 significant bits,
    'tf32' to nearest (ties away from zero) with 11, written out on the bit patterns."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    if kind == "bf16":
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    else:
        u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(x))


def _split(x, kind):
    """(hi, lo) with hi = round(x), lo = round(x - hi): the operand halves of a 3-term split product."""
    x = np.asarray(x, np.float32)
    h = _round_half(x, kind)
    return h, _round_half((x - h).astype(np.float32), kind)


def _fp32_chain(p, lo, hi, pl, pu, xl, xu, A_pre, order, seed=0, split=None):
    """The coefficient chain of the CROWN bound evaluated in FP32 (numpy float32, one rounding per multiply and
    per add, products summed in `order`: 'fwd', 'rev' or 'perm'), with the oracle's relaxation choices (lower line
    where the oracle's pre-relaxation coefficient is >= 0) and every constant term and the concretization taken
    in FP64 from the FP32 coefficients.  split = 'bf16' or 'tf32': every product A W is the 3-term split product
    A_hi W_hi + A_hi W_lo + A_lo W_hi instead, its terms accumulated in FP32.  Returns the bound per box; its
    distance from the FP64 bound is the rounding the margin has to cover."""
    f32 = np.float32
    layers = W.unpack_params(p)
    L, s, k, H, rho = len(layers), p["s"], p["k"], p["H"], float(p["rho"])
    dims = p["dims"]
    hoff = np.concatenate([[0], np.cumsum(dims[1:-1])]).astype(int)
    x0 = np.asarray(p["x0"], np.float64)
    goal = np.asarray(p["goal"], np.float64)
    rng = np.random.default_rng(seed)
    n = lo.shape[0]

    def prod(A, Wl):  # A [n, K] float32 times Wl [K, J]: sum over K in the chosen order
        K = Wl.shape[0]
        idx = np.arange(K) if order == "fwd" else (np.arange(K)[::-1] if order == "rev" else rng.permutation(K))
        acc = np.zeros((A.shape[0], Wl.shape[1]), f32)
        W32 = Wl.astype(f32)
        if split is None:
            terms = [(A, W32)]
        else:
            (Ah, Al), (Wh, Wlo) = _split(A, split), _split(W32, split)
            terms = [(Ah, Wh), (Ah, Wlo), (Al, Wh)]
        for kk in idx:
            for a_, w_ in terms:
                acc = (acc + (a_[:, kk:kk + 1] * w_[kk][None, :]).astype(f32)).astype(f32)
        return acc

    out = np.zeros(n)
    for b in range(n):
        cst = 0.0
        m = 0.5 * (xl[b, H] + xu[b, H]) - goal
        lam = (2 * m).astype(f32)[None, :]
        cst += float(np.sum(-2 * m * goal - m * m))
        mu = np.zeros(k * H)
        for t in range(H - 1, -1, -1):
            Wl_, bl_ = layers[L - 1]
            A = lam.copy()
            cst += float(A[0].astype(np.float64) @ bl_)
            A = prod(A, Wl_)  # W_L is [d_L, d_{L-1}]: A W_L
            for l in range(L - 1, 0, -1):
                Wl_, bl_ = layers[l - 1]
                zl = pl[b, t, hoff[l - 1]:hoff[l - 1] + dims[l]]
                zu = pu[b, t, hoff[l - 1]:hoff[l - 1] + dims[l]]
                Ao = A_pre[b, t, hoff[l - 1]:hoff[l - 1] + dims[l]]
                D = np.where(zl >= 0, 1.0, np.where(zu <= 0, 0.0, np.where(Ao >= 0, np.where(zu >= -zl, 1.0, 0.0),
                                                                            zu / np.where(zu > zl, zu - zl, 1.0))))
                c = np.where((zl < 0) & (zu > 0) & (Ao < 0), -zu * zl / np.where(zu > zl, zu - zl, 1.0), 0.0)
                cst += float(A[0].astype(np.float64) @ c)
                A = (A * D.astype(f32)[None, :]).astype(f32)
                cst += float(A[0].astype(np.float64) @ bl_)
                A = prod(A, Wl_)
            mu[t * k:(t + 1) * k] = A[0, s:s + k]
            at = np.zeros(s, f32)
            if t >= 1:
                mt = 0.5 * (xl[b, t] + xu[b, t]) - goal
                at = (2 * mt).astype(f32)
                cst += float(np.sum(-2 * mt * goal - mt * mt))
            lam = ((lam[0] + A[0, :s]).astype(f32) + at).astype(f32)[None, :]
        cst += float(lam[0].astype(np.float64) @ x0)
        for j in range(k * H):
            if rho > 0:
                u = min(max(-mu[j] / (2 * rho), lo[b, j]), hi[b, j])
            else:
                u = lo[b, j] if mu[j] >= 0 else hi[b, j]
            cst += mu[j] * u + rho * u * u
        out[b] = cst
    return out


@pytest.mark.parametrize("s,k,hidden,H,rho,wscale,maxw", [(4, 2, [32, 32], 5, 0.0, 0.3, 1.0),
                                                          (4, 2, [32, 32], 5, 0.01, 1.0, 0.5),
                                                          (8, 2, [128, 128], 3, 0.01, 0.3, 1.0)])
def test_margin_covers_fp32_evaluations(oracle, s, k, hidden, H, rho, wscale, maxw):
    """The margin of an FP32 evaluation covers the rounding of the coefficient chain in any summation order:
    the FP32 chain's bound minus the margin never exceeds the exact FP64 bound (checked in three orders)."""
    p = W.make_problem(s, k, hidden, H, rho, seed=31, weight_scale=wscale)
    lo, hi, _ = W.random_boxes(k * H, 6, seed=32, min_width=0.1, max_width=maxw)
    _, pl, pu, xl, xu = oracle.ibp(p, lo, hi)
    o = oracle.crown(p, lo, hi)
    r = oracle.crown_margin(p, lo, hi)
    np.testing.assert_allclose(r["lb"], o["lb"], rtol=1e-14, atol=1e-12)
    assert np.all(r["margin"] > 0)
    worst = 0.0
    for order in ("fwd", "rev", "perm"):
        v32 = _fp32_chain(p, lo, hi, pl, pu, xl, xu, o["A_pre"], order)
        assert np.all(v32 - r["margin"] <= r["lb"] + 1e-12 * np.abs(r["lb"])), order
        worst = max(worst, float(np.max(np.abs(v32 - r["lb"]) / r["margin"])))
    assert worst > 0  # the FP32 chain does round: the check is not vacuous
    # the split-BF16 margin charges 3.1 * 2^-16 per product term on top of its FP32 accumulation: larger
    r1 = oracle.crown_margin(p, lo, hi, prec=1)
    assert np.all(r1["margin"] > 10 * r["margin"])
    # the split-TF32 margin charges 3.1 * 2^-22 and accumulation at unit 2^-23: between the two
    r2 = oracle.crown_margin(p, lo, hi, prec=2)
    assert np.all(r2["margin"] > r["margin"]) and np.all(r2["margin"] < r1["margin"])


@pytest.mark.parametrize("prec,split", [(1, "bf16"), (2, "tf32")])
@pytest.mark.parametrize("s,k,hidden,H,rho,wscale,maxw", [(4, 2, [32, 32], 5, 0.0, 0.3, 1.0),
                                                          (8, 2, [128, 128], 3, 0.01, 0.3, 1.0)])
def test_margin_covers_split_evaluations(oracle, prec, split, s, k, hidden, H, rho, wscale, maxw):
    """The margin of a 3-term split evaluation covers the chain with every product evaluated as
    A_hi W_hi + A_hi W_lo + A_lo W_hi from BF16 or TF32 halves (accumulated in FP32, in two orders), and the
    chain does differ from the exact bound by more than the FP32 chain's rounding alone."""
    p = W.make_problem(s, k, hidden, H, rho, seed=33, weight_scale=wscale)
    lo, hi, _ = W.random_boxes(k * H, 5, seed=34, min_width=0.1, max_width=maxw)
    _, pl, pu, xl, xu = oracle.ibp(p, lo, hi)
    o = oracle.crown(p, lo, hi)
    r = oracle.crown_margin(p, lo, hi, prec=prec)
    np.testing.assert_allclose(r["lb"], o["lb"], rtol=1e-14, atol=1e-12)
    worst = 0.0
    for order in ("fwd", "rev"):
        v = _fp32_chain(p, lo, hi, pl, pu, xl, xu, o["A_pre"], order, split=split)
        assert np.all(v - r["margin"] <= r["lb"] + 1e-12 * np.abs(r["lb"])), order
        worst = max(worst, float(np.max(np.abs(v - r["lb"]) / r["margin"])))
    assert worst > 0


def test_split_halves_representation_error():
    """The halves the split margins assume: |x - hi| <= 2^-(p) |x| and |x - hi - lo| <= 2^-(2p) |x| with p = 8
    (BF16) and 11 (TF32) significant bits, hi and lo exactly representable in the half format (low bits zero)."""
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(20000) * np.exp2(rng.integers(-30, 30, 20000))).astype(np.float32)
    for kind, pbits, low in (("bf16", 8, 0xFFFF), ("tf32", 11, 0x1FFF)):
        h, l = _split(x, kind)
        xd, hd, ld = x.astype(np.float64), h.astype(np.float64), l.astype(np.float64)
        assert np.all(np.abs(xd - hd) <= 2.0 ** -pbits * np.abs(xd))
        assert np.all(np.abs(xd - hd - ld) <= 2.0 ** (-2 * pbits) * np.abs(xd))
        assert np.all((h.view(np.uint32) & low) == 0) and np.all((l.view(np.uint32) & low) == 0)


def test_margin_single_step_linear_closed_form(oracle):
    """One step of a network without hidden layers (x_1 = x_0 + W [x_0; u_0] + b), rho = 0: the tangent
    coefficient lam = 2 m of ||x_1 - g||^2 is carried through W once, so the margin is the FP32 product bound
    gamma_4 |lam|^T |W| amax (amax = [|x_0|; max(|lo|, |hi|)], Higham's gamma_n = n u / (1 - n u), u = 2^-24, over
    the 4 terms of a 3-wide product rounded up to a multiple of 4) plus the state update lam + lam W_x charged
    at 2^-23 against |x_0|."""
    rng = np.random.default_rng(5)
    s, k = 3, 2
    Wm = rng.uniform(-0.5, 0.5, size=(s, s + k))
    b = rng.normal(0, 0.1, size=s)
    p = dict(dims=[s + k, s], params=W.pack_params([(Wm, b)]), x0=np.array([0.3, -1.2, 0.7]),
             goal=np.array([1.0, 0.5, -0.25]), H=1, rho=0.0, s=s, k=k)
    lo = np.array([[-0.4, 0.1]])
    hi = np.array([[0.2, 0.9]])
    x0 = p["x0"]
    c = x0 + Wm[:, :s] @ x0 + Wm[:, s:] @ (0.5 * (lo[0] + hi[0])) + b
    r_ = np.abs(Wm[:, s:]) @ (0.5 * (hi[0] - lo[0]))
    m = c - p["goal"]  # midpoint of [c - r, c + r] - g
    lam = 2 * m
    amax = np.concatenate([np.abs(x0), np.maximum(np.abs(lo[0]), np.abs(hi[0]))])
    u = 2.0 ** -24
    g4 = 4 * u / (1 - 4 * u)
    expect = g4 * np.abs(lam) @ np.abs(Wm) @ amax + 2.0 ** -23 * (np.abs(lam) + np.abs(lam @ Wm[:, :s])) @ np.abs(x0)
    got = oracle.crown_margin(p, lo, hi)["margin"][0]
    assert got == pytest.approx(expect, rel=1e-12)
    assert r_.shape == (s,)
    # 3-term TF32 split: 3.1 * 2^-22 plus gamma_8 with unit 2^-23 (3 terms rounded up to a multiple of 8)
    g8 = 3.1 * 2.0 ** -22 + 8 * 2.0 ** -23 / (1 - 8 * 2.0 ** -23)
    expect2 = g8 * np.abs(lam) @ np.abs(Wm) @ amax + 2.0 ** -23 * (np.abs(lam) + np.abs(lam @ Wm[:, :s])) @ np.abs(x0)
    assert oracle.crown_margin(p, lo, hi, prec=2)["margin"][0] == pytest.approx(expect2, rel=1e-12)


def test_margin_scales_with_square_of_homogeneous_scaling(oracle):
    """The ReLU network is positively homogeneous once its biases scale too: scaling x_0, the goal, the boxes
    and every bias by c > 0 scales every state, pre-activation and coefficient by c and the objective by c^2,
    so every margin term (a coefficient times a variable's magnitude) scales by c^2."""
    p = W.make_problem(4, 2, [32, 32], 5, 0.01, seed=40, weight_scale=0.5)
    lo, hi, _ = W.random_boxes(10, 4, seed=41, min_width=0.2, max_width=1.0)
    r = oracle.crown_margin(p, lo, hi)
    cfac = 4.0  # a power of two: the scaled inputs are exact
    q = dict(p)
    q["x0"] = np.asarray(p["x0"], np.float64) * cfac
    q["goal"] = np.asarray(p["goal"], np.float64) * cfac
    q["params"] = W.pack_params([(Wl, bl * cfac) for Wl, bl in W.unpack_params(p)])
    rq = oracle.crown_margin(q, lo * cfac, hi * cfac)
    np.testing.assert_allclose(rq["lb"], r["lb"] * cfac ** 2, rtol=1e-12)
    np.testing.assert_allclose(rq["margin"], r["margin"] * cfac ** 2, rtol=1e-12)


def test_margin_one_hidden_layer_closed_form(oracle):
    """One step through a 2-2-1 network (s = k = 1) whose first hidden neuron is active and whose second is
    unstable with a negative coefficient (the chord of Lemma 1), with rho > 0 and the minimiser of mu u + rho u^2
    outside the box: every term of the margin is present and each is written out here from the intervals by
    hand: gamma_4 |lam| S^(2) for the output layer, gamma_4 sum_q |A'_q| S^(1)_q for the hidden layer,
    2^-23 |A'_1| max(-l_1, u_1) for the chord's slope product, 2^-23 (|lam| + |A_x|) |x_0| for the state update
    and rho (2^-23 u_c)^2 for the face of the box."""
    rng = np.random.default_rng(11)
    gam4 = 4 * 2.0 ** -24 / (1 - 4 * 2.0 ** -24)
    tu = 2.0 ** -23
    for _ in range(2000):
        W1 = rng.uniform(-1, 1, size=(2, 2))
        b1 = rng.uniform(-0.5, 0.5, size=2)
        W2 = rng.uniform(-1, 1, size=(1, 2))
        b2 = rng.uniform(-0.2, 0.2, size=1)
        x0, g = rng.uniform(-1, 1), rng.uniform(-1, 1)
        lo, hi = sorted(rng.uniform(-1, 1, size=2))
        rho = 1e-3
        # interval bounds by hand (centre / radius)
        c0, r0 = np.array([x0, 0.5 * (lo + hi)]), np.array([0.0, 0.5 * (hi - lo)])
        zc, zr = W1 @ c0 + b1, np.abs(W1) @ r0
        l1, u1 = zc - zr, zc + zr
        a_lo, a_hi = np.maximum(l1, 0), np.maximum(u1, 0)
        c1, r1 = 0.5 * (a_lo + a_hi), 0.5 * (a_hi - a_lo)
        x1l = x0 + (W2 @ c1 + b2 - np.abs(W2) @ r1)[0]
        x1u = x0 + (W2 @ c1 + b2 + np.abs(W2) @ r1)[0]
        lam = 2 * (0.5 * (x1l + x1u) - g)
        A = lam * W2[0]
        if not (l1[0] > 0 and l1[1] < 0 < u1[1] and A[1] < 0):
            continue
        D1 = u1[1] / (u1[1] - l1[1])
        Ap = np.array([A[0], A[1] * D1])
        Ax, Au = Ap @ W1[:, 0], Ap @ W1[:, 1]
        uc = -Au / (2 * rho)
        if lo <= uc <= hi:
            continue
        S2 = np.abs(W2[0]) @ a_hi
        S1 = np.abs(W1) @ np.array([abs(x0), max(abs(lo), abs(hi))])
        expect = (gam4 * abs(lam) * S2 + gam4 * np.abs(Ap) @ S1 + tu * abs(Ap[1]) * max(-l1[1], u1[1])
                  + tu * (abs(lam) + abs(Ax)) * abs(x0) + rho * (tu * uc) ** 2)
        p = dict(dims=[2, 2, 1], params=W.pack_params([(W1, b1), (W2, b2)]), x0=np.array([x0]), goal=np.array([g]),
                 H=1, rho=rho, s=1, k=1)
        got = oracle.crown_margin(p, np.array([[lo]]), np.array([[hi]]))["margin"][0]
        assert got == pytest.approx(expect, rel=1e-12)
        return
    pytest.fail("no network with the wanted neuron pattern was drawn")


def _ru32(x):
    """float64 values rounded up to float32."""
    y = np.asarray(x, np.float64).astype(np.float32)
    return np.where(y.astype(np.float64) < x, np.nextafter(y, np.float32(np.inf)), y)


def _rd32(x):
    """float64 values rounded down to float32."""
    y = np.asarray(x, np.float64).astype(np.float32)
    return np.where(y.astype(np.float64) > x, np.nextafter(y, np.float32(-np.inf)), y)


def _sum32(terms, order, rng):
    """Sum of terms [T][...] in float32, one rounding to nearest per addition, in 'fwd', 'rev' or 'perm' order."""
    idx = np.arange(terms.shape[0])
    if order == "rev":
        idx = idx[::-1]
    elif order == "perm":
        idx = rng.permutation(idx)
    acc = np.zeros(terms.shape[1:], np.float32)
    for i in idx:
        acc = (acc + terms[i]).astype(np.float32)
    return acc


@pytest.mark.parametrize("kind,K", [("bf16", 16), ("bf16", 36), ("bf16", 256), ("tf32", 8), ("tf32", 36),
                                    ("tf32", 256)])
def test_interval_split_margin_contains_exact_layer_interval(kind, K):
    """One layer of the tensor-core interval bounds (the intermediate bounds of Lemma 1, Appendix B.1), written
    out on the CPU in the kernel's steps: each input interval [l, u] in centre-radius form (c rounded to nearest,
    r and |c| + r rounded up), c and r as hi and lo halves (BF16 or TF32), W and |W| the same; zc = W c and
    zr = |W| r as 3-term split products and zs = |W|_hi (|c| + r)_hi, each accumulated in float32 in three orders;
    S' = zs (1 + 2^-6) for BF16 halves, (1 + 2^-9) for TF32, and the interval [zc + b - zr - eps S',
    zc + b + zr + eps S'] with every addition rounded outward, eps = 3.1 2^-16 (BF16) or 3.1 2^-22 (TF32) plus
    K' 2^-23 / (1 - K' 2^-23), K' = K rounded up to 16 (BF16) or 8 (TF32).  It must contain the exact interval
    sum_k min(W_jk l_k, W_jk u_k) + b_j .. sum_k max(..) + b_j (each sum by math.fsum over the exact float64
    products of float32 values), for boxes of every width down to points and weights over five binades; without
    the eps S' term it does not, and the TF32 widening is at most half the BF16 one.  Planted in a copy: the BF16
    halves charged the TF32 representation term, |W| replaced by W in zr, or the W_lo c_hi term dropped each
    fail."""
    import math
    rng = np.random.default_rng(100 + K + (0 if kind == "bf16" else 1000))
    nout, nbox = 48, 40
    Wm = (rng.standard_normal((nout, K)) * np.exp2(rng.integers(-3, 2, (nout, K)))).astype(np.float32)
    b = rng.standard_normal(nout).astype(np.float32)
    c0 = rng.uniform(-4.0, 4.0, (nbox, K))
    w = rng.uniform(0.0, 2.0, (nbox, K)) * (rng.random((nbox, K)) < 0.8)
    l, u = (c0 - w).astype(np.float32), (c0 + w).astype(np.float32)
    assert np.all(l <= u)
    # exact interval of W a + b over the box
    lo_x = np.empty((nbox, nout))
    hi_x = np.empty((nbox, nout))
    Wd, ld, ud = Wm.astype(np.float64), l.astype(np.float64), u.astype(np.float64)
    for n in range(nbox):
        p1, p2 = Wd * ld[n][None, :], Wd * ud[n][None, :]
        mn, mx = np.minimum(p1, p2), np.maximum(p1, p2)
        for j in range(nout):
            lo_x[n, j] = math.fsum(list(mn[j]) + [float(b[j])])
            hi_x[n, j] = math.fsum(list(mx[j]) + [float(b[j])])

    def layer(kind_, widen=True, order="fwd"):
        f32 = np.float32
        c = (f32(0.5) * (l + u).astype(f32)).astype(f32)
        r = np.maximum(_ru32(ud - c.astype(np.float64)), _ru32(c.astype(np.float64) - ld))
        m = _ru32(np.abs(c).astype(np.float64) + r.astype(np.float64))
        ch, cl = _split(c, kind_)
        rh, rl = _split(r, kind_)
        mh = _round_half(m, kind_)
        Wh, Wl = _split(Wm, kind_)
        Ah, Al = _split(np.abs(Wm), kind_)
        # products [K][box][out]: exact in float32 (8 + 8 or 11 + 11 significant bits)
        pr = lambda A, x: (x.T[:, :, None] * A.T[:, None, :]).astype(f32)
        zc = _sum32(np.concatenate([pr(Wh, ch), pr(Wl, ch), pr(Wh, cl)]), order, rng)
        zr = _sum32(np.concatenate([pr(Ah, rh), pr(Al, rh), pr(Ah, rl)]), order, rng)
        zs = _sum32(pr(Ah, mh), order, rng)
        if kind_ == "bf16":
            Kp, rep, s_up = (K + 15) // 16 * 16, 3.1 * 2.0 ** -16, 1 + 2.0 ** -6
        else:
            Kp, rep, s_up = (K + 7) // 8 * 8, 3.1 * 2.0 ** -22, 1 + 2.0 ** -9
        eps = np.float32(rep + Kp * 2.0 ** -23 / (1 - Kp * 2.0 ** -23))
        Sp = _ru32(zs.astype(np.float64) * s_up)
        es = _ru32(np.float64(eps) * Sp.astype(np.float64)) if widen else np.zeros_like(Sp)
        rad = _ru32(zr.astype(np.float64) + es.astype(np.float64))
        zb_d = _rd32(zc.astype(np.float64) + b.astype(np.float64)[None, :])
        zb_u = _ru32(zc.astype(np.float64) + b.astype(np.float64)[None, :])
        return (_rd32(zb_d.astype(np.float64) - rad.astype(np.float64)).astype(np.float64),
                _ru32(zb_u.astype(np.float64) + rad.astype(np.float64)).astype(np.float64))

    for order in ("fwd", "rev", "perm"):
        lo_g, hi_g = layer(kind, order=order)
        assert np.all(lo_g <= lo_x) and np.all(hi_g >= hi_x), order
    lo_n, hi_n = layer(kind, widen=False)
    assert np.any(lo_n > lo_x) or np.any(hi_n < hi_x)  # the margin is needed
    if K >= 32:
        wide = {}
        for k_ in ("bf16", "tf32"):
            lo_g, hi_g = layer(k_)
            wide[k_] = float(np.sum((hi_g - lo_g) - (hi_x - lo_x)))
        assert 0.0 < wide["tf32"] <= 0.5 * wide["bf16"]


def test_fast_upper_slope_is_at_least_the_chord():
    """Reading of Lemma 1's upper line in the feature-major CROWN: any slope at least the chord u / (u - l) gives
    an upper line through (l, 0).  The kernel's slope: den = u - l rounded down, a quotient u / den from a fast
    division modelled at the low end of its documented 2-ulp range for normal results and as 0 below 2^-126
    (flushed), times 1 + 2^-20 rounded up, raised to at least 2^-99, capped at 1; slope 1 outside
    den < 1e36, u > 1e-30.  Checked exactly (rationals) over neurons whose chord spans 2^-140 .. 1; without the
    2^-99 floor a flushed quotient gives slope 0, below the chord."""
    from fractions import Fraction
    rng = np.random.default_rng(12)
    f32 = np.float32

    def slope(zl, zu, floor=True):
        den = _rd32(np.float64(zu) - np.float64(zl))
        if not (den < f32(1e36) and zu > f32(1e-30)):
            return f32(1.0)
        q = Fraction(float(zu)) / Fraction(float(den))
        if q < Fraction(2) ** -126:
            qf = f32(0.0)
        else:
            qf = _rd32(float(q))
            for _ in range(2):  # two units in the last place below
                qf = np.nextafter(qf, f32(-np.inf))
        s = _ru32(np.float64(qf) * (1 + 2.0 ** -20))
        if floor:
            s = max(s, f32(2.0 ** -99))
        return min(s, f32(1.0))

    cases = []
    for _ in range(3000):
        zu = f32(np.exp2(rng.uniform(-99.5, 20)))
        zl = -f32(np.exp2(rng.uniform(-99.5, 120)))
        cases.append((zl, zu))
    cases += [(f32(-1e20), f32(1e-20)), (f32(-1e35), f32(2e-30)), (f32(-3.0), f32(1e-29)), (f32(-1.0), f32(1.0))]
    flushed = 0
    for zl, zu in cases:
        chord = Fraction(float(zu)) / (Fraction(float(zu)) - Fraction(float(zl)))
        s = slope(zl, zu)
        assert Fraction(float(s)) >= chord, (zl, zu)
        den = _rd32(np.float64(zu) - np.float64(zl))
        if den < f32(1e36) and zu > f32(1e-30) and Fraction(float(zu)) / Fraction(float(den)) < Fraction(2) ** -126:
            flushed += 1
            assert Fraction(float(slope(zl, zu, floor=False))) < chord  # the floor is what keeps it valid
    assert flushed > 0
