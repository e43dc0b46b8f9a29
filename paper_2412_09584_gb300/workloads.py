"""Seeded synthetic workloads shaped like the paper's planning problems.

This module only draws inputs: network weights, start state, goal and boxes.
It holds none of the method's arithmetic, so both the CUDA path and the oracle
can take their inputs from it.  All draws use numpy's PCG64 with a fixed seed.

Workloads (see ``CONFIGS``):

* ``tiny``      state 4, action 2, MLP 6-32-32-4, H=5, 64 boxes from a 2x grid
                over the first 6 action coordinates, 256 samples per box.
* ``pushing``   state 8 (4 planar keypoints), action 2, MLP 10-128-128-128-8,
                H=20, rho=0.01, 4096 boxes per iteration, 1024 samples per box.
                Stands in for the paper's pushing-with-obstacles task
                (Section 4, Appendix D), whose trained models are not public.
* ``alpha``     ``tiny`` with 4096 boxes and 20 alpha steps per iteration.
* ``manip``     state 32 (16 planar points), action 4, MLP 36-256x4-32, H=40,
                rho=0.01, 16384 boxes, 4 samples per box (65536 rollouts).
* ``batched``   64 independent ``tiny``-architecture problems, horizons 10..80.

Weights follow Kaiming-uniform with gain scaled by 0.1: W ~ U(-b, b) with
b = 0.1 * sqrt(6 / fan_in); biases ~ N(0, 0.01^2).  x_0 and the goal are
N(0, 1) per coordinate.  The action box is [-1, 1]^(kH).
"""
from __future__ import annotations

import numpy as np

CONFIGS = {
    "tiny": dict(s=4, k=2, hidden=[32, 32], H=5, rho=0.0, boxes=64, samples=256, grid_dims=6),
    "pushing": dict(s=8, k=2, hidden=[128, 128, 128], H=20, rho=0.01, boxes=4096, samples=1024, grid_dims=12),
    "alpha": dict(s=4, k=2, hidden=[32, 32], H=5, rho=0.0, boxes=4096, samples=256, grid_dims=10,
                  alpha_steps=20, alpha_lr=0.1),
    "manip": dict(s=32, k=4, hidden=[256, 256, 256, 256], H=40, rho=0.01, boxes=16384, samples=4, grid_dims=14),
    # many concurrent plans of the tiny architecture: horizons uniform in [H_lo, H_hi], each problem with its own
    # seed-drawn weights, start and goal
    "batched": dict(s=4, k=2, hidden=[32, 32], rho=0.0, problems=64, H_lo=10, H_hi=80, samples=256, alpha_steps=20,
                    alpha_lr=0.1, rows_lo=256, rows_hi=8192),
}


def layer_dims(s, k, hidden):
    return [s + k] + list(hidden) + [s]


def make_problem(s, k, hidden, H, rho, seed, weight_scale=0.1, bias_std=0.01):
    """Random network and start/goal states for one planning problem.

    Returns a dict with dims (L+1 ints), params (float32, packed per layer as
    W_l row-major [dims[l], dims[l-1]] followed by b_l), x0, goal (float32),
    H, rho, s, k."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = layer_dims(s, k, hidden)
    parts = []
    for l in range(1, len(dims)):
        fan_in = dims[l - 1]
        bound = weight_scale * np.sqrt(6.0 / fan_in)
        W = rng.uniform(-bound, bound, size=(dims[l], fan_in))
        b = rng.normal(0.0, bias_std, size=dims[l])
        parts += [W.ravel(), b]
    params = np.concatenate(parts).astype(np.float32)
    x0 = rng.normal(0.0, 1.0, size=s).astype(np.float32)
    goal = rng.normal(0.0, 1.0, size=s).astype(np.float32)
    return dict(dims=dims, params=params, x0=x0, goal=goal, H=int(H), rho=float(rho), s=int(s), k=int(k))


def config_problem(name, seed=0):
    c = CONFIGS[name]
    return make_problem(c["s"], c["k"], c["hidden"], c["H"], c["rho"], seed)


def unpack_params(problem):
    """List of (W, b) float32 arrays from the packed vector."""
    dims = problem["dims"]
    p = problem["params"]
    out, off = [], 0
    for l in range(1, len(dims)):
        n = dims[l] * dims[l - 1]
        W = p[off:off + n].reshape(dims[l], dims[l - 1])
        off += n
        b = p[off:off + dims[l]]
        off += dims[l]
        out.append((W, b))
    return out


def pack_params(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers]).astype(np.float32)


def grid_boxes(d, levels, lo=-1.0, hi=1.0):
    """The 2^levels boxes of the grid that halves each of the first `levels`
    coordinates of [lo, hi]^d, with heap identifiers 2^levels + b, where bit
    (levels-1-j) of b is 1 for the upper half of coordinate j.

    Returns (lo [n,d] f32, hi [n,d] f32, id [n] u64)."""
    assert levels <= d
    n = 1 << levels
    mid = np.float32(0.5) * (np.float32(lo) + np.float32(hi))
    blo = np.full((n, d), lo, dtype=np.float32)
    bhi = np.full((n, d), hi, dtype=np.float32)
    ids = np.zeros(n, dtype=np.uint64)
    for b in range(n):
        code = 0
        for j in range(levels):
            upper = (b >> j) & 1
            if upper:
                blo[b, j] = mid
            else:
                bhi[b, j] = mid
            code |= upper << (levels - 1 - j)
        ids[b] = n + code
    return blo, bhi, ids


def random_boxes(d, n, seed, min_width=0.0, max_width=2.0, lo=-1.0, hi=1.0):
    """n random axis-aligned sub-boxes of [lo, hi]^d with per-coordinate widths
    uniform in [min_width, max_width] (clipped to the domain)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.uniform(min_width, max_width, size=(n, d))
    w = np.minimum(w, hi - lo)
    a = lo + rng.uniform(0.0, 1.0, size=(n, d)) * (hi - lo - w)
    blo = a.astype(np.float32)
    bhi = np.minimum((a + w).astype(np.float32), np.float32(hi))
    bhi = np.maximum(bhi, blo)
    ids = (np.arange(n, dtype=np.uint64) + np.uint64(1) + np.uint64(seed % 1000) * np.uint64(1 << 20))
    return blo, bhi, ids


def dyadic_boxes(d, n, seed, max_depth=4):
    """n random dyadic sub-boxes of [-1, 1]^d (each coordinate an interval of
    width 2^(1-q), q <= max_depth, on the dyadic grid), as bisection makes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.integers(0, max_depth + 1, size=(n, d))
    w = 2.0 ** (1 - q)
    pos = np.floor(rng.uniform(0.0, 1.0, size=(n, d)) * (2.0 ** q))
    blo = (-1.0 + pos * w).astype(np.float32)
    bhi = (-1.0 + (pos + 1) * w).astype(np.float32)
    ids = np.arange(1, n + 1, dtype=np.uint64) + np.uint64(seed % 997) * np.uint64(1 << 24)
    return blo, bhi, ids


def pool_values(n, seed, nan_frac=0.0, tie_frac=0.0):
    """Random (lb, ub) pairs for prune/branch tests: lb <= ub, optional NaN
    lower bounds and repeated values (ties)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lb = rng.normal(10.0, 3.0, size=n).astype(np.float32)
    ub = (lb + np.abs(rng.normal(2.0, 1.0, size=n))).astype(np.float32)
    if tie_frac > 0 and n > 1:
        t = rng.uniform(size=n) < tie_frac
        lb[t] = lb[0]
        ub[t] = ub[0]
    if nan_frac > 0:
        lb[rng.uniform(size=n) < nan_frac] = np.nan
    return lb, ub


def batch_problems(P, seed, s=4, k=2, hidden=(32, 32), H_lo=10, H_hi=80, rho=0.0):
    """P independent problems of one architecture, problem p drawn by make_problem with seed (seed, p) and a
    horizon uniform in [H_lo, H_hi].  Returns (list of problem dicts, horizons int32 [P])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Hs = rng.integers(H_lo, H_hi + 1, size=P).astype(np.int32)
    probs = [make_problem(s, k, list(hidden), int(Hs[p]), rho, seed=int(seed) * 100003 + p) for p in range(P)]
    return probs, Hs


def pack_batch(problems):
    """Stacked per-problem arrays: params [P][n_params], x0 [P][s], goal [P][s], H int32 [P], rho f32 [P]."""
    return (np.stack([p["params"] for p in problems]), np.stack([p["x0"] for p in problems]),
            np.stack([p["goal"] for p in problems]), np.array([p["H"] for p in problems], dtype=np.int32),
            np.array([p["rho"] for p in problems], dtype=np.float32))


def batch_grid_boxes(problems, levels, d_stride):
    """Each problem's [-1, 1]^(k H_p) cut into the 2^levels grid of grid_boxes, rows grouped by problem, the
    coordinates beyond k H_p set to 0.  Returns (lo, hi [n][d_stride] f32, id u64 [n], prob int32 [n])."""
    los, his, ids, prob = [], [], [], []
    for i, p in enumerate(problems):
        dp = p["k"] * p["H"]
        lo, hi, idp = grid_boxes(dp, min(levels, dp))
        pad = np.zeros((lo.shape[0], d_stride - dp), dtype=np.float32)
        los.append(np.concatenate([lo, pad], axis=1))
        his.append(np.concatenate([hi, pad], axis=1))
        ids.append(idp)
        prob.append(np.full(lo.shape[0], i, dtype=np.int32))
    return np.concatenate(los), np.concatenate(his), np.concatenate(ids), np.concatenate(prob)


def batch_random_boxes(problems, rows, d_stride, seed, min_width=0.1, max_width=1.0):
    """rows[p] random sub-boxes of problem p's [-1, 1]^(k H_p) (random_boxes), then all rows shuffled across
    problems.  Returns (lo, hi [n][d_stride] f32, id u64 [n] distinct, prob int32 [n])."""
    los, his, prob = [], [], []
    for i, p in enumerate(problems):
        dp = p["k"] * p["H"]
        lo, hi, _ = random_boxes(dp, int(rows[i]), seed=seed * 7919 + i, min_width=min_width, max_width=max_width)
        pad = np.zeros((lo.shape[0], d_stride - dp), dtype=np.float32)
        los.append(np.concatenate([lo, pad], axis=1))
        his.append(np.concatenate([hi, pad], axis=1))
        prob.append(np.full(lo.shape[0], i, dtype=np.int32))
    lo, hi, prob = np.concatenate(los), np.concatenate(his), np.concatenate(prob)
    order = np.random.Generator(np.random.PCG64(seed)).permutation(lo.shape[0])
    ids = (np.arange(lo.shape[0], dtype=np.uint64) + np.uint64(1000))
    return lo[order], hi[order], ids, prob[order]


def obstacle_cost(H, seed, n_obs=3, lam=10.0):
    """The pushing-with-obstacles cost of Appendix D.4 for a pushing-scale problem (state: 4 planar keypoints,
    action: the planar pusher motion): weights w_t = t / H increasing with time, penalty lam, n_obs obstacles
    with centres N(0, 1) and radii U(0.3, 0.8), pusher start (0, 0).  Returns dict(w, lam, obstacles, p0)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    obs = [(float(rng.normal()), float(rng.normal()), float(rng.uniform(0.3, 0.8))) for _ in range(n_obs)]
    w = [(t + 1) / H for t in range(H)]
    return dict(w=np.array(w, dtype=np.float64), lam=float(lam), obstacles=obs, p0=(0.0, 0.0))
