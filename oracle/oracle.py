"""Python face of the FP64 CPU oracle (``bab_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the checker for the CUDA library:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and reference
(``--impl reference``) legs of ``bench.py`` may import it.  It shares no code with the CUDA path.

Each function converts its numpy inputs to the C layout (float64 for real
inputs; the FP32 boxes stay FP32 where the method fixes FP32 arithmetic, i.e.
the sample draw and the bisection midpoint) and calls the C routine.  The
citations are to arXiv 2412.09584 (BaB-ND):

* ``objective``     Section 3, Eq. (trajop)
* ``rollout``       Section 3.3 (batch_search, uniform samples)
* ``ibp``           interval intermediate bounds used by Lemma 1
* ``crown``         Appendix B.1, Lemma 1, Theorem 1, Theorem 2 (box form)
* ``crown_margin``  the same bound with the outward rounding margin of an FP32 / split-BF16 / split-TF32 evaluation
* ``alpha_grad``    gradient of the Theorem 1/2 bound in the Lemma 1 slopes
* ``alpha_optimize`` the Adam loop on those slopes (``adam_ascent``: one projected Adam step)
* ``box_grad``      gradient of the bound in the box faces, the relaxation choices held fixed
* ``search_bounds`` Section 3.2: per box the extremes over its samples of every pre-activation and state
* ``crown_given``   Appendix B.2, Algorithm 3: CROWN on given intermediate bounds with propagation early stop
* ``prune_branch``  Section 3 overview (Pruner), Section 3.1 (pick out, split)
* ``prune_branch_heuristic``, ``split_dims``  Section 3.1: pick-out by upper bound plus softmax sampling over
  scaled lower bounds; split dimension by the sample imbalance of the top samples
* ``bab``           Algorithm 2 (search, bound, incumbent, prune, pick, split)
* ``objective_f32`` Eq. (trajop) in FP32 (the precision the search ranks in)
* ``cem``           Section 3.3 (batch_search with the cross-entropy method)
* ``set_cost``      Appendix D.4, Eq. (pushing_cost): weighted norm and obstacle penalties
* ``synth_*``       Section 4, synthetic example f(u) = sum 5 u_i^2 + cos(50 u_i)

Every function is pinned in ``tests/test_oracle_pins.py`` against closed forms, brute force, invariants or
hand-worked values (``tests/golden/``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bab_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_float_p = ctypes.POINTER(ctypes.c_float)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_u64_p = ctypes.POINTER(ctypes.c_uint64)
_c_u8_p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE double, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.oracle_objective.restype = ctypes.c_double
        L.oracle_splitmix64.restype = ctypes.c_uint64
        L.oracle_splitmix64.argtypes = [ctypes.c_uint64]
        L.oracle_sample.restype = ctypes.c_float
        L.oracle_sample.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_float, ctypes.c_float]
        L.oracle_sq_tangent.restype = ctypes.c_double
        L.oracle_sq_tangent.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_sq_chord.restype = ctypes.c_double
        L.oracle_sq_chord.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_relu_relax.restype = None
        L.oracle_relu_relax.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        _c_double_p, _c_double_p]
        L.oracle_adam_ascent.restype = None
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_c_double_p)


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_c_float_p)


def _optd(a):
    if a is None:
        return None, None
    return _d(a)


class Net:
    """Network shape and packed parameters (W_1, b_1, ..., W_L, b_L)."""

    def __init__(self, dims, params, s, k):
        self.dims = np.ascontiguousarray(dims, dtype=np.int32)
        self.L = len(dims) - 1
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        self.s, self.k = int(s), int(k)
        self.sumh = int(sum(dims[1:-1]))

    def cargs(self):
        return (ctypes.c_int(self.L), self.dims.ctypes.data_as(_c_int_p), self.params.ctypes.data_as(_c_double_p),
                ctypes.c_int(self.s), ctypes.c_int(self.k))


def net_of(problem) -> Net:
    return Net(problem["dims"], problem["params"], problem["s"], problem["k"])


def _prob(problem):
    net = net_of(problem)
    x0, px0 = _d(problem["x0"])
    g, pg = _d(problem["goal"])
    return net, (x0, g), (ctypes.c_int(int(problem["H"])), ctypes.c_double(float(problem["rho"])), px0, pg)


def objective(problem, u, with_traj=False):
    """f(u) in FP64 (Section 3, Eq. trajop); optionally the trajectory and hidden pre-activations."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    u, pu = _d(u)
    H = int(problem["H"])
    traj = np.zeros((H + 1, net.s)) if with_traj else None
    pre = np.zeros((H, max(net.sumh, 1))) if with_traj else None
    f = lib().oracle_objective(*net.cargs(), cH, crho, px0, pg, pu,
                               traj.ctypes.data_as(_c_double_p) if with_traj else None,
                               pre.ctypes.data_as(_c_double_p) if with_traj else None)
    if with_traj:
        return f, traj, pre[:, :net.sumh]
    return f


def sample(seed, box_id, m, j, lo, hi):
    return lib().oracle_sample(seed, box_id, m, j, lo, hi)


def rollout(problem, lo, hi, ids, samples, seed):
    """Best of `samples` uniform samples per box (Section 3.3): (ub FP64, best_u FP32, best_m)."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    lo, plo = _f(lo)
    hi, phi = _f(hi)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    n, d = lo.shape
    ub = np.zeros(n)
    best_u = np.zeros((n, d), dtype=np.float32)
    best_m = np.zeros(n, dtype=np.int32)
    rc = lib().oracle_rollout(*net.cargs(), cH, crho, px0, pg, ctypes.c_int(n), plo, phi,
                              ids.ctypes.data_as(_c_u64_p), ctypes.c_int(samples), ctypes.c_uint64(seed),
                              ub.ctypes.data_as(_c_double_p), best_u.ctypes.data_as(_c_float_p),
                              best_m.ctypes.data_as(_c_int_p))
    assert rc == 0
    return ub, best_u, best_m


def ibp(problem, lo, hi):
    """Interval bounds: (lb_ibp [n], pre_lo/pre_hi [n,H,sumh], x_lo/x_hi [n,H+1,s])."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    lo, plo = _d(lo)
    hi, phi = _d(hi)
    n = lo.shape[0]
    H = int(problem["H"])
    pl = np.zeros((n, H, max(net.sumh, 1)))
    pu = np.zeros_like(pl)
    xl = np.zeros((n, H + 1, net.s))
    xu = np.zeros_like(xl)
    lb = np.zeros(n)
    rc = lib().oracle_ibp(*net.cargs(), cH, crho, px0, pg, ctypes.c_int(n), plo, phi,
                          pl.ctypes.data_as(_c_double_p), pu.ctypes.data_as(_c_double_p),
                          xl.ctypes.data_as(_c_double_p), xu.ctypes.data_as(_c_double_p),
                          lb.ctypes.data_as(_c_double_p))
    assert rc == 0
    return lb, pl[:, :, :net.sumh], pu[:, :, :net.sumh], xl, xu


def crown(problem, lo, hi, alpha=None):
    """CROWN bound per box (Appendix B.1): dict with lb, lin_coef, lin_const, ustar, A_pre."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    lo, plo = _d(lo)
    hi, phi = _d(hi)
    n, d = lo.shape
    H = int(problem["H"])
    alpha_a, palpha = _optd(alpha)
    lb = np.zeros(n)
    mu = np.zeros((n, d))
    cst = np.zeros(n)
    us = np.zeros((n, d))
    Ap = np.zeros((n, H, max(net.sumh, 1)))
    scale = np.zeros(n)
    rc = lib().oracle_crown(*net.cargs(), cH, crho, px0, pg, ctypes.c_int(n), plo, phi, palpha,
                            lb.ctypes.data_as(_c_double_p), mu.ctypes.data_as(_c_double_p),
                            cst.ctypes.data_as(_c_double_p), us.ctypes.data_as(_c_double_p),
                            Ap.ctypes.data_as(_c_double_p), scale.ctypes.data_as(_c_double_p))
    assert rc == 0
    return {"lb": lb, "lin_coef": mu, "lin_const": cst, "ustar": us, "A_pre": Ap[:, :, :net.sumh],
            "scale": scale}


def alpha_grad(problem, lo, hi, alpha=None):
    """(lb, dlb/dalpha [n,H,sumh], relaxed-network objective at u*) per box; the relaxed objective is NaN for
    the obstacle cost."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    lo, plo = _d(lo)
    hi, phi = _d(hi)
    n, d = lo.shape
    H = int(problem["H"])
    alpha_a, palpha = _optd(alpha)
    lb = np.zeros(n)
    g = np.zeros((n, H, max(net.sumh, 1)))
    robj = np.zeros(n)
    rc = lib().oracle_alpha_grad(*net.cargs(), cH, crho, px0, pg, ctypes.c_int(n), plo, phi, palpha,
                                 lb.ctypes.data_as(_c_double_p), g.ctypes.data_as(_c_double_p),
                                 robj.ctypes.data_as(_c_double_p))
    assert rc == 0
    return lb, g[:, :, :net.sumh], robj


def box_grad(problem, lo, hi, alpha=None):
    """(lb, dlb/dlo [n,d], dlb/dhi [n,d]) per box, alpha held fixed (None: adaptive slopes)."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    lo, plo = _d(lo)
    hi, phi = _d(hi)
    n, d = lo.shape
    alpha_a, palpha = _optd(alpha)
    lb = np.zeros(n)
    glo = np.zeros((n, d))
    ghi = np.zeros((n, d))
    rc = lib().oracle_box_grad(*net.cargs(), cH, crho, px0, pg, ctypes.c_int(n), plo, phi, palpha,
                               lb.ctypes.data_as(_c_double_p), glo.ctypes.data_as(_c_double_p),
                               ghi.ctypes.data_as(_c_double_p))
    assert rc == 0
    return lb, glo, ghi


def search_bounds(problem, lo, hi, ids, samples, seed):
    """Search-integrated bounds (Section 3.2): per box the min / max over the rollout samples of every hidden
    pre-activation ([n,H,sumh]) and state ([n,H+1,s])."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    lo, plo = _f(lo)
    hi, phi = _f(hi)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    n, d = lo.shape
    H = int(problem["H"])
    pl = np.zeros((n, H, max(net.sumh, 1)))
    pu = np.zeros_like(pl)
    xl = np.zeros((n, H + 1, net.s))
    xu = np.zeros_like(xl)
    rc = lib().oracle_search_bounds(*net.cargs(), cH, crho, px0, pg, ctypes.c_int(n), plo, phi,
                                    ids.ctypes.data_as(_c_u64_p), ctypes.c_int(samples), ctypes.c_uint64(seed),
                                    pl.ctypes.data_as(_c_double_p), pu.ctypes.data_as(_c_double_p),
                                    xl.ctypes.data_as(_c_double_p), xu.ctypes.data_as(_c_double_p))
    assert rc == 0
    return pl[:, :, :net.sumh], pu[:, :, :net.sumh], xl, xu


def crown_given(problem, lo, hi, pre_lo, pre_hi, x_lo, x_hi, t_stop=0):
    """CROWN with given intermediate bounds and propagation early-stop at step t_stop (Algorithm 3)."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    lo, plo = _d(lo)
    hi, phi = _d(hi)
    n = lo.shape[0]
    H = int(problem["H"])
    sh = max(net.sumh, 1)
    pl = np.zeros((n, H, sh))
    pu = np.zeros((n, H, sh))
    pl[:, :, :net.sumh] = pre_lo
    pu[:, :, :net.sumh] = pre_hi
    xl = np.ascontiguousarray(x_lo, dtype=np.float64)
    xu = np.ascontiguousarray(x_hi, dtype=np.float64)
    lb = np.zeros(n)
    rc = lib().oracle_crown_given(*net.cargs(), cH, crho, px0, pg, ctypes.c_int(n), plo, phi,
                                  pl.ctypes.data_as(_c_double_p), pu.ctypes.data_as(_c_double_p),
                                  xl.ctypes.data_as(_c_double_p), xu.ctypes.data_as(_c_double_p),
                                  ctypes.c_int(int(t_stop)), lb.ctypes.data_as(_c_double_p))
    assert rc == 0
    return lb


def crown_margin(problem, lo, hi, intervals=None, alpha=None, prec=0):
    """CROWN bound with the outward rounding margin of an FP32 (prec 0), 3-term BF16 split (prec 1) or 3-term TF32
    split (prec 2) evaluation, in FP64: dict with lb (no margin subtracted), margin and scale.  `intervals` = (pre_lo, pre_hi,
    x_lo, x_hi) gives the intermediate bounds (else the oracle's interval bounds); alpha: lower slopes or None
    (adaptive)."""
    net, keep, (cH, crho, px0, pg) = _prob(problem)
    lo, plo = _d(lo)
    hi, phi = _d(hi)
    n = lo.shape[0]
    H = int(problem["H"])
    sh = max(net.sumh, 1)
    ptrs = [None, None, None, None]
    held = []
    if intervals is not None:
        pre_lo, pre_hi, x_lo, x_hi = intervals
        pl = np.zeros((n, H, sh))
        pu = np.zeros((n, H, sh))
        pl[:, :, :net.sumh] = pre_lo
        pu[:, :, :net.sumh] = pre_hi
        xl = np.ascontiguousarray(x_lo, dtype=np.float64)
        xu = np.ascontiguousarray(x_hi, dtype=np.float64)
        held = [pl, pu, xl, xu]
        ptrs = [a.ctypes.data_as(_c_double_p) for a in held]
    alpha_a, palpha = _optd(alpha)
    lb = np.zeros(n)
    mg = np.zeros(n)
    scale = np.zeros(n)
    rc = lib().oracle_crown_margin(*net.cargs(), cH, crho, px0, pg, ctypes.c_int(n), plo, phi, *ptrs, palpha,
                                   ctypes.c_int(int(prec)), lb.ctypes.data_as(_c_double_p),
                                   mg.ctypes.data_as(_c_double_p), scale.ctypes.data_as(_c_double_p))
    assert rc == 0
    return {"lb": lb, "margin": mg, "scale": scale}


def adaptive_alpha(problem, lo, hi):
    """The adaptive lower slopes (1 where u >= -l, else 0) of every neuron, from the oracle's IBP bounds."""
    _, pl, pu, _, _ = ibp(problem, lo, hi)
    return np.where(pu >= -pl, 1.0, 0.0)


def adam_ascent(param, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, clamp=(0.0, 1.0)):
    """One projected Adam ascent step, in place on float64 arrays."""
    for a in (param, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    lib().oracle_adam_ascent(ctypes.c_int(param.size), param.ctypes.data_as(_c_double_p),
                             m.ctypes.data_as(_c_double_p), v.ctypes.data_as(_c_double_p),
                             grad.ctypes.data_as(_c_double_p), ctypes.c_int(step), ctypes.c_double(lr),
                             ctypes.c_double(beta1), ctypes.c_double(beta2), ctypes.c_double(eps),
                             ctypes.c_double(clamp[0]), ctypes.c_double(clamp[1]))


def alpha_optimize(problem, lo, hi, steps, lr, alpha0=None):
    """`steps` rounds of (bound and gradient at alpha, keep the best bound, Adam ascent step)."""
    alpha = adaptive_alpha(problem, lo, hi) if alpha0 is None else np.array(alpha0, dtype=np.float64)
    alpha = np.ascontiguousarray(alpha)
    m = np.zeros_like(alpha)
    v = np.zeros_like(alpha)
    best = np.full(alpha.shape[0], -np.inf)
    for step in range(1, steps + 1):
        lb, g, _ = alpha_grad(problem, lo, hi, alpha)
        best = np.maximum(best, lb)
        adam_ascent(alpha, m, v, g, step, lr)
    return best, alpha, m, v


def relu_relax(l, u, alpha, which):
    D = ctypes.c_double()
    c = ctypes.c_double()
    lib().oracle_relu_relax(l, u, alpha, which, ctypes.byref(D), ctypes.byref(c))
    return D.value, c.value


def sq_tangent(m, s):
    return lib().oracle_sq_tangent(m, s)


def sq_chord(L, U, s):
    return lib().oracle_sq_chord(L, U, s)


def prune_branch(lo, hi, lb, ub, ids, inc_val, n_pick, eta=0.75):
    """Prune, pick out, bisect (see bab_oracle.c). Returns dict of outputs."""
    lo, plo = _f(lo)
    hi, phi = _f(hi)
    lb, plb = _f(lb)
    ub, pub = _f(ub)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    n, d = lo.shape
    cap = 2 * n + 1
    out_lo = np.zeros((cap, d), dtype=np.float32)
    out_hi = np.zeros_like(out_lo)
    out_lb = np.zeros(cap, dtype=np.float32)
    out_ub = np.zeros(cap, dtype=np.float32)
    out_id = np.zeros(cap, dtype=np.uint64)
    keep = np.zeros(max(n, 1), dtype=np.uint8)
    nc = ctypes.c_int()
    nr = ctypes.c_int()
    rc = lib().oracle_prune_branch(ctypes.c_int(n), ctypes.c_int(d), plo, phi, plb, pub,
                                   ids.ctypes.data_as(_c_u64_p), ctypes.c_double(inc_val), ctypes.c_int(n_pick),
                                   ctypes.c_double(eta), out_lo.ctypes.data_as(_c_float_p),
                                   out_hi.ctypes.data_as(_c_float_p), out_lb.ctypes.data_as(_c_float_p),
                                   out_ub.ctypes.data_as(_c_float_p), out_id.ctypes.data_as(_c_u64_p),
                                   keep.ctypes.data_as(_c_u8_p), ctypes.byref(nc), ctypes.byref(nr))
    m = nc.value + nr.value
    return {"rc": rc, "keep": keep[:n], "n_children": nc.value, "n_rest": nr.value, "lo": out_lo[:m],
            "hi": out_hi[:m], "lb": out_lb[:m], "ub": out_ub[:m], "id": out_id[:m]}


def log_det(x):
    """The oracle's FP32 natural logarithm from basic operations (same bits on every IEEE implementation)."""
    L = lib()
    L.oracle_log_det.restype = ctypes.c_float
    L.oracle_log_det.argtypes = [ctypes.c_float]
    return float(L.oracle_log_det(float(x)))


def pick_key(lb, lb_min, lb_max, temperature, seed, box_id):
    """Softmax pick-out race key of one candidate (see bab_oracle.c)."""
    L = lib()
    L.oracle_pick_key.restype = ctypes.c_float
    L.oracle_pick_key.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                  ctypes.c_uint64]
    return float(L.oracle_pick_key(lb, lb_min, lb_max, temperature, int(seed), int(box_id)))


def split_dims(lo, hi, ids, seed, costs, top_k):
    """Dimension to split per box by the sample-imbalance score over the top_k samples (Section 3.1)."""
    lo, plo = _f(lo)
    hi, phi = _f(hi)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    costs = np.ascontiguousarray(costs, dtype=np.float32)
    n, d = lo.shape
    M = costs.shape[1]
    out = np.zeros(n, dtype=np.int32)
    rc = lib().oracle_split_dims(ctypes.c_int(n), ctypes.c_int(d), plo, phi, ids.ctypes.data_as(_c_u64_p),
                                 ctypes.c_uint64(seed), costs.ctypes.data_as(_c_float_p), ctypes.c_int(M),
                                 ctypes.c_int(top_k), out.ctypes.data_as(_c_int_p))
    assert rc == 0
    return out


def prune_branch_heuristic(lo, hi, lb, ub, ids, inc_val, n_pick, eta=0.75, pick_rule=1, temperature=0.05,
                           pick_seed=0, split_dim=None):
    """prune_branch with the softmax pick-out (pick_rule 1) and given split dimensions (None: widest)."""
    lo, plo = _f(lo)
    hi, phi = _f(hi)
    lb, plb = _f(lb)
    ub, pub = _f(ub)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    n, d = lo.shape
    cap = 2 * n + 1
    out_lo = np.zeros((cap, d), dtype=np.float32)
    out_hi = np.zeros_like(out_lo)
    out_lb = np.zeros(cap, dtype=np.float32)
    out_ub = np.zeros(cap, dtype=np.float32)
    out_id = np.zeros(cap, dtype=np.uint64)
    keep = np.zeros(max(n, 1), dtype=np.uint8)
    sd = None if split_dim is None else np.ascontiguousarray(split_dim, dtype=np.int32)
    nc = ctypes.c_int()
    nr = ctypes.c_int()
    rc = lib().oracle_prune_branch_heuristic(
        ctypes.c_int(n), ctypes.c_int(d), plo, phi, plb, pub, ids.ctypes.data_as(_c_u64_p), ctypes.c_double(inc_val),
        ctypes.c_int(n_pick), ctypes.c_double(eta), ctypes.c_int(pick_rule), ctypes.c_float(temperature),
        ctypes.c_uint64(pick_seed), None if sd is None else sd.ctypes.data_as(_c_int_p),
        out_lo.ctypes.data_as(_c_float_p), out_hi.ctypes.data_as(_c_float_p), out_lb.ctypes.data_as(_c_float_p),
        out_ub.ctypes.data_as(_c_float_p), out_id.ctypes.data_as(_c_u64_p), keep.ctypes.data_as(_c_u8_p),
        ctypes.byref(nc), ctypes.byref(nr))
    m = nc.value + nr.value
    return {"rc": rc, "keep": keep[:n], "n_children": nc.value, "n_rest": nr.value, "lo": out_lo[:m],
            "hi": out_hi[:m], "lb": out_lb[:m], "ub": out_ub[:m], "id": out_id[:m]}


def bab(problem, lo, hi, ids, iters, n_pick, samples, seed, alpha_steps=0, alpha_lr=0.1, eta=0.75):
    """Algorithm 2 on the host: search and bound the initial boxes, then per iteration prune the pool
    against the incumbent, pick out and split, search and bound the children, update the incumbent.

    Returns (inc_val, inc_u, history) where history holds one dict per iteration."""
    lo = np.asarray(lo, dtype=np.float32)
    hi = np.asarray(hi, dtype=np.float32)
    ids = np.asarray(ids, dtype=np.uint64)
    inc_val, inc_u = np.inf, None

    def search_and_bound(lo, hi, ids):
        nonlocal inc_val, inc_u
        ub, bu, _ = rollout(problem, lo, hi, ids, samples, seed)
        if alpha_steps > 0:
            lb, *_ = alpha_optimize(problem, lo, hi, alpha_steps, alpha_lr)
        else:
            lb = crown(problem, lo, hi)["lb"]
        if len(ub):
            i = int(np.argmin(ub))
            if ub[i] < inc_val:
                inc_val, inc_u = float(ub[i]), bu[i].copy()
        return lb.astype(np.float32), ub.astype(np.float32)

    lb, ub = search_and_bound(lo, hi, ids)
    hist = []
    for it in range(iters):
        out = prune_branch(lo, hi, lb, ub, ids, inc_val, n_pick, eta)
        nc = out["n_children"]
        lo, hi, ids = out["lo"], out["hi"], out["id"]
        lb, ub = out["lb"].copy(), out["ub"].copy()
        if nc:
            clb, cub = search_and_bound(lo[:nc], hi[:nc], ids[:nc])
            lb[:nc], ub[:nc] = clb, cub
        live_lb = float(np.min(lb)) if len(lb) else np.inf
        hist.append({"iter": it, "pool": len(lb), "children": nc, "pruned": int((out["keep"] == 0).sum()),
                     "inc_val": inc_val, "global_lb": live_lb})
        if len(lb) == 0:
            break
    return inc_val, inc_u, hist


def objective_f32(problem, u):
    """Eq. (trajop) in FP32 with one rounding per operation (dot products as fused multiply-add chains in input
    order): the value the search ranks samples by."""
    net = net_of(problem)
    u = np.ascontiguousarray(u, dtype=np.float32)
    x0f = np.ascontiguousarray(problem["x0"], dtype=np.float32)
    gf = np.ascontiguousarray(problem["goal"], dtype=np.float32)
    fn = lib().oracle_objective_f32
    fn.restype = ctypes.c_float
    return float(fn(*net.cargs(), ctypes.c_int(int(problem["H"])), ctypes.c_float(float(problem["rho"])),
                    x0f.ctypes.data_as(_c_float_p), gf.ctypes.data_as(_c_float_p), u.ctypes.data_as(_c_float_p)))


def cem_normal(seed, box_id, it, m, j):
    fn = lib().oracle_cem_normal
    fn.restype = ctypes.c_float
    fn.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
    return float(fn(seed, box_id, it, m, j))


def cem_sample(seed, box_id, it, m, j, mu, sigma, lo, hi):
    fn = lib().oracle_cem_sample
    fn.restype = ctypes.c_float
    fn.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                   ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    return float(fn(seed, box_id, it, m, j, mu, sigma, lo, hi))


def cem(problem, lo, hi, ids, samples, iters, elites, jitter, seed, warm_u=None, with_trace=False):
    """Cross-entropy search of each box (Section 3.3): returns ub [n] (FP32 objective of the best sample), best_u
    [n, d] and, with_trace, mu after every refit [n, iters, d]."""
    net = net_of(problem)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    n, d = lo.shape
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    x0f = np.ascontiguousarray(problem["x0"], dtype=np.float32)
    gf = np.ascontiguousarray(problem["goal"], dtype=np.float32)
    warm = None if warm_u is None else np.ascontiguousarray(warm_u, dtype=np.float32)
    ub = np.empty(n, dtype=np.float32)
    bu = np.empty((n, d), dtype=np.float32)
    tr = np.empty((n, iters, d), dtype=np.float32) if with_trace else None
    fn = lib().oracle_cem
    fn.restype = ctypes.c_int
    rc = fn(*net.cargs(), ctypes.c_int(int(problem["H"])), ctypes.c_float(float(problem["rho"])),
            x0f.ctypes.data_as(_c_float_p), gf.ctypes.data_as(_c_float_p), n, lo.ctypes.data_as(_c_float_p),
            hi.ctypes.data_as(_c_float_p), ids.ctypes.data_as(_c_u64_p),
            None if warm is None else warm.ctypes.data_as(_c_float_p), samples, iters, elites,
            ctypes.c_float(jitter), ctypes.c_uint64(seed), ub.ctypes.data_as(_c_float_p),
            bu.ctypes.data_as(_c_float_p), None if tr is None else tr.ctypes.data_as(_c_float_p))
    if rc != 0:
        raise ValueError("oracle_cem: bad arguments")
    return (ub, bu, tr) if with_trace else (ub, bu)


def synth_f(u):
    """Section 4, synthetic example: f(u) = sum_i 5 u_i^2 + cos(50 u_i) in FP64."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    fn = lib().oracle_synth_f
    fn.restype = ctypes.c_double
    return float(fn(int(u.size), u.ctypes.data_as(_c_double_p)))


def cos_min(a, b):
    fn = lib().oracle_cos_min
    fn.restype = ctypes.c_double
    fn.argtypes = [ctypes.c_double, ctypes.c_double]
    return float(fn(a, b))


def synth_bound(lo, hi):
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    n, d = lo.shape
    lb = np.empty(n)
    lib().oracle_synth_bound(n, d, lo.ctypes.data_as(_c_float_p), hi.ctypes.data_as(_c_float_p),
                             lb.ctypes.data_as(_c_double_p))
    return lb


def synth_search(lo, hi, ids, samples, seed):
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    n, d = lo.shape
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    ub = np.empty(n)
    bu = np.empty((n, d), dtype=np.float32)
    lib().oracle_synth_search(n, d, lo.ctypes.data_as(_c_float_p), hi.ctypes.data_as(_c_float_p),
                              ids.ctypes.data_as(_c_u64_p), int(samples), ctypes.c_uint64(seed),
                              ub.ctypes.data_as(_c_double_p), bu.ctypes.data_as(_c_float_p))
    return ub, bu


def set_cost(kind=0, w=None, lam=0.0, obstacles=(), p0=(0.0, 0.0)):
    """Select the state cost of every oracle function (Appendix D.4): kind 0 the squared distance, kind 1 the
    pushing-with-obstacles cost with weights w [H] (w_1..w_H), lam, obstacles [(x, y, size)], pusher start p0."""
    if kind == 0:
        lib().oracle_set_cost(0, 0, None, ctypes.c_double(0.0), 0, None, None)
        return
    w = np.ascontiguousarray(w, dtype=np.float64)
    obs = np.ascontiguousarray(np.asarray(obstacles, dtype=np.float64).reshape(-1, 3))
    p0 = np.ascontiguousarray(p0, dtype=np.float64)
    rc = lib().oracle_set_cost(int(kind), int(w.size), w.ctypes.data_as(_c_double_p), ctypes.c_double(lam),
                               int(obs.shape[0]), obs.ctypes.data_as(_c_double_p), p0.ctypes.data_as(_c_double_p))
    if rc != 0:
        raise ValueError("oracle_set_cost: bad arguments")


def relu_dist_lower(l0, u0, l1, u1, cx, cy, size):
    """The linear lower bound a . q + b of ReLU(size - ||q - c||) on a box (Appendix D.4 penalty): (used, a0, a1, b)."""
    a0, a1, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    fn = lib().oracle_relu_dist_lower
    fn.argtypes = [ctypes.c_double] * 7 + [_c_double_p] * 3
    used = fn(l0, u0, l1, u1, cx, cy, size, ctypes.byref(a0), ctypes.byref(a1), ctypes.byref(b))
    return int(used), a0.value, a1.value, b.value
