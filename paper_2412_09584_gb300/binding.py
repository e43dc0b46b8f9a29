"""Thin Python binding of libbab (include/bab.h), same names as the C entry points.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays are torch CUDA tensors (device memory and streams come from
PyTorch); the binding checks dtype, device and contiguity, passes raw
pointers and the current CUDA stream, and raises BabError on a nonzero status.
If libbab.so is missing the import fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbab.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "bab.h")

BAB_OK = 0
ERRORS = {-1: "BAB_ERR_INVALID_ARG", -2: "BAB_ERR_SHAPE", -3: "BAB_ERR_CUDA", -4: "BAB_ERR_OOM",
          -5: "BAB_ERR_TIMEOUT", -6: "BAB_ERR_NUMERIC", -7: "BAB_ERR_UNSUPPORTED"}
PREC_FP32, PREC_BF16X3, PREC_BF16, PREC_TF32X3 = 0, 1, 2, 3
SPLIT_WIDEST = 0
PICK_LB, PICK_SOFTMAX = 0, 1
KERNEL_ROLLOUT_FP32, KERNEL_ALPHA_FUSED, KERNEL_ROLLOUT_TC, KERNEL_CROWN_TC = 0, 1, 2, 3


class BabError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float


def header_symbols():
    """Names of the functions declared in include/bab.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(bab_\w+)\s*\(", text, re.M)))


def load(path: str = LIB_PATH):
    """Load libbab.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_2412_09584_gb300.build_lib.build()")
    L = ctypes.CDLL(path)
    L.bab_version.restype = _I
    L.bab_load_dynamics.argtypes = [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_F), _I, _I,
                                    ctypes.c_uint]
    L.bab_destroy.argtypes = [_P]
    L.bab_last_error.argtypes = [_P]
    L.bab_last_error.restype = ctypes.c_char_p
    L.bab_status.argtypes = [_P, _P]
    L.bab_rollout.argtypes = [_P, _P, _P, _I, _F, _P, _P, _P, _I, _P, _I, ctypes.c_uint64, _I, _P, _P, _P, _P, _P]
    L.bab_bound_ibp.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _P, _P, _P, _P, _P, _P]
    L.bab_bound_crown.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _P, _I, _P, _P, _P, _P, _P]
    L.bab_alpha_init.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _P, _P]
    L.bab_alpha_step.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _P, _P, _P, _I, _F, _I, _P, _P, _P, _P]
    L.bab_alpha_grad.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _P, _I, _P, _P, _P]
    L.bab_alpha_optimize.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _I, _F, _I, _P, _P, _P]
    L.bab_prune_branch.argtypes = [_P, _I, _P, _P, _P, _P, _P, _I, _P, _P, _I, _F, _I, _I, _P, _P, _P, _P, _P, _P, _P,
                                   _P]
    L.bab_bound_crown_static.argtypes = [_I, ctypes.POINTER(_I), _P, _I, _I, _P, _P, _I, _F, _P, _P, _I, _P, _P, _P]
    L.bab_probe_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P]
    L.bab_set_scratch_limit.argtypes = [_P, ctypes.c_size_t]
    L.bab_set_interval_precision.argtypes = [_P, ctypes.c_int]
    L.bab_load_dynamics_batch.argtypes = [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_F), _I,
                                          _I, ctypes.c_uint]
    L.bab_rollout_batch.argtypes = [_P, _P, _P, _P, _P, _I, _I, _P, _P, _P, _P, _I, _P, _I, ctypes.c_uint64, _I, _P,
                                    _P, _P, _P, _P]
    L.bab_bound_batch.argtypes = [_P, _P, _P, _P, _P, _I, _I, _P, _P, _P, _I, _P, _I, _F, _P, _P, _P]
    L.bab_prune_branch_batch.argtypes = [_P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _I, _P, _P, _P, _I, _F, _I, _I, _P,
                                         _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.bab_update_incumbent.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _P, _P, _P]
    L.bab_box_grad.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _P, _P, _P, _P, _P]
    L.bab_rollout_search_bounds.argtypes = [_P, _P, _P, _I, _F, _P, _P, _P, _I, _P, _I, ctypes.c_uint64, _P, _P, _P,
                                            _P, _P, _P, _P, _P, _P]
    L.bab_bound_crown_given.argtypes = [_P, _P, _P, _I, _F, _P, _P, _I, _P, _P, _P, _P, _P, _I, _P, _P]
    L.bab_context_create.argtypes = [ctypes.POINTER(_P)]
    L.bab_synth_search.argtypes = [_P, _I, _P, _P, _P, _I, _P, _I, ctypes.c_uint64, _I, _I, _F, _P, _P, _P, _P, _P,
                                   _P]
    L.bab_synth_bound.argtypes = [_P, _I, _P, _P, _I, _P, _P, _P]
    L.bab_set_cost.argtypes = [_P, _I, _I, _P, _F, _I, _P, _P]
    L.bab_rollout_cem.argtypes = [_P, _P, _P, _I, _F, _P, _P, _P, _I, _P, _I, _I, _I, _F, ctypes.c_uint64, _I, _P,
                                  _P, _P, _P, _P, _P]
    L.bab_prune_branch_heuristic.argtypes = [_P, _I, _P, _P, _P, _P, _P, _I, _P, _P, _I, _F, _I, _F, ctypes.c_uint64,
                                             _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.bab_split_dims.argtypes = [_P, _I, _P, _P, _P, _I, _P, ctypes.c_uint64, _P, _I, _I, _P, _P]
    L.bab_rollout_split.argtypes = [_P, _P, _P, _I, _F, _P, _P, _P, _I, _P, _I, ctypes.c_uint64, _I, _F, _P, _P, _P,
                                    _P, _P, _P, _P]
    L.bab_set_variant.argtypes = [_P, _I, _I]
    L.bab_set_rescore_topk.argtypes = [_P, _I]
    L.bab_get_variant.argtypes = [_P, _I, ctypes.POINTER(_I)]
    L.bab_autotune.argtypes = [_P, _P, _P, _I, _F, _P, _P, _P, _I, _I, _I, _P]
    _lib = L
    return L


def _ptr(t, dtype=None, name="array", allow_none=True):
    if t is None:
        if not allow_none:
            raise ValueError(f"{name} is required")
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is torch.uint64 and t.dtype == torch.int64:
        dtype = torch.int64  # box identifiers: the same 64 bits either way
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check(ctx, rc):
    if rc != BAB_OK:
        raise BabError(rc, load().bab_last_error(ctx).decode())


def bab_version():
    return load().bab_version()


def bab_load_dynamics(dims, params, state_dim, action_dim, flags=0):
    """Create a context from host parameters (packed W_1, b_1, ..., W_L, b_L). Returns an opaque handle."""
    L = load()
    dims_a = (_I * len(dims))(*[int(x) for x in dims])
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    out = _P()
    rc = L.bab_load_dynamics(ctypes.byref(out), len(dims) - 1, dims_a, p.ctypes.data_as(ctypes.POINTER(_F)),
                             int(state_dim), int(action_dim), int(flags))
    if rc != BAB_OK:
        raise BabError(rc, "bab_load_dynamics failed")
    return out.value


def bab_destroy(ctx):
    load().bab_destroy(ctx)


def bab_status(ctx, stream=None):
    return load().bab_status(ctx, _stream(stream))


def bab_rollout(ctx, x0, goal, horizon, rho, lo, hi, ids, n, samples, seed, precision, ub, best_u=None,
                inc_val=None, inc_u=None, d_n=None, stream=None):
    f32, u64 = torch.float32, torch.uint64
    rc = load().bab_rollout(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), int(horizon), float(rho),
                            _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), _ptr(ids, u64, "id"), int(n),
                            _ptr(d_n, torch.int32, "d_n"), int(samples), ctypes.c_uint64(int(seed)), int(precision),
                            _ptr(ub, f32, "ub"), _ptr(best_u, f32, "best_u"), _ptr(inc_val, torch.float64, "inc_val"),
                            _ptr(inc_u, f32, "inc_u"), _stream(stream))
    _check(ctx, rc)


def bab_bound_ibp(ctx, x0, goal, horizon, rho, lo, hi, n, lb_ibp=None, pre_lo=None, pre_hi=None, x_lo=None,
                  x_hi=None, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_bound_ibp(ctx, _ptr(x0, f32), _ptr(goal, f32), int(horizon), float(rho), _ptr(lo, f32),
                              _ptr(hi, f32), int(n), _ptr(d_n, torch.int32), _ptr(lb_ibp, f32), _ptr(pre_lo, f32),
                              _ptr(pre_hi, f32), _ptr(x_lo, f32), _ptr(x_hi, f32), _stream(stream))
    _check(ctx, rc)


def bab_bound_crown(ctx, x0, goal, horizon, rho, lo, hi, n, lb, alpha=None, precision=PREC_FP32, margin=None,
                    lin_coef=None, lin_const=None, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_bound_crown(ctx, _ptr(x0, f32), _ptr(goal, f32), int(horizon), float(rho), _ptr(lo, f32),
                                _ptr(hi, f32), int(n), _ptr(d_n, torch.int32), _ptr(alpha, f32), int(precision),
                                _ptr(lb, f32), _ptr(margin, f32), _ptr(lin_coef, f32), _ptr(lin_const, f32),
                                _stream(stream))
    _check(ctx, rc)


def bab_alpha_init(ctx, x0, goal, horizon, rho, lo, hi, n, alpha, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_alpha_init(ctx, _ptr(x0, f32), _ptr(goal, f32), int(horizon), float(rho), _ptr(lo, f32),
                               _ptr(hi, f32), int(n), _ptr(d_n, torch.int32), _ptr(alpha, f32), _stream(stream))
    _check(ctx, rc)


def bab_alpha_step(ctx, x0, goal, horizon, rho, lo, hi, n, alpha, adam_m, adam_v, step, lr, lb=None, lb_best=None,
                   grad_alpha=None, precision=PREC_FP32, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_alpha_step(ctx, _ptr(x0, f32), _ptr(goal, f32), int(horizon), float(rho), _ptr(lo, f32),
                               _ptr(hi, f32), int(n), _ptr(d_n, torch.int32), _ptr(alpha, f32), _ptr(adam_m, f32),
                               _ptr(adam_v, f32), int(step), float(lr), int(precision), _ptr(lb, f32),
                               _ptr(lb_best, f32), _ptr(grad_alpha, f32), _stream(stream))
    _check(ctx, rc)


def bab_alpha_grad(ctx, x0, goal, horizon, rho, lo, hi, n, alpha, lb, grad_alpha, precision=PREC_FP32, d_n=None,
                   stream=None):
    f32 = torch.float32
    rc = load().bab_alpha_grad(ctx, _ptr(x0, f32), _ptr(goal, f32), int(horizon), float(rho), _ptr(lo, f32),
                               _ptr(hi, f32), int(n), _ptr(d_n, torch.int32), _ptr(alpha, f32), int(precision),
                               _ptr(lb, f32), _ptr(grad_alpha, f32), _stream(stream))
    _check(ctx, rc)


def bab_prune_branch(ctx, d, lo, hi, lb, ub, ids, n, inc_val, n_pick, eta, cap_out, out_lo, out_hi, out_lb, out_ub,
                     out_id, keep, d_counts, split_rule=SPLIT_WIDEST, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_prune_branch(ctx, int(d), _ptr(lo, f32), _ptr(hi, f32), _ptr(lb, f32), _ptr(ub, f32),
                                 _ptr(ids, torch.uint64), int(n), _ptr(d_n, torch.int32),
                                 _ptr(inc_val, torch.float64), int(n_pick), float(eta), int(split_rule), int(cap_out),
                                 _ptr(out_lo, f32), _ptr(out_hi, f32), _ptr(out_lb, f32), _ptr(out_ub, f32),
                                 _ptr(out_id, torch.uint64), _ptr(keep, torch.uint8), _ptr(d_counts, torch.int32),
                                 _stream(stream))
    _check(ctx, rc)


def bab_bound_crown_static(dims, params, state_dim, action_dim, x0, goal, horizon, rho, lo, hi, n, lb, margin=None,
                           stream=None):
    """The CROWN bound without device allocation (no context): `params` is a CUDA tensor holding the packed
    network; returns the library's status code instead of raising, so callers can test for BAB_ERR_SHAPE."""
    f32 = torch.float32
    dims_a = (_I * len(dims))(*[int(x) for x in dims])
    return load().bab_bound_crown_static(len(dims) - 1, dims_a, _ptr(params, f32, "params"), int(state_dim),
                                         int(action_dim), _ptr(x0, f32), _ptr(goal, f32), int(horizon), float(rho),
                                         _ptr(lo, f32), _ptr(hi, f32), int(n), _ptr(lb, f32), _ptr(margin, f32),
                                         _stream(stream))


def bab_probe_fp32_peak(stream=None):
    """Measured FP32 FMA rate of the current GPU in TFLOP/s: (scalar FMAs, paired FMAs)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = load().bab_probe_fp32_peak(ctypes.byref(a), ctypes.byref(b), _stream(stream))
    if rc != BAB_OK:
        raise BabError(rc, "bab_probe_fp32_peak failed")
    return a.value, b.value


def bab_alpha_optimize(ctx, x0, goal, horizon, rho, lo, hi, n, steps, lr, lb_best, alpha=None, precision=PREC_FP32,
                       d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_alpha_optimize(ctx, _ptr(x0, f32), _ptr(goal, f32), int(horizon), float(rho), _ptr(lo, f32),
                                   _ptr(hi, f32), int(n), _ptr(d_n, torch.int32), int(steps), float(lr),
                                   int(precision), _ptr(alpha, f32), _ptr(lb_best, f32), _stream(stream))
    _check(ctx, rc)


def bab_set_variant(ctx, kernel, variant):
    _check(ctx, load().bab_set_variant(ctx, int(kernel), int(variant)))


def bab_set_scratch_limit(ctx, nbytes):
    _check(ctx, load().bab_set_scratch_limit(ctx, ctypes.c_size_t(int(nbytes))))


def bab_set_interval_precision(ctx, precision):
    _check(ctx, load().bab_set_interval_precision(ctx, int(precision)))


def bab_set_rescore_topk(ctx, k):
    _check(ctx, load().bab_set_rescore_topk(ctx, int(k)))


def bab_get_variant(ctx, kernel):
    v = _I()
    _check(ctx, load().bab_get_variant(ctx, int(kernel), ctypes.byref(v)))
    return v.value


def bab_autotune(ctx, x0, goal, horizon, rho, lo, hi, ids, n, samples, alpha_steps=0, stream=None):
    f32 = torch.float32
    rc = load().bab_autotune(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), int(horizon), float(rho),
                             _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), _ptr(ids, torch.uint64, "id"), int(n),
                             int(samples), int(alpha_steps), _stream(stream))
    _check(ctx, rc)


def bab_load_dynamics_batch(dims, params, state_dim, action_dim, flags=0):
    """Context for P problems of one architecture: params is [P][n_params] (host). Returns an opaque handle."""
    L = load()
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    if p.ndim != 2:
        raise ValueError("params must be [n_problems][n_params]")
    dims_a = (_I * len(dims))(*[int(x) for x in dims])
    out = _P()
    rc = L.bab_load_dynamics_batch(ctypes.byref(out), p.shape[0], len(dims) - 1, dims_a,
                                   p.ctypes.data_as(ctypes.POINTER(_F)), int(state_dim), int(action_dim), int(flags))
    if rc != BAB_OK:
        raise BabError(rc, "bab_load_dynamics_batch failed")
    return out.value


def bab_rollout_batch(ctx, x0, goal, horizon, rho, max_horizon, d_stride, lo, hi, ids, prob, n, samples, seed, ub,
                      best_u=None, inc_val=None, inc_u=None, d_n=None, precision=PREC_FP32, stream=None):
    f32, i32 = torch.float32, torch.int32
    rc = load().bab_rollout_batch(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), _ptr(horizon, i32, "horizon"),
                                  _ptr(rho, f32, "rho"), int(max_horizon), int(d_stride), _ptr(lo, f32, "lo"),
                                  _ptr(hi, f32, "hi"), _ptr(ids, torch.uint64, "id"), _ptr(prob, i32, "prob"), int(n),
                                  _ptr(d_n, i32), int(samples), int(seed), int(precision), _ptr(ub, f32, "ub"),
                                  _ptr(best_u, f32), _ptr(inc_val, torch.float64), _ptr(inc_u, f32), _stream(stream))
    _check(ctx, rc)


def bab_bound_batch(ctx, x0, goal, horizon, rho, max_horizon, d_stride, lo, hi, prob, n, lb, alpha_steps=0, lr=0.1,
                    lb_ibp=None, d_n=None, stream=None):
    f32, i32 = torch.float32, torch.int32
    rc = load().bab_bound_batch(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), _ptr(horizon, i32, "horizon"),
                                _ptr(rho, f32, "rho"), int(max_horizon), int(d_stride), _ptr(lo, f32, "lo"),
                                _ptr(hi, f32, "hi"), _ptr(prob, i32, "prob"), int(n), _ptr(d_n, i32),
                                int(alpha_steps), float(lr), _ptr(lb, f32, "lb"), _ptr(lb_ibp, f32), _stream(stream))
    _check(ctx, rc)


def bab_prune_branch_batch(ctx, d_stride, horizon, max_horizon, lo, hi, lb, ub, ids, prob, n, inc_val, n_pick,
                           max_pick_total, eta, cap_out, out_lo, out_hi, out_lb, out_ub, out_id, out_prob, keep,
                           d_counts, d_pcounts=None, d_n=None, split_rule=SPLIT_WIDEST, stream=None):
    f32, i32 = torch.float32, torch.int32
    rc = load().bab_prune_branch_batch(
        ctx, int(d_stride), _ptr(horizon, i32, "horizon"), int(max_horizon), _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"),
        _ptr(lb, f32, "lb"), _ptr(ub, f32, "ub"), _ptr(ids, torch.uint64, "id"), _ptr(prob, i32, "prob"), int(n),
        _ptr(d_n, i32), _ptr(inc_val, torch.float64, "inc_val"), _ptr(n_pick, i32, "n_pick"), int(max_pick_total),
        float(eta), int(split_rule), int(cap_out), _ptr(out_lo, f32), _ptr(out_hi, f32), _ptr(out_lb, f32),
        _ptr(out_ub, f32), _ptr(out_id, torch.uint64), _ptr(out_prob, i32), _ptr(keep, torch.uint8),
        _ptr(d_counts, i32, "d_counts"), _ptr(d_pcounts, i32), _stream(stream))
    _check(ctx, rc)


def bab_update_incumbent(ctx, x0, goal, horizon, rho, ub, best_u, n, inc_val, inc_u, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_update_incumbent(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), int(horizon), float(rho),
                                     _ptr(ub, f32, "ub"), _ptr(best_u, f32, "best_u"), int(n), _ptr(d_n, torch.int32),
                                     _ptr(inc_val, torch.float64, "inc_val"), _ptr(inc_u, f32, "inc_u"),
                                     _stream(stream))
    _check(ctx, rc)


def bab_box_grad(ctx, x0, goal, horizon, rho, lo, hi, n, lb, grad_lo, grad_hi, alpha=None, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_box_grad(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), int(horizon), float(rho),
                             _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), int(n), _ptr(d_n, torch.int32),
                             _ptr(alpha, f32), _ptr(lb, f32, "lb"), _ptr(grad_lo, f32, "grad_lo"),
                             _ptr(grad_hi, f32, "grad_hi"), _stream(stream))
    _check(ctx, rc)


def bab_rollout_search_bounds(ctx, x0, goal, horizon, rho, lo, hi, ids, n, samples, seed, ub, pre_lo, pre_hi, x_lo,
                              x_hi, best_u=None, inc_val=None, inc_u=None, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_rollout_search_bounds(
        ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), int(horizon), float(rho), _ptr(lo, f32, "lo"),
        _ptr(hi, f32, "hi"), _ptr(ids, torch.uint64, "id"), int(n), _ptr(d_n, torch.int32), int(samples), int(seed),
        _ptr(ub, f32, "ub"), _ptr(best_u, f32), _ptr(inc_val, torch.float64), _ptr(inc_u, f32),
        _ptr(pre_lo, f32, "pre_lo"), _ptr(pre_hi, f32, "pre_hi"), _ptr(x_lo, f32, "x_lo"), _ptr(x_hi, f32, "x_hi"),
        _stream(stream))
    _check(ctx, rc)


def bab_bound_crown_given(ctx, x0, goal, horizon, rho, lo, hi, n, pre_lo, pre_hi, x_lo, x_hi, t_stop, lb, d_n=None,
                          stream=None):
    f32 = torch.float32
    rc = load().bab_bound_crown_given(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), int(horizon), float(rho),
                                      _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), int(n), _ptr(d_n, torch.int32),
                                      _ptr(pre_lo, f32, "pre_lo"), _ptr(pre_hi, f32, "pre_hi"),
                                      _ptr(x_lo, f32, "x_lo"), _ptr(x_hi, f32, "x_hi"), int(t_stop),
                                      _ptr(lb, f32, "lb"), _stream(stream))
    _check(ctx, rc)


def bab_prune_branch_heuristic(ctx, d, lo, hi, lb, ub, ids, n, inc_val, n_pick, eta, pick_rule, temperature, pick_seed,
                               cap_out, out_lo, out_hi, out_lb, out_ub, out_id, keep, d_counts, split_dim=None,
                               out_split_dim=None, row_u=None, out_row_u=None, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_prune_branch_heuristic(
        ctx, int(d), _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), _ptr(lb, f32, "lb"), _ptr(ub, f32, "ub"),
        _ptr(ids, torch.uint64, "id"), int(n), _ptr(d_n, torch.int32), _ptr(inc_val, torch.float64, "inc_val"),
        int(n_pick), float(eta), int(pick_rule), float(temperature), int(pick_seed), _ptr(split_dim, torch.int32),
        int(cap_out), _ptr(out_lo, f32), _ptr(out_hi, f32), _ptr(out_lb, f32), _ptr(out_ub, f32),
        _ptr(out_id, torch.uint64), _ptr(out_split_dim, torch.int32), _ptr(row_u, f32), _ptr(out_row_u, f32),
        _ptr(keep, torch.uint8),
        _ptr(d_counts, torch.int32, "d_counts"), _stream(stream))
    _check(ctx, rc)


def bab_split_dims(ctx, d, lo, hi, ids, n, seed, costs, samples, top_k, split_dim, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_split_dims(ctx, int(d), _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), _ptr(ids, torch.uint64, "id"),
                               int(n), _ptr(d_n, torch.int32), int(seed), _ptr(costs, f32, "costs"), int(samples),
                               int(top_k), _ptr(split_dim, torch.int32, "split_dim"), _stream(stream))
    _check(ctx, rc)


def bab_rollout_split(ctx, x0, goal, horizon, rho, lo, hi, ids, n, samples, seed, precision, top_pct, ub, split_dim,
                      best_u=None, inc_val=None, inc_u=None, costs=None, d_n=None, stream=None):
    f32 = torch.float32
    rc = load().bab_rollout_split(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), int(horizon), float(rho),
                                  _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), _ptr(ids, torch.uint64, "id"), int(n),
                                  _ptr(d_n, torch.int32), int(samples), int(seed), int(precision), float(top_pct),
                                  _ptr(ub, f32, "ub"), _ptr(best_u, f32), _ptr(inc_val, torch.float64),
                                  _ptr(inc_u, f32), _ptr(costs, f32), _ptr(split_dim, torch.int32, "split_dim"),
                                  _stream(stream))
    _check(ctx, rc)


CEM_MAX_SAMPLES = 4096


def bab_rollout_cem(ctx, x0, goal, horizon, rho, lo, hi, ids, n, samples, iters, elites, jitter, seed, precision, ub,
                    best_u, warm_u=None, inc_val=None, inc_u=None, d_n=None, stream=None):
    """Cross-entropy search of each box (Section 3.3 batch_search with CEM); see include/bab.h."""
    f32 = torch.float32
    rc = load().bab_rollout_cem(ctx, _ptr(x0, f32, "x0"), _ptr(goal, f32, "goal"), int(horizon), float(rho),
                                _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), _ptr(ids, torch.uint64, "id"), int(n),
                                _ptr(d_n, torch.int32), int(samples), int(iters), int(elites), float(jitter),
                                int(seed), int(precision), _ptr(warm_u, f32), _ptr(ub, f32, "ub"),
                                _ptr(best_u, f32, "best_u"), _ptr(inc_val, torch.float64), _ptr(inc_u, f32),
                                _stream(stream))
    _check(ctx, rc)


def bab_context_create():
    """A context without a network (the synthetic objective and the prune / branch calls)."""
    out = _P()
    rc = load().bab_context_create(ctypes.byref(out))
    if rc != BAB_OK:
        raise BabError(rc, "bab_context_create failed")
    return out.value


def bab_synth_search(ctx, d, lo, hi, ids, n, samples, seed, ub, best_u, iters=0, elites=10, jitter=1e-3,
                     warm_u=None, inc_val=None, inc_u=None, d_n=None, stream=None):
    """The synthetic objective sum 5 u^2 + cos(50 u) (Section 4): sampled search; see include/bab.h."""
    f32 = torch.float32
    rc = load().bab_synth_search(ctx, int(d), _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), _ptr(ids, torch.uint64, "id"),
                                 int(n), _ptr(d_n, torch.int32), int(samples), int(seed), int(iters), int(elites),
                                 float(jitter), _ptr(warm_u, f32), _ptr(ub, f32, "ub"), _ptr(best_u, f32, "best_u"),
                                 _ptr(inc_val, torch.float64), _ptr(inc_u, f32), _stream(stream))
    _check(ctx, rc)


def bab_synth_bound(ctx, d, lo, hi, n, lb, d_n=None, stream=None):
    """Sound lower bound of the synthetic objective over each box (Section 4); see include/bab.h."""
    f32 = torch.float32
    rc = load().bab_synth_bound(ctx, int(d), _ptr(lo, f32, "lo"), _ptr(hi, f32, "hi"), int(n), _ptr(d_n, torch.int32),
                                _ptr(lb, f32, "lb"), _stream(stream))
    _check(ctx, rc)


COST_SQUARED = 0
COST_PUSHING_OBSTACLES = 1


def bab_set_cost(ctx, kind, w=None, lam=0.0, obstacles=(), p0=(0.0, 0.0)):
    """Select the state cost (Appendix D.4 pushing-with-obstacles, or the squared distance); see include/bab.h.
    w: the weights w_1..w_H (host), obstacles: [(x, y, size)], p0: the pusher start."""
    L = load()
    if kind == COST_SQUARED:
        _check(ctx, L.bab_set_cost(ctx, 0, 0, None, 0.0, 0, None, None))
        return
    wa = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
    ob = np.ascontiguousarray(np.asarray(obstacles, dtype=np.float32).reshape(-1, 3))
    pa = np.ascontiguousarray(np.asarray(p0, dtype=np.float32))
    _check(ctx, L.bab_set_cost(ctx, int(kind), int(wa.size), wa.ctypes.data, float(lam), int(ob.shape[0]),
                               ob.ctypes.data if ob.size else None, pa.ctypes.data))
