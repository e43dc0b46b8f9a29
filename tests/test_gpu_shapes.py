"""Network shapes beyond the named workloads, through every bound and search path, against the FP64 oracle:
a one-hidden-layer network with one state and one action, widths that are multiples of 32 but not of 64 (one tile
slot and no column split in the tensor-core epilogue), 16 and 20 states (the 16- and 32-register state paths),
eight actions (the widest action block of the tensor-core input row), and widths that are not multiples of 32
(the FP32 paths serve them; the tensor-core paths refuse with BAB_ERR_UNSUPPORTED)."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5
REL_TC = 5e-5

# name, s, k, hidden widths, H, rho, tensor-core paths available
SHAPES = [("one_hidden", 1, 1, [32], 3, 0.0, True),
          ("odd_widths", 3, 3, [96, 64], 7, 0.05, True),
          ("wide_narrow", 16, 4, [160, 32, 64], 4, 0.01, True),
          ("state20_action8", 20, 8, [64, 64], 2, 0.0, True),
          ("not_mult_32", 5, 2, [48, 40], 3, 0.01, False)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def ibp_error_bound(p, lo, hi, pl_o, pu_o, xl_o, xu_o):
    """A priori bound on how far outward-rounded FP32 interval bounds can lie from the exact ones: per layer the
    directed-rounding error of each sum (at most K + 2 roundings of 2^-23 relative to sum |W| max(|l|, |h|) + |b|)
    plus the widening of the layer's inputs carried through |W|; per step the state's widening carried forward
    and the rounding of the residual add.  Returns (bound for the hidden pre-activations, bound for the states)."""
    dims = p["dims"]
    L, s, k, H = len(dims) - 1, p["s"], p["k"], p["H"]
    par = p["params"].astype(np.float64)
    Ws, bs, off = [], [], 0
    for l in range(1, L + 1):
        Ws.append(np.abs(par[off:off + dims[l] * dims[l - 1]].reshape(dims[l], dims[l - 1])))
        off += dims[l] * dims[l - 1]
        bs.append(np.abs(par[off:off + dims[l]]))
        off += dims[l]
    u = 2.0 ** -23
    n = lo.shape[0]
    e_pre, e_x = np.zeros_like(pl_o), np.zeros_like(xl_o)
    ex = np.zeros((n, s))
    for t in range(H):
        a_l = np.concatenate([xl_o[:, t], lo[:, t * k:(t + 1) * k]], axis=1)
        a_h = np.concatenate([xu_o[:, t], hi[:, t * k:(t + 1) * k]], axis=1)
        e_in = np.concatenate([ex, np.zeros((n, k))], axis=1)
        hoff = 0
        for l in range(1, L + 1):
            S = (np.maximum(np.abs(a_l), np.abs(a_h)) + e_in) @ Ws[l - 1].T + bs[l - 1]
            e = e_in @ Ws[l - 1].T + (dims[l - 1] + 2) * u * S
            if l < L:
                e_pre[:, t, hoff:hoff + dims[l]] = e
                a_l = np.maximum(pl_o[:, t, hoff:hoff + dims[l]], 0.0)
                a_h = np.maximum(pu_o[:, t, hoff:hoff + dims[l]], 0.0)
                e_in = e
                hoff += dims[l]
            else:
                mag = np.maximum(np.abs(xl_o[:, t + 1]), np.abs(xu_o[:, t + 1])) + ex + e
                ex = ex + e + 2 * u * mag
                e_x[:, t + 1] = ex
    return e_pre, e_x


def _setup(shape, seed):
    name, s, k, hidden, H, rho, tc = shape
    p = W.make_problem(s, k, hidden, H, rho, seed=seed)
    lo, hi, ids = W.random_boxes(k * H, 37, seed=seed + 1, min_width=0.0, max_width=1.0)
    return p, lo, hi, ids, tc


@pytest.mark.parametrize("shape", SHAPES, ids=[s[0] for s in SHAPES])
def test_shape_rollouts(oracle, gp, shape):
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, tc = _setup(shape, 40)
    g = gp(p)
    M = 200
    ub_o, _, _ = oracle.rollout(p, lo, hi, ids, M, 5)
    r = g.rollout(lo, hi, ids, M=M, seed=5, incumbent=True)
    np.testing.assert_allclose(r["ub"], ub_o, rtol=REL, atol=REL)
    assert r["inc_val"] == pytest.approx(oracle.objective(p, r["inc_u"].astype(np.float64)), rel=1e-10)
    if tc:
        rt = g.rollout(lo, hi, ids, M=M, seed=5, precision=B.PREC_BF16X3, incumbent=True)
        np.testing.assert_allclose(rt["ub"], ub_o, rtol=REL, atol=REL)
        assert rt["inc_val"] == pytest.approx(oracle.objective(p, rt["inc_u"].astype(np.float64)), rel=1e-10)
    else:
        with pytest.raises(B.BabError) as e:
            g.rollout(lo, hi, ids, M=M, seed=5, precision=B.PREC_BF16X3)
        assert e.value.code == -7


@pytest.mark.parametrize("shape", SHAPES, ids=[s[0] for s in SHAPES])
def test_shape_bounds(oracle, gp, shape):
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, ids, tc = _setup(shape, 50)
    g = gp(p)
    # interval bounds: within rounding of the oracle's and containing them
    lb, pl, pu, xl, xu = g.ibp(lo, hi)
    lb_o, pl_o, pu_o, xl_o, xu_o = oracle.ibp(p, lo, hi)
    e_pre, e_x = ibp_error_bound(p, lo, hi, pl_o, pu_o, xl_o, xu_o)
    for gv, ov, e in ((pl, pl_o, e_pre), (pu, pu_o, e_pre), (xl, xl_o, e_x), (xu, xu_o, e_x)):
        assert np.all(np.abs(gv - ov) <= e + 1e-30), np.max(np.abs(gv - ov) / (e + 1e-30))
    assert np.all(pl <= pl_o + 1e-12 * np.abs(pl_o)) and np.all(pu >= pu_o - 1e-12 * np.abs(pu_o))
    assert np.all(lb <= lb_o + 1e-12 * np.abs(lb_o))
    # CROWN: within rounding (FP32) or the split band (BF16x3) of the oracle's, never above it
    o = oracle.crown(p, lo, hi)
    scale = np.maximum(o["scale"], 1.0)
    r = g.crown(lo, hi)
    assert np.all(np.abs(r["lb"].astype(np.float64) + r["margin"] - o["lb"]) <= REL * scale)
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))
    if tc:
        rt = g.crown(lo, hi, precision=B.PREC_BF16X3)
        assert np.all(np.abs(rt["lb"].astype(np.float64) + rt["margin"] - o["lb"]) <= REL_TC * scale)
        assert np.all(rt["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))
    else:
        with pytest.raises(B.BabError) as e:
            g.crown(lo, hi, precision=B.PREC_BF16X3)
        assert e.value.code == -7
    # one alpha step: the adjoint gradient at the adaptive slopes against the oracle's
    best, alpha, hist = g.alpha_steps(lo, hi, steps=1, lr=0.1)
    a0 = oracle.adaptive_alpha(p, lo, hi)
    lb_a, grad_o, _ = oracle.alpha_grad(p, lo, hi, a0)
    gs = np.maximum(np.abs(grad_o).max(axis=(1, 2), keepdims=True), 1e-30)
    assert np.all(np.abs(hist[0]["grad"] - grad_o) <= 1e-4 * gs)
    assert np.all(np.abs(hist[0]["lb"] - lb_a) <= REL * scale)
