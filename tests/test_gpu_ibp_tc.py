"""Interval bounds on tensor cores (bab_set_interval_precision(BAB_PREC_BF16X3 or BAB_PREC_TF32X3)): W c and |W| r
as 3-term BF16 or TF32 split products with a computed margin.  Checked against the FP64 oracle's interval bounds (they must contain them:
the margin is sound), for the tiny, pushing and object-manipulation networks, ragged tiles included; the CROWN bound
on these intervals stays sound (below the oracle's bound on exact intervals and below sampled objectives) and close
to it at the pushing scale; the interval bound of the cost stays below the oracle's.  The TF32 halves widen the
intervals by less than the BF16 ones."""
import numpy as np
import pytest

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


SPLITS = ["bf16x3", "tf32x3"]


def _prec(B, split):
    return B.PREC_TF32X3 if split == "tf32x3" else B.PREC_BF16X3


@pytest.mark.parametrize("split", SPLITS)
@pytest.mark.parametrize("name,n,maxw", [("tiny", 64, 0.5), ("tiny", 37, 2.0), ("pushing", 19, 0.5),
                                         ("pushing", 70, 0.05), ("manip", 5, 0.02)])
def test_tc_intervals_contain_the_oracle(oracle, gp, name, n, maxw, split):
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 2)
    d = p["k"] * p["H"]
    lo, hi, _ = W.random_boxes(d, n, seed=4, min_width=0.0, max_width=maxw)
    g = gp(p)
    B.bab_set_interval_precision(g.ctx, _prec(B, split))
    lb, pl, pu, xl, xu = g.ibp(lo, hi)
    assert B.bab_status(g.ctx) == 0
    lb_o, pl_o, pu_o, xl_o, xu_o = oracle.ibp(p, lo, hi)
    assert np.all(pl <= pl_o) and np.all(pu >= pu_o)
    assert np.all(xl <= xl_o) and np.all(xu >= xu_o)
    assert np.all(lb <= lb_o + 1e-12 * np.abs(lb_o))
    if name != "manip":
        # the margin's widening: about gamma_split |W| (|c| + r) per layer, compounding over the unrolled steps
        scale = np.maximum(np.abs(pl_o) + np.abs(pu_o), 1.0)
        assert np.max(((pu - pl) - (pu_o - pl_o)) / scale) <= 2e-3


@pytest.mark.parametrize("split", SPLITS)
@pytest.mark.parametrize("name,n,maxw", [("pushing", 21, 0.2), ("pushing", 200, 2.0), ("tiny", 64, 2.0)])
def test_crown_on_tc_intervals(oracle, gp, name, n, maxw, split):
    """The tensor-core CROWN on the tensor-core intervals: at most the oracle's bound on exact intervals, within
    1e-4 of its scale at these depths, and below sampled objectives."""
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 3)
    d = p["k"] * p["H"]
    lo, hi, _ = W.random_boxes(d, n, seed=n, min_width=0.0, max_width=maxw)
    g = gp(p)
    B.bab_set_interval_precision(g.ctx, _prec(B, split))
    r = g.crown(lo, hi, precision=B.PREC_BF16X3)
    assert B.bab_status(g.ctx) == 0
    o = oracle.crown(p, lo, hi)
    scale = np.maximum(o["scale"], 1.0)
    assert np.all(r["lb"] <= o["lb"] + 1e-12 * np.abs(o["lb"]))
    assert np.all(r["lb"] + r["margin"] >= o["lb"] - 1e-4 * scale)
    rng = np.random.default_rng(1)
    for i in range(0, n, max(1, n // 8)):
        us = lo[i] + rng.uniform(size=(64, d)) * (hi[i] - lo[i])
        assert r["lb"][i] <= min(oracle.objective(p, u.astype(np.float64)) for u in us)


def test_interval_precision_settings(gp):
    from paper_2412_09584_gb300 import binding as B
    g = gp(W.config_problem("tiny", 1))
    with pytest.raises(B.BabError) as e:
        B.bab_set_interval_precision(g.ctx, 7)
    assert e.value.code == -1
    B.bab_set_interval_precision(g.ctx, B.PREC_BF16X3)
    B.bab_set_interval_precision(g.ctx, B.PREC_TF32X3)
    B.bab_set_interval_precision(g.ctx, B.PREC_FP32)
    # several problems in one context: the tensor-core intervals are refused, the FP32 ones stay
    probs, _ = W.batch_problems(3, 5, H_lo=2, H_hi=4)
    params, _, _, _, _ = W.pack_batch(probs)
    ctx = B.bab_load_dynamics_batch(probs[0]["dims"], params, probs[0]["s"], probs[0]["k"])
    try:
        for prec in (B.PREC_BF16X3, B.PREC_TF32X3):
            with pytest.raises(B.BabError) as e:
                B.bab_set_interval_precision(ctx, prec)
            assert e.value.code == -7
        B.bab_set_interval_precision(ctx, B.PREC_FP32)
    finally:
        B.bab_destroy(ctx)


@pytest.mark.parametrize("split", SPLITS)
def test_tc_intervals_chunked_bit_identical(gp, split):
    """Under a scratch limit the boxes are bounded in chunks, each box on its own: the tensor-core intervals and the
    CROWN bound on them equal the one-pass results bit for bit (a box's column of the products and its epilogue do
    not depend on its neighbours in the tile)."""
    import torch
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 2)
    g = gp(p)
    n = 150
    lo, hi, _ = W.random_boxes(g.d, n, seed=9, min_width=0.0, max_width=1.0)
    B.bab_set_interval_precision(g.ctx, _prec(B, split))
    per_box = (3 * g.H * g.sumh + 2 * (g.H + 1) * p["s"] + g.H * (g.sumh + p["s"]) + 2 * g.d + 4) * 4
    outs = []
    for limit in (0, 64 * 1024 + 37 * per_box):
        B.bab_set_scratch_limit(g.ctx, limit)
        lb, mg = torch.empty(n, device=DEV), torch.empty(n, device=DEV)
        B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, lb, precision=B.PREC_BF16X3, margin=mg)
        torch.cuda.synchronize()
        outs.append((lb.cpu().numpy().view(np.uint32).copy(), mg.cpu().numpy().view(np.uint32).copy()))
    B.bab_set_scratch_limit(g.ctx, 0)
    assert B.bab_status(g.ctx) == 0
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name,n,maxw", [("tiny", 64, 2.0), ("pushing", 70, 0.5), ("manip", 5, 0.02)])
def test_tf32_intervals_tighter_than_bf16(oracle, gp, name, n, maxw):
    """Both splits contain the oracle's exact intervals; the TF32 one's widening beyond them (eps S' per layer,
    eps = 3.1 2^-22 + K 2^-23 / (1 - K 2^-23) against 3.1 2^-16 + the same term) is at most half the BF16 one's,
    summed over every interval of every box."""
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 2)
    lo, hi, _ = W.random_boxes(p["k"] * p["H"], n, seed=11, min_width=0.0, max_width=maxw)
    g = gp(p)
    _, pl_o, pu_o, _, _ = oracle.ibp(p, lo, hi)
    excess = {}
    for split in SPLITS:
        B.bab_set_interval_precision(g.ctx, _prec(B, split))
        _, pl, pu, _, _ = g.ibp(lo, hi)
        assert B.bab_status(g.ctx) == 0
        assert np.all(pl <= pl_o) and np.all(pu >= pu_o)
        excess[split] = float(np.sum((pu - pl) - (pu_o - pl_o)))
    B.bab_set_interval_precision(g.ctx, B.PREC_FP32)
    assert 0.0 <= excess["tf32x3"] <= 0.5 * excess["bf16x3"]
