"""Bounding under a scratch limit (bab_set_scratch_limit): the boxes go through in chunks whose working set fits,
each chunk's interval bounds recomputed instead of held for every box, and every output is bit-identical to the
one-pass call (each box is bounded on its own).  Covers the CROWN bound in its three precisions, the box gradient, the
whole alpha optimisation (the adjoint's stored coefficients are the largest per-box state), a device-side live
count, and the object-manipulation configuration with alpha-CROWN at its full 16384 boxes."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _bits(t):
    return t.detach().cpu().numpy().view(np.uint32).copy()


def _limit_for(g, rows):
    """A limit that fits `rows` boxes of the alpha optimisation (the largest per-box working set of the three)."""
    N, H, d = g.p, g.H, g.d
    s, sumh = N["s"], g.sumh
    per = (2 * H * sumh + 2 * (H + 1) * s + H * (sumh + s) + 2 * H * sumh + d + 2 + 3 * H * sumh + (H + 1) * s +
           2 * d) * 4
    return 32 * 256 + rows * per


@pytest.mark.parametrize("name,n,prec", [("pushing", 200, 0), ("pushing", 130, 1), ("tiny", 300, 0),
                                         ("pushing", 150, 3)])
def test_crown_chunked_bit_identical(gp, name, n, prec):
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 2)
    g = gp(p)
    lo, hi, _ = W.random_boxes(g.d, n, seed=n, min_width=0.0, max_width=1.0)
    tlo, thi = T(lo), T(hi)
    outs = []
    for limit in (0, _limit_for(g, 37)):
        B.bab_set_scratch_limit(g.ctx, limit)
        lb, mg = torch.empty(n, device=DEV), torch.empty(n, device=DEV)
        mu, cst = torch.empty(n, g.d, device=DEV), torch.empty(n, device=DEV)
        B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, tlo, thi, n, lb, precision=prec, margin=mg, lin_coef=mu,
                          lin_const=cst)
        torch.cuda.synchronize()
        outs.append([_bits(x) for x in (lb, mg, mu, cst)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_box_grad_chunked_bit_identical(gp):
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 3)
    g = gp(p)
    n = 90
    lo, hi, _ = W.random_boxes(g.d, n, seed=5, min_width=0.05, max_width=0.5)
    outs = []
    for limit in (0, _limit_for(g, 16)):
        B.bab_set_scratch_limit(g.ctx, limit)
        lb, gl, gh = torch.empty(n, device=DEV), torch.empty(n, g.d, device=DEV), torch.empty(n, g.d, device=DEV)
        B.bab_box_grad(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, lb, gl, gh)
        torch.cuda.synchronize()
        outs.append([_bits(x) for x in (lb, gl, gh)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name,n,variant", [("tiny", 500, -1), ("tiny", 300, -2), ("pushing", 150, -1)])
def test_alpha_optimize_chunked_bit_identical(gp, name, n, variant):
    """The whole Adam loop (warp-per-box launch, or separate bound / adjoint / Adam launches) with a limit that
    leaves a few dozen boxes a chunk; alpha and the best bound equal bit for bit."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem(name, 4)
    g = gp(p)
    B.bab_set_variant(g.ctx, B.KERNEL_ALPHA_FUSED, variant)
    lo, hi, _ = W.random_boxes(g.d, n, seed=7, min_width=0.1, max_width=1.0)
    outs = []
    for limit in (0, _limit_for(g, 41)):
        B.bab_set_scratch_limit(g.ctx, limit)
        alpha = torch.empty(n, g.H, g.sumh, device=DEV)
        B.bab_alpha_init(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, alpha)
        best = torch.empty(n, device=DEV)
        B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, 6, 0.1, best, alpha=alpha)
        torch.cuda.synchronize()
        assert B.bab_status(g.ctx) == 0
        outs.append([_bits(best), _bits(alpha)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_chunked_with_device_count(gp):
    """A device-side live count below n: each chunk reads it relative to its first row, so rows beyond the count
    are left untouched in both modes and the live rows agree bit for bit."""
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("tiny", 5)
    g = gp(p)
    n, live = 400, 233
    lo, hi, _ = W.random_boxes(g.d, n, seed=9, min_width=0.0, max_width=1.0)
    dn = torch.tensor([live], dtype=torch.int32, device=DEV)
    outs = []
    for limit in (0, _limit_for(g, 50)):
        B.bab_set_scratch_limit(g.ctx, limit)
        lb = torch.full((n,), 7.0, device=DEV)
        best = torch.full((n,), 7.0, device=DEV)
        B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, lb, d_n=dn)
        B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), n, 3, 0.1, best, d_n=dn)
        torch.cuda.synchronize()
        assert bool((lb[live:] == 7.0).all()) and bool(torch.isfinite(lb[:live]).all())
        outs.append([_bits(lb), _bits(best[:live])])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_limit_below_one_box_is_refused(gp):
    from gpu_util import DEV, T
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 6)
    g = gp(p)
    lo, hi, _ = W.random_boxes(g.d, 4, seed=1, min_width=0.1, max_width=0.2)
    B.bab_set_scratch_limit(g.ctx, 64 * 1024)  # far below one box's working set at this size
    lb = torch.empty(4, device=DEV)
    with pytest.raises(B.BabError) as e:
        B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, T(lo), T(hi), 4, lb)
    assert e.value.code == -4


def test_manip_alpha_full_batch_under_a_limit():
    """The object-manipulation configuration (MLP 36-256x4-32, H = 40) with alpha-CROWN at 16384 boxes: about
    1.3 MB of adjoint state a box (21 GB for the batch) held in one pass, or chunks of a 2 GiB limit; the two
    agree bit for bit, every bound is finite and at least the plain CROWN bound's value minus its rounding."""
    from gpu_util import DEV, T, GpuProblem
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("manip", 0)
    g = GpuProblem(p)
    try:
        n = 16384
        lo, hi, _ = W.random_boxes(160, n, seed=6, min_width=0.002, max_width=0.05)
        tlo, thi = T(lo), T(hi)
        outs = []
        for limit in (2 << 30, 0):
            B.bab_set_scratch_limit(g.ctx, limit)
            best = torch.empty(n, device=DEV)
            B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, tlo, thi, n, 2, 0.1, best)
            torch.cuda.synchronize()
            assert B.bab_status(g.ctx) == 0
            outs.append(_bits(best))
        assert np.array_equal(outs[0], outs[1])
        best = torch.from_numpy(outs[0].view(np.float32)).to(DEV)
        B.bab_set_scratch_limit(g.ctx, 2 << 30)
        lb = torch.empty(n, device=DEV)
        mg = torch.empty(n, device=DEV)
        B.bab_bound_crown(g.ctx, g.x0, g.goal, g.H, g.rho, tlo, thi, n, lb, margin=mg)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(best).all())
        # the first Adam step's bound is the adaptive-slope CROWN bound; the best over the steps is at least it
        assert bool((best >= lb - mg.abs() - 1e-6 * lb.abs()).all())
    finally:
        B.bab_set_scratch_limit(g.ctx, 0)
        g.close()
