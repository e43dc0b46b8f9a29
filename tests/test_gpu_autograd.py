"""alpha-CROWN through torch.autograd (CrownBound over bab_alpha_grad), checked against the FP64 oracle, whose
gradient is itself pinned by central finite differences."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _setup(seed=12, n=24):
    from gpu_util import GpuProblem, T
    p = W.make_problem(4, 2, [32, 32], 5, 0.01, seed=seed, weight_scale=0.3)
    lo, hi, _ = W.random_boxes(10, n, seed=seed + 1, min_width=0.3, max_width=1.0)
    g = GpuProblem(p)
    return p, lo, hi, g, T(lo), T(hi)


@pytest.mark.parametrize("prec_name,tol", [("fp32", 1e-4), ("bf16x3", 1e-3), ("tf32x3", 1e-4)])
def test_autograd_gradient_matches_oracle(oracle, prec_name, tol):
    from paper_2412_09584_gb300 import binding as B
    from paper_2412_09584_gb300.autograd import CrownProblem, crown_bound
    prec = {"fp32": B.PREC_FP32, "bf16x3": B.PREC_BF16X3, "tf32x3": B.PREC_TF32X3}[prec_name]
    p, lo, hi, g, tlo, thi = _setup()
    try:
        a0 = oracle.adaptive_alpha(p, lo, hi)
        alpha = torch.tensor(a0, dtype=torch.float32, device="cuda", requires_grad=True)
        prob = CrownProblem(g.ctx, g.x0, g.goal, g.H, g.rho, tlo, thi, precision=prec)
        lb = crown_bound(alpha, prob)
        w = torch.linspace(0.5, 1.5, lb.shape[0], device="cuda")
        (gr,) = torch.autograd.grad((w * lb).sum(), alpha)
        lb_o, g_o, _ = oracle.alpha_grad(p, lo, hi, a0)
        expect = g_o * w.cpu().numpy()[:, None, None]
        scale = np.maximum(np.abs(expect).max(axis=(1, 2), keepdims=True), 1e-30)
        assert np.all(np.abs(gr.cpu().numpy() - expect) <= tol * scale)
        # the forward value is the library's bound at alpha (margin subtracted): below the oracle's
        assert np.all(lb.detach().cpu().numpy() <= lb_o + 1e-9)
        r = g.crown(lo, hi, alpha=a0.astype(np.float32), precision=prec)
        np.testing.assert_array_equal(lb.detach().cpu().numpy(), r["lb"])
    finally:
        g.close()


def test_autograd_adam_raises_sound_bounds(oracle):
    from paper_2412_09584_gb300.autograd import CrownProblem, crown_bound
    p, lo, hi, g, tlo, thi = _setup(seed=30, n=16)
    try:
        alpha = torch.tensor(oracle.adaptive_alpha(p, lo, hi), dtype=torch.float32, device="cuda",
                             requires_grad=True)
        prob = CrownProblem(g.ctx, g.x0, g.goal, g.H, g.rho, tlo, thi)
        opt = torch.optim.Adam([alpha], lr=0.1, maximize=True)
        first = None
        best = None
        for _ in range(10):
            lb = crown_bound(alpha, prob)
            best = lb.detach() if best is None else torch.maximum(best, lb.detach())
            first = lb.detach().clone() if first is None else first
            opt.zero_grad()
            lb.sum().backward()
            opt.step()
            with torch.no_grad():
                alpha.clamp_(0.0, 1.0)
        assert float(best.sum()) >= float(first.sum())
        bestn = best.cpu().numpy()
        rng = np.random.default_rng(3)
        for i in range(16):
            u = lo[i] + rng.uniform(size=(50, 10)) * (hi[i] - lo[i])
            assert bestn[i] <= min(oracle.objective(p, x.astype(np.float64)) for x in u)
    finally:
        g.close()


@pytest.mark.parametrize("prec_name", ["fp32", "bf16x3", "tf32x3"])
def test_alpha_optimize_matches_oracle(oracle, prec_name):
    """bab_alpha_optimize (interval bounds once, 20 Adam steps on the device) against the oracle's 20 steps."""
    from paper_2412_09584_gb300 import binding as B
    prec = {"fp32": B.PREC_FP32, "bf16x3": B.PREC_BF16X3, "tf32x3": B.PREC_TF32X3}[prec_name]
    p, lo, hi, g, tlo, thi = _setup(seed=40, n=32)
    try:
        n = lo.shape[0]
        best = torch.empty(n, device="cuda")
        B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, tlo, thi, n, 20, 0.1, best, precision=prec)
        torch.cuda.synchronize()
        best_o, _, _, _ = oracle.alpha_optimize(p, lo, hi, 20, 0.1)
        b = best.cpu().numpy()
        scale = np.maximum(oracle.crown(p, lo, hi)["scale"], 1.0)
        assert np.all(np.abs(b - best_o) <= 1e-3 * scale)
        lb0 = oracle.crown(p, lo, hi)["lb"]
        assert np.all(b >= lb0 - 1e-4 * scale)  # never worse than the adaptive slopes
        rng = np.random.default_rng(4)
        for i in range(n):
            u = lo[i] + rng.uniform(size=(40, 10)) * (hi[i] - lo[i])
            assert b[i] <= min(oracle.objective(p, x.astype(np.float64)) for x in u)
    finally:
        g.close()


@pytest.mark.parametrize("fixed_alpha", [False, True])
def test_box_gradient_matches_oracle(oracle, fixed_alpha):
    """d lb / d (lo, hi) from bab_box_grad against the oracle's (itself pinned by central differences)."""
    from paper_2412_09584_gb300 import binding as B
    p, lo, hi, g, tlo, thi = _setup(seed=70, n=40)
    try:
        n = lo.shape[0]
        alpha = None
        if fixed_alpha:
            alpha = np.random.default_rng(3).uniform(0.05, 0.95, size=(n, g.H, g.sumh)).astype(np.float32)
        lb = torch.empty(n, device="cuda")
        glo, ghi = torch.empty_like(tlo), torch.empty_like(thi)
        ta = None if alpha is None else torch.tensor(alpha, device="cuda")
        B.bab_box_grad(g.ctx, g.x0, g.goal, g.H, g.rho, tlo, thi, n, lb, glo, ghi, alpha=ta)
        torch.cuda.synchronize()
        lb_o, glo_o, ghi_o = oracle.box_grad(p, lo, hi, None if alpha is None else alpha.astype(np.float64))
        r = g.crown(lo, hi, alpha=alpha)
        np.testing.assert_array_equal(lb.cpu().numpy(), r["lb"])  # the same bound as bab_bound_crown
        for got, want in ((glo.cpu().numpy(), glo_o), (ghi.cpu().numpy(), ghi_o)):
            scale = np.maximum(np.abs(want).max(axis=1, keepdims=True), 1e-30)
            assert np.all(np.abs(got - want) <= 1e-3 * scale), np.max(np.abs(got - want) / scale)
    finally:
        g.close()


def test_box_gradient_through_autograd(oracle):
    from paper_2412_09584_gb300.autograd import CrownProblem, crown_box_bound
    p, lo, hi, g, tlo, thi = _setup(seed=71, n=16)
    try:
        l_ = tlo.clone().requires_grad_(True)
        h_ = thi.clone().requires_grad_(True)
        prob = CrownProblem(g.ctx, g.x0, g.goal, g.H, g.rho, tlo, thi)
        lb = crown_box_bound(l_, h_, prob)
        w = torch.linspace(0.5, 1.5, lb.shape[0], device="cuda")
        gl, gh = torch.autograd.grad((w * lb).sum(), (l_, h_))
        _, glo_o, ghi_o = oracle.box_grad(p, lo, hi)
        wn = w.cpu().numpy()[:, None]
        for got, want in ((gl.cpu().numpy(), glo_o * wn), (gh.cpu().numpy(), ghi_o * wn)):
            scale = np.maximum(np.abs(want).max(axis=1, keepdims=True), 1e-30)
            assert np.all(np.abs(got - want) <= 1e-3 * scale)
        # the forward value is the library's sound bound: never above the oracle's exact CROWN bound
        assert np.all(lb.detach().cpu().numpy() <= oracle.crown(p, lo, hi)["lb"] + 1e-9)
    finally:
        g.close()
