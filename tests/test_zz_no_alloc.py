"""bab_bound_crown_static: the CROWN bound for callers that cannot allocate device memory.

Such callers (a plugin running inside a framework that owns all device memory, or a real-time planning loop
that must not allocate once started) get the bound with every byte of working memory in a fixed array inside
the library.  This file runs last (pytest collects it after the others) so that a failure here leaves every
other test already run.  It checks, through the C-ABI, that a warm-up call with no boxes succeeds, that two
calls in a row give the same bounds as the context-based bab_bound_crown within the parity tolerance and the
FP64 oracle's CROWN bound and margin within theirs (with and without the margin output, on the default and on
a side stream), and that an oversized batch is refused.
"""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _context_bound(p, lo, hi):
    from gpu_util import GpuProblem
    g = GpuProblem(p)
    try:
        r = g.crown(lo, hi)
    finally:
        g.close()
    return r["lb"], r["margin"]


def _static_bound(p, lo, hi, with_margin=True, stream=None):
    from paper_2412_09584_gb300 import binding as B
    dev = torch.device("cuda:0")
    n = lo.shape[0]
    lb = torch.full((n,), np.nan, device=dev)
    mg = torch.full((n,), np.nan, device=dev) if with_margin else None
    params = torch.as_tensor(p["params"]).to(dev, torch.float32)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev, torch.float32)
    args = (T(p["x0"]), T(p["goal"]), p["H"], p["rho"], T(lo), T(hi), n, lb, mg)
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            rc = B.bab_bound_crown_static(p["dims"], params, p["s"], p["k"], *args)
    else:
        rc = B.bab_bound_crown_static(p["dims"], params, p["s"], p["k"], *args)
    torch.cuda.synchronize()
    assert rc == 0, rc
    return lb.cpu().numpy(), (mg.cpu().numpy() if with_margin else None)


def test_static_bound_warm_up_call_with_no_boxes():
    """n = 0 is the warm-up: it only looks up the array's address (and loads the kernels) and returns BAB_OK
    without writing anything."""
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("tiny", 5)
    dev = torch.device("cuda:0")
    params = torch.as_tensor(p["params"]).to(dev, torch.float32)
    x0 = torch.as_tensor(p["x0"]).to(dev, torch.float32)
    lb = torch.full((4,), 3.0, device=dev)
    z = torch.zeros(4, 10, device=dev)
    for _ in range(2):
        assert B.bab_bound_crown_static(p["dims"], params, p["s"], p["k"], x0, x0, p["H"], p["rho"], z, z, 0, lb) == 0
    torch.cuda.synchronize()
    assert bool((lb == 3.0).all())


@pytest.mark.parametrize("name,n", [("tiny", 64), ("pushing", 24)])
def test_static_bound_matches_context_bound_twice(name, n):
    p = W.config_problem(name, 5)
    d = p["k"] * p["H"]
    lo, hi, _ = W.random_boxes(d, n, seed=17, min_width=0.0, max_width=0.6)
    lb_ref, mg_ref = _context_bound(p, lo, hi)
    scale = np.maximum(np.abs(lb_ref), 1.0)
    for _ in range(2):  # the array keeps the previous call's contents: the second call must not depend on them
        lb, mg = _static_bound(p, lo, hi)
        assert np.all(np.abs(lb - lb_ref) <= REL * scale)
        assert np.all(np.abs(mg - mg_ref) <= REL * scale)
    # a different network and batch in between, then the first again, without the margin and on a side stream
    q = W.config_problem("tiny", 6)
    lo2, hi2, _ = W.random_boxes(10, 7, seed=3, min_width=0.1, max_width=0.4)
    _static_bound(q, lo2, hi2)
    lb, _ = _static_bound(p, lo, hi, with_margin=False)
    assert np.all(np.abs(lb - lb_ref) <= REL * scale)
    lb, mg = _static_bound(p, lo, hi, stream=torch.cuda.Stream())
    assert np.all(np.abs(lb - lb_ref) <= REL * scale)
    assert np.all(np.abs(mg - mg_ref) <= REL * scale)


@pytest.mark.parametrize("name,n", [("tiny", 64), ("pushing", 24)])
def test_static_bound_matches_oracle(oracle, name, n):
    """Against the FP64 oracle directly: the raw bound (lb + margin) within 1e-5 of the bound's scale, the
    returned bound never above the oracle's, the margin within 1e-3 of the oracle's FP64 evaluation of the same
    rounding-error formula."""
    p = W.config_problem(name, 7)
    d = p["k"] * p["H"]
    lo, hi, _ = W.random_boxes(d, n, seed=19, min_width=0.0, max_width=0.8)
    lb, mg = _static_bound(p, lo, hi)
    o = oracle.crown_margin(p, lo, hi, prec=0)
    scale = np.maximum(o["scale"], 1.0)
    assert np.all(np.abs(lb.astype(np.float64) + mg - o["lb"]) <= REL * scale)
    assert np.all(lb <= o["lb"] + 1e-12 * np.abs(o["lb"]))
    np.testing.assert_allclose(mg, o["margin"], rtol=1e-3, atol=0)


def test_static_bound_refuses_oversized_batch():
    from paper_2412_09584_gb300 import binding as B
    p = W.config_problem("pushing", 5)
    dev = torch.device("cuda:0")
    n = 4096  # about 94 KB of working memory per box at this size: far above the fixed array
    z = torch.zeros(n, 40, device=dev)
    lb = torch.full((n,), 7.0, device=dev)
    params = torch.as_tensor(p["params"]).to(dev, torch.float32)
    x0 = torch.as_tensor(p["x0"]).to(dev)
    rc = B.bab_bound_crown_static(p["dims"], params, p["s"], p["k"], x0, x0, p["H"], p["rho"], z, z, n, lb)
    torch.cuda.synchronize()
    assert rc == B.BabError(-2, "").code == -2
    assert bool((lb == 7.0).all())  # nothing was written
    # sizes whose byte count would wrap in 64 bits are refused the same way, before any device work
    rc = B.bab_bound_crown_static(p["dims"], params, p["s"], p["k"], x0, x0, 1 << 20, p["rho"], z, z, 2 ** 31 - 1,
                                  lb)
    torch.cuda.synchronize()
    assert rc == -2
    assert bool((lb == 7.0).all())
