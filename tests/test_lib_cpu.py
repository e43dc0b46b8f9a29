"""Host-side checks of the C-ABI library that need no GPU: it builds for sm_103a, loads, exports every symbol
include/bab.h declares, and rejects bad arguments before touching the device."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2412_09584_gb300 import build_lib
    build_lib.build()
    from paper_2412_09584_gb300 import binding
    return binding.load()


def test_exports_every_header_symbol(lib):
    from paper_2412_09584_gb300 import binding
    names = binding.header_symbols()
    assert {"bab_load_dynamics", "bab_rollout", "bab_bound_ibp", "bab_bound_crown", "bab_alpha_step",
            "bab_prune_branch"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_version(lib):
    assert lib.bab_version() >= 10000


def test_rejects_bad_arguments_without_device_work(lib):
    from paper_2412_09584_gb300 import binding
    # null context
    assert lib.bab_rollout(None, None, None, 5, 0.0, None, None, None, 1, None, 1, 0, 0, None, None, None, None,
                           None) == -1
    assert lib.bab_prune_branch(None, 2, None, None, None, None, None, 0, None, None, 0, 0.5, 0, 0, None, None, None,
                                None, None, None, None, None) == -1
    # shapes are checked before any allocation
    out = ctypes.c_void_p()
    dims = (ctypes.c_int * 3)(6, 8, 5)  # output width must equal the state dimension (4)
    params = (ctypes.c_float * 100)()
    assert lib.bab_load_dynamics(ctypes.byref(out), 2, dims, params, 4, 2, 0) == -2
    dims = (ctypes.c_int * 3)(6, 300, 4)  # wider than the build limit
    assert lib.bab_load_dynamics(ctypes.byref(out), 2, dims, params, 4, 2, 0) == -2
    assert lib.bab_load_dynamics(ctypes.byref(out), 0, dims, params, 4, 2, 0) == -2
    assert lib.bab_load_dynamics(ctypes.byref(out), 2, dims, params, 4, 2, 7) == -1
    with pytest.raises(TypeError):
        binding._ptr([1, 2, 3], None, "x")
