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


def test_static_bound_refuses_sizes_beyond_its_array_on_the_host(lib):
    """bab_bound_crown_static sizes its working set per box first and refuses any batch that would not fit its
    fixed array before forming a total or touching the device, so even sizes whose byte count would wrap in
    64 bits (n near 2^31 with H = 2^20) come back as BAB_ERR_SHAPE; the pointers are never dereferenced here."""
    lib.bab_bound_crown_static.restype = ctypes.c_int
    dims = (ctypes.c_int * 5)(10, 128, 128, 128, 8)
    fake = ctypes.c_void_p(0x1000)  # stands in for device pointers: never read when the shape is refused
    for n, H in ((2 ** 31 - 1, 1 << 20), (1, 1 << 20), (4096, 20), (200, 20)):
        rc = lib.bab_bound_crown_static(4, dims, fake, 8, 2, fake, fake, H, ctypes.c_float(0.01), fake, fake, n,
                                        fake, None, None)
        assert rc == -2, (n, H)
    # the horizon limit and argument checks come first
    assert lib.bab_bound_crown_static(4, dims, fake, 8, 2, fake, fake, (1 << 20) + 1, ctypes.c_float(0.0), fake,
                                      fake, 1, fake, None, None) == -2
    assert lib.bab_bound_crown_static(4, dims, fake, 8, 2, fake, fake, 20, ctypes.c_float(-1.0), fake, fake, 1,
                                      fake, None, None) == -1


def test_binding_constants_match_the_header():
    """Every numeric #define of include/bab.h that the binding mirrors (BAB_<NAME> as <NAME>, the error codes in
    ERRORS) has the same value on both sides."""
    import os
    import re
    from paper_2412_09584_gb300 import binding
    text = open(binding.HEADER).read()
    defines = {}
    for name, val in re.findall(r"^#define (BAB_[A-Z0-9_]+)\s+\(?(-?\d+)u?\)?", text, flags=re.M):
        defines[name] = int(val)
    assert defines["BAB_PREC_TF32X3"] == 3 and defines["BAB_ERR_UNSUPPORTED"] == -7
    mirrored = 0
    for name, val in defines.items():
        short = name[len("BAB_"):]
        if hasattr(binding, short):
            assert getattr(binding, short) == val, name
            mirrored += 1
        if name.startswith("BAB_ERR_"):
            assert binding.ERRORS[val] == name
    assert defines["BAB_OK"] == binding.BAB_OK
    assert mirrored >= 12
    assert os.path.exists(binding.HEADER)
