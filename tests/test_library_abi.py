"""CPU checks of the C ABI library (no GPU needed): it builds, loads, and
exports every function include/hdg.h declares, with the status codes the
header defines. No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hdg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hdg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_09907_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hdg_setup", "hdg_setup_batch", "hdg_get_maps", "hdg_condense_rhs", "hdg_apply_trace",
                     "hdg_gmg_vcycle", "hdg_solve", "hdg_recover_local", "hdg_adjoint_grad", "hdg_destroy"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults(lib):
    lib.hdg_error_string.restype = ctypes.c_char_p
    assert lib.hdg_error_string(0) == b"ok"
    assert b"invalid" in lib.hdg_error_string(1)
    from paper_1705_09907_gb300 import hdg
    o = hdg.default_options()
    assert (o.nu1, o.nu2, o.coarse_n, o.tau, o.cheb_degree) == (2, 2, 2, 1.0, 2)


def test_invalid_arguments_rejected_before_any_device_work(lib):
    from paper_1705_09907_gb300 import hdg
    ctx = ctypes.c_void_p()
    m = hdg.hdg_mesh(1, 4, 0.0, 0.0, 1.0, 1.0)              # nx < 2
    assert hdg.hdg_setup(ctypes.byref(m), 1, ctypes.c_void_p(16), None, None, ctypes.byref(ctx)) == hdg.HDG_ERR_INVALID_ARG
    m = hdg.hdg_mesh(4, 4, 0.0, 0.0, 1.0, 1.0)
    assert hdg.hdg_setup(ctypes.byref(m), 8, ctypes.c_void_p(16), None, None, ctypes.byref(ctx)) == hdg.HDG_ERR_INVALID_ARG
    assert hdg.hdg_setup(ctypes.byref(m), 1, None, None, None, ctypes.byref(ctx)) == hdg.HDG_ERR_INVALID_ARG
    assert hdg.hdg_apply_trace(None, None, None, 1, 0, None) == hdg.HDG_ERR_INVALID_ARG
    assert hdg.hdg_solve(None, None, None, 1, 1e-10, 10, 0, None, None) == hdg.HDG_ERR_INVALID_ARG


def test_setup_batch_rejects_bad_arguments_before_any_device_work(lib):
    from paper_1705_09907_gb300 import hdg
    out = (ctypes.c_void_p * 2)()
    ms = (hdg.hdg_mesh * 2)(hdg.hdg_mesh(1, 4, 0.0, 0.0, 1.0, 1.0), hdg.hdg_mesh(4, 4, 0.0, 0.0, 1.0, 1.0))
    ks = (ctypes.c_int * 2)(1, 1)
    kp = (ctypes.c_void_p * 2)(16, 16)
    assert hdg.hdg_setup_batch(0, ms, ks, kp, None, None, out) == hdg.HDG_ERR_INVALID_ARG
    assert hdg.hdg_setup_batch(17, ms, ks, kp, None, None, out) == hdg.HDG_ERR_INVALID_ARG
    assert hdg.hdg_setup_batch(2, None, ks, kp, None, None, out) == hdg.HDG_ERR_INVALID_ARG
    # the first instance is invalid (nx < 2): rejected before anything is set up
    assert hdg.hdg_setup_batch(2, ms, ks, kp, None, None, out) == hdg.HDG_ERR_INVALID_ARG
    assert out[0] is None and out[1] is None


def test_options_validated_before_any_device_work(lib):
    """Out-of-range options are rejected by hdg_setup before it touches a
    device (the kappa pointer is never read); the defaults are the documented
    ones."""
    from paper_1705_09907_gb300 import hdg
    d = hdg.default_options()
    assert (d.nu1, d.nu2, d.coarse_n, d.tau, d.cheb_degree, d.mixed, d.use_graphs, d.autotune, d.reduced,
            d.tau_kappa, d.smoother, d.tensor_apply, d.fmg_start, d.max_device_bytes, d.wait_probe,
            d.coarse_fuse, d.top_accum) == (2, 2, 2, 1.0, 2, 1, 1, 1, 1, 0, 0, 1, 0, 0, 0, 1, 1)
    ctx = ctypes.c_void_p()
    m = hdg.hdg_mesh(4, 4, 0.0, 0.0, 1.0, 1.0)
    for bad in ({"reduced": 3}, {"reduced": -1}, {"tau_kappa": 2}, {"tau": 0.0}, {"nu1": 0},
                {"cheb_degree": 9}, {"coarse_n": 1}, {"wait_probe": -1}, {"wait_probe": 65},
                {"smoother": 2}, {"smoother": -1}, {"fmg_start": -1}, {"fmg_start": 17},
                {"tensor_apply": 2}, {"coarse_fuse": -1}, {"coarse_fuse": 2}, {"top_accum": 2}):
        o = hdg.default_options(**bad)
        st = hdg.hdg_setup(ctypes.byref(m), 1, ctypes.c_void_p(16), ctypes.byref(o), None, ctypes.byref(ctx))
        assert st == hdg.HDG_ERR_INVALID_ARG, bad


def test_options_struct_matches_header(lib):
    """The binding's hdg_options has the header's field order and size: the
    defaults written by the library land in the right fields."""
    from paper_1705_09907_gb300 import hdg
    o = hdg.hdg_options()
    ctypes.memset(ctypes.byref(o), 0xFF, ctypes.sizeof(o))
    lib.hdg_default_options(ctypes.byref(o))
    assert o.max_device_bytes == 0 and o.wait_probe == 0 and o.tau_kappa == 0 and o.coarse_fuse == 1 and o.top_accum == 1
