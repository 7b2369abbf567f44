"""The C ABI library loads and exports every symbol the public header declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(chase_bse_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_10557_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["chase_bse_solve", "chase_bse_filter", "chase_bse_rr", "chase_bse_grad", "chase_bse_strerror"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    for name in _declared():
        assert hasattr(lib, name), name
    # pure host functions are safe to call without a GPU
    assert lib.chase_bse_version() >= 100
    assert lib.chase_bse_strerror(-1) == b"invalid argument"
    assert lib.chase_bse_strerror(1).startswith(b"not converged")


def test_binding_exports_cover_header(lib):
    from paper_2601_10557_gb300 import _lib
    for name in _declared():
        assert name in _lib.EXPORTS


def test_bad_arguments_rejected_without_touching_device(lib):
    import ctypes
    # NULL pointers / nonsense sizes are rejected before any CUDA call
    assert lib.chase_bse_solve(None, None, 0, 1, 0, 1, 1e-10, None, None, None, None) == -1
    assert lib.chase_bse_rr(None, None, 4, None, 3, None, None, None) == -1
    assert lib.chase_bse_grad(None, None, 4, 1, None, None, None) == -1


def test_gemm_timer_host_side(lib):
    """The filter-GEMM event record answers without a GPU while it holds nothing, and
    rejects a NULL pointer or an unknown kind."""
    import ctypes
    ms, fl, cnt = ctypes.c_double(1.0), ctypes.c_double(1.0), ctypes.c_int64(7)
    lib.chase_bse_gemm_timer(0)
    args = (ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(cnt))
    assert lib.chase_bse_gemm_time(0, *args) == 0
    assert (ms.value, fl.value, cnt.value) == (0.0, 0.0, 0)
    assert lib.chase_bse_gemm_time(2, *args) == 0
    assert lib.chase_bse_gemm_time(3, *args) == -1
    assert lib.chase_bse_gemm_time(0, None, ctypes.byref(fl), ctypes.byref(cnt)) == -1
