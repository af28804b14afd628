"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point declared in include/harp_gb300.h."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "harp_gb300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1702_03781_gb300 import build
    return build.build()


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("harp_ctx_create", "harp_ctx_destroy", "harp_fill", "mbf_solve",
              "harp_fill_adjoint", "harp_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ct.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    L = ct.CDLL(libpath)
    L.harp_status_string.restype = ct.c_char_p
    L.harp_status_string.argtypes = [ct.c_int]
    assert L.harp_status_string(0) == b"ok"
    assert b"invalid" in L.harp_status_string(-3)
    assert b"coincident" in L.harp_status_string(0x40000001)
    assert b"zero pivot" in L.harp_status_string(17)


def test_invalid_arguments_rejected_before_any_device_work(libpath):
    """Null context and bad sizes come back as -i without touching a GPU."""
    L = ct.CDLL(libpath)
    vp = ct.c_void_p
    L.harp_fill.argtypes = [vp, ct.c_int, ct.c_int, ct.c_int, ct.c_int, vp, ct.c_double, vp, vp,
                            ct.c_long, vp, ct.c_int, ct.c_int, vp]
    assert L.harp_fill(None, 4, 2, 1, 1, None, 1e8, None, None, 0, None, 8, 0, None) == -1
    L.mbf_solve.argtypes = [vp, ct.c_int, vp, ct.c_int, vp, ct.c_int, ct.c_int, vp, ct.c_int,
                            ct.c_char, ct.c_int, ct.c_double, ct.c_int, vp, vp, vp]
    assert L.mbf_solve(None, 4, None, 4, None, 4, 1, None, 4, b"N", 0, 0.0, 1, None, None,
                       None) == -1
    L.harp_ctx_create.argtypes = [ct.POINTER(vp), ct.c_int, ct.c_int, ct.c_int]
    assert L.harp_ctx_create(None, 0, 16, 4) == -1
    L.harp_residual.argtypes = [vp, ct.c_int, vp, ct.c_int, vp, ct.c_int, vp, ct.c_int, ct.c_int,
                                vp, ct.c_int, ct.c_char, vp]
    assert L.harp_residual(None, 4, None, 4, None, 4, None, 4, 1, None, 4, b"N", None) == -1
    L.harp_ctx_set_option.argtypes = [vp, ct.c_int, ct.c_int]
    assert L.harp_ctx_set_option(None, 1, 0) == -1
    L.harp_ctx_get_option.argtypes = [vp, ct.c_int, vp]
    assert L.harp_ctx_get_option(None, 1, None) == -1
    L.harp_wait_check.argtypes = [vp, ct.c_int, vp]
    assert L.harp_wait_check(None, 0, None) == -1
