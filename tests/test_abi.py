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


def test_empty_and_degenerate_sizes_rejected_on_the_host(libpath):
    """Empty inputs (Na = 0, Nm = 0, nrhs = 0), out-of-range orders, null
    buffers, short leading dimensions and unknown precisions come back as
    -i (the argument's 1-based position) before any device work. A zeroed
    host buffer stands in for every non-null pointer and for the opaque
    context: none of these checks reads it."""
    L = ct.CDLL(libpath)
    buf = ct.create_string_buffer(1 << 16)
    h = ct.c_void_p(ct.addressof(buf))  # any non-null address
    vp, i, d, l = ct.c_void_p, ct.c_int, ct.c_double, ct.c_long
    L.harp_fill.argtypes = [vp, i, i, i, i, vp, d, vp, vp, l, vp, i, i, vp]
    ok = dict(Na=4, Nm=2, P=1, Q=1, pos=h, f=1e8, coef=h, sb=h, stride=4, Z=h, ldz=8, prec=0)

    def fill(**kw):
        a = dict(ok, **kw)
        return L.harp_fill(h, a["Na"], a["Nm"], a["P"], a["Q"], a["pos"], a["f"], a["coef"],
                           a["sb"], a["stride"], a["Z"], a["ldz"], a["prec"], None)

    assert fill(Na=0) == -2
    assert fill(Nm=0) == -3
    assert fill(P=-1) == -4 and fill(P=65) == -4
    assert fill(Q=-1) == -5 and fill(Q=65) == -5
    assert fill(pos=None) == -6
    assert fill(f=0.0) == -7 and fill(f=float("nan")) == -7
    assert fill(coef=None) == -8
    assert fill(sb=None) == -9
    assert fill(stride=-1) == -10
    assert fill(Z=None) == -11
    assert fill(ldz=7) == -12
    assert fill(prec=9) == -13

    L.harp_fill_adjoint_noalloc.argtypes = [i, i, i, i, vp, d, vp, vp, vp, i, i, vp, i, vp]
    adj = dict(Na=4, Nm=2, P=1, Q=1, pos=h, f=1e8, coef=h, Lam=h, X=h, ld=8, nrhs=4, g=h)

    def noalloc(**kw):
        a = dict(adj, **kw)
        return L.harp_fill_adjoint_noalloc(a["Na"], a["Nm"], a["P"], a["Q"], a["pos"], a["f"],
                                           a["coef"], a["Lam"], a["X"], a["ld"], a["nrhs"],
                                           a["g"], 0, None)

    assert noalloc(Na=0) == -1
    assert noalloc(Nm=0) == -2
    assert noalloc(P=-1) == -3
    assert noalloc(Q=65) == -4
    assert noalloc(pos=None) == -5
    assert noalloc(f=-1.0) == -6
    assert noalloc(coef=None) == -7
    assert noalloc(Lam=None) == -8
    assert noalloc(X=None) == -9
    assert noalloc(ld=7) == -10
    assert noalloc(nrhs=0) == -11
    assert noalloc(g=None) == -12

    L.harp_port_objective.argtypes = [i, i, vp, i, vp, vp, vp, i, vp]
    assert L.harp_port_objective(0, 2, h, 8, h, h, h, 8, None) == -1
    assert L.harp_port_objective(4, 0, h, 8, h, h, h, 8, None) == -2
    assert L.harp_port_objective(4, 2, None, 8, h, h, h, 8, None) == -3
    assert L.harp_port_objective(4, 2, h, 7, h, h, h, 8, None) == -4
    assert L.harp_port_objective(4, 2, h, 8, h, None, h, 8, None) == -6
    assert L.harp_port_objective(4, 2, h, 8, h, h, h, 7, None) == -8

    L.harp_port_impedance.argtypes = [vp, i, i, vp, i, vp, i, vp, vp, i, vp, i, vp]
    imp = dict(ctx=h, Na=4, Nm=2, P=h, ldp=4, Y=h, ldy=4, J=h, G=h, ldg=4, W=h, ldw=8)

    def impedance(**kw):
        a = dict(imp, **kw)
        return L.harp_port_impedance(a["ctx"], a["Na"], a["Nm"], a["P"], a["ldp"], a["Y"],
                                     a["ldy"], a["J"], a["G"], a["ldg"], a["W"], a["ldw"], None)

    assert impedance(ctx=None) == -1
    assert impedance(Na=0) == -2
    assert impedance(Nm=0) == -3
    assert impedance(P=None) == -4
    assert impedance(ldp=3) == -5
    assert impedance(Y=None) == -6
    assert impedance(ldy=3) == -7
    assert impedance(J=None) == -8
    assert impedance(G=None) == -9
    assert impedance(ldg=3) == -10
    assert impedance(W=None) == -11
    assert impedance(ldw=7) == -12
