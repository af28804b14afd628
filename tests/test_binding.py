"""The Python binding is marshalling only: no CPU fallback, no host pointers
handed to kernels, no dependence on the oracle, and the column-major layout
the C ABI expects. Runs without a GPU."""
import ctypes as ct
import os
import re
import subprocess
import sys

import pytest
import torch

from paper_1702_03781_gb300 import harp as H
from paper_1702_03781_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1702_03781_gb300")


@pytest.fixture(scope="module")
def built():
    from paper_1702_03781_gb300 import build
    return build.build()


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(H, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(H, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        H.lib()


def test_host_tensors_are_refused():
    assert H._ptr(None).value is None
    with pytest.raises(ValueError, match="CUDA tensor"):
        H._ptr(torch.zeros(4, dtype=torch.float64))


def test_fill_and_solve_refuse_host_tensors_before_any_library_call(built):
    # a context object that never reached the library: the refusal must come
    # from the binding, before a pointer crosses the ABI
    h = object.__new__(H.Harp)
    h._h, h.device, h.max_N, h.max_nrhs = ct.c_void_p(0), 0, 64, 16
    p = synth.tiny()
    pos, coef, sb = (torch.from_numpy(p.pos), torch.from_numpy(p.coef),
                     torch.from_numpy(p.self_blocks))
    with pytest.raises(ValueError, match="CUDA tensor"):
        h.fill(pos, p.freq_hz, coef, sb, prec="fp64")
    Z = torch.zeros((p.N, p.N), dtype=torch.complex128)
    with pytest.raises(ValueError, match="CUDA tensor"):
        h.solve(Z, None, nrhs=p.Na, prec="fp64", out=H.colmajor_empty(p.N, p.Na,
                                                                        torch.complex128, "cpu"))
    with pytest.raises(ValueError, match="CUDA tensor"):
        H.port_objective(torch.zeros((p.N, p.Na), dtype=torch.complex128), p.Na, p.Nm)


def test_noalloc_refuses_host_tensors_before_any_library_call(monkeypatch):
    """The context-free adjoint runs on the current device: every tensor must
    be device memory, checked in the binding before the library is even
    loaded."""
    def no_library():
        raise AssertionError("the library was reached")
    monkeypatch.setattr(H, "lib", no_library)
    p = synth.tiny()
    pos, coef = torch.from_numpy(p.pos), torch.from_numpy(p.coef)
    X = torch.zeros((p.N, p.Na), dtype=torch.complex128)
    with pytest.raises(ValueError, match="pos must be a CUDA tensor"):
        H.fill_adjoint_noalloc(pos, p.freq_hz, coef, X, X)


def test_colmajor_layout():
    Z = H.colmajor_empty(5, 3, torch.complex64, "cpu")
    assert Z.shape == (5, 3) and Z.stride() == (1, 5)
    assert H._ld(Z) == 5
    assert H.as_colmajor(Z) is Z
    R = torch.arange(15, dtype=torch.float64).reshape(5, 3)  # row-major
    C = H.as_colmajor(R)
    assert C.stride() == (1, 5)
    assert torch.equal(C, R)
    # a column-major view with padding keeps its leading dimension
    big = H.colmajor_empty(8, 3, torch.float64, "cpu")
    view = big[:5, :]
    assert H.as_colmajor(view) is view and H._ld(view) == 8


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
    code = ("import sys; import paper_1702_03781_gb300.harp, paper_1702_03781_gb300.synthesis, "
            "paper_1702_03781_gb300.replicas, paper_1702_03781_gb300.roofline; "
            "assert 'oracle' not in sys.modules, 'oracle imported'")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)


def test_library_sources_do_not_reference_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        src = open(os.path.join(csrc, f), errors="replace").read()
        assert "oracle" not in src.lower(), f


class _FakeCudaTensor:
    """Stands in for a CUDA tensor: only the two members the marshalling reads."""
    is_cuda = True

    def __init__(self, addr):
        self.addr = addr

    def data_ptr(self):
        return self.addr


def test_batch_descriptor_carries_the_device_addresses():
    addrs = [0x7F0000001000, 0x7F0000002000, 0x7F0000003000, 0x7F0000004000]
    pos, coef, sb, X = (_FakeCudaTensor(a) for a in addrs)
    pr = H.HarpProblem(4, 2, 1, 1, H._ptr(pos).value, 1e8, H._ptr(coef).value,
                       H._ptr(sb).value, 4, H._ptr(X).value, 8, 0, 0, 0.0)
    assert (pr.pos, pr.coef, pr.self_blocks, pr.X) == tuple(addrs)
    assert (pr.Na, pr.Nm, pr.P, pr.Q, pr.self_stride, pr.ldx) == (4, 2, 1, 1, 4, 8)


def test_batch_descriptor_matches_the_c_layout(tmp_path):
    """The ctypes mirror of harp_problem has the C compiler's field offsets
    and size (gcc on the header itself)."""
    names = [n for n, _ in H.HarpProblem._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "harp_gb300.h"\n'
        "int main(void) {\n"
        + "".join(f'  printf("%zu\\n", offsetof(harp_problem, {n}));\n' for n in names)
        + '  printf("%zu\\n", sizeof(harp_problem));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog),
                           "-o", str(exe)])
    c = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    py = [getattr(H.HarpProblem, n).offset for n in names] + [ct.sizeof(H.HarpProblem)]
    assert py == c, dict(zip(names + ["sizeof"], zip(py, c)))


def _header_prototypes():
    src = open(os.path.join(ROOT, "include", "harp_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
    protos = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(\w+)\s*\(([^;{}]*?)\)\s*;", src, flags=re.S):
        ret, name, params = " ".join(m.group(1).split()), m.group(2), " ".join(m.group(3).split())
        if name in ("if", "while") or ret.startswith("typedef"):
            continue
        args = [] if params in ("", "void") else [a.strip() for a in params.split(",")]
        protos[name] = (ret, args)
    return protos


def _kind_of_c(decl: str) -> str:
    if "*" in decl:
        return "ptr"
    toks = decl.replace("const", "").split()
    base = " ".join(toks[:-1]) if len(toks) > 1 else toks[0]
    return {"int": "int", "long": "long", "double": "double", "char": "char",
            "unsigned": "uint", "size_t": "size_t", "harp_prec": "int"}[base]


def _kind_of_ctype(t) -> str:
    if t in (ct.c_void_p, ct.c_char_p) or (isinstance(t, type) and issubclass(t, ct._Pointer)):
        return "ptr"
    for k, v in (("int", ct.c_int), ("long", ct.c_long), ("double", ct.c_double),
                 ("char", ct.c_char), ("uint", ct.c_uint), ("size_t", ct.c_size_t)):
        if t is v:
            return k
    raise AssertionError(f"unmapped ctypes type {t}")


def test_binding_signatures_match_the_header(built):
    protos = _header_prototypes()
    L = H.lib()
    checked = 0
    for name, (ret, args) in protos.items():
        fn = getattr(L, name)
        if fn.argtypes is None:
            assert not args, f"{name}: the binding sets no argtypes for {len(args)} arguments"
            continue
        want = [_kind_of_c(a) for a in args]
        got = [_kind_of_ctype(t) for t in fn.argtypes]
        assert got == want, f"{name}: binding {got} vs header {want}"
        checked += 1
    assert checked >= 15
    # non-int results
    assert L.harp_status_string.restype is ct.c_char_p
    assert L.harp_kernel_launches.restype is ct.c_ulonglong


def test_outputs_must_have_the_layout_the_library_writes():
    h = object.__new__(H.Harp)
    h._h, h.device, h.max_N, h.max_nrhs = ct.c_void_p(0), 0, 64, 16
    p = synth.tiny()
    pos, coef, sb = (torch.from_numpy(p.pos), torch.from_numpy(p.coef),
                     torch.from_numpy(p.self_blocks))
    # row-major, wrong dtype, wrong shape: refused before anything else
    for bad in (torch.empty((p.N, p.N), dtype=torch.complex64),
                H.colmajor_empty(p.N, p.N, torch.complex128, "cpu"),
                H.colmajor_empty(p.N, p.N - 1, torch.complex64, "cpu")):
        with pytest.raises(ValueError, match="out must be"):
            h.fill(pos, p.freq_hz, coef, sb, prec="mixed", out=bad)
    Z = H.colmajor_empty(p.N, p.N, torch.complex128, "cpu")
    with pytest.raises(ValueError, match="out must be"):
        h.solve(Z, None, nrhs=p.Na, prec="fp64", out=torch.empty((p.N, p.Na), dtype=torch.complex128))
    # a padded column-major view is accepted (the host-tensor refusal comes next)
    big = H.colmajor_empty(p.N + 8, p.Na, torch.complex128, "cpu")
    with pytest.raises(ValueError, match="CUDA tensor"):
        h.solve(Z, None, nrhs=p.Na, prec="fp64", out=big[:p.N, :])
    assert H._check_out(big[:p.N, :], p.N, p.Na, torch.complex128) is not None


def test_solve_refuses_a_matrix_of_the_wrong_precision():
    h = object.__new__(H.Harp)
    h._h, h.device, h.max_N, h.max_nrhs = ct.c_void_p(0), 0, 64, 16
    Z128 = H.colmajor_empty(8, 8, torch.complex128, "cpu")
    Z64 = H.colmajor_empty(8, 8, torch.complex64, "cpu")
    with pytest.raises(ValueError, match="complex64"):
        h.solve(Z128, None, nrhs=2, prec="mixed")
    with pytest.raises(ValueError, match="complex128"):
        h.solve(Z64, None, nrhs=2, prec="fp64")
    # the matching precision reaches the pointer marshalling (host tensors refused there)
    with pytest.raises(ValueError, match="CUDA tensor"):
        h.solve(Z64, None, nrhs=2, prec="mixed")


def test_malformed_shapes_are_refused_before_the_library_reads_them():
    """A self-block table for fewer antennas, a coefficient table of another
    Nm, or vectors of the wrong length would make a kernel read past a
    device buffer: the binding refuses them first."""
    h = object.__new__(H.Harp)
    h._h, h.device, h.max_N, h.max_nrhs = ct.c_void_p(0), 0, 64, 16
    p = synth.tiny()
    pos, coef, sb = (torch.from_numpy(p.pos), torch.from_numpy(p.coef),
                     torch.from_numpy(p.self_blocks))
    cases = [
        (dict(self_blocks=sb[:-1]), "self_blocks must be"),
        (dict(self_blocks=sb[:, :-1, :]), "self_blocks must be"),
        (dict(coef=coef[:, :-1]), "coef must be"),
        (dict(coef=coef[:, :, :-1]), "coef must be"),
        (dict(pos=pos[:, :1]), "pos must be"),
        (dict(pos=pos[:0]), "pos must be"),
    ]
    for kw, msg in cases:
        a = dict(pos=pos, coef=coef, self_blocks=sb)
        a.update(kw)
        with pytest.raises(ValueError, match=msg):
            h.fill(a["pos"], p.freq_hz, a["coef"], a["self_blocks"], prec="fp64")
        with pytest.raises(ValueError, match=msg):
            H.BatchItem(a["pos"], p.freq_hz, a["coef"], a["self_blocks"])
    # one shared block and one block per antenna are both accepted
    assert H._self_layout(sb[0], p.Na, p.Nm)[1] == 0
    assert H._self_layout(sb, p.Na, p.Nm)[1] == p.Nm * p.Nm

    X = torch.zeros((p.N, p.Na), dtype=torch.complex128)
    with pytest.raises(ValueError, match="X must be"):
        H.port_objective(X[:-1], p.Na, p.Nm)
    with pytest.raises(ValueError, match="X must be"):
        h.fill_adjoint(pos, p.freq_hz, coef, X, X[:-1])
    with pytest.raises(ValueError, match="Lam must be"):
        h.fill_adjoint(pos, p.freq_hz, coef, X[:, :-1], X)
    with pytest.raises(ValueError, match="Lam must be"):
        H.fill_adjoint_noalloc(pos, p.freq_hz, coef, X[:, :-1], X)
    with pytest.raises(ValueError, match="out must be"):
        H.fill_adjoint_noalloc(pos, p.freq_hz, coef, X, X,
                               out=torch.empty((p.Na, 3), dtype=torch.float64))
    Z = H.colmajor_empty(p.N, p.N, torch.complex128, "cpu")
    with pytest.raises(ValueError, match="square"):
        h.solve(Z[:, :-1], None, nrhs=p.Na, prec="fp64")
    with pytest.raises(ValueError, match="V must be"):
        h.solve(Z, X[:-1], prec="fp64")
    with pytest.raises(ValueError, match="V must be"):
        h.residual(Z, X.to(torch.complex64), X[:, :-1])


def test_valid_calls_pass_every_check_up_to_the_device_pointers():
    """The shapes the tests and the bench use pass validation: with host
    tensors the only refusal left is the device-memory one."""
    h = object.__new__(H.Harp)
    h._h, h.device, h.max_N, h.max_nrhs = ct.c_void_p(0), 0, 64, 16
    p = synth.tiny()
    pos, coef, sb = (torch.from_numpy(p.pos), torch.from_numpy(p.coef),
                     torch.from_numpy(p.self_blocks))
    X = H.colmajor_empty(p.N, p.Na, torch.complex128, "cpu")
    Z64 = H.colmajor_empty(p.N, p.N, torch.complex128, "cpu")
    Z32 = H.colmajor_empty(p.N, p.N, torch.complex64, "cpu")
    calls = [
        lambda: h.fill(pos, p.freq_hz, coef, sb, prec="fp64"),
        lambda: h.fill(pos, p.freq_hz, coef, sb[0], prec="mixed"),
        lambda: h.fill(pos, p.freq_hz, coef, sb, prec="mixed", out=Z32),
        lambda: h.solve(Z64, None, nrhs=p.Na, prec="fp64", out=X),
        lambda: h.solve(Z32, None, nrhs=p.Na, prec="mixed", max_iter=10),
        lambda: h.solve(Z32, torch.zeros((p.N, 9), dtype=torch.complex128), prec="mixed"),
        lambda: h.solve(None, torch.zeros((p.N, 9), dtype=torch.complex128), prec="fp64",
                        trans="T"),
        lambda: h.residual(Z64, X.to(torch.complex64), X),
        lambda: h.fill_adjoint(pos, p.freq_hz, coef, X, X),
        lambda: H.fill_adjoint_noalloc(pos, p.freq_hz, coef, X, X),
        lambda: H.port_objective(X, p.Na, p.Nm),
        lambda: H.solve_batch([], [H.BatchItem(pos, p.freq_hz, coef, sb)]),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="CUDA tensor"):
            call()
