"""Python binding of libharp_gb300.so (argument marshalling only).

Every step of the fill, the solve and the adjoint runs in the library's CUDA
kernels; this module only moves torch tensors (device memory) and streams
across the C ABI declared in include/harp_gb300.h. It never falls back to a
CPU path: if the library is missing or fails to load, `lib()` raises.

Matrices are column-major at the ABI. A column-major N x N buffer appears in
torch as the transpose view of a row-major tensor, so the tensors returned
here index naturally (Z[i, j] is row i, column j) with strides (1, ld).
"""
from __future__ import annotations

import ctypes as ct
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libharp_gb300.so")

FP64, MIXED_3XTF32, MIXED_TF32, FP32 = 0, 1, 2, 3
PREC = {"fp64": FP64, "mixed": MIXED_3XTF32, "mixed_3xtf32": MIXED_3XTF32,
        "mixed_tf32": MIXED_TF32, "fp32": FP32}

HARP_OK = 0
HARP_E_COINCIDENT = 0x40000001
HARP_E_NOCONV = 0x40000002
HARP_E_TIMEOUT = 0x40000003
HARP_E_CUDA = 0x40000004
HARP_E_NOMEM = 0x40000005
HARP_E_UNSUPPORTED = 0x40000006
HARP_E_STATE = 0x40000007
HARP_E_NONFINITE = 0x40000008

# harp_ctx_set_option: how the mixed refinement forms its FP64 residual, and
# how the FP32 factorisation pivots its panels
HARP_OPT_RESIDUAL = 1
RESIDUAL = {"slices": 0, "ff": 1}
HARP_OPT_PIVOT = 2
PIVOT = {"partial": 0, "tournament": 1, "block": 2}
HARP_OPT_PIVOT_FALLBACKS = 3
# tile-shape knobs of a context (the autotuner's search space) and the
# device time of the last batch
HARP_OPT_PANEL_ROWS = 4
HARP_OPT_FILL_CHUNK = 5
HARP_OPT_SPLITK_MAX = 6
HARP_OPT_BATCH_DEVICE_US = 7
HARP_OPT_TC_FALLBACKS = 8
HARP_OPT_INVERSES = 9
HARP_OPT_FILL_CLUSTERS = 10
HARP_OPT_FILL64 = 11
HARP_OPT_ADJOINT_G = 12
KNOBS = {"panel_rows": HARP_OPT_PANEL_ROWS, "fill_chunk": HARP_OPT_FILL_CHUNK,
         "splitk_max": HARP_OPT_SPLITK_MAX, "inverses": HARP_OPT_INVERSES,
         "fill_clusters": HARP_OPT_FILL_CLUSTERS, "fill64": HARP_OPT_FILL64,
         "adjoint_g": HARP_OPT_ADJOINT_G}

_lib = None


class HarpProblem(ct.Structure):
    """Mirror of the C struct harp_problem (one problem of a batch)."""
    _fields_ = [("Na", ct.c_int), ("Nm", ct.c_int), ("P", ct.c_int), ("Q", ct.c_int),
                ("pos", ct.c_void_p), ("freq_hz", ct.c_double), ("coef", ct.c_void_p),
                ("self_blocks", ct.c_void_p), ("self_stride", ct.c_long), ("X", ct.c_void_p),
                ("ldx", ct.c_int), ("status", ct.c_int), ("iters", ct.c_int),
                ("resid", ct.c_double)]


class HarpError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        msg = lib().harp_status_string(status).decode()
        extra = ""
        if status == HARP_E_CUDA:
            extra = f" (cuda error {lib().harp_last_cuda_error()})"
        super().__init__(f"{fn} returned {status:#x}: {msg}{extra}")


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run python -m paper_1702_03781_gb300.build)")
        L = ct.CDLL(LIB_PATH)
        vp, i, d, l = ct.c_void_p, ct.c_int, ct.c_double, ct.c_long
        L.harp_status_string.argtypes = [i]
        L.harp_status_string.restype = ct.c_char_p
        L.harp_last_cuda_error.restype = i
        L.harp_kernel_launches.restype = ct.c_ulonglong
        L.harp_ctx_create.argtypes = [ct.POINTER(vp), i, i, i]
        L.harp_ctx_destroy.argtypes = [vp]
        L.harp_ctx_z64.argtypes = [vp, ct.POINTER(vp), ct.POINTER(i)]
        L.harp_fill.argtypes = [vp, i, i, i, i, vp, d, vp, vp, l, vp, i, i, vp]
        L.mbf_solve.argtypes = [vp, i, vp, i, vp, i, i, vp, i, ct.c_char, i, d, i,
                                ct.POINTER(i), ct.POINTER(d), vp]
        L.harp_fill_adjoint.argtypes = [vp, i, i, i, i, vp, d, vp, vp, vp, i, i, vp, i, vp]
        L.harp_solve_batch.argtypes = [ct.POINTER(vp), i, ct.POINTER(HarpProblem), i, i, d, i]
        L.harp_solve_batch.restype = i
        L.harp_port_objective.argtypes = [i, i, vp, i, vp, vp, vp, i, vp]
        L.harp_port_objective.restype = i
        L.harp_port_impedance.argtypes = [vp, i, i, vp, i, vp, i, vp, vp, i, vp, i, vp]
        L.harp_port_impedance.restype = i
        L.harp_fill_adjoint_noalloc.argtypes = [i, i, i, i, vp, d, vp, vp, vp, i, i, vp, i, vp]
        L.harp_fill_adjoint_noalloc.restype = i
        L.harp_profile_begin.argtypes = [vp, ct.c_uint]
        L.harp_profile_end.argtypes = [vp, vp, vp, vp]
        L.harp_ctx_set_option.argtypes = [vp, i, i]
        L.harp_ctx_get_option.argtypes = [vp, i, ct.POINTER(i)]
        L.harp_residual.argtypes = [vp, i, vp, i, vp, i, vp, i, i, vp, i, ct.c_char, vp]
        L.harp_wait_check.argtypes = [vp, i, vp]
        L.harp_ctx_sync.argtypes = [vp, vp]
        L.harp_eep.argtypes = [vp, i, i, vp, d, vp, i, i, i, vp, vp, vp, vp, vp]
        L.harp_eep.restype = i
        L.harp_pattern_error.argtypes = [l, vp, vp, d, vp, vp]
        L.harp_pattern_error.restype = i
        L.harp_model_fit.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp]
        L.harp_model_fit.restype = i
        L.harp_tessellate.argtypes = [i, vp, d, d, i, vp, vp, vp, vp, vp, l, ct.POINTER(i),
                                      ct.POINTER(l), vp]
        L.harp_tessellate.restype = i
        L.harp_solve_tessellated.argtypes = [ct.POINTER(vp), i, i, i, i, i, vp, d, vp, vp, l, i,
                                             vp, vp, vp, vp, vp, i, i, d, i]
        L.harp_solve_tessellated.restype = i
        L.harp_ri_pairs.argtypes = [i, vp, d, l, vp, vp, ct.POINTER(l), vp]
        L.harp_ri_pairs.restype = i
        L.harp_ri_fill.argtypes = [i, i, i, i, vp, d, vp, vp, l, vp, vp, l, vp, i, vp, vp]
        L.harp_ri_fill.restype = i
        L.harp_bsr_to_dense.argtypes = [i, i, vp, vp, l, vp, i, vp, i, vp]
        L.harp_bsr_to_dense.restype = i
        for fn in ("harp_ctx_create", "harp_ctx_destroy", "harp_ctx_sync", "harp_ctx_z64",
                   "harp_fill",
                   "mbf_solve", "harp_fill_adjoint", "harp_profile_begin", "harp_profile_end",
                   "harp_ctx_set_option", "harp_ctx_get_option", "harp_residual",
                   "harp_wait_check"):
            getattr(L, fn).restype = i
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernels the library has launched so far in this process."""
    return int(lib().harp_kernel_launches())


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


def _stream(stream) -> ct.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ct.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ct.c_void_p:
    """Device address of a CUDA tensor (NULL for None). Every tensor argument
    of the ABI is device memory; a host tensor is refused here, never handed
    to a kernel."""
    if t is None:
        return ct.c_void_p(0)
    if not t.is_cuda:
        raise ValueError(f"expected a CUDA tensor (device memory), got one on {t.device}")
    return ct.c_void_p(t.data_ptr())


def colmajor_empty(rows: int, cols: int, dtype, device) -> torch.Tensor:
    """An uninitialised column-major (rows x cols) tensor (strides (1, rows))."""
    return torch.empty((cols, rows), dtype=dtype, device=device).T


def as_colmajor(x: torch.Tensor) -> torch.Tensor:
    """x itself if it is column-major with unit row stride, else a copy."""
    if x.dim() == 2 and x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0]):
        return x
    return x.T.contiguous().T


def _model_shape(pos: torch.Tensor, coef: torch.Tensor) -> tuple[int, int, int, int]:
    """(Na, Nm, P, Q) of positions (Na, 2) and a coefficient table
    (Nm, Nm, 2P+1, Q+1); anything else is refused before the library reads
    past a buffer."""
    if pos.dim() != 2 or pos.shape[1] != 2 or pos.shape[0] < 1:
        raise ValueError(f"pos must be (Na, 2) with Na >= 1, got {tuple(pos.shape)}")
    if coef.dim() != 4 or coef.shape[0] != coef.shape[1] or coef.shape[0] < 1 \
            or coef.shape[2] % 2 != 1 or coef.shape[3] < 1:
        raise ValueError(f"coef must be (Nm, Nm, 2P+1, Q+1), got {tuple(coef.shape)}")
    return pos.shape[0], coef.shape[0], (coef.shape[2] - 1) // 2, coef.shape[3] - 1


def _self_layout(self_blocks: torch.Tensor, Na: int, Nm: int) -> tuple[torch.Tensor, int]:
    """Self blocks in ABI layout (column-major per antenna) and their stride:
    (Na, Nm, Nm) [antenna, T, S], or one shared (Nm, Nm) block (stride 0)."""
    if tuple(self_blocks.shape) == (Nm, Nm):
        return self_blocks.to(torch.complex128).T.contiguous(), 0
    if tuple(self_blocks.shape) == (Na, Nm, Nm):
        return self_blocks.to(torch.complex128).transpose(1, 2).contiguous(), Nm * Nm
    raise ValueError(f"self_blocks must be ({Na}, {Nm}, {Nm}) or ({Nm}, {Nm}), "
                     f"got {tuple(self_blocks.shape)}")


def _expect_shape(name: str, t: torch.Tensor, shape: tuple) -> None:
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be {tuple(shape)}, got {tuple(t.shape)}")


def _check_out(out: torch.Tensor, rows: int, cols: int, dtype) -> torch.Tensor:
    """A caller-given output: rows x cols of `dtype`, column-major with a
    leading dimension >= rows (the layout the library writes)."""
    if tuple(out.shape) != (rows, cols) or out.dtype != dtype:
        raise ValueError(f"out must be {rows} x {cols} {dtype}, got {tuple(out.shape)} {out.dtype}")
    if out.stride(0) != 1 or out.stride(1) < max(1, rows):
        raise ValueError(f"out must be column-major (strides (1, ld >= {rows})), "
                         f"got strides {tuple(out.stride())}")
    return out


def _ld(x: torch.Tensor) -> int:
    return max(int(x.stride(1)), int(x.shape[0]), 1)


def _check(fn: str, status: int, ok=(HARP_OK,)):
    if status not in ok:
        raise HarpError(fn, status)
    return status


class Harp:
    """A library context on one CUDA device: owns the device workspace for
    systems of up to max_N unknowns and max_nrhs right-hand sides."""

    def __init__(self, device: int | None = None, max_N: int = 3072, max_nrhs: int = 256):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        self.max_N = int(max_N)
        self.max_nrhs = int(max_nrhs)
        h = ct.c_void_p()
        _check("harp_ctx_create", lib().harp_ctx_create(ct.byref(h), self.device, self.max_N,
                                                         self.max_nrhs))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().harp_ctx_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ct.c_void_p:
        return self._h

    def sync(self, stream=None) -> None:
        """Wait for the work enqueued on `stream` and raise HarpError on the
        context's pending device status (coincident antennas or non-finite
        entries found by fill(), a bounded wait that gave up), clearing it."""
        _check("harp_ctx_sync", lib().harp_ctx_sync(self._h, _stream(stream)))

    def z64(self, N: int) -> torch.Tensor:
        """The context's FP64 reduced matrix as a column-major (N x N) view."""
        p, ld = ct.c_void_p(), ct.c_int()
        _check("harp_ctx_z64", lib().harp_ctx_z64(self._h, ct.byref(p), ct.byref(ld)))
        # Wrap the raw device pointer without copying.
        storage = _alias_storage(p.value, ld.value * self.max_N * 16, self.device)
        full = torch.empty(0, dtype=torch.complex128, device=f"cuda:{self.device}")
        full.set_(storage, 0, (self.max_N, ld.value), (ld.value, 1))
        return full.T[:N, :N]

    # -- fill ---------------------------------------------------------------
    def fill(self, pos: torch.Tensor, freq_hz: float, coef: torch.Tensor,
             self_blocks: torch.Tensor, prec="fp64", out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
        """Reduced MBF matrix: complex128 (fp64) or complex64 (other modes),
        column-major N x N. self_blocks: (Na, Nm, Nm) [antenna, T, S] or one
        shared (Nm, Nm) block. Asynchronous: coincident antennas or
        non-finite entries are raised by the next solve() or by sync()."""
        pr = _prec(prec)
        Na, Nm, P, Q = _model_shape(pos, coef)
        pos = pos.to(torch.float64).contiguous()
        coef = coef.to(torch.complex128).contiguous()
        N = Na * Nm
        sb, stride = _self_layout(self_blocks, Na, Nm)
        dt = torch.complex128 if pr == FP64 else torch.complex64
        Z = colmajor_empty(N, N, dt, pos.device) if out is None else _check_out(out, N, N, dt)
        _check("harp_fill", lib().harp_fill(self._h, Na, Nm, P, Q, _ptr(pos), float(freq_hz),
                                            _ptr(coef), _ptr(sb), stride, _ptr(Z), _ld(Z), pr,
                                            _stream(stream)))
        return Z

    # -- solve --------------------------------------------------------------
    def solve(self, Z: torch.Tensor | None, V: torch.Tensor | None = None, nrhs: int | None = None,
              prec="fp64", trans: str = "N", tol: float = 0.0, max_iter: int = 10,
              out: torch.Tensor | None = None, stream=None, allow_noconv: bool = False):
        """X (complex128, column-major N x nrhs) and {'iters', 'resid', 'status'}.
        V = None solves for the port excitations (nrhs ports)."""
        pr = _prec(prec)
        if Z is not None:
            # the library reads c128 for FP64 and c64 for the other modes
            want = torch.complex128 if pr == FP64 else torch.complex64
            if Z.dtype != want:
                raise ValueError(f"Z must be {want} for prec={prec!r}, got {Z.dtype}")
            if Z.dim() != 2 or Z.shape[0] != Z.shape[1]:
                raise ValueError(f"Z must be square, got {tuple(Z.shape)}")
            Z = as_colmajor(Z)
            N = Z.shape[0]
        elif V is not None:
            N = V.shape[0]
        else:
            raise ValueError("need Z or V to know N")
        if V is not None:
            if V.dim() != 2 or V.shape[0] != N:
                raise ValueError(f"V must be ({N}, nrhs), got {tuple(V.shape)}")
            V = as_colmajor(V.to(torch.complex128))
            nrhs = V.shape[1]
        if nrhs is None:
            raise ValueError("nrhs is required when V is None")
        dev = Z.device if Z is not None else V.device
        X = (colmajor_empty(N, nrhs, torch.complex128, dev) if out is None
             else _check_out(out, N, nrhs, torch.complex128))
        it, res = ct.c_int(0), ct.c_double(0.0)
        st = lib().mbf_solve(self._h, N, _ptr(Z), _ld(Z) if Z is not None else N, _ptr(V),
                             _ld(V) if V is not None else N, nrhs, _ptr(X), _ld(X),
                             trans.encode(), pr, float(tol), int(max_iter), ct.byref(it),
                             ct.byref(res), _stream(stream))
        ok = (HARP_OK, HARP_E_NOCONV) if allow_noconv else (HARP_OK,)
        _check("mbf_solve", st, ok)
        return X, {"iters": it.value, "resid": res.value, "status": st}

    # -- refinement residual -------------------------------------------------
    def set_residual(self, method: str):
        """'slices' (tensor cores, exact integer digits) or 'ff' (float-float)."""
        _check("harp_ctx_set_option",
               lib().harp_ctx_set_option(self._h, HARP_OPT_RESIDUAL, RESIDUAL[method]))

    def residual_method(self) -> str:
        v = ct.c_int(-1)
        _check("harp_ctx_get_option", lib().harp_ctx_get_option(self._h, HARP_OPT_RESIDUAL,
                                                                ct.byref(v)))
        return {k: m for m, k in RESIDUAL.items()}[v.value]

    def set_pivot(self, rule: str):
        """Pivot rule of the FP32 factorisation's panels: 'partial',
        'tournament' (communication-avoiding LU) or 'block' (restricted to
        the diagonal blocks, checked by the refinement)."""
        _check("harp_ctx_set_option",
               lib().harp_ctx_set_option(self._h, HARP_OPT_PIVOT, PIVOT[rule]))

    def pivot_rule(self) -> str:
        v = ct.c_int(-1)
        _check("harp_ctx_get_option", lib().harp_ctx_get_option(self._h, HARP_OPT_PIVOT,
                                                                ct.byref(v)))
        return {k: m for m, k in PIVOT.items()}[v.value]

    def set_knob(self, name: str, value: int):
        """A scheduling knob: 'panel_rows', 'fill_chunk', 'splitk_max' (tile
        shapes), 'inverses' (0 after, 1 beside, 2 beside unless batched) or
        'fill_clusters' (GPC-sized clusters of the background FP64 fill, 0:
        about half) or 'fill64' (how the background fill forms the
        FP64-accurate matrix: 0 float-float, 1 exact digit products on the
        tensor cores, 2 digit products inside a batch of several contexts)
        or 'adjoint_g' (the mixed adjoint's G = Lambda X^T: 1 digit products
        on the tensor cores, 0 double-float on the CUDA cores)."""
        _check("harp_ctx_set_option",
               lib().harp_ctx_set_option(self._h, KNOBS[name], int(value)))

    def knob(self, name: str) -> int:
        v = ct.c_int(-1)
        _check("harp_ctx_get_option", lib().harp_ctx_get_option(self._h, KNOBS[name],
                                                                ct.byref(v)))
        return v.value

    def batch_device_ms(self) -> float:
        """Device time of the last solve_batch led by this context."""
        v = ct.c_int(-1)
        _check("harp_ctx_get_option", lib().harp_ctx_get_option(
            self._h, HARP_OPT_BATCH_DEVICE_US, ct.byref(v)))
        return v.value / 1e3

    def tc_fallbacks(self) -> int:
        """Process-wide count of FP32 products of tensor-core shape that ran
        on the CUDA cores (0 when every workspace and tensor map was fine)."""
        v = ct.c_int(-1)
        _check("harp_ctx_get_option", lib().harp_ctx_get_option(
            self._h, HARP_OPT_TC_FALLBACKS, ct.byref(v)))
        return v.value

    def pivot_fallbacks(self) -> int:
        """Factorisations of this context whose block-restricted pivots were
        redone with partial pivoting."""
        v = ct.c_int(-1)
        _check("harp_ctx_get_option", lib().harp_ctx_get_option(
            self._h, HARP_OPT_PIVOT_FALLBACKS, ct.byref(v)))
        return v.value

    def residual(self, Z: torch.Tensor, X: torch.Tensor, V: torch.Tensor, trans: str = "N",
                 stream=None) -> torch.Tensor:
        """R = V - op(Z) X (complex128) for FP64 Z, FP32 X (complex64), FP64 V."""
        if X.dim() != 2:
            raise ValueError(f"X must be (N, nrhs), got {tuple(X.shape)}")
        N, nrhs = X.shape
        _expect_shape("Z", Z, (N, N))
        _expect_shape("V", V, (N, nrhs))
        Z = as_colmajor(Z.to(torch.complex128))
        X = as_colmajor(X.to(torch.complex64))
        V = as_colmajor(V.to(torch.complex128))
        R = colmajor_empty(N, nrhs, torch.complex128, X.device)
        _check("harp_residual", lib().harp_residual(
            self._h, N, _ptr(Z), _ld(Z), _ptr(X), _ld(X), _ptr(V), _ld(V), nrhs, _ptr(R), _ld(R),
            trans.encode(), _stream(stream)))
        return R

    def wait_check(self, release: bool, stream=None) -> int:
        """Status of one bounded device wait on an mbarrier that is released
        (HARP_OK) or never arrived at (HARP_E_TIMEOUT after ~0.5 s)."""
        return lib().harp_wait_check(self._h, 1 if release else 0, _stream(stream))

    # -- patterns (Section II-C) --------------------------------------------
    def eep(self, pos: torch.Tensor, freq_hz: float, X: torch.Tensor, Nm: int,
            ux: torch.Tensor, uy: torch.Tensor, F: torch.Tensor, out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
        """Embedded element patterns (2, nports, D) complex64 of the ports
        whose MBF coefficients are the columns of X (N x nports), for the
        directions (ux, uy) and the MBF patterns F (2, D, Nm)."""
        if pos.dim() != 2 or pos.shape[1] != 2:
            raise ValueError(f"pos must be (Na, 2), got {tuple(pos.shape)}")
        Na = pos.shape[0]
        if X.dim() != 2 or X.shape[0] != Na * Nm:
            raise ValueError(f"X must be ({Na * Nm}, nports), got {tuple(X.shape)}")
        if ux.dim() != 1 or tuple(uy.shape) != tuple(ux.shape):
            raise ValueError("ux and uy must be (D,)")
        D = ux.shape[0]
        _expect_shape("F", F, (2, D, Nm))
        nports = X.shape[1]
        pos = pos.to(torch.float64).contiguous()
        X = as_colmajor(X.to(torch.complex128))
        ux = ux.to(torch.float64).contiguous()
        uy = uy.to(torch.float64).contiguous()
        F = F.to(torch.complex128).contiguous()
        if out is None:
            out = torch.empty((2, nports, D), dtype=torch.complex64, device=pos.device)
        elif tuple(out.shape) != (2, nports, D) or out.dtype != torch.complex64 \
                or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous (2, {nports}, {D}) complex64 tensor")
        _check("harp_eep", lib().harp_eep(
            self._h, Na, Nm, _ptr(pos), float(freq_hz), _ptr(X), _ld(X), nports, D, _ptr(ux),
            _ptr(uy), _ptr(F), _ptr(out), _stream(stream)))
        return out

    # -- adjoint ------------------------------------------------------------
    def fill_adjoint(self, pos: torch.Tensor, freq_hz: float, coef: torch.Tensor,
                     Lam: torch.Tensor, X: torch.Tensor, prec="fp64", stream=None) -> torch.Tensor:
        """grad (Na, 2) float64 of J from the adjoint Lambda and solution X."""
        pr = _prec(prec)
        Na, Nm, P, Q = _model_shape(pos, coef)
        if X.dim() != 2 or X.shape[0] != Na * Nm:
            raise ValueError(f"X must be ({Na * Nm}, nrhs), got {tuple(X.shape)}")
        _expect_shape("Lam", Lam, tuple(X.shape))
        pos = pos.to(torch.float64).contiguous()
        coef = coef.to(torch.complex128).contiguous()
        Lam = as_colmajor(Lam.to(torch.complex128))
        X = as_colmajor(X.to(torch.complex128))
        if _ld(Lam) != _ld(X):
            Lam, X = Lam.T.contiguous().T, X.T.contiguous().T
        ld = _ld(X)
        grad = torch.empty((Na, 2), dtype=torch.float64, device=pos.device)
        _check("harp_fill_adjoint", lib().harp_fill_adjoint(
            self._h, Na, Nm, P, Q, _ptr(pos), float(freq_hz), _ptr(coef), _ptr(Lam), _ptr(X), ld,
            X.shape[1], _ptr(grad), pr, _stream(stream)))
        return grad


def _alias_storage(ptr: int, nbytes: int, device: int):
    # torch.from_dlpack over a DLPack capsule would also work; a cuda array
    # interface dict is the simplest zero-copy alias.
    class _A:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                    "version": 3, "strides": None}
    t = torch.as_tensor(_A(), device=f"cuda:{device}")
    return t.untyped_storage()


class BatchItem:
    """One problem of solve_batch, with its device inputs in ABI layout and
    its output X (column-major N x Na complex128)."""

    def __init__(self, pos, freq_hz, coef, self_blocks):
        self.Na, self.Nm, self.P, self.Q = _model_shape(pos, coef)
        self.pos = pos.to(torch.float64).contiguous()
        self.coef = coef.to(torch.complex128).contiguous()
        self.freq_hz = float(freq_hz)
        self.sb, self.stride = _self_layout(self_blocks, self.Na, self.Nm)
        self.N = self.Na * self.Nm
        self.X = colmajor_empty(self.N, self.Na, torch.complex128, self.pos.device)
        self.status = self.iters = 0
        self.resid = 0.0


def solve_batch(contexts, items, prec="mixed", tol: float = 0.0, max_iter: int = 10,
                check: bool = True):
    """Fill and solve every item (each for its port excitations) with the
    library's batch scheduler: one worker thread and stream per context."""
    arr = (HarpProblem * len(items))()
    for k, it in enumerate(items):
        arr[k] = HarpProblem(it.Na, it.Nm, it.P, it.Q, _ptr(it.pos).value, it.freq_hz,
                             _ptr(it.coef).value, _ptr(it.sb).value, it.stride,
                             _ptr(it.X).value, _ld(it.X), 0, 0, 0.0)
    hs = (ct.c_void_p * len(contexts))(*[c.handle.value for c in contexts])
    torch.cuda.synchronize()  # inputs prepared on torch's stream are ready
    st = lib().harp_solve_batch(hs, len(contexts), arr, len(items), _prec(prec), float(tol),
                                int(max_iter))
    for k, it in enumerate(items):
        it.status, it.iters, it.resid = arr[k].status, arr[k].iters, arr[k].resid
    if check:
        _check("harp_solve_batch", st)
    return st


def port_objective(X: torch.Tensor, Na: int, Nm: int, want_P: bool = True, want_W: bool = True,
                   stream=None):
    """(P, J, W) of the port objective: P = E^T X (Na x Na), J = sum |P|^2
    (0-d float64 tensor on the device), W = E conj(P) (N x Na, the adjoint
    right-hand side). Computed by the library's kernels."""
    _expect_shape("X", X, (Na * Nm, Na))
    X = as_colmajor(X.to(torch.complex128))
    dev = X.device
    N = Na * Nm
    P = colmajor_empty(Na, Na, torch.complex128, dev) if want_P else None
    W = colmajor_empty(N, Na, torch.complex128, dev) if want_W else None
    J = torch.empty((), dtype=torch.float64, device=dev)
    _check("harp_port_objective", lib().harp_port_objective(
        Na, Nm, _ptr(X), _ld(X), _ptr(P), _ptr(J), _ptr(W), _ld(W) if W is not None else N,
        _stream(stream)))
    return P, J, W


def port_impedance(ctx: "Harp", P: torch.Tensor, Nm: int, stream=None):
    """(Y, J, G, W) of the impedance reading of the port objective: Y = P^-1
    (FP64 solve on `ctx`, whose factorisation it replaces), J = sum |Y|^2
    (0-d float64 tensor), G = -Y^H Y Y^H, W = E conj(G) (N x Na, the adjoint
    right-hand side). Computed by the library's kernels."""
    if P.dim() != 2 or P.shape[0] != P.shape[1]:
        raise ValueError(f"P must be square, got {tuple(P.shape)}")
    Na = P.shape[0]
    P = as_colmajor(P.to(torch.complex128))
    dev = P.device
    Y = colmajor_empty(Na, Na, torch.complex128, dev)
    G = colmajor_empty(Na, Na, torch.complex128, dev)
    W = colmajor_empty(Na * Nm, Na, torch.complex128, dev)
    J = torch.empty((), dtype=torch.float64, device=dev)
    _check("harp_port_impedance", lib().harp_port_impedance(
        ctx.handle, Na, Nm, _ptr(P), _ld(P), _ptr(Y), _ld(Y), _ptr(J), _ptr(G), _ld(G), _ptr(W),
        _ld(W), _stream(stream)))
    return Y, J, G, W


NOALLOC_MAX_NA = 512


def fill_adjoint_noalloc(pos: torch.Tensor, freq_hz: float, coef: torch.Tensor, Lam: torch.Tensor,
                         X: torch.Tensor, prec="fp64", out: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """The adjoint gradient through the allocation-free entry point (no
    context; per-pair scratch in a fixed device array of the library, at
    most NOALLOC_MAX_NA antennas). `out` (Na, 2) float64 may be given so the
    call itself allocates nothing either."""
    pr = _prec(prec)
    Na, Nm, P, Q = _model_shape(pos, coef)
    if X.dim() != 2 or X.shape[0] != Na * Nm:
        raise ValueError(f"X must be ({Na * Nm}, nrhs), got {tuple(X.shape)}")
    _expect_shape("Lam", Lam, tuple(X.shape))
    if out is not None and (tuple(out.shape) != (Na, 2) or out.dtype != torch.float64
                            or not out.is_contiguous()):
        raise ValueError(f"out must be a contiguous ({Na}, 2) float64 tensor")
    # The entry point has no context: it runs on the current CUDA device and
    # takes that device's scratch array, so every tensor (and the stream) must
    # live on one device, which is made current for the call.
    named = {"pos": pos, "coef": coef, "Lam": Lam, "X": X}
    if out is not None:
        named["out"] = out
    for name, t in named.items():
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor (device memory), got one on {t.device}")
    devs = {t.device for t in named.values()}
    if len(devs) != 1:
        raise ValueError("pos, coef, Lam, X and out must be on one CUDA device, got "
                         + ", ".join(f"{n}: {t.device}" for n, t in named.items()))
    dev = pos.device
    if stream is not None and stream.device != dev:
        raise ValueError(f"stream is on {stream.device}, the tensors on {dev}")
    with torch.cuda.device(dev):
        pos = pos.to(torch.float64).contiguous()
        coef = coef.to(torch.complex128).contiguous()
        Lam = as_colmajor(Lam.to(torch.complex128))
        X = as_colmajor(X.to(torch.complex128))
        if _ld(Lam) != _ld(X):
            Lam, X = Lam.T.contiguous().T, X.T.contiguous().T
        grad = torch.empty((Na, 2), dtype=torch.float64, device=dev) if out is None else out
        _check("harp_fill_adjoint_noalloc", lib().harp_fill_adjoint_noalloc(
            Na, Nm, P, Q, _ptr(pos), float(freq_hz), _ptr(coef), _ptr(Lam), _ptr(X), _ld(X),
            X.shape[1], _ptr(grad), pr, _stream(stream)))
    return grad


def pattern_error(E: torch.Tensor, Eref: torch.Tensor, norm: float, stream=None) -> torch.Tensor:
    """Eq. 8 per direction: sqrt(|dE_theta|^2 + |dE_phi|^2) / norm for
    complex64 patterns (2, ...) of the same shape; float32 (...)."""
    if E.shape != Eref.shape or E.dim() < 1 or E.shape[0] != 2:
        raise ValueError("E and Eref must have the same shape (2, ...)")
    if E.dtype != torch.complex64 or Eref.dtype != torch.complex64:
        raise ValueError("E and Eref must be complex64")
    E, Eref = E.contiguous(), Eref.contiguous()
    eps = torch.empty(E.shape[1:], dtype=torch.float32, device=E.device)
    n = eps.numel()
    _check("harp_pattern_error", lib().harp_pattern_error(n, _ptr(E), _ptr(Eref), float(norm),
                                                          _ptr(eps), _stream(stream)))
    return eps


def model_fit(d: torch.Tensor, B: torch.Tensor, P: int, Q: int, stream=None):
    """HARP model construction: coefficients (Nm, Nm, 2P+1, Q+1) complex128
    and the rms residual (Nm, Nm) from samples B (Nm, Nm, Nd, N_alpha) on
    the grid d (Nd,) x alpha_a = 2 pi a / N_alpha."""
    if B.dim() != 4 or B.shape[0] != B.shape[1]:
        raise ValueError(f"B must be (Nm, Nm, Nd, N_alpha), got {tuple(B.shape)}")
    Nm, _, Nd, Nal = B.shape
    _expect_shape("d", d, (Nd,))
    if not B.is_cuda or not d.is_cuda:
        raise ValueError("expected CUDA tensors (device memory)")
    d = d.to(torch.float64).contiguous()
    B = B.to(torch.complex128).contiguous()
    coef = torch.empty((Nm, Nm, 2 * P + 1, Q + 1), dtype=torch.complex128, device=B.device)
    rms = torch.empty((Nm, Nm), dtype=torch.float64, device=B.device)
    _check("harp_model_fit", lib().harp_model_fit(Nm, P, Q, Nd, Nal, _ptr(d), _ptr(B),
                                                  _ptr(coef), _ptr(rms), _stream(stream)))
    return coef, rms


class Tessellation:
    """Tiles (T, 2) int32 and the CSR lists of the tiles' inner members and
    subarrays (device int32 tensors), from harp_tessellate."""

    def __init__(self, tiles, inner_ptr, inner_idx, outer_ptr, outer_idx):
        self.tiles, self.inner_ptr, self.inner_idx = tiles, inner_ptr, inner_idx
        self.outer_ptr, self.outer_idx = outer_ptr, outer_idx

    @property
    def n_tiles(self) -> int:
        return self.tiles.shape[0]

    def sizes(self):
        """Subarray sizes (antennas) per tile, on the host."""
        op = self.outer_ptr.cpu()
        return (op[1:] - op[:-1]).tolist()


def tessellate(pos: torch.Tensor, R_in: float, R_ext: float, stream=None) -> Tessellation:
    """Hexagonal tiles of the array (inner circumradius R_in, extension
    R_ext) with their inner members and subarrays."""
    if pos.dim() != 2 or pos.shape[1] != 2 or pos.shape[0] < 1:
        raise ValueError(f"pos must be (Na, 2), got {tuple(pos.shape)}")
    pos = pos.to(torch.float64).contiguous()
    Na, dev = pos.shape[0], pos.device
    max_t, cap = max(16, Na), 4 * Na
    for _ in range(3):
        tiles = torch.empty((max_t, 2), dtype=torch.int32, device=dev)
        ip = torch.empty(max_t + 1, dtype=torch.int32, device=dev)
        ii = torch.empty(Na, dtype=torch.int32, device=dev)
        op = torch.empty(max_t + 1, dtype=torch.int32, device=dev)
        oi = torch.empty(max(1, cap), dtype=torch.int32, device=dev)
        nt, tot = ct.c_int(0), ct.c_long(0)
        st = lib().harp_tessellate(Na, _ptr(pos), float(R_in), float(R_ext), max_t, _ptr(tiles),
                                   _ptr(ip), _ptr(ii), _ptr(op), _ptr(oi), cap, ct.byref(nt),
                                   ct.byref(tot), _stream(stream))
        if st == HARP_E_UNSUPPORTED and (nt.value > max_t or tot.value > cap):
            max_t, cap = max(max_t, nt.value), max(cap, tot.value)
            continue
        _check("harp_tessellate", st)
        T = nt.value
        return Tessellation(tiles[:T], ip[:T + 1], ii, op[:T + 1], oi[:tot.value])
    raise RuntimeError("harp_tessellate: list sizes did not settle")


def solve_tessellated(contexts, tess: Tessellation, pos: torch.Tensor, freq_hz: float,
                      coef: torch.Tensor, self_blocks: torch.Tensor, prec="mixed",
                      tol: float = 0.0, max_iter: int = 10) -> torch.Tensor:
    """The (Na Nm) x Na currents of every port by the tessellation approach
    (each column nonzero on its tile's subarray only)."""
    Na, Nm, P, Q = _model_shape(pos, coef)
    pos = pos.to(torch.float64).contiguous()
    coef = coef.to(torch.complex128).contiguous()
    sb, stride = _self_layout(self_blocks, Na, Nm)
    X = colmajor_empty(Na * Nm, Na, torch.complex128, pos.device)
    hs = (ct.c_void_p * len(contexts))(*[c.handle.value for c in contexts])
    torch.cuda.synchronize()  # inputs prepared on torch's stream are ready
    _check("harp_solve_tessellated", lib().harp_solve_tessellated(
        hs, len(contexts), Na, Nm, P, Q, _ptr(pos), float(freq_hz), _ptr(coef), _ptr(sb), stride,
        tess.n_tiles, _ptr(tess.inner_ptr), _ptr(tess.inner_idx), _ptr(tess.outer_ptr),
        _ptr(tess.outer_idx), _ptr(X), _ld(X), _prec(prec), float(tol), int(max_iter)))
    return X


def ri_pairs(pos: torch.Tensor, RI: float, stream=None):
    """Block-CSR structure (row_ptr int64 (Na+1,), col_idx int32 (nnzb,)) of
    the kept blocks under a radius of influence RI."""
    if pos.dim() != 2 or pos.shape[1] != 2 or pos.shape[0] < 1:
        raise ValueError(f"pos must be (Na, 2), got {tuple(pos.shape)}")
    pos = pos.to(torch.float64).contiguous()
    Na = pos.shape[0]
    cap = Na * Na
    row_ptr = torch.empty(Na + 1, dtype=torch.int64, device=pos.device)
    col_idx = torch.empty(cap, dtype=torch.int32, device=pos.device)
    nnzb = ct.c_long(0)
    _check("harp_ri_pairs", lib().harp_ri_pairs(Na, _ptr(pos), float(RI), cap, _ptr(row_ptr),
                                                _ptr(col_idx), ct.byref(nnzb), _stream(stream)))
    return row_ptr, col_idx[:nnzb.value].clone()


def ri_fill(pos, freq_hz, coef, self_blocks, row_ptr, col_idx, prec="fp64", stream=None):
    """The kept blocks' values (nnzb, Nm, Nm) (each block column-major:
    [b, S, T] in torch's row-major view), complex128 for fp64, complex64
    otherwise; raises on coincident antennas or non-finite entries."""
    Na, Nm, P, Q = _model_shape(pos, coef)
    pos = pos.to(torch.float64).contiguous()
    coef = coef.to(torch.complex128).contiguous()
    sb, stride = _self_layout(self_blocks, Na, Nm)
    pr = _prec(prec)
    nnzb = col_idx.shape[0]
    dt = torch.complex128 if pr == FP64 else torch.complex64
    vals = torch.empty((nnzb, Nm, Nm), dtype=dt, device=pos.device)
    flag = torch.zeros(1, dtype=torch.int32, device=pos.device)
    _check("harp_ri_fill", lib().harp_ri_fill(
        Na, Nm, P, Q, _ptr(pos), float(freq_hz), _ptr(coef), _ptr(sb), stride, _ptr(row_ptr),
        _ptr(col_idx), nnzb, _ptr(vals), pr, _ptr(flag), _stream(stream)))
    f = int(flag.item())
    if f & 1:
        raise HarpError("harp_ri_fill", HARP_E_COINCIDENT)
    if f & 2:
        raise HarpError("harp_ri_fill", HARP_E_NONFINITE)
    return vals


def bsr_to_dense(row_ptr, col_idx, vals, Na: int, out: torch.Tensor | None = None, stream=None):
    """The block-sparse matrix in dense column-major storage (N x N)."""
    nnzb, Nm, _ = vals.shape
    N = Na * Nm
    pr = FP64 if vals.dtype == torch.complex128 else FP32
    Z = colmajor_empty(N, N, vals.dtype, vals.device) if out is None else out
    _check("harp_bsr_to_dense", lib().harp_bsr_to_dense(
        Na, Nm, _ptr(row_ptr), _ptr(col_idx), nnzb, _ptr(vals.contiguous()), pr, _ptr(Z), _ld(Z),
        _stream(stream)))
    return Z
