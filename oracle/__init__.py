"""FP64 CPU oracle for the HARP fill and MBF solve -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package. The product path (the CUDA library and its binding)
never imports it, and it never imports the product path.

Thin ctypes wrapper over liboracle.so (harp_oracle.c); numpy arrays in and
out. Matrices cross the boundary column-major (Fortran order).
"""
from __future__ import annotations

import ctypes as ct
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB points the wrapper at another build of harp_oracle.c
        # (the mutation tests load deliberately broken copies this way).
        path = os.environ.get("ORACLE_LIB") or _build.build(quiet=True)
        L = ct.CDLL(path)
        dp, ip, vp = ct.POINTER(ct.c_double), ct.POINTER(ct.c_int), ct.c_void_p
        L.oracle_fill.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int, vp, ct.c_double, vp, vp,
                                  ct.c_int, vp, ct.c_long, vp, ct.c_long]
        L.oracle_fill.restype = ct.c_int
        L.oracle_lu.argtypes = [ct.c_int, vp, ct.c_long, vp]
        L.oracle_lu.restype = ct.c_int
        L.oracle_lu_solve.argtypes = [ct.c_int, vp, ct.c_long, vp, ct.c_int, vp, ct.c_long, ct.c_char]
        L.oracle_lu_solve.restype = None
        L.oracle_port_objective.argtypes = [ct.c_int, ct.c_int, vp, ct.c_long, vp]
        L.oracle_port_objective.restype = ct.c_double
        L.oracle_grad_from_adjoint.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int, vp, ct.c_double,
                                               vp, ct.c_int, vp, vp, ct.c_long, ct.c_int, vp]
        L.oracle_grad_from_adjoint.restype = None
        L.oracle_port_objective_grad.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int, vp,
                                                 ct.c_double, vp, ct.c_int, vp, ct.c_long, vp, vp]
        L.oracle_port_objective_grad.restype = ct.c_int
        L.oracle_eep.argtypes = [ct.c_int, ct.c_int, vp, ct.c_double, vp, ct.c_long, ct.c_int,
                                 ct.c_int, vp, vp, vp, vp]
        L.oracle_eep.restype = None
        L.oracle_pattern_error.argtypes = [ct.c_int, vp, vp, ct.c_double, vp]
        L.oracle_pattern_error.restype = None
        L.oracle_wavenumber.argtypes = [ct.c_double]
        L.oracle_wavenumber.restype = ct.c_double
        L.oracle_num_threads.restype = ct.c_int
        L.oracle_set_threads.argtypes = [ct.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ct.c_void_p) if a is not None else None


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def wavenumber(freq_hz: float) -> float:
    """k = 2 pi f / c0 of the phase factor e^{-jkr} (Eq. 1, 4)."""
    return float(lib().oracle_wavenumber(freq_hz))


def _self_cm(self_blocks: np.ndarray) -> tuple[np.ndarray, int]:
    """(Na, Nm, Nm) [a, T, S] -> column-major per antenna, stride Nm*Nm.
    A single (Nm, Nm) block is shared by every antenna (stride 0)."""
    if self_blocks.ndim == 2:
        return np.ascontiguousarray(self_blocks.T, dtype=np.complex128), 0
    sb = np.ascontiguousarray(self_blocks.transpose(0, 2, 1), dtype=np.complex128)
    return sb, sb.shape[1] * sb.shape[2]


def fill(pos, freq_hz, coef, self_blocks, ff=None, dvar: int = 1) -> np.ndarray:
    """Reduced matrix Z (N x N complex128, Fortran order): Eq. 1, 3, 4."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.complex128)
    Nm, _, np_, nq = coef.shape
    P, Q = (np_ - 1) // 2, nq - 1
    Na = pos.shape[0]
    N = Na * Nm
    sb, stride = _self_cm(self_blocks)
    ffa = None if ff is None else np.ascontiguousarray(ff, dtype=np.complex128)
    Z = np.zeros((N, N), dtype=np.complex128, order="F")
    rc = lib().oracle_fill(Na, Nm, P, Q, _p(pos), float(freq_hz), _p(coef), _p(ffa), int(dvar),
                           _p(sb), stride, _p(Z), N)
    if rc != 0:
        raise ValueError("oracle_fill: coincident antennas (r == 0)")
    return Z


def lu(Z: np.ndarray):
    """(LU, ipiv, info): partial-pivot LU of a copy of Z, the direct solve of
    the reduced system (Section II-B); textbook right-looking elimination."""
    A = np.array(Z, dtype=np.complex128, order="F", copy=True)
    N = A.shape[0]
    ipiv = np.zeros(N, dtype=np.int32)
    info = lib().oracle_lu(N, _p(A), N, _p(ipiv))
    return A, ipiv, int(info)


def lu_solve(LU, ipiv, B, trans: str = "N") -> np.ndarray:
    """X with op(Z) X = B from the factors of `lu` (forward and back
    substitution; trans 'T' solves with Z^T for the adjoint)."""
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    N = LU.shape[0]
    lib().oracle_lu_solve(N, _p(LU), N, _p(ipiv), X.shape[1], _p(X), N, trans.encode())
    return X


def solve(Z, V, trans: str = "N") -> np.ndarray:
    """Z X = V (or Z^T X = V) for every right-hand side: the MBF coefficients
    for each port excitation (Section II-B, II-C)."""
    A, ipiv, info = lu(Z)
    if info:
        raise np.linalg.LinAlgError(f"oracle_lu: zero pivot at column {info - 1}")
    return lu_solve(A, ipiv, V, trans)


def port_objective(X, Na: int, Nm: int):
    """(J, P): the port response P = E^T X (row m*Nm of column n, MBF 0 of
    each antenna) and J = sum |P_mn|^2, the synthesis objective (Section V)."""
    X = np.asarray(X, dtype=np.complex128, order="F")
    Pm = np.zeros((Na, Na), dtype=np.complex128, order="F")
    J = lib().oracle_port_objective(Na, Nm, _p(X), X.shape[0], _p(Pm))
    return float(J), Pm


def grad_from_adjoint(pos, freq_hz, coef, Lam, X, dvar: int = 1) -> np.ndarray:
    """dJ/d(positions) (Na, 2) from the adjoint Lambda and the solution X:
    -2 Re sum over pair blocks of (Lambda X^T) . dZ/dDelta, with dZ from Eq. 3, 4
    differentiated in r and alpha."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.complex128)
    Nm, _, np_, nq = coef.shape
    Lam = np.asarray(Lam, dtype=np.complex128, order="F")
    X = np.asarray(X, dtype=np.complex128, order="F")
    g = np.zeros((pos.shape[0], 2), dtype=np.float64)
    lib().oracle_grad_from_adjoint(pos.shape[0], Nm, (np_ - 1) // 2, nq - 1, _p(pos), float(freq_hz),
                                   _p(coef), int(dvar), _p(Lam), _p(X), X.shape[0], X.shape[1], _p(g))
    return g


def port_objective_grad(pos, freq_hz, coef, self_blocks, dvar: int = 1, want_grad: bool = True):
    """(J, grad (Na, 2) or None) for J = sum |(E^T Z^{-1} E)_mn|^2."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.complex128)
    Nm, _, np_, nq = coef.shape
    sb, stride = _self_cm(self_blocks)
    J = ct.c_double(0.0)
    g = np.zeros((pos.shape[0], 2), dtype=np.float64) if want_grad else None
    rc = lib().oracle_port_objective_grad(pos.shape[0], Nm, (np_ - 1) // 2, nq - 1, _p(pos),
                                          float(freq_hz), _p(coef), int(dvar), _p(sb), stride,
                                          ct.byref(J), _p(g))
    if rc != 0:
        raise ValueError(f"oracle_port_objective_grad failed: {rc}")
    return J.value, g


def port_impedance_objective_grad(pos, freq_hz, coef, self_blocks, dvar: int = 1,
                                  want_grad: bool = True):
    """(J, grad (Na, 2) or None) for the impedance reading of the synthesis
    objective (Section V): J = sum_mn |(P^{-1})_mn|^2, where P = E^T Z^{-1} E
    is the port response and E selects MBF 0 of every antenna.

    Forward, step by step: X = Z^{-1} E and Y = P^{-1}, both with this
    oracle's LU.

    Adjoint: dY = -Y dP Y gives dJ = 2 Re tr(G^H dP) with G = -Y^H Y Y^H.
    Since dP = -E^T Z^{-1} dZ X, the adjoint is Lambda = Z^{-T} E conj(G), and
    the gradient is the same contraction as for the admittance reading, with
    E conj(G) in place of E conj(P)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    Na, Nm = pos.shape[0], np.shape(coef)[0]
    Z = fill(pos, freq_hz, coef, self_blocks, dvar=dvar)
    A, ipiv, info = lu(Z)
    if info:
        raise np.linalg.LinAlgError(f"oracle_lu: zero pivot at column {info - 1}")
    E = np.zeros((Na * Nm, Na), dtype=np.complex128)
    E[np.arange(Na) * Nm, np.arange(Na)] = 1.0
    X = lu_solve(A, ipiv, E)
    P = E.T @ X
    Y = solve(P, np.eye(Na, dtype=np.complex128))
    J = float(np.sum(np.abs(Y) ** 2))
    if not want_grad:
        return J, None
    G = -(Y.conj().T @ Y @ Y.conj().T)
    Lam = lu_solve(A, ipiv, E @ np.conj(G), trans="T")
    return J, grad_from_adjoint(pos, freq_hz, coef, Lam, X, dvar=dvar)


def relerr(a, b) -> float:
    """Frobenius relative error ||a - b|| / ||b||."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def eep(pos, freq_hz, X, Nm: int, ux, uy, F) -> np.ndarray:
    """Embedded element patterns of every column (port) of X, Eq. 5 term by
    term (Section II-C): E[comp, m, d] for comp 0 = theta, 1 = phi.
    X: (Na*Nm, nports); ux, uy: (D,) direction cosines; F: (2, D, Nm) MBF
    patterns."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    X = np.asfortranarray(X, dtype=np.complex128)
    ux = np.ascontiguousarray(ux, dtype=np.float64)
    uy = np.ascontiguousarray(uy, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.complex128)
    Na, nports, D = pos.shape[0], X.shape[1], ux.shape[0]
    assert X.shape[0] == Na * Nm and F.shape == (2, D, Nm) and uy.shape == (D,)
    E = np.zeros((2, nports, D), dtype=np.complex128)
    lib().oracle_eep(Na, Nm, _p(pos), float(freq_hz), _p(X), X.shape[0], nports, D, _p(ux),
                     _p(uy), _p(F), _p(E))
    return E


def pattern_error(E, Eref, norm: float) -> np.ndarray:
    """Eq. 8 (Section III-A): sqrt(|dE_theta|^2 + |dE_phi|^2) / norm per
    direction; E, Eref: (2, ...) theta and phi components."""
    E = np.ascontiguousarray(E, dtype=np.complex128)
    Eref = np.ascontiguousarray(Eref, dtype=np.complex128)
    assert E.shape == Eref.shape and E.shape[0] == 2
    n = E[0].size
    eps = np.zeros(n)
    lib().oracle_pattern_error(n, _p(E), _p(Eref), float(norm), _p(eps))
    return eps.reshape(E.shape[1:])


def model_fit(d, B, P: int, Q: int):
    """HARP model construction (Section II-A, Eq. 2-3; Section II-B for the
    sampling and the DFT): from samples B[T, S, l, a] of the complementary
    interaction on a polar grid -- d_l regular in d = 1/r, alpha_a = 2 pi a /
    N_alpha regular in angle -- the coefficients c[T, S, p + P, q] of
    B(d, alpha) = sum_p e^{j p alpha} sum_q c_pq d^q:
      1. the DFT over alpha gives each harmonic's radial samples,
         b_p(d_l) = (1 / N_alpha) sum_a B(d_l, alpha_a) e^{-j p alpha_a};
      2. a least-squares polynomial fit in d (library QR/SVD solve of the
         Vandermonde system V[l, q] = d_l^q) gives c_pq.
    Returns (coef, rms) with rms[T, S] the root-mean-square residual of the
    fitted model on the samples."""
    d = np.asarray(d, dtype=np.float64)
    B = np.asarray(B, dtype=np.complex128)
    Nm, Nm2, Nd, Na_ = B.shape
    assert Nm == Nm2 and Nd == d.size
    alpha = 2.0 * np.pi * np.arange(Na_) / Na_
    ps = np.arange(-P, P + 1)
    W = np.exp(-1j * np.outer(alpha, ps)) / Na_            # (N_alpha, 2P+1)
    V = d[:, None] ** np.arange(Q + 1)[None, :]             # (Nd, Q+1)
    coef = np.zeros((Nm, Nm, 2 * P + 1, Q + 1), dtype=np.complex128)
    rms = np.zeros((Nm, Nm))
    Ea = np.exp(1j * np.outer(alpha, ps))                   # (N_alpha, 2P+1)
    for T in range(Nm):
        for S in range(Nm):
            b = B[T, S] @ W                                  # (Nd, 2P+1)
            for k in range(2 * P + 1):
                coef[T, S, k] = np.linalg.lstsq(V, b[:, k], rcond=None)[0]
            model = (V @ coef[T, S].T) @ Ea.T                # (Nd, N_alpha)
            rms[T, S] = np.sqrt(np.mean(np.abs(model - B[T, S]) ** 2))
    return coef, rms


# ---- Tessellation (Section II-D, Fig. 3; Section IV-B) -------------------
# Reading: hexagons are flat-topped with circumradius R (vertex distance);
# the inner hexagons of circumradius R_in tile the plane with centres
# x = 1.5 R_in i, y = sqrt(3) R_in (j + (i mod 2) / 2); an antenna belongs
# to the tile of the nearest centre (smallest (i, j) on ties), and a tile's
# subarray is every antenna inside the concentric hexagon of circumradius
# R_in + R_ext (boundary included). The arithmetic below is plain IEEE FP64
# without fused multiply-adds, the same sequence the library uses, so the
# membership decisions are identical.
SQRT3 = 1.7320508075688772


def hex_center(i: int, j: int, R: float):
    return 1.5 * R * i, SQRT3 * R * (j + 0.5 * (i & 1))


def in_hexagon(dx: float, dy: float, R: float) -> bool:
    """Inside the flat-topped hexagon of circumradius R (or on its edge)."""
    ax, ay = abs(dx), abs(dy)
    return ay <= 0.5 * SQRT3 * R and SQRT3 * ax + ay <= SQRT3 * R


def hex_tile(x: float, y: float, R: float):
    """(i, j) of the nearest centre of the R-hexagon lattice."""
    i0 = math.floor(x / (1.5 * R))
    best = None
    for i in (i0 - 1, i0, i0 + 1, i0 + 2):
        j0 = math.floor(y / (SQRT3 * R) - 0.5 * (i & 1))
        for j in (j0 - 1, j0, j0 + 1, j0 + 2):
            cx, cy = hex_center(i, j, R)
            ddx, ddy = x - cx, y - cy
            d2 = ddx * ddx + ddy * ddy
            if best is None or d2 < best[0] or (d2 == best[0] and (i, j) < best[1]):
                best = (d2, (i, j))
    return best[1]


def tessellate(pos, R_in: float, R_ext: float):
    """Tiles (i, j) sorted, and per tile the sorted antenna indices of its
    inner part and of its subarray (inner and extended parts)."""
    pos = np.asarray(pos, dtype=np.float64)
    tij = [hex_tile(float(x), float(y), R_in) for x, y in pos]
    tiles = sorted(set(tij))
    inner = [[a for a in range(len(pos)) if tij[a] == t] for t in tiles]
    outer = []
    for t in tiles:
        cx, cy = hex_center(t[0], t[1], R_in)
        outer.append([a for a in range(len(pos))
                      if in_hexagon(float(pos[a, 0]) - cx, float(pos[a, 1]) - cy, R_in + R_ext)])
    return tiles, inner, outer


def solve_tessellated(pos, freq_hz, coef, self_blocks, R_in: float, R_ext: float):
    """The currents of every port by the tessellation approach: each tile's
    subarray filled (Eq. 3-4) and solved for the excitation of each of its
    inner antennas; column m of the result holds the currents of port m on
    the subarray of m's tile (zero elsewhere)."""
    pos = np.asarray(pos, dtype=np.float64)
    Na, Nm = pos.shape[0], coef.shape[0]
    X = np.zeros((Na * Nm, Na), dtype=np.complex128)
    tiles, inner, outer = tessellate(pos, R_in, R_ext)
    for t in range(len(tiles)):
        sub = outer[t]
        sb = self_blocks if self_blocks.ndim == 2 else self_blocks[sub]
        Z = fill(pos[sub], freq_hz, coef, sb)
        rows = (np.asarray(sub)[:, None] * Nm + np.arange(Nm)[None, :]).ravel()
        for m in inner[t]:
            v = np.zeros(len(sub) * Nm, dtype=np.complex128)
            v[sub.index(m) * Nm] = 1.0
            X[rows, m] = solve(Z, v[:, None])[:, 0]
    return X


# ---- Radius of influence (Section II-D, Section IV-A) ---------------------
def ri_pairs(pos, RI: float):
    """Block-sparse structure of the reduced matrix under a radius of
    influence: block (m, n) is kept when m == n or the antennas are closer
    than RI (r^2 < RI^2 with r^2 = dx*dx + dy*dy, each operation rounded in
    FP64). Returns CSR (row_ptr (Na+1,), col_idx) with each row's columns
    in increasing order."""
    pos = np.asarray(pos, dtype=np.float64)
    Na = pos.shape[0]
    R2 = float(RI) * float(RI)
    row_ptr, cols = [0], []
    for m in range(Na):
        for n in range(Na):
            dx = float(pos[m, 0]) - float(pos[n, 0])
            dy = float(pos[m, 1]) - float(pos[n, 1])
            if m == n or dx * dx + dy * dy < R2:
                cols.append(n)
        row_ptr.append(len(cols))
    return np.array(row_ptr, dtype=np.int64), np.array(cols, dtype=np.int64)


def ri_fill(pos, freq_hz, coef, self_blocks, RI: float):
    """The reduced matrix under the radius of influence: the full fill with
    every block (m, n) of pairs at r >= RI set to zero."""
    Z = fill(pos, freq_hz, coef, self_blocks)
    Nm = coef.shape[0]
    row_ptr, cols = ri_pairs(pos, RI)
    keep = np.zeros((len(row_ptr) - 1,) * 2, dtype=bool)
    for m in range(len(row_ptr) - 1):
        keep[m, cols[row_ptr[m]:row_ptr[m + 1]]] = True
    return Z * np.kron(keep, np.ones((Nm, Nm), dtype=bool))
