"""Seeded synthetic inputs for the HARP fill + MBF solve path.

This module is shared by the oracle tests and the CUDA path. It holds no
arithmetic of the method itself (no basis, no fill, no solve): only random
layouts, random coefficient tables, random self blocks and the port
right-hand sides, drawn from numpy's PCG64 so that every consumer sees the
same bytes for the same seed.

Stand-ins (the paper's SKALA element model and station layouts are not
available):

* layouts: random sequential addition in a disc with a minimum separation,
  the shape of the 256-element SKA station of Section II (Fig. 2) and the
  1500-element arrays of Section IV;
* HARP coefficients c_pq^{TS} of Eq. 3: complex normal CN(0, 1) scaled by
  2^-q (q the polynomial power), harmonic p in [-P, P], q in [0, Q];
* self blocks (diagonal blocks of the reduced matrix): CN(0, 1) with the
  off-diagonal absolute row sum plus one added to each diagonal entry;
* right-hand sides: unit voltage on MBF 0 of each antenna port (one column
  per port), the "excitation at each port" of Section II-C.

Array conventions (all arrays complex128 unless stated):

* pos: (Na, 2) float64 metres.
* coef: (Nm, Nm, 2P+1, Q+1), index [T, S, p+P, q].
* self_blocks: (Na, Nm, Nm), index [antenna, T, S].
* V: (N, Na) with N = Na * Nm; row i = m*Nm + T.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C0 = 299_792_458.0  # speed of light in vacuum, m/s


def wavelength(freq_hz: float) -> float:
    return C0 / freq_hz


def disc_layout(Na: int, radius: float, min_sep: float, seed: int,
                max_draws: int = 10_000_000) -> np.ndarray:
    """Random sequential addition of Na points in a disc of `radius` metres.

    A draw (rho = R sqrt(u), theta = 2 pi v) is rejected when it lies closer
    than `min_sep` to an accepted point. Returns (Na, 2) float64.
    """
    rng = np.random.default_rng(seed)
    cell = min_sep
    grid: dict[tuple[int, int], list[int]] = {}
    pts = np.empty((Na, 2), dtype=np.float64)
    n = 0
    draws = 0
    min_sep2 = min_sep * min_sep
    while n < Na:
        if draws >= max_draws:
            raise RuntimeError(f"disc_layout: could not place {Na} points "
                               f"(R={radius}, min_sep={min_sep}) in {max_draws} draws")
        u, v = rng.random(2)
        draws += 1
        rho = radius * math.sqrt(u)
        th = 2.0 * math.pi * v
        x, y = rho * math.cos(th), rho * math.sin(th)
        gx, gy = int(math.floor(x / cell)), int(math.floor(y / cell))
        ok = True
        for ix in range(gx - 1, gx + 2):
            for iy in range(gy - 1, gy + 2):
                for j in grid.get((ix, iy), ()):
                    dx, dy = x - pts[j, 0], y - pts[j, 1]
                    if dx * dx + dy * dy < min_sep2:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pts[n] = (x, y)
            grid.setdefault((gx, gy), []).append(n)
            n += 1
    return pts


def complex_normal(rng: np.random.Generator, shape) -> np.ndarray:
    """CN(0, 1): (N(0,1) + j N(0,1)) / sqrt(2)."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / math.sqrt(2.0)


def harp_coefficients(Nm: int, P: int, Q: int, seed: int) -> np.ndarray:
    """c[T, S, p+P, q] ~ CN(0, 1) * 2^-q, complex128, C-contiguous."""
    rng = np.random.default_rng(seed)
    c = complex_normal(rng, (Nm, Nm, 2 * P + 1, Q + 1))
    c *= (2.0 ** -np.arange(Q + 1))[None, None, None, :]
    return np.ascontiguousarray(c)


def self_blocks(Na: int, Nm: int, seed: int) -> np.ndarray:
    """(Na, Nm, Nm) blocks [antenna, T, S]: CN(0, 1) entries with the real margin
    sum_{S != T} |A_TS| + 1 added to each diagonal entry."""
    rng = np.random.default_rng(seed)
    A = complex_normal(rng, (Na, Nm, Nm))
    absrow = np.abs(A).sum(axis=2) - np.abs(np.diagonal(A, axis1=1, axis2=2))
    idx = np.arange(Nm)
    A[:, idx, idx] += absrow + 1.0
    return np.ascontiguousarray(A)


def port_rhs(Na: int, Nm: int) -> np.ndarray:
    """V = E: (N, Na) with a unit entry at row m*Nm (MBF 0 of antenna m)."""
    V = np.zeros((Na * Nm, Na), dtype=np.complex128)
    V[np.arange(Na) * Nm, np.arange(Na)] = 1.0
    return V


@dataclass
class Problem:
    """One frequency of one layout: everything the fill and solve consume."""
    name: str
    pos: np.ndarray
    freq_hz: float
    Nm: int
    P: int
    Q: int
    coef: np.ndarray
    self_blocks: np.ndarray
    V: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def Na(self) -> int:
        return self.pos.shape[0]

    @property
    def N(self) -> int:
        return self.Na * self.Nm

    @property
    def K(self) -> int:
        return (2 * self.P + 1) * (self.Q + 1)


# Seed plan: config c, layout l -> layout seed 1000c + l; coefficients of
# frequency i -> 1000c + 100 + i; self blocks of frequency i -> 1000c + 200 + i.
def _seeds(c: int, layout: int = 0, freq_index: int = 0):
    return 1000 * c + layout, 1000 * c + 100 + freq_index, 1000 * c + 200 + freq_index


def make_problem(name: str, Na: int, radius: float, min_sep: float, freq_hz: float,
                 Nm: int, P: int, Q: int, cfg: int, layout: int = 0,
                 freq_index: int = 0, pos: np.ndarray | None = None) -> Problem:
    s_lay, s_coef, s_self = _seeds(cfg, layout, freq_index)
    if pos is None:
        pos = disc_layout(Na, radius, min_sep, s_lay)
    coef = harp_coefficients(Nm, P, Q, s_coef)
    sb = self_blocks(pos.shape[0], Nm, s_self)
    V = port_rhs(pos.shape[0], Nm)
    return Problem(name, pos, freq_hz, Nm, P, Q, coef, sb, V,
                   meta=dict(cfg=cfg, layout=layout, freq_index=freq_index,
                             radius=radius, min_sep=min_sep))


F110 = 110e6


def tiny(layout: int = 0) -> Problem:
    """16 antennas in a disc of radius 3 lambda (110 MHz), min separation
    lambda/2, 4 MBFs, P = 4, Q = 3: a 64 x 64 system with 16 port RHS."""
    lam = wavelength(F110)
    return make_problem("tiny-16x4", 16, 3 * lam, 0.5 * lam, F110, 4, 4, 3, cfg=1, layout=layout)


def station(layout: int = 0, Nm: int = 12) -> Problem:
    """SKA-like station at 110 MHz: 256 antennas in a 38 m disc, min
    separation 1.5 m, 12 MBFs, P = 8, Q = 5: a 3072 x 3072 system, 256 RHS."""
    return make_problem("station-256x12", 256, 19.0, 1.5, F110, Nm, 8, 5, cfg=2, layout=layout)


def wideband_plan(n_freq: int = 64, f_lo: float = 50e6, f_hi: float = 350e6,
                  nm_lo: int = 6, nm_hi: int = 20):
    """(freq_hz, Nm) per frequency: linear in the frequency index."""
    out = []
    for i in range(n_freq):
        t = i / (n_freq - 1) if n_freq > 1 else 0.0
        out.append((f_lo + (f_hi - f_lo) * t, int(round(nm_lo + (nm_hi - nm_lo) * t))))
    return out


def wideband(n_freq: int = 64) -> list[Problem]:
    """The station layout at n_freq frequencies over 50-350 MHz, Nm 6..20."""
    pos = disc_layout(256, 19.0, 1.5, _seeds(2)[0])
    probs = []
    for i, (f, nm) in enumerate(wideband_plan(n_freq)):
        probs.append(make_problem(f"wideband-{i}", 256, 19.0, 1.5, f, nm, 8, 5,
                                  cfg=3, freq_index=i, pos=pos))
    return probs


def large(layout: int = 0) -> Problem:
    """1024 antennas in a 76 m disc, min separation 1.5 m, 16 MBFs at 110
    MHz: a 16384 x 16384 system with 1024 RHS."""
    return make_problem("large-1024x16", 1024, 38.0, 1.5, F110, 16, 8, 5, cfg=5, layout=layout)


def physical(p: Problem) -> Problem:
    """The same problem with c_{p0} = 0 for every harmonic p and MBF pair:
    without the distance-independent q = 0 part of Eq. 3, every coupling
    block decays at least as d = 1/r."""
    coef = p.coef.copy()
    coef[..., 0] = 0.0
    return Problem(p.name + "-physical", p.pos, p.freq_hz, p.Nm, p.P, p.Q,
                   np.ascontiguousarray(coef), p.self_blocks, p.V,
                   meta=dict(p.meta, physical=True))


def small(Na: int, Nm: int, P: int = 3, Q: int = 2, seed_cfg: int = 9,
          layout: int = 0, freq_hz: float = F110, min_sep: float = 1.5) -> Problem:
    """A small random problem of any shape, in a disc sized for ~40% cover."""
    radius = max(2.0 * min_sep, min_sep * math.sqrt(Na / 0.4) / 2.0 * 1.05)
    return make_problem(f"small-{Na}x{Nm}", Na, radius, min_sep, freq_hz, Nm, P, Q,
                        cfg=seed_cfg, layout=layout)


# ---- Pattern inputs (Section II-C): directions and synthetic MBF patterns.
# The SKALA MBF patterns are not available; smooth seeded stand-ins take
# their place.

def direction_grid(d_theta_deg: float = 1.0, d_phi_deg: float = 1.0):
    """Upper-hemisphere grid theta in [0, 90] deg, phi in [0, 360) deg:
    (theta, phi) in radians and the direction cosines (ux, uy), each (D,),
    theta major."""
    th = np.deg2rad(np.arange(0.0, 90.0 + 1e-9, d_theta_deg))
    ph = np.deg2rad(np.arange(0.0, 360.0 - 1e-9, d_phi_deg))
    T, Ph = np.meshgrid(th, ph, indexing="ij")
    T, Ph = T.ravel(), Ph.ravel()
    return T, Ph, np.sin(T) * np.cos(Ph), np.sin(T) * np.sin(Ph)


def mbf_patterns(Nm: int, theta: np.ndarray, phi: np.ndarray, seed: int) -> np.ndarray:
    """(2, D, Nm) complex128 patterns [comp][d][j] (comp 0 = theta, 1 = phi):
    F_j = sum_{l=0..2} a_jl cos(theta)^l e^{i m_j phi}, with seeded
    a_jl ~ CN(0,1) per component and m_j = j mod 3, smooth in both angles
    like the patterns of small antennas."""
    rng = np.random.default_rng(seed)
    a = complex_normal(rng, (2, Nm, 3))
    m = np.arange(Nm) % 3
    ct = np.cos(theta)
    powers = np.stack([np.ones_like(ct), ct, ct * ct], axis=1)  # (D, 3)
    F = np.einsum("dl,cjl->cdj", powers, a) * np.exp(1j * np.outer(phi, m))[None]
    return np.ascontiguousarray(F)


def model_grid(r_min: float = 1.5, r_max: float = 40.0, n_d: int = 24, n_alpha: int = 32):
    """The sampling grid of a HARP model build (Section II-B): n_d radii
    regular in d = 1/r between 1/r_max and 1/r_min, and n_alpha angles
    regular on [0, 2 pi). Returns d (n_d,), alpha (n_alpha,)."""
    d = np.linspace(1.0 / r_max, 1.0 / r_min, n_d)
    alpha = 2.0 * np.pi * np.arange(n_alpha) / n_alpha
    return d, alpha
