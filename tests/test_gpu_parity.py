"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances (written here, derived in the design notes):
  * FP64 fill: every entry within 1e-13 of the largest entry (the GPU forms
    e^{j p alpha} by repeated multiplication, the oracle by cexp).
  * FP32 fill: Frobenius relative error <= 1e-5.
  * solutions (FP64 and mixed with refinement): Frobenius relative error
    <= 1e-10 against the oracle's X.
  * self blocks and the block index mapping: bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def harp():
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300.harp import Harp
    h = Harp(0, max_N=3072, max_nrhs=256)
    yield h
    h.close()


def _dev(p):
    d = "cuda:0"
    return (torch.from_numpy(p.pos).to(d), torch.from_numpy(p.coef).to(d),
            torch.from_numpy(p.self_blocks).to(d))


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mk", [lambda: synth.tiny(), lambda: synth.small(37, 5, P=3, Q=2),
                                lambda: synth.small(70, 3, P=2, Q=4, seed_cfg=21),
                                lambda: synth.physical(synth.small(37, 5, P=3, Q=2))])
def test_fill_fp64_matches_oracle(harp, mk):
    p = mk()
    pos, coef, sb = _dev(p)
    Z = _np(harp.fill(pos, p.freq_hz, coef, sb, prec="fp64"))
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert np.max(np.abs(Z - Zo)) <= 1e-13 * np.max(np.abs(Zo))
    # self blocks bit-exact
    for a in range(p.Na):
        sl = slice(a * p.Nm, (a + 1) * p.Nm)
        assert np.array_equal(Z[sl, sl], p.self_blocks[a])


def test_fill_fp32_matches_oracle(harp):
    p = synth.station()
    pos, coef, sb = _dev(p)
    Z = _np(harp.fill(pos, p.freq_hz, coef, sb, prec="fp32")).astype(np.complex128)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert _rel(Z, Zo) <= 1e-5


def test_fill_mixed_writes_fp32_matrix_and_fp64_accurate_z64(harp):
    """The mixed fill returns the FP32 evaluation (the factorisation's input)
    and fills the context's Z64 on its own stream; harp_ctx_z64 (harp.z64)
    waits for that fill, which must then be FP64-accurate."""
    p = synth.station()
    pos, coef, sb = _dev(p)
    Z32 = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    Zf = harp.fill(pos, p.freq_hz, coef, sb, prec="fp32")
    Z64 = harp.z64(p.N)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    z64 = _np(Z64)
    assert np.max(np.abs(z64 - Zo)) <= 1e-13 * np.max(np.abs(Zo))
    assert torch.equal(Z32, Zf)
    assert _rel(_np(Z32).astype(np.complex128), Zo) <= 1e-5


def test_fill_shared_self_block(harp):
    p = synth.small(20, 3)
    pos, coef, _ = _dev(p)
    shared = torch.from_numpy(p.self_blocks[7]).to("cuda:0")
    Z = _np(harp.fill(pos, p.freq_hz, coef, shared, prec="fp64"))
    for a in range(p.Na):
        sl = slice(a * 3, a * 3 + 3)
        assert np.array_equal(Z[sl, sl], p.self_blocks[7])


def test_fill_coincident_antennas_reported(harp):
    """The fill does not synchronise: coincident antennas are the context's
    pending status, returned by the next solve or by harp_ctx_sync."""
    from paper_1702_03781_gb300.harp import HarpError, HARP_E_COINCIDENT
    p = synth.small(6, 2)
    pos = p.pos.copy()
    pos[4] = pos[1]
    args = (torch.from_numpy(pos).cuda(), p.freq_hz, torch.from_numpy(p.coef).cuda(),
            torch.from_numpy(p.self_blocks).cuda())
    harp.fill(*args, prec="fp64")
    with pytest.raises(HarpError) as e:
        harp.sync()
    assert e.value.status == HARP_E_COINCIDENT
    harp.sync()  # reported once, then cleared
    for prec in ("fp64", "mixed"):
        Z = harp.fill(*args, prec=prec)
        with pytest.raises(HarpError) as e:
            harp.solve(Z, None, nrhs=p.Na, prec=prec)
        assert e.value.status == HARP_E_COINCIDENT
    harp.sync()


@pytest.mark.parametrize("mk", [lambda: synth.tiny(), lambda: synth.small(37, 5, P=3, Q=2),
                                lambda: synth.small(23, 7, P=2, Q=2, seed_cfg=22)])
def test_solve_fp64_matches_oracle(harp, mk):
    p = mk()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="fp64")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="fp64")
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xo = oracle.solve(Zo, p.V)
    assert _rel(_np(X), Xo) <= 1e-10


@pytest.mark.parametrize("mk", [lambda: synth.tiny(), lambda: synth.small(37, 5, P=3, Q=2),
                                lambda: synth.physical(synth.small(37, 5, P=3, Q=2))])
def test_solve_mixed_refined_matches_oracle(harp, mk):
    p = mk()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xo = oracle.solve(Zo, p.V)
    assert info["iters"] >= 1
    assert _rel(_np(X), Xo) <= 1e-10


def test_solve_general_rhs_and_transpose(harp):
    p = synth.small(30, 4, P=2, Q=2, seed_cfg=23)
    pos, coef, sb = _dev(p)
    rng = np.random.default_rng(1)
    V = synth.complex_normal(rng, (p.N, 9))
    Vt = torch.from_numpy(V).cuda()
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    for prec, zprec in (("fp64", "fp64"), ("mixed", "mixed")):
        Z = harp.fill(pos, p.freq_hz, coef, sb, prec=zprec)
        X, _ = harp.solve(Z, Vt, prec=prec)
        assert _rel(_np(X), oracle.solve(Zo, V)) <= 1e-10
        Xt, _ = harp.solve(None, Vt, prec=prec, trans="T")
        assert _rel(_np(Xt), oracle.solve(Zo, V, trans="T")) <= 1e-10


def test_zero_pivot_reported(harp):
    from paper_1702_03781_gb300.harp import HarpError
    p = synth.small(10, 3, seed_cfg=24)
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="fp64")
    Z[:, 13] = 0
    with pytest.raises(HarpError) as e:
        harp.solve(Z, None, nrhs=p.Na, prec="fp64")
    assert 1 <= e.value.status <= p.N


def test_station_fp64_and_mixed_match_oracle(harp):
    """The 256-antenna, 12-MBF station at 110 MHz in the launch configuration
    the benchmark times: both paths within 1e-10 of the oracle's X."""
    p = synth.station()
    pos, coef, sb = _dev(p)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xo = oracle.solve(Zo, p.V)
    Z64 = harp.fill(pos, p.freq_hz, coef, sb, prec="fp64")
    X64, _ = harp.solve(Z64, None, nrhs=p.Na, prec="fp64")
    assert _rel(_np(X64), Xo) <= 1e-10
    Z32 = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    Xm, info = harp.solve(Z32, None, nrhs=p.Na, prec="mixed", max_iter=10)
    assert _rel(_np(Xm), Xo) <= 1e-10
    assert info["resid"] <= np.sqrt(p.N) * 2.0 ** -53


def test_adjoint_fp64_matches_oracle_gradient(harp):
    p = synth.small(24, 3, P=2, Q=2, seed_cfg=25)
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="fp64")
    X, _ = harp.solve(Z, None, nrhs=p.Na, prec="fp64")
    Pm = _np(X)[0::p.Nm, :]
    W = np.zeros((p.N, p.Na), np.complex128)
    W[0::p.Nm, :] = np.conj(Pm)
    Lam, _ = harp.solve(None, torch.from_numpy(W).cuda(), prec="fp64", trans="T")
    g = _np(harp.fill_adjoint(pos, p.freq_hz, coef, Lam, X, prec="fp64"))
    _, go = oracle.port_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert _rel(g, go) <= 1e-10


def test_background_fill_reads_its_own_copy_of_the_inputs(harp):
    """The mixed fill's FP64 matrix is made on the context's own stream after
    harp_fill returns. The binding hands it temporaries (the self blocks in
    column-major order, a contiguous copy of a strided coefficient table)
    that go back to the allocator when fill() returns; the allocations below
    reuse and overwrite them on the caller's stream at once. Z64 must still be
    the oracle's matrix: the library works from its own copies."""
    p = synth.small(110, 7, P=2, Q=2, seed_cfg=62)
    pos, coef, sb = _dev(p)
    coef_strided = coef.permute(1, 0, 2, 3).contiguous().permute(1, 0, 2, 3)
    assert not coef_strided.is_contiguous()
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    for _ in range(3):
        harp.fill(pos, p.freq_hz, coef_strided, sb, prec="mixed")
        junk = [torch.full(t.shape, complex(1e30, -1e30), dtype=torch.complex128, device="cuda:0")
                for t in (sb, coef) for _ in range(4)]
        z64 = _np(harp.z64(p.N))
        del junk
        assert np.max(np.abs(z64 - Zo)) <= 1e-13 * np.max(np.abs(Zo))
