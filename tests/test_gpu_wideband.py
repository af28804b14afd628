"""GPU parity of the batched wideband solve: the station layout at several
of the 64 frequencies over 50-350 MHz (MBF count 6..20, so uneven systems of
1536..5120 unknowns), solved together by the batch scheduler on several
workers, each against the FP64 oracle (relative error <= 1e-10)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("inverses", [2, 1])
def test_wideband_batch_matches_oracle(inverses):
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300 import harp as H
    probs = synth.wideband(64)
    pick = [63, 40, 20, 0, 9]  # Nm 20, 15, 10, 6, 8: largest first
    d = "cuda:0"
    items = [H.BatchItem(torch.from_numpy(probs[i].pos).to(d), probs[i].freq_hz,
                         torch.from_numpy(probs[i].coef).to(d),
                         torch.from_numpy(probs[i].self_blocks).to(d)) for i in pick]
    max_N = max(it.N for it in items)
    ctxs = [H.Harp(0, max_N=max_N, max_nrhs=256) for _ in range(3)]
    for c in ctxs:
        c.set_knob("inverses", inverses)  # 1: built beside each factorisation
    H.solve_batch(ctxs, items, prec="mixed")
    for i, it in zip(pick, items):
        p = probs[i]
        assert it.status == 0 and it.iters >= 1
        Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
        Xo = oracle.solve(Zo, p.V)
        X = it.X.cpu().numpy()
        assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-10, (i, p.Nm)
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("i", [10, 21, 32, 50, 63])
def test_wideband_products_stay_on_tensor_cores(i):
    """Every FP32 product of tensor-core shape in the factorisation, the
    factor inverses built beside it and the refinement runs on the tensor
    cores at sizes whose N / 64 is not a multiple of 3 (the workspace split
    in three for the side stream and the two inverse chains must keep each
    part's TMA base 16-byte aligned), and the result meets the parity bar."""
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300 import harp as H
    p = synth.wideband(64)[i]
    d = "cuda:0"
    with H.Harp(0, max_N=p.N, max_nrhs=p.Na) as h:
        before = h.tc_fallbacks()
        Z = h.fill(torch.from_numpy(p.pos).to(d), p.freq_hz, torch.from_numpy(p.coef).to(d),
                   torch.from_numpy(p.self_blocks).to(d), prec="mixed")
        X, info = h.solve(Z, None, nrhs=p.Na, prec="mixed")
        assert h.tc_fallbacks() == before, (i, p.N)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xo = oracle.solve(Zo, p.V)
    Xg = X.cpu().numpy()
    assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= 1e-10
