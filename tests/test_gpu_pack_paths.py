"""Operand packing paths of the tensor-core engine.  By default the packs of
t2 views copy from the BF16 image of t2 made once per residual, and sources
contiguous along k go through the warp-per-row kernel; DCSD_PACK_GENERIC=1
sends every pack through the tiled FP64 kernel.  Both make the same BF16
operands (the image holds exactly the parts the FP64 kernel computes), so the
residuals must be identical bit for bit: one to six split products, CCSD and
DCSD, both references, shapes with ragged k runs (V not a multiple of 8)."""
import os

import numpy as np
import pytest

from synth import make_system, random_amplitudes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


def _residual(P, s, T, prec, method, ref, generic):
    old = os.environ.get("DCSD_PACK_GENERIC")
    os.environ["DCSD_PACK_GENERIC"] = "1" if generic else "0"
    try:
        eng = P.Engine.from_system(s)
    finally:
        if old is None:
            del os.environ["DCSD_PACK_GENERIC"]
        else:
            os.environ["DCSD_PACK_GENERIC"] = old
    R, W, dE = eng.residual(eng.to_device(T), ref=ref, method=method, precision=prec)
    out = [x.cpu().numpy() for x in R], W, dE
    eng.close()
    return out


@pytest.mark.parametrize("dims,seed", [((6, 40, 64), 5), ((5, 29, 45), 7)])
@pytest.mark.parametrize("prec", [1, 2, 4])
@pytest.mark.parametrize("method,ref", [(0, 0), (1, 0), (1, 1)])
def test_pack_paths_give_identical_residuals(P, dims, seed, prec, method, ref):
    s = make_system(dims, seed=seed)
    T = random_amplitudes(s, seed=seed + 100, ref=ref, scale1=0.02, scale2=0.02)
    R1, W1, E1 = _residual(P, s, T, prec, method, ref, False)
    R0, W0, E0 = _residual(P, s, T, prec, method, ref, True)
    for a, b in zip(R1, R0):
        assert np.array_equal(a, b)
    assert W1 == W0 and E1 == E0
