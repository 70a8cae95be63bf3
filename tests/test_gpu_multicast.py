"""The ladder contraction in clusters of two CTAs sharing each B tile by TMA
multicast (the default) against the one-CTA kernel (DCSD_TC_MULTICAST=0):
both run the same MMAs in the same order per output tile, so the residuals
must be identical bit for bit.  Sizes with an even and an odd number of
128-row tiles of stacked amplitudes (the odd one leaves the second CTA of
the last pair without rows), one to six split products, CCSD and DCSD; and
the result against the oracle."""
import os

import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import twod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


def _residual(P, s, T, prec, method, multicast):
    old = os.environ.get("DCSD_TC_MULTICAST")
    os.environ["DCSD_TC_MULTICAST"] = "1" if multicast else "0"
    try:
        eng = P.Engine.from_system(s)
    finally:
        if old is None:
            del os.environ["DCSD_TC_MULTICAST"]
        else:
            os.environ["DCSD_TC_MULTICAST"] = old
    R, W, dE = eng.residual(eng.to_device(T), method=method, precision=prec)
    out = [x.cpu().numpy() for x in R], W, dE
    eng.close()
    return out


# stacked rows 2 C(O,2) + 2 O^2: O = 8 -> 184 (2 tiles), O = 10 -> 290 (3 tiles)
@pytest.mark.parametrize("dims,seed", [((6, 40, 64), 5), ((8, 37, 50), 6)])
@pytest.mark.parametrize("prec", [1, 2, 4])
@pytest.mark.parametrize("method", [0, 1])
def test_multicast_ladder_is_bitwise_identical(P, dims, seed, prec, method):
    s = make_system(dims, seed=seed)
    T = random_amplitudes(s, seed=seed + 100, scale1=0.02, scale2=0.02)
    R1, W1, E1 = _residual(P, s, T, prec, method, True)
    R0, W0, E0 = _residual(P, s, T, prec, method, False)
    for a, b in zip(R1, R0):
        assert np.array_equal(a, b)
    assert W1 == W0 and E1 == E0
    if prec == 4:
        Ro, Wo, _ = twod.residual(s, 0, method, T)
        rmax = max(np.abs(x).max() for x in Ro)
        assert max(float(np.abs(a - b).max()) for a, b in zip(R1, Ro)) < 2e-5 * rmax
