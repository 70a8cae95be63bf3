"""The tensor-core ladder in symmetric / antisymmetric form (the default:
M+-_ab[cd] = (ac|bd) +- (ad|bc) over the pairs c <= d, with the amplitude
combinations (t_cd +- t_dc) / 2) against the contraction over all (c, d)
(DCSD_LADDER_SA=0) and against the oracle.  V up to 302 covers one, two and three
128-wide c/d blocks (the off-diagonal block tiles of the producer),
ragged V (not a multiple of 8), both references and one to six split
products.  The two forms round differently, so they agree to the precision
of the split, not bit for bit."""
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


def _residual(P, s, T, prec, method, ref, sa):
    old = os.environ.get("DCSD_LADDER_SA")
    os.environ["DCSD_LADDER_SA"] = "1" if sa else "0"
    try:
        eng = P.Engine.from_system(s)
    finally:
        if old is None:
            del os.environ["DCSD_LADDER_SA"]
        else:
            os.environ["DCSD_LADDER_SA"] = old
    R, W, dE = eng.residual(eng.to_device(T), ref=ref, method=method, precision=prec)
    out = [x.cpu().numpy() for x in R], W, dE
    eng.close()
    return out


def _dev(R, Rref):
    return max(float(np.abs(a - b).max()) for a, b in zip(R, Rref))


# relative to max|R|: BF16 products 2e-2, split (hi + mid) 2e-4, FP32-class 2e-5
RTOL = {1: 2e-2, 2: 2e-4, 4: 2e-5}


@pytest.mark.parametrize("dims,seed", [((6, 40, 64), 5), ((5, 29, 45), 7), ((4, 130, 60), 8)])
@pytest.mark.parametrize("prec", [1, 2, 4])
@pytest.mark.parametrize("method,ref", [(0, 0), (1, 1)])
def test_sa_ladder_matches_oracle_and_full_form(P, dims, seed, prec, method, ref):
    s = make_system(dims, seed=seed)
    T = random_amplitudes(s, seed=seed + 100, ref=ref, scale1=0.02, scale2=0.02)
    R1, W1, E1 = _residual(P, s, T, prec, method, ref, True)
    R0, W0, E0 = _residual(P, s, T, prec, method, ref, False)
    Ro, Wo, _ = twod.residual(s, ref, method, T)
    rmax = max(float(np.abs(x).max()) for x in Ro)
    assert _dev(R1, Ro) < RTOL[prec] * rmax
    assert _dev(R1, R0) < RTOL[prec] * rmax
    assert abs(W1 - Wo) < RTOL[prec] * rmax
    assert E1 == E0


# three c/d blocks (V = 302): the two forms against each other only (the
# oracle residual at this size takes minutes)
@pytest.mark.parametrize("prec", [1, 4])
def test_sa_ladder_three_blocks(P, prec):
    s = make_system((2, 300, 40), seed=9)
    T = random_amplitudes(s, seed=109, scale1=0.02, scale2=0.02)
    R1, W1, _ = _residual(P, s, T, prec, 1, 0, True)
    R0, W0, _ = _residual(P, s, T, prec, 1, 0, False)
    rmax = max(float(np.abs(x).max()) for x in R0)
    assert _dev(R1, R0) < RTOL[prec] * rmax
    assert abs(W1 - W0) < RTOL[prec] * rmax
