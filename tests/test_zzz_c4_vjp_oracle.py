"""Reverse mode at the adjoint workload (12+2 occupied/open, 160 virtuals,
naux 480, FP64) against the oracle.  The cotangent is one-hot at a sampled,
symmetry-allowed element q of R2ab, so <T_bar, d> from dcsd_vjp must equal
the derivative of the single element R_q along the direction d, which the
element-wise oracle (oracle/element.py) gives by the fourth-order central
stencil [8 (R(h) - R(-h)) - (R(2h) - R(-2h))] / (12 h) (R_q is a polynomial
in the amplitudes).  d is random over all five amplitude arrays,
antisymmetric in the same-spin blocks.  Collected after the other GPU tests."""
import numpy as np
import pytest

from oracle import element
from oracle.vjp import antisym
from synth import make_system, random_amplitudes

pytestmark = pytest.mark.gpu

Q = (4, 4, 0, 0)        # R2ab element: i, j core, a = b = the active virtual of each spin
H = 1e-3


def oracle_directional(s, method, T, d, block, idx, h=H):
    """d/de R_q(T + e d) at e = 0 by the fourth-order central stencil."""
    def r(e):
        Te = tuple(t + e * x for t, x in zip(T, d))
        return element.residual_element(element.ElementOracle(s, 0, method, Te), block, idx)
    return (8.0 * (r(h) - r(-h)) - (r(2 * h) - r(-2 * h))) / (12.0 * h)


def inputs():
    s = make_system("c4")
    T = random_amplitudes(s, seed=81, scale1=0.02, scale2=0.02)
    rng = np.random.default_rng(82)
    d = [rng.normal(0, 1, t.shape) for t in T]
    d[2], d[3] = antisym(d[2]), antisym(d[3])
    return s, T, d


def test_c4_vjp_matches_element_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    s, T, d = inputs()
    Rb = [np.zeros_like(t) for t in T]
    Rb[4][Q] = 1.0
    eng = P.Engine.from_system(s)
    Tb, _, _, _ = eng.vjp(eng.to_device(T), Rbar=eng.to_device(Rb), Ebar=0.0, Wbar=0.0, ref=0, method=P.DCSD)
    torch.cuda.synchronize()
    gpu = sum(float((g.cpu().numpy() * x).sum()) for g, x in zip(Tb, d))
    eng.close()
    ora = oracle_directional(s, 1, T, d, 4, Q)
    assert abs(ora) > 1e-6
    assert abs(gpu - ora) < 1e-8 * max(1.0, abs(ora)), (gpu, ora)
