"""The incomplete-active-space case (t and u in the same irrep, Section II)
on the GPU against the oracle (pinned in tests/test_ias_oracle.py): the
internal singles do not vanish, the A->B doubles element follows the
C-condition and W carries the internal-singles products.

FP64 residuals to 1e-9 (both frames, CCSD and DCSD), tensor-core residuals
within precision, converged energies to 1e-10 Eh, and the reverse mode
(which differentiates through the C-condition and W) against the oracle's
per-element gradient.
"""
import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import solve as osolve
from oracle import twod
from oracle import vjp as ovjp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


@pytest.mark.parametrize("dims,seed", [((0, 3, 7), 1), ((2, 5, 12), 3), ((6, 13, 40), 5)])
@pytest.mark.parametrize("ref", [0, 1])
@pytest.mark.parametrize("method", [0, 1])
def test_ias_residual_fp64_matches_oracle(P, dims, seed, ref, method):
    s = make_system(dims, seed=seed, ias=True)
    T = random_amplitudes(s, seed=seed + 100, ref=ref, scale1=0.03, scale2=0.03)
    o = s.o
    assert abs(T[0][o - 1, 0]) > 1e-4 and abs(T[1][o - 1, 0]) > 1e-4
    eng = P.Engine.from_system(s)
    R, W, dE = eng.residual(eng.to_device(T), ref=ref, method=method)
    R = [x.cpu().numpy() for x in R]
    Ro, Wo, dEo = twod.residual(s, ref, method, T)
    assert max(float(np.abs(r - ro).max()) for r, ro in zip(R, Ro)) < 1e-9
    assert abs(W - Wo) < 1e-10 and abs(dE - dEo) < 1e-10
    eng.close()


@pytest.mark.parametrize("prec,rtol", [(1, 2e-2), (4, 2e-5)])
def test_ias_residual_tensor_core_within_precision(P, prec, rtol):
    s = make_system((6, 40, 64), seed=5, ias=True)
    T = random_amplitudes(s, seed=105, scale1=0.02, scale2=0.02)
    eng = P.Engine.from_system(s)
    R, W, dE = eng.residual(eng.to_device(T), method=1, precision=prec)
    Ro, Wo, dEo = twod.residual(s, 0, 1, T)
    rmax = max(np.abs(x).max() for x in Ro)
    assert max(float(np.abs(r.cpu().numpy() - ro).max()) for r, ro in zip(R, Ro)) < rtol * rmax
    assert abs(W - Wo) < rtol * rmax
    eng.close()


@pytest.mark.parametrize("method", [0, 1])
def test_ias_solve_matches_oracle(P, method):
    s = make_system((4, 20, 60), seed=1, ias=True)
    To, info = osolve.solve(s, method, tol=1e-10)
    assert info["converged"]
    eng = P.Engine.from_system(s)
    T, res = eng.solve(method=method, tol=1e-10, maxiter=100)
    eng.close()
    assert res.converged
    assert abs(res.E_S - info["E_S"]) < 1e-10 and abs(res.E_T - info["E_T"]) < 1e-10
    Tn = [x.cpu().numpy() for x in T]
    o = s.o
    # the returned amplitudes satisfy the C-condition, with internal singles present
    assert abs(Tn[4][o - 1, o - 1, 0, 0] + Tn[0][o - 1, 0] * Tn[1][o - 1, 0]) < 1e-15
    assert abs(Tn[0][o - 1, 0]) > 1e-6


@pytest.mark.parametrize("dims,seed", [((0, 2, 5), 1), ((1, 2, 6), 2)])
@pytest.mark.parametrize("ref", [0, 1])
def test_ias_vjp_gradient_matches_oracle(P, dims, seed, ref):
    import torch
    s = make_system(dims, seed=seed, ias=True)
    T = random_amplitudes(s, seed=seed + 20, ref=ref, scale1=0.05, scale2=0.05)
    rng = np.random.default_rng(seed)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    Eb, Wb = 0.3, -0.8
    eng = P.Engine.from_system(s)
    Tb, _, _, _ = eng.vjp(eng.to_device(T), Rbar=eng.to_device(Rb), Ebar=Eb, Wbar=Wb, ref=ref, method=1)
    torch.cuda.synchronize()
    G = [x.cpu().numpy() for x in Tb]
    eng.close()
    Go = ovjp.gradient_T(s, ref, 1, T, Rb, Eb, Wb)
    scale = max(float(np.abs(g).max()) for g in Go)
    for g, go in zip(ovjp.project(G), ovjp.project(Go)):
        assert np.abs(g - go).max() < 1e-8 * scale
    # the internal singles' gradients include the C-condition and W terms
    o = s.o
    assert abs(Go[0][o - 1, 0]) > 1e-3
