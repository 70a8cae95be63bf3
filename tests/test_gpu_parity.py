"""GPU path vs CPU oracle (parity tests proper; call the C ABI).

The FP64 path must match the oracle to 1e-9 in max |R| and 1e-10 in W and
dE_A (residual at random amplitudes) and to 1e-10 Eh in converged energies.
Sizes span several 64-wide tiles of the contraction kernels with ragged
tails; edge cases: no core orbitals (two electrons), one external virtual.
"""
import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import solve as osolve
from oracle import twod

pytestmark = pytest.mark.gpu

TOL_R, TOL_E = 1e-9, 1e-10


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


def _cmp(R, Ro):
    return max(float(np.abs(np.asarray(r) - ro).max()) for r, ro in zip(R, Ro))


CASES = [((0, 3, 7), 1), ((1, 1, 5), 2), ((2, 5, 12), 3), ((4, 20, 30), 4), ((6, 13, 40), 5)]


@pytest.mark.parametrize("dims,seed", CASES)
@pytest.mark.parametrize("ref", [0, 1])
@pytest.mark.parametrize("method", [0, 1])
def test_residual_fp64_matches_oracle(P, dims, seed, ref, method):
    s = make_system(dims, seed=seed)
    T = random_amplitudes(s, seed=seed + 100, ref=ref, scale1=0.03, scale2=0.03)
    eng = P.Engine.from_system(s)
    R, W, dE = eng.residual(eng.to_device(T), ref=ref, method=method)
    R = [x.cpu().numpy() for x in R]
    Ro, Wo, dEo = twod.residual(s, ref, method, T)
    assert _cmp(R, Ro) < TOL_R
    assert abs(W - Wo) < TOL_E and abs(dE - dEo) < TOL_E
    eng.close()


def test_residual_host_memory_path(P):
    s = make_system((3, 9, 20), seed=8)
    T = random_amplitudes(s, seed=9)
    eng = P.Engine.from_system(s)
    R, W, dE = eng.residual_host(T, method=P.DCSD)
    Ro, Wo, dEo = twod.residual(s, 0, twod.DCSD, T)
    assert _cmp(R, Ro) < TOL_R and abs(W - Wo) < TOL_E
    dE2, W2 = eng.energy(eng.to_device(T), method=P.DCSD)
    assert abs(dE2 - dEo) < TOL_E and abs(W2 - Wo) < TOL_E
    eng.close()


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("ref", [0, 1])
def test_solve_c1_matches_oracle(P, method, ref):
    s = make_system("c1")
    _, info = osolve.solve(s, method, ref=0, tol=1e-10)
    eng = P.Engine.from_system(s)
    T, res = eng.solve(method=method, ref=ref, tol=1e-10, maxiter=100)
    assert res.converged
    assert abs(res.dEA - info["dEA"]) < TOL_E
    assert abs(res.W - info["W"]) < TOL_E
    assert abs(res.E_S - info["E_S"]) < TOL_E and abs(res.E_T - info["E_T"]) < TOL_E
    # converged amplitudes give a zero oracle residual
    Tn = [x.cpu().numpy() for x in T]
    Ro, _, _ = twod.residual(s, ref, method, tuple(Tn))
    assert max(np.abs(x).max() for x in Ro) < 1e-9
    H, ev, si = P.dcsd_heff(res.dEA, res.W)
    assert abs(ev[si] - info["E_S"]) < TOL_E
    eng.close()


def test_invalid_arguments_rejected(P):
    s = make_system((1, 2, 4), seed=1)
    eng = P.Engine.from_system(s)
    T = eng.zeros()
    with pytest.raises(P.DcsdError):
        eng.residual(T, ref=2)
    with pytest.raises(P.DcsdError):
        eng.residual(T, precision=9)
    eng.close()


# Tensor-core paths.  BF16 has a unit roundoff of 2^-9; with FP32 accumulation
# over K terms the residual error is bounded by ~K^(1/2) 2^-9 times the size of
# the largest contributing products, observed <= 5e-3 max|R|: tolerance 2e-2
# max|R|.  The split (hi+lo) products carry 2^-17 relative error per product;
# FP32 accumulation then dominates: tolerance 2e-4 max|R|.
# (4, 60, 200): long DF contractions onto few output tiles take the split-K
# tensor-core path
@pytest.mark.parametrize("dims,seed", [((2, 5, 12), 3), ((4, 20, 30), 4), ((6, 40, 64), 5), ((4, 60, 200), 6)])
@pytest.mark.parametrize("prec,rtol", [(1, 2e-2), (2, 2e-4), (4, 2e-5)])
@pytest.mark.parametrize("method", [0, 1])
def test_residual_tensor_core_within_precision(P, dims, seed, prec, rtol, method):
    s = make_system(dims, seed=seed)
    T = random_amplitudes(s, seed=seed + 100, scale1=0.02, scale2=0.02)
    eng = P.Engine.from_system(s)
    Td = eng.to_device(T)
    R, W, dE = eng.residual(Td, method=method, precision=prec)
    R = [x.cpu().numpy() for x in R]
    Ro, Wo, dEo = twod.residual(s, 0, method, T)
    rmax = max(np.abs(x).max() for x in Ro)
    assert _cmp(R, Ro) < rtol * rmax
    assert abs(W - Wo) < rtol * rmax
    assert abs(dE - dEo) < 1e-12  # the energy is always FP64
    eng.close()


def test_integer_unit_conversions_match_hardware(P):
    """The tensor-core modes convert between FP64 and FP32 on the integer
    units; every binary32 value and 2^28 binary64 patterns (all exponents,
    ties, near-ties) must convert exactly as the hardware does."""
    from paper_2401_11935_gb300 import _lib
    assert _lib.dcsd_selftest_conversions() == 0


def test_mixed_solve_matches_fp64_c2(P):
    """The mixed-precision solve (BF16, BF16X6, FP64 polish) reaches the FP64
    solution: singlet and triplet energies within 1e-6 Eh (here far below)."""
    s = make_system("c2")
    eng = P.Engine.from_system(s)
    _, f = eng.solve(method=1, precision=P.PREC_FP64, tol=1e-8, maxiter=80)
    _, m = eng.solve(method=1, precision=P.PREC_MIXED, tol=1e-8, maxiter=80)
    eng.close()
    assert f.converged and m.converged
    assert m.switched_at > 0 and m.polished_at > m.switched_at
    assert abs(m.E_S - f.E_S) < 1e-6 and abs(m.E_T - f.E_T) < 1e-6
    assert m.seconds < f.seconds
