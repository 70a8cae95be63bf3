"""Contexts made from FCIDUMP files (dcsd_init_fcidump, Section III) against
the oracle evaluated directly on the file's four-index integrals (no
factorisation on the oracle side).

The file holds a small synthetic system (core Hamiltonian and integrals, 4
or 3 correlated core orbitals after freezing, 10 virtuals).  FP64 residuals
at random amplitudes: 1e-9 in max |R|, 1e-10 in W and dE_A, with the
factorised ladder and with the stored four-index ladder; converged 2D-DCSD
energies to 1e-10 Eh, and total energies e_ref + dE_A +- W.
"""
import numpy as np
import pytest

from synth import make_pin_system, random_amplitudes
from synth import fcidump as wfcidump
from oracle import fcidump as ofcidump
from oracle import solve as osolve
from oracle import twod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


@pytest.fixture(scope="module")
def path(tmp_path_factory):
    s = make_pin_system(3, 10, 24, seed=4, b_sigma=0.08)
    p = str(tmp_path_factory.mktemp("fcidump") / "FCIDUMP")
    wfcidump.write(p, s.h, wfcidump.eri_from_factors(s.B), 2 * s.n_c + 2, 0, ecore=0.5,
                   orbsym=[1 + int(x) for x in s.parity])
    return p


@pytest.mark.parametrize("n_frozen", [0, 1])
@pytest.mark.parametrize("stored", [False, True])
@pytest.mark.parametrize("ref,method", [(0, 1), (1, 0), (0, 3)])
def test_fcidump_residual_matches_oracle(P, path, n_frozen, stored, ref, method):
    so, _ = ofcidump.system(path, n_frozen=n_frozen)
    eng = P.Engine.from_fcidump(path, n_frozen=n_frozen, stored_ladder=stored)
    assert (eng.n_c, eng.n_v) == (so.n_c, so.n_v)
    T = random_amplitudes(so, seed=11 + ref, ref=ref, scale1=0.03, scale2=0.03)
    R, W, dE = eng.residual(eng.to_device(T), ref=ref, method=method)
    R = [x.cpu().numpy() for x in R]
    if method >= 2:
        from oracle import fr
        Ro, Wo, dEo = fr.residual(so, ref, method % 2, T, 1.0)
    else:
        Ro, Wo, dEo = twod.residual(so, ref, method, T)
    assert max(float(np.abs(r - ro).max()) for r, ro in zip(R, Ro)) < 1e-9
    assert abs(W - Wo) < 1e-10 and abs(dE - dEo) < 1e-10
    eng.close()


def test_fcidump_bf16_residual_within_precision(P, path):
    so, _ = ofcidump.system(path)
    eng = P.Engine.from_fcidump(path)
    T = random_amplitudes(so, seed=21, scale1=0.02, scale2=0.02)
    R, W, dE = eng.residual(eng.to_device(T), method=1, precision=P.PREC_BF16X6)
    Ro, Wo, dEo = twod.residual(so, 0, 1, T)
    rmax = max(np.abs(x).max() for x in Ro)
    assert max(float(np.abs(r.cpu().numpy() - ro).max()) for r, ro in zip(R, Ro)) < 2e-5 * rmax
    assert abs(dE - dEo) < 1e-12
    eng.close()


@pytest.mark.parametrize("n_frozen", [0, 1])
def test_fcidump_solve_matches_oracle(P, path, n_frozen):
    so, eref = ofcidump.system(path, n_frozen=n_frozen)
    _, info = osolve.solve(so, 1, tol=1e-10)
    assert info["converged"]
    eng = P.Engine.from_fcidump(path, n_frozen=n_frozen)
    _, res = eng.solve(method=1, tol=1e-10, maxiter=100)
    assert res.converged
    assert abs(res.E_S - info["E_S"]) < 1e-10 and abs(res.E_T - info["E_T"]) < 1e-10
    assert abs(eng.fcidump.e_ref - eref) < 1e-12
    # total energies of the two states
    assert abs((eng.fcidump.e_ref + res.E_S) - (eref + info["E_S"])) < 1e-10
    eng.close()
