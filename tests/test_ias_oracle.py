"""The incomplete-active-space (IAS) case of Section II: the open orbitals t
and u in the same irrep, so the internal singles t alpha -> u alpha and
u beta -> t beta do not vanish and the two ionic determinants lie outside
the model space {Phi_A, Phi_B}.

The reading (oracle/twod.py): the Jeziorski-Monkhorst wave operator with
intermediate normalisation, <B|exp(T_A)|A> = 0 (the C-condition: the A->B
doubles element equals minus the product of the internal singles), and the
coupling W = <B|H_N exp(T_A)|A>, which adds to the residual element of the
A->B double the products of the internal singles with their residuals.  In
the CAS case both additions vanish and the equations are those of the CAS
tests.

  I1  two electrons: with T complete, the Bloch equations are exact, so
      2D-CCSD's dE_A +- W equal the two FCI eigenvalues whose eigenvectors
      are dominated by Phi_A and Phi_B (brute-force diagonalisation) --
      and leaving out either addition (the internal-singles products in W,
      or the C-condition) breaks that;
  I2  the working-equation residual equals the Bloch form evaluated with
      CI vectors at random IAS amplitudes (both frames);
  I3  reference B gives the same energies; the C-condition holds in the
      converged amplitudes.
"""
import numpy as np
import pytest

from synth import make_pin_system, make_system, random_amplitudes
from oracle import brute, ccsd, solve, twod
from oracle.spinorb import fock_from_h, flip_abi, pack, unpack


def _pin(nc, nv, X, seed, b_sigma=0.1):
    s = make_pin_system(nc, nv, X, seed=seed, ias=True, b_sigma=b_sigma)
    fa, fb, e = fock_from_h(s.h, s.B, nc)
    s.fock_a, s.fock_b = fa, fb
    return s, e


def _fci_pair(s):
    space, w, V = brute.fci_two_electron(s)
    fr, fro = twod.frames(s, 0)
    ia, ib = space.index[twod.frame_det(fr)], space.index[twod.frame_det(fro)]
    top = np.argsort(-(V[ia] ** 2 + V[ib] ** 2))[:2]
    return {("S" if V[ia, k] * V[ib, k] > 0 else "T"): w[k] for k in top}


@pytest.mark.parametrize("nv,X,seed", [(4, 10, 11), (5, 12, 12), (6, 12, 13)])
def test_i1_two_electrons_equal_fci(nv, X, seed):
    s, eref = _pin(0, nv, X, seed)
    _, info = solve.solve(s, twod.CCSD, tol=1e-12, maxiter=400)
    assert info["converged"]
    fci = _fci_pair(s)
    assert abs(eref + info["E_S"] - fci["S"]) < 1e-10
    assert abs(eref + info["E_T"] - fci["T"]) < 1e-10
    # the internal singles are not negligible here
    Ts, _ = solve.solve(s, twod.CCSD, tol=1e-12, maxiter=400)
    assert abs(Ts[0][0, 0] * Ts[1][0, 0]) > 1e-4


def _solve_variant(s, drop):
    """The same iterations with one IAS addition left out (CPU, test only)."""
    orig_cc, orig_so = twod.c_condition, twod._c_condition_so
    orig_res = twod.residual_so
    try:
        if drop == "c-condition":
            twod._c_condition_so = lambda fr, t1, t2: t2
            twod.c_condition = lambda T: tuple(np.array(x) for x in T)
        else:
            def no_singles_w(fr, fro, method, t1, t2, t1o, t2o):
                R1, R2, W, dE, R1x, R2x = orig_res(fr, fro, method, t1, t2, t1o, t2o)
                i, j, a, b = fr.q_ab()
                W0 = R2x[i, j, a, b]
                c1, c2 = twod.c_other(fr, fro, t1o, twod._c_condition_so(fro, t1o, t2o))
                tc = ccsd.P_ij(ccsd.P_ab(np.einsum("ia,jb->ijab", t1, c1)))
                R1 = R1x - W0 * c1
                R2 = R2x - W0 * (c2 - tc)
                for (p, q, r, u) in ((i, j, a, b), (j, i, a, b), (i, j, b, a), (j, i, b, a)):
                    R2[p, q, r, u] = 0.0
                return R1, R2, W0, dE, R1x, R2x
            solve.residual_so = no_singles_w
        _, info = solve.solve(s, twod.CCSD, tol=1e-11, maxiter=400)
    finally:
        twod.c_condition, twod._c_condition_so = orig_cc, orig_so
        solve.residual_so = orig_res
    return info


@pytest.mark.parametrize("drop", ["c-condition", "internal singles in W"])
def test_i1_each_addition_is_needed(drop):
    s, eref = _pin(0, 4, 10, 11)
    info = _solve_variant(s, drop)
    fci = _fci_pair(s)
    err = max(abs(eref + info["E_S"] - fci["S"]), abs(eref + info["E_T"] - fci["T"]))
    assert err > 1e-8, (drop, err)  # the complete treatment agrees to 1e-10


@pytest.mark.parametrize("nc,nv,X,seed", [(1, 2, 6, 3), (2, 3, 8, 4), (1, 3, 8, 5)])
@pytest.mark.parametrize("ref", [0, 1])
def test_i2_residual_vs_bloch_form(nc, nv, X, seed, ref):
    s, _ = _pin(nc, nv, X, seed)
    T = twod.c_condition(random_amplitudes(s, seed=seed + 7, ref=ref, scale1=0.05, scale2=0.05))
    o = s.o
    assert abs(T[0][o - 1, 0]) > 1e-3 and abs(T[1][o - 1, 0]) > 1e-3  # internal singles present
    fr, fro = twod.frames(s, ref)
    t1, t2 = unpack(fr.o, fr.v, T)
    t1o, t2o = unpack(fr.o, fr.v, flip_abi(T))
    d = brute.Brute(s).twod(ref, t1, t2, t1o, t2o)
    R1, R2, W, dE, _, _ = twod.residual_so(fr, fro, twod.CCSD, t1, t2, t1o, t2o)
    assert abs(W - d["W"]) < 1e-13 and abs(dE - d["dEA"]) < 1e-13
    assert np.abs(R1 - d["R1"]).max() < 1e-13 and np.abs(R2 - d["R2"]).max() < 1e-13


@pytest.mark.parametrize("method", [twod.CCSD, twod.DCSD])
def test_i3_reference_b_and_c_condition(method):
    s = make_system((3, 6, 16), seed=9, ias=True)
    T = random_amplitudes(s, seed=5)
    RA, WA, EA = twod.residual(s, 0, method, T)
    RB, WB, EB = twod.residual(s, 1, method, flip_abi(T))
    for x, y in zip(flip_abi(RA), RB):
        assert np.abs(x - y).max() < 1e-15
    assert abs(WA - WB) < 1e-15 and abs(EA - EB) < 1e-15
    Ta, ia = solve.solve(s, method, ref=0, tol=1e-11)
    _, ib = solve.solve(s, method, ref=1, tol=1e-11)
    assert ia["converged"] and ib["converged"]
    assert abs(ia["E_S"] - ib["E_S"]) < 1e-12 and abs(ia["E_T"] - ib["E_T"]) < 1e-12
    o = s.o
    assert Ta[4][o - 1, o - 1, 0, 0] == -Ta[0][o - 1, 0] * Ta[1][o - 1, 0]
    assert abs(Ta[0][o - 1, 0]) > 1e-5
