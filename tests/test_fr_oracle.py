"""Pins of the fixed-reference (FR) oracle (oracle/fr.py): FR-CCSD / FR-DCSD
hold the A->B doubles amplitude at +1 (singlet) or -1 (M_s = 0 triplet)
and solve the single-reference equations for the rest (the approach of the
paper's introduction, Section I).

  F0  two electrons: the FR-CCSD wave function spans the whole M_s = 0
      space, and a solution of definite spin-flip parity also satisfies the
      one projection the method leaves out; so FR-CCSD with +1 (-1) gives
      the FCI singlet (triplet) energy exactly (brute-force diagonalisation);
  F1  the FR residual equals <q| exp(-T) H_N exp(T) |Phi> from explicit CI
      vectors with the fixed amplitude inside T (CCSD), for both frames;
  F2  with every relaxed amplitude zero, the FR energy is +-(tu|ut), the
      exchange splitting of the two open-shell configurations, and the
      fixed values label the states: <S^2> of Phi_A + Phi_B is 0, of
      Phi_A - Phi_B it is 2;
  F3  at convergence the wave function exp(T) Phi_A satisfies the
      projected Schroedinger equations <q|(H - E)|Psi> = 0 for every single
      and double q other than the fixed one, with E from <Phi_A|H|Psi>
      (explicit CI vectors);
  F4  reference B gives the same FR energies (the spin flip maps the
      singlet and the M_s = 0 triplet onto themselves);
  F5  FR-DCSD differs from FR-CCSD by exactly the DC modification.
"""
import numpy as np
import pytest

from synth import make_pin_system, make_system, random_amplitudes
from oracle import brute, ccsd, fr, solve, twod
from oracle.spinorb import fock_from_h, flip_abi, pack, unpack

TINY = [(1, 2, 6, True), (1, 3, 8, False), (2, 3, 10, True), (2, 2, 7, False)]


def _pin(nc, nv, X, z2, seed=7):
    s = make_pin_system(nc, nv, X, seed=seed, z2=z2)
    fa, fb, e = fock_from_h(s.h, s.B, nc)
    s.fock_a, s.fock_b = fa, fb
    return s, e


@pytest.mark.parametrize("nc,nv,X,z2", TINY)
@pytest.mark.parametrize("ref", [0, 1])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_f1_fr_residual_vs_ci_vectors(nc, nv, X, z2, ref, sign):
    s, _ = _pin(nc, nv, X, z2)
    T = random_amplitudes(s, seed=3, z2=z2, scale1=0.05, scale2=0.05)
    R, Rq, dE = fr.residual(s, ref, twod.CCSD, T, sign)
    frm, _ = twod.frames(s, ref)
    t1, t2 = unpack(frm.o, frm.v, fr.with_fixed(T, sign))
    B1, B2 = brute.Brute(s).ccsd_residual(ref, t1, t2)
    i, j, a, b = frm.q_ab()
    assert abs(B2[i, j, a, b] - Rq) < 1e-13
    for (p, q, r, u) in ((i, j, a, b), (j, i, a, b), (i, j, b, a), (j, i, b, a)):
        B2[p, q, r, u] = 0.0
    for x, y in zip(R, pack(frm.o, frm.v, B1, B2)):
        assert np.abs(x - y).max() < 1e-13
    assert np.abs(B2).max() > 1e-2
    # the energy <Phi| H_N exp(T) |Phi> from CI vectors
    d = brute.Brute(s).twod(ref, t1, t2, t1, t2)
    assert abs(dE - d["dEA"]) < 1e-13


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_f2_zeroth_order_energy_and_state_labels(sign):
    s = make_system((3, 6, 16), seed=9)
    zero = tuple(np.zeros(x.shape) for x in random_amplitudes(s, seed=1))
    _, _, dE = fr.residual(s, 0, twod.CCSD, zero, sign)
    t, u = s.n_c, s.n_c + 1
    K = float(np.sum(s.B[:, t, u] * s.B[:, u, t]))
    assert K > 1e-3
    assert abs(dE - sign * K) < 1e-15
    p, _ = _pin(1, 2, 4, True)
    frm, fro = twod.frames(p, 0)
    dA, dB = twod.frame_det(frm), twod.frame_det(fro)
    assert abs(brute.s_squared(p.n, {dA: 1.0, dB: sign}) - (0.0 if sign > 0 else 2.0)) < 1e-14


@pytest.mark.parametrize("nv,X,seed", [(3, 8, 11), (6, 8, 11), (5, 12, 21)])
def test_f0_two_electrons_fr_ccsd_equals_fci(nv, X, seed):
    s, eref = _pin(0, nv, X, True, seed=seed)
    space, w, V = brute.fci_two_electron(s)
    frm, fro = twod.frames(s, 0)
    ia, ib = space.index[twod.frame_det(frm)], space.index[twod.frame_det(fro)]
    weight = V[ia] ** 2 + V[ib] ** 2
    top = np.argsort(-weight)[:2]
    got = {("S" if V[ia, k] * V[ib, k] > 0 else "T"): w[k] for k in top}
    for sign, lab in ((1.0, "S"), (-1.0, "T")):
        _, info = solve.solve(s, twod.CCSD, tol=1e-12, maxiter=400, fixed=sign)
        assert info["converged"]
        assert abs(eref + info["E"] - got[lab]) < 1e-10, (lab, eref + info["E"], got[lab])


@pytest.mark.parametrize("nc,nv,X,z2,seed", [(1, 3, 8, True, 7), (2, 3, 10, True, 7), (1, 3, 8, False, 3)])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_f3_converged_fr_ccsd_solves_projected_equations(nc, nv, X, z2, seed, sign):
    s, _ = _pin(nc, nv, X, z2, seed=seed)
    T, info = solve.solve(s, twod.CCSD, tol=1e-12, maxiter=400, fixed=sign)
    assert info["converged"]
    frm, _ = twod.frames(s, 0)
    t1, t2 = unpack(frm.o, frm.v, T)
    assert T[4][s.o - 1, s.o - 1, 0, 0] == sign
    b = brute.Brute(s)
    det = twod.frame_det(frm)
    x0 = b.space.vec(det)
    psi = brute.expm_apply(brute.cluster_operator(b.space, frm, t1, t2), x0)
    hpsi = b.H @ psi
    E = x0 @ hpsi  # <Phi_A|H|Psi>, intermediate normalisation <Phi_A|Psi> = 1
    eref = x0 @ b.H @ x0
    assert abs((E - eref) - info["E"]) < 1e-11
    h1, h2 = brute.project_singles_doubles(b.space, frm, det, hpsi - E * psi)
    i, j, a, bb = frm.q_ab()
    fixed_val = h2[i, j, a, bb]
    for (p, q, r, u) in ((i, j, a, bb), (j, i, a, bb), (i, j, bb, a), (j, i, bb, a)):
        h2[p, q, r, u] = 0.0
    assert np.abs(h1).max() < 1e-10 and np.abs(h2).max() < 1e-10
    # the fixed projection is not an equation of the method: it does not vanish
    assert abs(fixed_val) > 1e-6, fixed_val


@pytest.mark.parametrize("method", [twod.CCSD, twod.DCSD])
def test_f4_reference_b_gives_same_energies(method):
    s = make_system((3, 6, 16), seed=9)
    T = random_amplitudes(s, seed=5)
    for sign in (1.0, -1.0):
        RA, qA, EA = fr.residual(s, 0, method, T, sign)
        RB, qB, EB = fr.residual(s, 1, method, flip_abi(T), sign)
        for x, y in zip(flip_abi(RA), RB):
            assert np.abs(x - y).max() < 1e-15
        assert abs(qA - qB) < 1e-15 and abs(EA - EB) < 1e-15
        _, ia = solve.solve(s, method, ref=0, tol=1e-11, fixed=sign)
        _, ib = solve.solve(s, method, ref=1, tol=1e-11, fixed=sign)
        assert ia["converged"] and ib["converged"]
        assert abs(ia["E"] - ib["E"]) < 1e-12


def test_f5_fr_dcsd_is_fr_ccsd_plus_dc_modification():
    s = make_system((2, 5, 12), seed=3)
    T = random_amplitudes(s, seed=2)
    Rc, _, Ec = fr.residual(s, 0, twod.CCSD, T, 1.0)
    Rd, _, Ed = fr.residual(s, 0, twod.DCSD, T, 1.0)
    frm, _ = twod.frames(s, 0)
    _, t2 = unpack(frm.o, frm.v, fr.with_fixed(T, 1.0))
    d = ccsd.dc_delta(frm, t2)
    i, j, a, b = frm.q_ab()
    for (p, q, r, u) in ((i, j, a, b), (j, i, a, b), (i, j, b, a), (j, i, b, a)):
        d[p, q, r, u] = 0.0
    _, dpk = (None, pack(frm.o, frm.v, np.zeros((2 * frm.o, 2 * frm.v)), d))
    for x, y, z in zip(Rc, Rd, dpk):
        assert np.abs(y - x - z).max() < 1e-15
    assert Ec == Ed
