"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself:
  P1  two electrons: full CC = FCI (Section I), so 2D-CCSD's dE_A +- W must
      equal the two FCI eigenvalues dominated by Phi_A, Phi_B;
  P2  the working-equation 2D residual (Eqs. 3-4) equals the Bloch-form
      Omega evaluated with explicit CI vectors, at random amplitudes;
  P3  the Stanton-Gauss CCSD residual equals <q|exp(-T) H_N exp(T)|0>
      evaluated with explicit CI vectors, at random amplitudes;
  P4  reference A and reference B give the same result (Section II);
  P5  energies are invariant under occupied-occupied and virtual-virtual
      rotations (CCSD and DCSD);
  P6  antisymmetry, zero A->B amplitude, symmetry-forbidden amplitudes;
  P7  DCSD with the DC modification switched off is CCSD, bit for bit;
  P8  zero residual at convergence;
  phase: <S^2> fixes which eigenvalue of H_eff is the singlet.
"""
import copy

import numpy as np
import pytest

from synth import make_pin_system, make_system, random_amplitudes
from oracle import brute, ccsd, solve, twod
from oracle.spinorb import Frame, fock_from_h, flip_abi, pack, unpack

TINY = [(1, 2, 6, True), (1, 3, 8, False), (2, 3, 10, True), (2, 2, 7, False)]


def _pin(nc, nv, X, z2, seed=7):
    s = make_pin_system(nc, nv, X, seed=seed, z2=z2)
    fa, fb, e = fock_from_h(s.h, s.B, nc)
    s.fock_a, s.fock_b = fa, fb
    return s, e


@pytest.mark.parametrize("nc,nv,X,z2", TINY)
@pytest.mark.parametrize("ref", [0, 1])
def test_p3_ccsd_residual_vs_ci_vectors(nc, nv, X, z2, ref):
    s, _ = _pin(nc, nv, X, z2)
    T = random_amplitudes(s, seed=3, z2=z2, scale1=0.05, scale2=0.05)
    fr = Frame(nc, nv, s.B, s.fock_a, s.fock_b, ref)
    t1, t2 = unpack(fr.o, fr.v, T)
    R1, R2 = ccsd.ccsd_residual(fr, t1, t2)
    B1, B2 = brute.Brute(s).ccsd_residual(ref, t1, t2)
    assert np.abs(R1 - B1).max() < 1e-13
    assert np.abs(R2 - B2).max() < 1e-13
    assert np.abs(B2).max() > 1e-2  # the check is not vacuous


@pytest.mark.parametrize("nc,nv,X,z2", TINY)
@pytest.mark.parametrize("ref", [0, 1])
def test_p2_twod_residual_vs_bloch_form(nc, nv, X, z2, ref):
    s, _ = _pin(nc, nv, X, z2)
    # the C-condition fixes the A->B element (non-zero for non-CAS amplitudes)
    T = twod.c_condition(random_amplitudes(s, seed=4, z2=z2, scale1=0.05, scale2=0.05))
    fr, fro = twod.frames(s, ref)
    t1, t2 = unpack(fr.o, fr.v, T)
    t1o, t2o = unpack(fr.o, fr.v, flip_abi(T))
    c1, c2 = twod.c_other(fr, fro, t1o, t2o)
    d = brute.Brute(s).twod(ref, t1, t2, t1o, t2o)
    assert np.abs(c1 - d["cB1"]).max() < 1e-14
    assert np.abs(c2 - d["cB2"]).max() < 1e-14
    R1, R2, W, dE, _, _ = twod.residual_so(fr, fro, twod.CCSD, t1, t2, t1o, t2o)
    assert abs(W - d["W"]) < 1e-13
    assert abs(dE - d["dEA"]) < 1e-13
    assert np.abs(R1 - d["R1"]).max() < 1e-13
    assert np.abs(R2 - d["R2"]).max() < 1e-13
    # the M*W coupling is not negligible in this check
    q = fr.q_ab()
    nz = np.abs(c2)
    nz[q] = 0.0
    assert np.abs(W) * nz.max() > 1e-5


@pytest.mark.parametrize("nv,X,seed", [(3, 8, 11), (6, 8, 11), (5, 12, 21)])
def test_p1_two_electrons_equal_fci(nv, X, seed):
    s, eref = _pin(0, nv, X, True, seed=seed)
    _, info = solve.solve(s, twod.CCSD, tol=1e-12, maxiter=400)
    assert info["converged"]
    space, w, V = brute.fci_two_electron(s)
    fr, fro = twod.frames(s, 0)
    ia, ib = space.index[twod.frame_det(fr)], space.index[twod.frame_det(fro)]
    weight = V[ia] ** 2 + V[ib] ** 2
    top = np.argsort(-weight)[:2]
    got = {}
    for k in top:
        got["S" if V[ia, k] * V[ib, k] > 0 else "T"] = w[k]
    assert abs(eref + info["E_S"] - got["S"]) < 1e-10
    assert abs(eref + info["E_T"] - got["T"]) < 1e-10


def test_singlet_phase_by_s_squared():
    for nc in (0, 1, 2):
        s, _ = _pin(nc, 2, 4, True)
        fr, fro = twod.frames(s, 0)
        dA, dB = twod.frame_det(fr), twod.frame_det(fro)
        assert abs(brute.s_squared(s.n, {dA: 1.0, dB: 1.0}) - 0.0) < 1e-14
        assert abs(brute.s_squared(s.n, {dA: 1.0, dB: -1.0}) - 2.0) < 1e-14
        # Phi_B (canonical order) is E_{A->B} Phi_A with a + sign
        i, j, a, b = fr.q_ab()
        d, sg = brute.excited(fr, dA, [i, j], [a, b], s.n)
        assert d == dB and sg == 1


@pytest.mark.parametrize("method", [twod.CCSD, twod.DCSD])
def test_p4_reference_b_is_spin_flip(method):
    s = make_system((3, 6, 16), seed=9)
    T = random_amplitudes(s, seed=5)
    RA, WA, EA = twod.residual(s, 0, method, T)
    RB, WB, EB = twod.residual(s, 1, method, flip_abi(T))
    for x, y in zip(flip_abi(RA), RB):
        assert np.abs(x - y).max() < 1e-15
    assert abs(WA - WB) < 1e-16 and abs(EA - EB) < 1e-16
    _, ia = solve.solve(s, method, ref=0, tol=1e-11)
    _, ib = solve.solve(s, method, ref=1, tol=1e-11)
    assert abs(ia["E_S"] - ib["E_S"]) < 1e-12 and abs(ia["E_T"] - ib["E_T"]) < 1e-12


def _rotated(s, seed):
    from scipy.stats import ortho_group
    U = np.eye(s.n)
    U[:s.n_c, :s.n_c] = ortho_group.rvs(s.n_c, random_state=seed)
    U[s.n_c + 2:, s.n_c + 2:] = ortho_group.rvs(s.n_v, random_state=seed + 1)
    r = copy.deepcopy(s)
    r.fock_a, r.fock_b = U.T @ s.fock_a @ U, U.T @ s.fock_b @ U
    r.B = np.einsum("pq,Lpr,rs->Lqs", U, s.B, U)
    return r


@pytest.mark.parametrize("method", [twod.CCSD, twod.DCSD])
def test_p5_rotation_invariance(method):
    s = make_system((3, 8, 20), seed=5)
    _, i1 = solve.solve(s, method, tol=1e-11)
    _, i2 = solve.solve(_rotated(s, 3), method, tol=1e-11)
    assert i1["converged"] and i2["converged"]
    assert abs(i1["dEA"] - i2["dEA"]) < 1e-10
    assert abs(i1["W"] - i2["W"]) < 1e-10


@pytest.mark.parametrize("method", [twod.CCSD, twod.DCSD])
def test_p6_p8_converged_amplitudes(method):
    s = make_system("c1")
    T, info = solve.solve(s, method, tol=1e-10)
    assert info["converged"] and info["max_r"] <= 1e-10  # P8
    R, W, dE = twod.residual(s, 0, method, T)
    assert max(np.abs(x).max() for x in R) <= 1e-10
    T1a, T1b, T2aa, T2bb, T2ab = T
    for t in (T2aa, T2bb):
        assert np.abs(t + t.transpose(1, 0, 2, 3)).max() < 1e-15
        assert np.abs(t + t.transpose(0, 1, 3, 2)).max() < 1e-15
    o = s.o
    assert T2ab[o - 1, o - 1, 0, 0] == 0.0
    # Z2: active-active singles vanish (CAS case, Section II)
    assert abs(T1a[o - 1, 0]) < 1e-14 and abs(T1b[o - 1, 0]) < 1e-14
    assert abs(info["E_S"] - (dE + W)) < 1e-9


def test_p7_dc_switch_off_is_ccsd():
    s = make_system((2, 5, 12), seed=3)
    T = random_amplitudes(s, seed=2)
    fr, fro = twod.frames(s, 0)
    t1, t2 = unpack(fr.o, fr.v, T)
    t1o, t2o = unpack(fr.o, fr.v, flip_abi(T))
    R1c, R2c = ccsd.ccsd_residual(fr, t1, t2)
    d = ccsd.dc_delta(fr, t2)
    *_, R1x, R2x = twod.residual_so(fr, fro, twod.DCSD, t1, t2, t1o, t2o)
    assert np.array_equal(R1x, R1c)
    assert np.array_equal(R2x, R2c + d)
    *_, R1y, R2y = twod.residual_so(fr, fro, twod.CCSD, t1, t2, t1o, t2o)
    assert np.array_equal(R2y, R2c)
    # the DC modification is homogeneous of degree two in t2 and antisymmetric
    assert np.abs(ccsd.dc_delta(fr, 2.0 * t2) - 4.0 * d).max() < 1e-15
    assert np.abs(d + d.transpose(1, 0, 2, 3)).max() < 1e-16
    assert np.abs(d + d.transpose(0, 1, 3, 2)).max() < 1e-16
    assert np.abs(d).max() > 1e-6


def test_pack_roundtrip():
    s = make_system((2, 4, 8), seed=1)
    T = random_amplitudes(s, seed=1)
    t1, t2 = unpack(s.o, s.v, T)
    for x, y in zip(T, pack(s.o, s.v, t1, t2)):
        assert np.array_equal(x, y)
    for x, y in zip(flip_abi(flip_abi(T)), T):
        assert np.array_equal(x, y)
