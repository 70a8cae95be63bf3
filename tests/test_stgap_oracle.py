"""Singlet-triplet gaps from one calculation or from two (Table 4's
comparison, Section IV.B), on the CPU oracle.

Orbital sets of one synthetic molecule are made by rotating its integrals
(occupied-virtual mixing within a symmetry label, standing in for the
relaxation between state-averaged and state-specific orbitals).

  G1  two electrons: 2D-CCSD is exact, so its total singlet and triplet
      energies do not depend on the orbitals: the gap from one calculation
      (2W) equals the gap from two calculations with different orbitals and
      the FCI gap;
  G2  with more electrons the total energies do depend on the orbitals (so
      the two ways of computing the gap differ, the effect the paper
      measures), while each single calculation still gives its gap as 2W.
"""
import numpy as np
import pytest

from synth import make_pin_system
from synth import fcidump as wfcidump
from oracle import brute
from oracle import fcidump as ofcidump
from oracle import solve, twod


def orbital_sets(nc, nv, X, seed, scale):
    """FCIDUMP contents (h, eri, parity) of three orbital sets: the original
    and two rotated ones."""
    s = make_pin_system(nc, nv, X, seed=seed, b_sigma=0.1)
    eri = wfcidump.eri_from_factors(s.B)
    sets = [(s.h, eri)]
    for k in (1, 2):
        U = wfcidump.random_ov_rotation(s.parity, nc + 2, scale, seed + 10 * k)
        sets.append(wfcidump.rotate(s.h, eri, U))
    return s, sets


def write_sets(tmp_path, s, sets):
    paths = []
    for k, (h, eri) in enumerate(sets):
        p = str(tmp_path / f"FCIDUMP.{k}")
        wfcidump.write(p, h, eri, 2 * s.n_c + 2, 0, ecore=0.75, orbsym=[1 + int(x) for x in s.parity])
        paths.append(p)
    return paths


def totals(path, method=twod.CCSD):
    so, eref = ofcidump.system(path)
    _, info = solve.solve(so, method, tol=1e-12, maxiter=400)
    assert info["converged"]
    return eref + info["E_S"], eref + info["E_T"], info["W"]


def test_g1_two_electrons_gap_independent_of_orbitals(tmp_path):
    s, sets = orbital_sets(0, 4, 10, 21, 0.1)
    paths = write_sets(tmp_path, s, sets)
    E = [totals(p) for p in paths]
    # FCI of the unrotated set (core energy 0.75)
    space, w, V = brute.fci_two_electron(s)
    fr, fro = twod.frames(s, 0)
    ia, ib = space.index[twod.frame_det(fr)], space.index[twod.frame_det(fro)]
    top = np.argsort(-(V[ia] ** 2 + V[ib] ** 2))[:2]
    fci = {("S" if V[ia, k] * V[ib, k] > 0 else "T"): w[k] + 0.75 for k in top}
    for (ES, ET, W) in E:
        assert abs(ES - fci["S"]) < 1e-10 and abs(ET - fci["T"]) < 1e-10
        assert abs((ES - ET) - 2 * W) < 1e-14
    # one calculation vs two (singlet from set 1, triplet from set 2)
    assert abs((E[0][0] - E[0][1]) - (E[1][0] - E[2][1])) < 1e-10
    # the rotations are not trivial: the reference energies differ
    refs = [ofcidump.system(p)[1] for p in paths]
    assert abs(refs[0] - refs[1]) > 1e-4 and abs(refs[0] - refs[2]) > 1e-4


def test_g2_more_electrons_totals_depend_on_orbitals(tmp_path):
    s, sets = orbital_sets(2, 5, 12, 22, 0.05)
    paths = write_sets(tmp_path, s, sets)
    E = [totals(p, twod.DCSD) for p in paths]
    for (ES, ET, W) in E:
        assert abs((ES - ET) - 2 * W) < 1e-14
    assert abs(E[0][0] - E[1][0]) > 1e-7
    single, two = E[0][0] - E[0][1], E[1][0] - E[2][1]
    assert abs(single - two) > 1e-7
