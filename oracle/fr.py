"""Fixed-reference (FR) CCSD and DCSD of an open-shell singlet or M_s = 0
triplet (oracle; test infrastructure only).

Section I of the paper (the fixed-reference approach it builds on): the
doubles amplitude of the excitation that takes Phi_A to Phi_B is held fixed
at one, and every other amplitude relaxes in an ordinary single-reference CC
calculation on Phi_A.  So the equations are the single-reference residuals

  R^X_q(T) = <Phi_q| exp(-T) H_N exp(T) |Phi_A> = 0,   q != A->B,

with X = CCSD or DCSD (the DC modification of ``ccsd.dc_delta``), and no
M*W terms; the energy is the single-reference one, Delta E = <Phi_A| H_N
exp(T) |Phi_A> (``ccsd.energy``), which now contains the fixed amplitude.

Reading (the paper states the value one for the singlet): with this
library's phase of Phi_B (E_{A->B} Phi_A, for which the singlet is
Phi_A + Phi_B), a fixed value of +1 targets the open-shell singlet and -1
the M_s = 0 triplet, Phi_A - Phi_B.
"""
from __future__ import annotations

import numpy as np

from . import ccsd
from .spinorb import pack, unpack
from .twod import DCSD, frames

SINGLET, TRIPLET = 1.0, -1.0


def with_fixed(T, sign):
    """Copy of the ABI amplitudes with the A->B doubles element set to sign."""
    T = tuple(np.array(x, dtype=float) for x in T)
    o = T[0].shape[0]
    T[4][o - 1, o - 1, 0, 0] = sign
    return T


def residual_so(fr, method, t1, t2):
    """Spin-orbital FR residual for amplitudes that already hold the fixed
    element; returns (R1, R2, Rq, dE) with Rq the single-reference residual
    element of the fixed excitation (not an equation; zeroed in R2)."""
    R1, R2 = ccsd.ccsd_residual(fr, t1, t2)
    if method == DCSD:
        R2 = R2 + ccsd.dc_delta(fr, t2)
    i, j, a, b = fr.q_ab()
    Rq = R2[i, j, a, b]
    for (p, q, r, s) in ((i, j, a, b), (j, i, a, b), (i, j, b, a), (j, i, b, a)):
        R2[p, q, r, s] = 0.0
    return R1, R2, Rq, ccsd.energy(fr, t1, t2)


def residual(sys, ref, method, T, sign):
    """ABI-level FR residual: (R, Rq, dE) for amplitudes T normal-ordered to
    the frame `ref`, with the fixed element set to sign (whatever T holds
    there)."""
    fr, _ = frames(sys, ref)
    t1, t2 = unpack(fr.o, fr.v, with_fixed(T, sign))
    R1, R2, Rq, dE = residual_so(fr, method, t1, t2)
    return pack(fr.o, fr.v, R1, R2), Rq, dE
