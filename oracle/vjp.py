"""Derivatives of the oracle residual (TEST INFRASTRUCTURE ONLY; see the
package docstring for who may import this).

The quantity differentiated is

    phi(T, B, f) = <R_bar, R(T)> + E_bar * dE_A(T) + W_bar * W(T)

with R, dE_A, W from ``twod.residual`` (Section II, Eqs. 2-4).  phi is a
polynomial in the amplitudes, the DF factors and the Fock matrices, so its
directional derivative is taken with the fourth-order central difference

    phi'(0) = [8 (phi(h) - phi(-h)) - (phi(2h) - phi(-2h))] / (12 h),

whose truncation error is h^4 phi^(5) / 30 (exact for polynomials of degree
four or less along the direction).  ``gradient_T`` applies it along every
unit direction of the stored amplitude arrays (tiny systems only).

The same-spin doubles are antisymmetric and B and f are symmetric, so only
derivatives along directions with those symmetries are defined independently
of how an implementation reads the stored arrays; the A->B doubles element
is set by the C-condition (``twod.c_condition``), so the derivative along it
is zero; ``project`` maps a gradient onto that subspace for comparisons.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import twod


def objective(sys, ref, method, T, Rbar, Ebar=0.0, Wbar=0.0):
    R, W, dE = twod.residual(sys, ref, method, T)
    v = Ebar * dE + Wbar * W
    if Rbar is not None:
        v += sum(float((np.asarray(r) * rb).sum()) for r, rb in zip(R, Rbar))
    return v


def directional(sys, ref, method, T, Rbar, Ebar=0.0, Wbar=0.0, dT=None, dB=None, dfa=None, dfb=None,
                h=1e-3):
    """d/de phi(T + e dT, B + e dB, f + e df) at e = 0 (fourth-order stencil)."""
    def phi(e):
        Tp = T if dT is None else tuple(t + e * d for t, d in zip(T, dT))
        sp = sys
        if dB is not None or dfa is not None or dfb is not None:
            sp = dataclasses.replace(
                sys,
                B=sys.B + e * dB if dB is not None else sys.B,
                fock_a=sys.fock_a + e * dfa if dfa is not None else sys.fock_a,
                fock_b=sys.fock_b + e * dfb if dfb is not None else sys.fock_b)
        return objective(sp, ref, method, Tp, Rbar, Ebar, Wbar)
    return (8.0 * (phi(h) - phi(-h)) - (phi(2 * h) - phi(-2 * h))) / (12.0 * h)


def gradient_T(sys, ref, method, T, Rbar, Ebar=0.0, Wbar=0.0, h=1e-3):
    """Gradient of phi with respect to every stored amplitude element."""
    G = []
    for k, t in enumerate(T):
        g = np.zeros_like(t)
        for idx in np.ndindex(t.shape):
            dT = [np.zeros_like(x) for x in T]
            dT[k][idx] = 1.0
            g[idx] = directional(sys, ref, method, T, Rbar, Ebar, Wbar, dT=dT, h=h)
        G.append(g)
    return tuple(G)


def antisym(x):
    """Projection of [o][o][v][v] onto arrays antisymmetric in (i,j) and (a,b)."""
    return 0.25 * (x - x.transpose(1, 0, 2, 3) - x.transpose(0, 1, 3, 2) + x.transpose(1, 0, 3, 2))


def project(G):
    """Gradient along symmetry-respecting directions: same-spin doubles
    antisymmetrised, the A->B doubles element (fixed by the C-condition, not
    a free amplitude) zero, everything else unchanged."""
    G4 = np.array(G[4], dtype=float)
    o = G4.shape[0]
    G4[o - 1, o - 1, 0, 0] = 0.0
    return (G[0], G[1], antisym(G[2]), antisym(G[3]), G4)
