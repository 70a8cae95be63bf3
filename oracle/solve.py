"""Amplitude iterations and the 2x2 effective Hamiltonian (oracle; test
infrastructure only).

The paper does not state its solver.  Reading used here: start from T = 0,
Jacobi steps T <- T - R/D with D the orbital-energy differences taken from
the diagonal of the frame's Fock matrix, Pulay DIIS on the packed residual
(up to 8 vectors), stop when max|R| <= tol.  Energies (Eq. 2 and the text
after Eq. 4): H_eff = [[dE_A, W], [W, dE_A]], singlet dE_A + W, triplet
dE_A - W.
"""
from __future__ import annotations

import numpy as np

from .spinorb import unpack, pack, flip_abi
from .twod import frames, residual_so


def denominators(fr):
    fo = np.diag(fr.f("oo"))
    fv = np.diag(fr.f("vv"))
    D1 = fv[None, :] - fo[:, None]
    D2 = fv[None, None, :, None] + fv[None, None, None, :] - fo[:, None, None, None] - fo[None, :, None, None]
    return D1, D2


def heff(dEA, W):
    """2x2 effective Hamiltonian, its eigenvalues (ascending) and the index
    of the singlet (eigenvector (1,1)/sqrt2 <-> dE_A + W)."""
    H = np.array([[dEA, W], [W, dEA]])
    ev = np.array(sorted([dEA - W, dEA + W]))
    singlet = int(np.argmin(np.abs(ev - (dEA + W))))
    return H, ev, singlet


def _vec(T):
    return np.concatenate([x.ravel() for x in T])


def _unvec(x, shapes):
    out, k = [], 0
    for s in shapes:
        m = int(np.prod(s))
        out.append(x[k:k + m].reshape(s))
        k += m
    return tuple(out)


def solve(sys, method, ref=0, tol=1e-10, maxiter=200, diis_n=8, T0=None, verbose=False, fixed=None):
    """Converge the 2D amplitude equations.  Returns (T, info).  With fixed =
    +1 or -1, the fixed-reference equations of ``fr`` instead (the A->B
    doubles amplitude held at that value, no M*W terms); info then has E,
    the single-reference energy, and W is the residual element of the fixed
    excitation."""
    from . import fr as frmod
    fr, fro = frames(sys, ref)
    o, v = fr.o, fr.v
    D1, D2 = denominators(fr)
    shapes = [(o, v), (o, v), (o, o, v, v), (o, o, v, v), (o, o, v, v)]
    if T0 is None:
        T = tuple(np.zeros(s) for s in shapes)
    else:
        T = tuple(np.array(x, dtype=float) for x in T0)
    if fixed is not None:
        T = frmod.with_fixed(T, fixed)
    hist_t, hist_e = [], []
    info = {}
    for it in range(1, maxiter + 1):
        if fixed is not None:
            T = frmod.with_fixed(T, fixed)
            t1, t2 = unpack(o, v, T)
            R1, R2, W, dE = frmod.residual_so(fr, method, t1, t2)
        else:
            t1, t2 = unpack(o, v, T)
            t1o, t2o = unpack(o, v, flip_abi(T))
            R1, R2, W, dE, _, _ = residual_so(fr, fro, method, t1, t2, t1o, t2o)
        Rp = pack(o, v, R1, R2)
        rmax = max(np.abs(x).max() for x in Rp)
        info = dict(iters=it, max_r=rmax, dEA=dE, W=W)
        if verbose:
            print(f"it {it:3d} max|R| {rmax:.3e} dEA {dE:.12f} W {W:.12f}")
        if rmax <= tol:
            break
        s1 = np.zeros_like(R1)
        nz1 = R1 != 0.0
        s1[nz1] = -R1[nz1] / D1[nz1]
        s2 = np.zeros_like(R2)
        nz = R2 != 0.0
        s2[nz] = -R2[nz] / D2[nz]
        step = pack(o, v, s1, s2)
        Tn = tuple(a + b for a, b in zip(T, step))
        hist_t.append(_vec(Tn))
        hist_e.append(_vec(step))
        if len(hist_t) > diis_n:
            hist_t.pop(0)
            hist_e.pop(0)
        m = len(hist_t)
        if m >= 2:
            Bm = np.empty((m + 1, m + 1))
            for a in range(m):
                for b in range(m):
                    Bm[a, b] = hist_e[a] @ hist_e[b]
            Bm[m, :] = -1.0
            Bm[:, m] = -1.0
            Bm[m, m] = 0.0
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            c = np.linalg.solve(Bm, rhs)[:m]
            Tn = _unvec(sum(ci * ti for ci, ti in zip(c, hist_t)), shapes)
        T = Tn
    if fixed is not None:
        info.update(E=info["dEA"], converged=info["max_r"] <= tol)
        return T, info
    from .twod import c_condition
    T = c_condition(T)
    H, ev, si = heff(info["dEA"], info["W"])
    info.update(E_S=info["dEA"] + info["W"], E_T=info["dEA"] - info["W"], H=H, evals=ev,
                singlet_index=si, converged=info["max_r"] <= tol)
    return T, info
