"""Determinant-space brute force (oracle pins; test infrastructure only).

Everything here works with explicit CI vectors over all M_s = 0 determinants
of a tiny system, so it shares no algebra with the working equations it is
used to pin:
  * H from the spin-free core Hamiltonian h and DF factors B;
  * exp(T) applied to vectors with T built from a+/a operators;
  * R^CC_q = <Phi_q| exp(-T) H_N exp(T) |Phi>            (Eqs. 3-4, first terms)
  * c^X_q  = <A_q| exp(T_X) |X>                           (Eqs. 3-4)
  * Omega_q = <A_q|H_N exp(T_A)|A> - c^A_q dE_A - c^B_q W  (Bloch form)
  * full CI eigenpairs and <S^2>.

Determinants: sorted tuples of spin-orbital ids gid = spin*n + spatial
(alpha string first); |D> = a+_{d1} a+_{d2} ... |vac> with d1 < d2 < ...
"""
from __future__ import annotations

import itertools
import numpy as np
import scipy.sparse as sp

from .twod import apply_excitation, frame_det, create, annihilate
from .spinorb import Frame


class DetSpace:
    def __init__(self, n, na, nb):
        self.n = n
        al = list(itertools.combinations(range(n), na))
        be = list(itertools.combinations(range(n), nb))
        self.dets = [tuple(a) + tuple(n + x for x in b) for a in al for b in be]
        self.index = {d: k for k, d in enumerate(self.dets)}
        self.dim = len(self.dets)
        self._E = {}

    def E(self, p, q):
        """Sparse matrix of a+_p a_q (gids)."""
        key = (p, q)
        if key not in self._E:
            rows, cols, vals = [], [], []
            for c, d in enumerate(self.dets):
                d1, s1 = annihilate(d, q)
                d2, s2 = create(d1, p)
                if d2 is not None:
                    rows.append(self.index[d2])
                    cols.append(c)
                    vals.append(s1 * s2)
            self._E[key] = sp.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim))
        return self._E[key]

    def vec(self, det, coef=1.0):
        x = np.zeros(self.dim)
        x[self.index[det]] = coef
        return x

    def hamiltonian(self, h, B):
        """H = sum_pq h_pq E_pq + 1/2 sum (pq|rs) a+_p a+_r a_s a_q
             = sum_pq [h - 1/2 sum_L B_L B_L]_pq E_pq + 1/2 sum_L O_L^2,
        O_L = sum_{pq,spin} B^L_pq E_pq."""
        n = self.n
        hp = h - 0.5 * np.einsum("Lpr,Lrq->pq", B, B)
        H = sp.csr_matrix((self.dim, self.dim))
        ops = {}
        for s in (0, 1):
            for p in range(n):
                for q in range(n):
                    ops[(s, p, q)] = self.E(s * n + p, s * n + q)
        for (s, p, q), Ep in ops.items():
            if hp[p, q] != 0.0:
                H = H + hp[p, q] * Ep
        for L in range(B.shape[0]):
            O = sp.csr_matrix((self.dim, self.dim))
            for (s, p, q), Ep in ops.items():
                if B[L, p, q] != 0.0:
                    O = O + B[L, p, q] * Ep
            H = H + 0.5 * (O @ O)
        return H.toarray()


def cluster_operator(space, fr: Frame, t1, t2):
    """T = sum t_ia a+_a a_i + sum_{i<j,a<b} t_ijab a+_a a+_b a_j a_i for the
    frame's spin-orbital ordering (a+_a a+_b a_j a_i = E_ai E_bj since the
    occupied and virtual sets are disjoint)."""
    n = space.n
    og = [int(s * n + p) for p, s in zip(fr.occ_sp, fr.occ_spin)]
    vg = [int(s * n + p) for p, s in zip(fr.vir_sp, fr.vir_spin)]
    T = sp.csr_matrix((space.dim, space.dim))
    for i, a in zip(*np.nonzero(t1)):
        T = T + t1[i, a] * space.E(vg[a], og[i])
    no, nv = len(og), len(vg)
    for i in range(no):
        for j in range(i + 1, no):
            for a in range(nv):
                for b in range(a + 1, nv):
                    x = t2[i, j, a, b]
                    if x != 0.0:
                        T = T + x * (space.E(vg[a], og[i]) @ space.E(vg[b], og[j]))
    return T


def expm_apply(T, x, nmax=64):
    out, term = x.copy(), x.copy()
    for k in range(1, nmax):
        term = T @ term / k
        if not np.any(term):
            break
        out += term
    return out


def excited(fr: Frame, det, holes, parts, n):
    og = [int(s * n + p) for p, s in zip(fr.occ_sp, fr.occ_spin)]
    vg = [int(s * n + p) for p, s in zip(fr.vir_sp, fr.vir_spin)]
    return apply_excitation(det, [og[i] for i in holes], [vg[a] for a in parts])


def project_singles_doubles(space, fr, det, vec):
    """<Phi_q|vec> for all singles [o,v] and doubles [o,o,v,v] of det
    (dense spin-orbital arrays)."""
    n = space.n
    no, nv = len(fr.occ_sp), len(fr.vir_sp)
    r1 = np.zeros((no, nv))
    r2 = np.zeros((no, no, nv, nv))
    for i in range(no):
        for a in range(nv):
            d, s = excited(fr, det, [i], [a], n)
            if d is not None and d in space.index:
                r1[i, a] = s * vec[space.index[d]]
    for i in range(no):
        for j in range(no):
            if i == j:
                continue
            for a in range(nv):
                for b in range(nv):
                    if a == b:
                        continue
                    d, s = excited(fr, det, [i, j], [a, b], n)
                    if d is not None and d in space.index:
                        r2[i, j, a, b] = s * vec[space.index[d]]
    return r1, r2


class Brute:
    """CI-vector evaluation of the 2D quantities for one tiny system."""

    def __init__(self, sys):
        self.sys = sys
        n = sys.n
        self.space = DetSpace(n, sys.n_c + 1, sys.n_c + 1)
        self.H = self.space.hamiltonian(sys.h, sys.B)

    def frame(self, ref):
        s = self.sys
        return Frame(s.n_c, s.n_v, s.B, s.fock_a, s.fock_b, ref)

    def ccsd_residual(self, ref, t1, t2):
        """R^CC_q = <Phi_q| exp(-T) (H - E_ref) exp(T) |Phi> (dense spin-orbital)."""
        fr = self.frame(ref)
        det = frame_det(fr)
        x0 = self.space.vec(det)
        eref = x0 @ self.H @ x0
        T = cluster_operator(self.space, fr, t1, t2)
        w = expm_apply(T, x0)
        w = self.H @ w - eref * w
        w = expm_apply(-T, w)
        return project_singles_doubles(self.space, fr, det, w)

    def twod(self, ref, t1, t2, t1o, t2o):
        """Omega1, Omega2 (Bloch form), c^A, c^B, W = <B|H_N exp(T_A)|A>,
        dE_A, and the residuals R1 = Omega1, R2 = Omega2 - A[t1 Omega1].  The
        amplitudes must satisfy the C-condition <B|exp(T_A)|A> = 0."""
        fr, fro = self.frame(ref), self.frame(1 - ref)
        detA, detB = frame_det(fr), frame_det(fro)
        xA = self.space.vec(detA)
        eref = xA @ self.H @ xA
        TA = cluster_operator(self.space, fr, t1, t2)
        TB = cluster_operator(self.space, fro, t1o, t2o)
        eA = expm_apply(TA, xA)
        eB = expm_apply(TB, self.space.vec(detB))
        hN = self.H @ eA - eref * eA
        dEA = xA @ hN
        hbar = expm_apply(-TA, hN)
        i, j, a, b = fr.q_ab()
        d, s = excited(fr, detA, [i, j], [a, b], self.space.n)
        # W = <B| H_N exp(T_A) |A> (the Bloch effective Hamiltonian with
        # intermediate normalisation, <B|exp(T_A)|A> = 0)
        W = s * hN[self.space.index[d]]
        h1, h2 = project_singles_doubles(self.space, fr, detA, hN)
        cA1, cA2 = project_singles_doubles(self.space, fr, detA, eA)
        cB1, cB2 = project_singles_doubles(self.space, fr, detA, eB)
        O1 = h1 - cA1 * dEA - cB1 * W
        O2 = h2 - cA2 * dEA - cB2 * W
        tO = np.einsum("ia,jb->ijab", t1, O1)
        tO = tO - tO.transpose(1, 0, 2, 3)
        tO = tO - tO.transpose(0, 1, 3, 2)
        R2 = O2 - tO
        for (p, q, r, s_) in ((i, j, a, b), (j, i, a, b), (i, j, b, a), (j, i, b, a)):
            R2[p, q, r, s_] = 0.0
        return dict(R1=O1, R2=R2, cB1=cB1, cB2=cB2, W=W, dEA=dEA, eref=eref)


def fci_two_electron(sys):
    """Eigenpairs of H in the M_s = 0 two-electron space (n_c = 0)."""
    space = DetSpace(sys.n, 1, 1)
    H = space.hamiltonian(sys.h, sys.B)
    w, V = np.linalg.eigh(H)
    return space, w, V


def s_squared(space_n, coeffs):
    """<S^2> of an M_s = 0 state given as {det: coef}: ||S+ Psi||^2 with
    S+ = sum_p a+_{p alpha} a_{p beta}."""
    n = space_n
    out = {}
    for d, c in coeffs.items():
        for p in range(n):
            d1, s1 = annihilate(d, n + p)
            d2, s2 = create(d1, p)
            if d2 is not None:
                out[d2] = out.get(d2, 0.0) + s1 * s2 * c
    norm = sum(c * c for c in coeffs.values())
    return sum(c * c for c in out.values()) / norm
