"""Spin-orbital bookkeeping for the oracle (test infrastructure only).

A *frame* is the determinant the amplitudes are normal-ordered to:
ref 0 = Phi_A (core^2, t alpha, u beta), ref 1 = Phi_B (core^2, u alpha,
t beta) -- the two determinants of Fig. 1, related by flipping the spins of
the open orbitals t and u (Section II).

Spin-orbital basis of a frame: occupied = [alpha-occ..., beta-occ...],
virtual = [alpha-vir..., beta-vir...], with the per-spin spatial lists of
``synth.frame_orbitals`` (core..., t|u) and (u|t, V...).

Antisymmetrised integrals <pq||rs> = (pr|qs) d(sp,sr) d(sq,ss)
                                    - (ps|qr) d(sp,ss) d(sq,sr),
with (pq|rs) = sum_L B[L,p,q] B[L,r,s] (density fitting).

The Fock matrices given as input are those of Phi_A.  For frame B the alpha
Fock matrix is the input beta one and vice versa: that is what a spin-free
Hamiltonian gives (the occupations of Phi_B are the spin flip of Phi_A's),
and it defines the method for general inputs.
"""
from __future__ import annotations

import numpy as np

from synth import frame_orbitals

ALPHA, BETA = 0, 1


class Frame:
    def __init__(self, n_c, n_v, B, fock_a, fock_b, ref, eri=None):
        self.n_c, self.n_v, self.ref = n_c, n_v, ref
        self.n = n_c + 2 + n_v
        self.o, self.v = n_c + 1, n_v + 1
        oa, ob, va, vb = frame_orbitals(n_c, n_v, ref)
        self.occ_sp = np.array(oa + ob)
        self.occ_spin = np.array([ALPHA] * len(oa) + [BETA] * len(ob))
        self.vir_sp = np.array(va + vb)
        self.vir_spin = np.array([ALPHA] * len(va) + [BETA] * len(vb))
        self.B = B
        self.eri = eri  # four-index (pq|rs) used instead of B when given
        fa, fb = (fock_a, fock_b) if ref == 0 else (fock_b, fock_a)
        self.fock = (fa, fb)
        self._cache = {}

    # --- index spaces -------------------------------------------------------
    def space(self, k):
        return (self.occ_sp, self.occ_spin) if k == "o" else (self.vir_sp, self.vir_spin)

    # --- Fock matrix in the spin-orbital basis ------------------------------
    def f(self, kinds):
        (sp, ss), (sq, sq_s) = self.space(kinds[0]), self.space(kinds[1])
        out = np.zeros((len(sp), len(sq)))
        for s in (ALPHA, BETA):
            mp, mq = ss == s, sq_s == s
            out[np.ix_(mp, mq)] = self.fock[s][np.ix_(sp[mp], sq[mq])]
        return out

    # --- <pq||rs> blocks -----------------------------------------------------
    def _coul(self, k1, k2, k3, k4):
        """<pq|rs> = (pr|qs) d(s_p,s_r) d(s_q,s_s) for p in k1, q in k2, r in k3, s in k4."""
        (p, ps), (q, qs), (r, rs), (s, ss) = (self.space(k) for k in (k1, k2, k3, k4))
        if self.eri is not None:
            g = self.eri[np.ix_(p, r, q, s)].transpose(0, 2, 1, 3).copy()
        else:
            Bpr = self.B[:, p][:, :, r]
            Bqs = self.B[:, q][:, :, s]
            g = np.einsum("Lpr,Lqs->pqrs", Bpr, Bqs, optimize=True)
        g *= (ps[:, None] == rs[None, :])[:, None, :, None]
        g *= (qs[:, None] == ss[None, :])[None, :, None, :]
        return g

    def g(self, kinds):
        """Antisymmetrised <pq||rs> for the index kinds, e.g. 'oovv'."""
        if kinds in self._cache:
            return self._cache[kinds]
        k1, k2, k3, k4 = kinds
        val = self._coul(k1, k2, k3, k4) - self._coul(k1, k2, k4, k3).transpose(0, 1, 3, 2)
        if kinds != "vvvv":
            self._cache[kinds] = val
        return val

    def g_direct(self, kinds):
        """The non-antisymmetrised <pq|rs> (direct Coulomb part) block."""
        return self._coul(*kinds)

    def g_vvvv_rows(self, a_idx):
        """<ab||ef> for the virtual indices a in a_idx (all b, e, f)."""
        (v, vs) = self.space("v")
        pa, psa = v[a_idx], vs[a_idx]
        if self.eri is not None:
            g1 = self.eri[np.ix_(pa, v, v, v)].transpose(0, 2, 1, 3).copy()
        else:
            Bae = self.B[:, pa][:, :, v]
            Bbf = self.B[:, v][:, :, v]
            g1 = np.einsum("Lae,Lbf->abef", Bae, Bbf, optimize=True)
        g1 *= (psa[:, None] == vs[None, :])[:, None, :, None]
        g1 *= (vs[:, None] == vs[None, :])[None, :, None, :]
        g2 = g1.transpose(0, 1, 3, 2)
        return g1 - g2

    # --- reference -> excitation positions ---------------------------------
    def q_ab(self):
        """Spin-orbital positions (i, j, a, b) of the double excitation that
        maps this frame's determinant onto the other one (t alpha -> u alpha,
        u beta -> t beta for Phi_A; the spin flip for Phi_B)."""
        o, v = self.o, self.v
        return (o - 1, o + o - 1, 0, v + 0)


# ----------------------------------------------------------------------------
# ABI layout <-> dense spin-orbital arrays
# ----------------------------------------------------------------------------

def unpack(o, v, T):
    """(T1a, T1b, T2aa, T2bb, T2ab) in the ABI layout -> t1[2o,2v], t2[2o,2o,2v,2v]."""
    T1a, T1b, T2aa, T2bb, T2ab = T
    t1 = np.zeros((2 * o, 2 * v))
    t1[:o, :v] = T1a
    t1[o:, v:] = T1b
    t2 = np.zeros((2 * o, 2 * o, 2 * v, 2 * v))
    t2[:o, :o, :v, :v] = T2aa
    t2[o:, o:, v:, v:] = T2bb
    t2[:o, o:, :v, v:] = T2ab
    t2[o:, :o, :v, v:] = -T2ab.transpose(1, 0, 2, 3)
    t2[:o, o:, v:, :v] = -T2ab.transpose(0, 1, 3, 2)
    t2[o:, :o, v:, :v] = T2ab.transpose(1, 0, 3, 2)
    return t1, t2


def pack(o, v, t1, t2):
    """Dense spin-orbital arrays -> ABI layout (alpha-alpha, beta-beta and
    alpha(occ i, vir a)-beta(occ j, vir b) blocks)."""
    return (t1[:o, :v].copy(), t1[o:, v:].copy(), t2[:o, :o, :v, :v].copy(),
            t2[o:, o:, v:, v:].copy(), t2[:o, o:, :v, v:].copy())


def flip_abi(T):
    """Amplitudes of the spin-flipped determinant: T_B = F T_A F^-1 with F the
    alpha<->beta substitution (Section II: amplitudes normal-ordered to one
    determinant follow from those of the other by flipping the spin).  In
    the ABI layout of the other frame this swaps the alpha and beta blocks
    and transposes the mixed one."""
    T1a, T1b, T2aa, T2bb, T2ab = T
    return (T1b.copy(), T1a.copy(), T2bb.copy(), T2aa.copy(),
            T2ab.transpose(1, 0, 3, 2).copy())


# ----------------------------------------------------------------------------
# Fock matrices and reference energy from a core Hamiltonian (pin systems)
# ----------------------------------------------------------------------------

def fock_from_h(h, B, n_c, ref=0):
    """f^sigma_pq = h_pq + sum_{k sigma' occ} [(pq|kk) - d(sigma,sigma') (pk|kq)]
    for the occupations of Phi_A (ref 0) or Phi_B (ref 1); also returns the
    reference energy <Phi|H|Phi> = sum_k h_kk + 1/2 sum_kl <kl||kl>."""
    n = h.shape[0]
    oa, ob, _, _ = frame_orbitals(n_c, n - n_c - 2, ref)
    J = np.einsum("Lpq,Lkk->pq", B, B[:, oa][:, :, oa]) + np.einsum("Lpq,Lkk->pq", B, B[:, ob][:, :, ob])
    Ka = np.einsum("Lpk,Lkq->pq", B[:, :, oa], B[:, oa, :])
    Kb = np.einsum("Lpk,Lkq->pq", B[:, :, ob], B[:, ob, :])
    fa = h + J - Ka
    fb = h + J - Kb
    e = np.trace(h[np.ix_(oa, oa)]) + np.trace(h[np.ix_(ob, ob)])
    e += 0.5 * (np.trace((J - Ka)[np.ix_(oa, oa)]) + np.trace((J - Kb)[np.ix_(ob, ob)]))
    return fa, fb, e
