"""Single elements of the 2D-CCSD / 2D-DCSD residual (oracle; test
infrastructure only).

The full oracle (``twod.residual``) forms every residual element at once
from dense spin-orbital integral blocks, which limits it to small systems.
This module evaluates chosen elements R1_ia and R2_ijab, for systems of any
size, from the same definitions:

* the connected residual R^X (first term of Eqs. 3 and 4, Section II) with
  the textbook spin-orbital CCSD intermediates of Stanton, Gauss, Watts and
  Bartlett (J. Chem. Phys. 94, 4334 (1991)), as in ``ccsd.ccsd_residual``,
  each term restated for one element;
* the DC modification of ``ccsd.dc_delta`` for one element;
* the coupling R = R^X - W c (M W terms of Eqs. 3-4) with
  c_q = <Phi_q| exp(T_other) |Phi_other> from the cluster-to-CI expansion of
  ``twod.expand`` for the one determinant E_q Phi, and W the residual
  element of the A->B double.

Integrals are never stored as four-index blocks: <pq|rs> = (pr|qs) with
(pq|rs) = sum_L B_pq^L B_rs^L, and every contraction over two integral
indices is done through the DF factors (amplitudes contracted into B first).
Spin-orbital indices follow ``spinorb.Frame``: occupied 0..2o-1 (alpha
then beta), virtual 0..2v-1.
"""
from __future__ import annotations

import numpy as np

from . import twod
from .spinorb import flip_abi

E = lambda s, *a: np.einsum(s, *a, optimize=True)  # noqa: E731


class DF:
    """Contractions with the spin-orbital DF block B[l,m,e] (l auxiliary, m
    occupied, e virtual), each written as a matrix product over a layout
    prepared once, so that no call copies the block."""

    def __init__(self, Bov):
        L, o, v = Bov.shape
        self.B = Bov
        self.F = Bov.reshape(L, o * v)                                   # [l, (m,e)]
        self.R = Bov.reshape(L * o, v)                                   # [(l,m), e]
        self.T = np.ascontiguousarray(Bov.transpose(1, 0, 2)).reshape(o, L * v)  # [m, (l,e)]
        self.L, self.o, self.v = L, o, v

    def lm_e(self, Y):
        """sum_{l,m} B[l,m,e] Y[l,m]"""
        return Y.reshape(-1) @ self.R

    def le_m(self, Z):
        """sum_{l,e} B[l,m,e] Z[l,e]"""
        return self.T @ Z.reshape(-1)

    def e(self, x):
        """sum_e B[l,m,e] x[e] -> [l,m]"""
        return (self.R @ x).reshape(self.L, self.o)

    def m(self, x):
        """sum_m x[m] B[l,m,e] -> [l,e]"""
        return (x @ self.T).reshape(self.L, self.v)

    def me(self, A):
        """sum_{m,e} A[..., m, e] B[l,m,e] -> [..., l]"""
        return A.reshape(-1, self.o * self.v) @ self.F.T if A.ndim > 2 else self.F @ A.reshape(-1)

    def me_f(self, A):
        """sum_{m,e} B[l,m,e] A[m,e,f] -> [l,f]"""
        return self.F @ A.reshape(self.o * self.v, -1)

    def mf_e(self, A):
        """sum_{m,f} A[m,e,f] B[l,m,f] -> [l,e]"""
        out = np.zeros((self.L, A.shape[1]))
        for m in range(self.o):
            out += self.B[:, m, :] @ A[m].T
        return out

    def f_right(self, Y):
        """sum_f B[l,m,f] Y[n,f] -> [l,m,n]"""
        return (self.R @ Y.T).reshape(self.L, self.o, -1)

    def ln_me(self, X):
        """sum_{l,n} X[l,m,n] B[l,n,e] -> [m,e]"""
        return np.ascontiguousarray(X.transpose(1, 0, 2)).reshape(X.shape[1], -1) @ self.R

    def sandwich_vv(self, M):
        """sum_{l,m,n} B[l,m,e] M[m,n] B[l,n,f] -> [e,f]"""
        MB = (M @ self.T).reshape(self.o, self.L, self.v)  # [m,l,f] = sum_n M[m,n] B[l,n,f]
        return self.R.T @ np.ascontiguousarray(MB.transpose(1, 0, 2)).reshape(self.L * self.o, self.v)

    def sandwich_oo(self, M):
        """sum_{l,e,f} B[l,m,e] M[e,f] B[l,n,f] -> [m,n]"""
        Y = np.ascontiguousarray((self.R @ M).reshape(self.L, self.o, -1).transpose(1, 0, 2)).reshape(self.o, -1)
        return Y @ self.T.T

    def trace4(self, A, C):
        """sum_{l,m,n,e,f} A[m,e] B[l,n,e] C[n,f] B[l,m,f]"""
        P = (self.R @ A.T).reshape(self.L, self.o, -1)  # [l,n,m] = sum_e B[l,n,e] A[m,e]
        Q = (self.R @ C.T).reshape(self.L, self.o, -1)  # [l,m,n] = sum_f B[l,m,f] C[n,f]
        return float(np.sum(P * Q.transpose(0, 2, 1)))


class Amplitudes:
    """Dense spin-orbital views of ABI amplitudes, built slice by slice.

    t2[p,q,r,s] for spin-orbital p, q (occupied) and r, s (virtual) from
    the alpha-alpha, beta-beta and alpha-beta blocks, with the signs of the
    antisymmetric spin-orbital tensor (as ``spinorb.unpack``)."""

    def __init__(self, fr, T):
        self.o, self.v = fr.o, fr.v
        self.T1a, self.T1b, self.T2aa, self.T2bb, self.T2ab = (np.asarray(x, dtype=float) for x in T)
        o, v = self.o, self.v
        self.t1 = np.zeros((2 * o, 2 * v))
        self.t1[:o, :v] = self.T1a
        self.t1[o:, v:] = self.T1b

    def t2(self, p, q, r, s):
        """Sub-array of t2 for index selections p, q, r, s: an int, or
        slice(None) for the whole axis (a selected int drops its axis)."""
        o, v = self.o, self.v
        sels = (p, q, r, s)
        for x in sels:
            assert isinstance(x, (int, np.integer)) or x == slice(None)
        full = (2 * o, 2 * o, 2 * v, 2 * v)
        out = np.zeros([full[k] for k in range(4) if isinstance(sels[k], slice)])
        blocks = (  # spins of (p, q, r, s) (1 = beta), source block, its axis order, sign
            ((0, 0, 0, 0), self.T2aa, (0, 1, 2, 3), 1.0),
            ((1, 1, 1, 1), self.T2bb, (0, 1, 2, 3), 1.0),
            ((0, 1, 0, 1), self.T2ab, (0, 1, 2, 3), 1.0),
            ((1, 0, 0, 1), self.T2ab, (1, 0, 2, 3), -1.0),
            ((0, 1, 1, 0), self.T2ab, (0, 1, 3, 2), -1.0),
            ((1, 0, 1, 0), self.T2ab, (1, 0, 3, 2), 1.0),
        )
        size = (o, o, v, v)
        for spins, src, tr, sign in blocks:
            dst, loc, ok = [], [], True
            for k in range(4):
                x = sels[k]
                if isinstance(x, slice):
                    dst.append(slice(spins[k] * size[k], (spins[k] + 1) * size[k]))
                    loc.append(slice(None))
                else:
                    if int(x) // size[k] != spins[k]:
                        ok = False
                        break
                    loc.append(int(x) % size[k])
            if not ok:
                continue
            # source indexed in its own axis order; then back to (p, q, r, s)
            order = [None] * 4
            for k in range(4):
                order[tr[k]] = loc[k]
            val = src[tuple(order)]
            kept = [k for k in range(4) if isinstance(loc[k], slice)]
            perm = sorted(range(len(kept)), key=lambda a: tr[kept[a]])  # axes of val, in source order
            val = val.transpose(np.argsort(perm)) if len(kept) > 1 else val
            out[tuple(dst)] = sign * val
        return out


class ElementOracle:
    """Residual elements of one frame (ref) for ABI amplitudes T."""

    def __init__(self, sys, ref, method, T):
        self.method = method
        self.fr, self.fro = twod.frames(sys, ref)
        fr = self.fr
        self.o, self.v = fr.o, fr.v
        T = twod.c_condition(T)
        self.T = Amplitudes(fr, T)
        self.To = Amplitudes(fr, flip_abi(T))  # T_other in this frame's ABI layout
        self.t1 = self.T.t1
        # spin-orbital DF factors: B_so[L][p][q] = B[L][sp(p)][sp(q)] if the spins agree
        osp, osn, vsp, vsn = fr.occ_sp, fr.occ_spin, fr.vir_sp, fr.vir_spin
        B = sys.B
        self.Boo = B[:, osp][:, :, osp] * (osn[:, None] == osn[None, :])
        self.Bov = B[:, osp][:, :, vsp] * (osn[:, None] == vsn[None, :])
        self._B, self._vsp, self._vsn = B, vsp, vsn
        self.df = df = DF(self.Bov)
        self.f_oo, self.f_ov, self.f_vv = fr.f("oo"), fr.f("ov"), fr.f("vv")
        self.f_vo = fr.f("vo")
        t1 = self.t1
        # c_L = sum_nf t_nf B_nf^L;  F_me = f_me + t_nf <mn||ef> = f_me + t_nf ((me|nf) - (mf|ne))
        self.cL = df.me(t1)
        self.Fme = self.f_ov + (self.cL @ df.F).reshape(df.o, df.v) - df.ln_me(df.f_right(t1))
        self._W = None
        self._cache = {}

    # --- integrals -----------------------------------------------------------
    def Bvv(self, x):
        """B_so[L][x][e] for virtual x and all virtual e."""
        return self._B[:, self._vsp[x]][:, self._vsp] * (self._vsn[x] == self._vsn)[None, :]

    def tau(self, p, q, r, s, half=False):
        """tau (half=False) or tau-tilde (half=True) sub-array:
        t2_pqrs + c (t_pr t_qs - t_ps t_qr), c = 1 or 1/2; selectors as for t2."""
        c = 0.5 if half else 1.0
        t1, sel, lab = self.t1, (p, q, r, s), "pqrs"
        out = "".join(lab[k] for k in range(4) if isinstance(sel[k], slice))
        prod = 0.0
        for (a1, b1, a2, b2), sg in (((0, 2, 1, 3), 1.0), ((0, 3, 1, 2), -1.0)):
            sx = "".join(lab[k] for k in (a1, b1) if isinstance(sel[k], slice))
            sy = "".join(lab[k] for k in (a2, b2) if isinstance(sel[k], slice))
            prod = prod + sg * np.einsum(f"{sx},{sy}->{out}", t1[sel[a1], sel[b1]], t1[sel[a2], sel[b2]])
        return self.T.t2(p, q, r, s) + c * prod

    # --- one-particle intermediates -------------------------------------------
    def Fae_row(self, x):
        """F_xe for all e: f_xe - 1/2 f_me t_mx + t_mf <mx||fe> - 1/2 tau~_mnxf <mn||ef>."""
        key = ("Fae", x)
        if key in self._cache:
            return self._cache[key]
        df, t1 = self.df, self.t1
        Bx = self.Bvv(x)
        r = self.f_vv[x].copy() - 0.5 * (t1[:, x] @ self.f_ov)
        # t_mf <mx||fe> = t_mf (mf|xe) - t_mf (me|xf)
        r += self.cL @ Bx - df.lm_e(Bx @ t1.T)
        tt = self.tau(slice(None), slice(None), x, slice(None), half=True)  # [m,n,f]
        # tau~_mnxf ((me|nf) - (mf|ne))
        r -= 0.5 * (df.lm_e(df.me(tt).T) - df.lm_e(df.me(tt.transpose(1, 0, 2)).T))
        self._cache[key] = r
        return r

    def Fmi_col(self, i):
        """F_mi for all m: f_mi + 1/2 t_ie f_me + t_ne <mn||ie> + 1/2 tau~_inef <mn||ef>."""
        key = ("Fmi", i)
        if key in self._cache:
            return self._cache[key]
        df, t1, Boo = self.df, self.t1, self.Boo
        r = self.f_oo[:, i] + 0.5 * (self.f_ov @ t1[i])
        # t_ne <mn||ie> = t_ne (mi|ne) - t_ne (me|ni)
        r += Boo[:, :, i].T @ self.cL - df.le_m(Boo[:, :, i] @ t1)
        tt = self.tau(i, slice(None), slice(None), slice(None), half=True)  # [n,e,f]
        # 1/2 tau~_inef ((me|nf) - (mf|ne))
        r += 0.5 * (df.le_m(df.mf_e(tt)) - df.le_m(df.me_f(tt)))
        self._cache[key] = r
        return r

    # --- the connected residual ----------------------------------------------
    def r1x(self, i, a):
        df, t1, Boo, Bov = self.df, self.t1, self.Boo, self.Bov
        Ba = self.Bvv(a)
        r = self.f_vo[a, i] + t1[i] @ self.Fae_row(a) - t1[:, a] @ self.Fmi_col(i)
        r += np.sum(self.T.t2(i, slice(None), a, slice(None)) * self.Fme)
        # - t_nf <na||if> = - t_nf ((ni|af) - (nf|ai))
        r -= np.sum((Boo[:, :, i] @ t1) * Ba) - self.cL @ Bov[:, i, a]
        # - 1/2 t_imef <ma||ef> = - 1/2 t_imef ((me|af) - (mf|ae))
        ti = self.T.t2(i, slice(None), slice(None), slice(None))  # [m,e,f]
        r -= 0.5 * (np.sum(df.me_f(ti) * Ba) - np.sum(df.mf_e(ti) * Ba))
        # - 1/2 t_mnae <nm||ei> = - 1/2 t_mnae ((ne|mi) - (ni|me))
        ta = self.T.t2(slice(None), slice(None), a, slice(None))  # [m,n,e]
        r -= 0.5 * (np.sum(df.me(ta).T * Boo[:, :, i]) - np.sum(df.me(ta.transpose(1, 0, 2)).T * Boo[:, :, i]))
        return float(r)

    def _Wmbej(self, s, q):
        """W_msEq for all m, e at virtual s and occupied q (Stanton-Gauss W_mbej)."""
        df, t1, Boo, Bov = self.df, self.t1, self.Boo, self.Bov
        Bs = self.Bvv(s)
        # <ms||eq> = (me|sq) - (mq|se)
        g = (Bov[:, q, s] @ df.F).reshape(df.o, df.v) - Boo[:, :, q].T @ Bs
        # + t_qf <ms||ef> = t_qf ((me|sf) - (mf|se))
        g2 = ((Bs @ t1[q]) @ df.F).reshape(df.o, df.v) - df.e(t1[q]).T @ Bs
        # - t_ns <mn||eq> = - t_ns ((me|nq) - (mq|ne))
        g3 = ((Boo[:, :, q] @ t1[:, s]) @ df.F).reshape(df.o, df.v) - Boo[:, :, q].T @ df.m(t1[:, s])
        Y = 0.5 * self.T.t2(q, slice(None), slice(None), s) + np.outer(t1[:, s], t1[q])  # [n,f]
        # - Y_nf <mn||ef> = - Y_nf ((me|nf) - (mf|ne))
        g4 = (df.me(Y) @ df.F).reshape(df.o, df.v) - df.ln_me(df.f_right(Y))
        return g + g2 - g3 - g4, g

    def _ring(self, p, q, r, s):
        """t_pmre W_msEq - t_pe t_mr <ms||eq> (one element of the ring term)."""
        W, g = self._Wmbej(s, q)
        return float(np.sum(self.T.t2(p, slice(None), r, slice(None)) * W) - self.t1[p] @ (self.t1[:, r] @ g))

    def _Wabef(self, a, b):
        """W_abef for all e, f: <ab||ef> - t_mb <am||ef> + t_ma <bm||ef> + 1/4 tau_mnab <mn||ef>."""
        df, t1 = self.df, self.t1
        Ba, Bb = self.Bvv(a), self.Bvv(b)
        W = Ba.T @ Bb - Bb.T @ Ba
        # t_mb <am||ef> = t_mb ((ae|mf) - (af|me))
        ub, ua = df.m(t1[:, b]), df.m(t1[:, a])
        W -= Ba.T @ ub - ub.T @ Ba
        W += Bb.T @ ua - ua.T @ Bb
        # 1/4 tau_mnab ((me|nf) - (mf|ne))
        X = df.sandwich_vv(self.tau(slice(None), slice(None), a, b))
        W += 0.25 * (X - X.T)
        return W

    def _Wmnij(self, i, j):
        """W_mnij for all m, n: <mn||ij> + P(ij) t_je <mn||ie> + 1/4 tau_ijef <mn||ef>."""
        df, t1, Boo = self.df, self.t1, self.Boo
        W = Boo[:, :, i].T @ Boo[:, :, j] - Boo[:, :, j].T @ Boo[:, :, i]

        def x(i_, j_):  # t_j_e <mn||i_ e> = t_j_e ((mi_|ne) - (me|ni_))
            u = df.e(t1[j_])  # [l,n] = sum_e B[l,n,e] t_j_e
            return Boo[:, :, i_].T @ u - u.T @ Boo[:, :, i_]
        W += x(i, j) - x(j, i)
        X = df.sandwich_oo(self.tau(i, j, slice(None), slice(None)))
        W += 0.25 * (X - X.T)
        return W

    def r2x(self, i, j, a, b):
        t1, Boo, Bov = self.t1, self.Boo, self.Bov
        Ba, Bb = self.Bvv(a), self.Bvv(b)
        r = float(Bov[:, i, a] @ Bov[:, j, b] - Bov[:, i, b] @ Bov[:, j, a])  # <ij||ab>

        def G(x):  # F_xe - 1/2 t_mx F_me
            return self.Fae_row(x) - 0.5 * self.t1[:, x] @ self.Fme

        r += self.T.t2(i, j, a, slice(None)) @ G(b) - self.T.t2(i, j, b, slice(None)) @ G(a)

        def H(y):  # F_my + 1/2 t_ye F_me
            return self.Fmi_col(y) + 0.5 * self.Fme @ t1[y]

        r -= self.T.t2(i, slice(None), a, b) @ H(j) - self.T.t2(j, slice(None), a, b) @ H(i)
        r += 0.5 * np.sum(self.tau(slice(None), slice(None), a, b) * self._Wmnij(i, j))
        r += 0.5 * np.sum(self.tau(i, j, slice(None), slice(None)) * self._Wabef(a, b))
        r += (self._ring(i, j, a, b) - self._ring(j, i, a, b) - self._ring(i, j, b, a) + self._ring(j, i, b, a))

        def X7(i_, j_):  # t_i_e <ab||e j_> = t_i_e ((ae|b j_) - (a j_|be))
            return t1[i_] @ (Ba.T @ Bov[:, j_, b]) - t1[i_] @ (Bb.T @ Bov[:, j_, a])
        r += X7(i, j) - X7(j, i)

        def X8(a_, b_):  # t_m a_ <m b_||ij> = t_m a_ ((mi|b_ j) - (mj|b_ i))
            return t1[:, a_] @ (Boo[:, :, i].T @ Bov[:, j, b_]) - t1[:, a_] @ (Boo[:, :, j].T @ Bov[:, i, b_])
        r -= X8(a, b) - X8(b, a)
        if self.method == twod.DCSD:
            r += self.dc(i, j, a, b)
        return float(r)

    def ladder(self, i, j, a, b):
        """The particle-particle ladder piece 1/2 sum_ef tau_ijef <ab||ef> of
        R2_ijab (the <ab||ef> part of the W_abef term above), one element.
        Used to show how much of an element a broken ladder would change."""
        Ba, Bb = self.Bvv(a), self.Bvv(b)
        g = Ba.T @ Bb - Bb.T @ Ba  # <ab||ef> = (ae|bf) - (af|be)
        return 0.5 * float(np.sum(self.tau(i, j, slice(None), slice(None)) * g))

    def dc(self, i, j, a, b):
        """DCSD - CCSD doubles (``ccsd.dc_delta``) at one element."""
        df = self.df
        t2 = self.T.t2
        sl = slice(None)

        def ring(p, q, r, s):  # t_pmre <mn|fe> t_qnsf, <mn|fe> = (mf|ne)
            return df.trace4(t2(p, sl, r, sl), t2(q, sl, s, sl))

        def Z(q):  # sum_nef t_qnef <mn||ef> = t_qnef ((me|nf) - (mf|ne)) for all m
            tq = t2(q, sl, sl, sl)
            return df.le_m(df.mf_e(tq)) - df.le_m(df.me_f(tq))

        def Zv(s):  # sum_mnf t_mnsf <mn||ef> = t_mnsf ((me|nf) - (mf|ne)) for all e
            ts = t2(sl, sl, s, sl)
            return df.lm_e(df.me(ts).T) - df.lm_e(df.me(ts.transpose(1, 0, 2)).T)

        def occ(p, q, r, s):
            return t2(p, sl, r, s) @ Z(q)

        def vir(p, q, r, s):
            return t2(p, q, r, sl) @ Zv(s)
        return float(0.5 * (ring(i, j, a, b) - ring(j, i, a, b) - ring(i, j, b, a) + ring(j, i, b, a))
                     + 0.25 * (occ(i, j, a, b) - occ(j, i, a, b)) + 0.25 * (vir(i, j, a, b) - vir(i, j, b, a)))

    # --- coupling ---------------------------------------------------------------
    def c(self, holes, parts):
        """c_q = <Phi_q| exp(T_other) |Phi_other> for q = holes -> parts (spin-orbital
        positions of this frame), by the cluster-to-CI expansion of the one
        determinant E_q Phi_this relative to Phi_other."""
        fr, fro, n = self.fr, self.fro, self.fr.n
        gid_o = [int(s * n + p) for p, s in zip(fr.occ_sp, fr.occ_spin)]
        gid_v = [int(s * n + p) for p, s in zip(fr.vir_sp, fr.vir_spin)]
        D, s1 = twod.apply_excitation(twod.frame_det(fr), [gid_o[h] for h in holes], [gid_v[p] for p in parts])
        if D is None:
            return 0.0
        det_o = twod.frame_det(fro)
        I = [g for g in det_o if g not in D]
        A = [g for g in D if g not in det_o]
        D2, s2 = twod.apply_excitation(det_o, I, A)
        assert D2 == D
        pos_o = {int(s * n + p): k for k, (p, s) in enumerate(zip(fro.occ_sp, fro.occ_spin))}
        pos_v = {int(s * n + p): k for k, (p, s) in enumerate(zip(fro.vir_sp, fro.vir_spin))}
        To = self.To
        total = 0.0
        for sg, facs in twod.expand(I, A):
            prod = float(sg)
            for f in facs:
                if f[0] == "t1":
                    prod *= To.t1[pos_o[f[1]], pos_v[f[2]]]
                else:
                    prod *= float(To.t2(pos_o[f[1]], pos_o[f[2]], pos_v[f[3]], pos_v[f[4]]))
                if prod == 0.0:
                    break
            total += prod
        return s1 * s2 * total

    def energy(self):
        """Delta E_A = f_ia t_ia + 1/4 <ij||ab> t_ijab + 1/2 <ij||ab> t_ia t_jb (first
        term of Eq. 2), summed one occupied spin-orbital i at a time."""
        df, t1, Bov = self.df, self.t1, self.Bov
        e = float(np.sum(self.f_ov * t1))
        for i in range(2 * self.o):
            ti = self.T.t2(i, slice(None), slice(None), slice(None))  # [j,a,b]
            # sum_jab <ij||ab> t_ijab = sum_jab ((ia|jb) - (ib|ja)) t_ijab
            direct = np.sum(Bov[:, i, :] * df.mf_e(ti))  # sum_{L,a} B_ia sum_{j,b} t_ijab B_jb
            exch = np.sum(Bov[:, i, :] * df.me_f(ti))    # sum_{L,b} B_ib sum_{j,a} B_ja t_ijab
            # sum_jab <ij||ab> t_ia t_jb = sum_L (B_ia t_ia)(B_jb t_jb) - sum_jab (ib|ja) t_ia t_jb
            P = Bov[:, i, :] @ t1.T                      # [L,j] = sum_b B_ib t_jb
            Q = df.e(t1[i])                              # [L,j] = sum_a B_ja t_ia
            tt = (Bov[:, i, :] @ t1[i]) @ self.cL - np.sum(P * Q)
            e += 0.25 * (direct - exch) + 0.5 * tt
        return e

    def W(self):
        """W = <B|H_N exp(T_A)|A>: the connected (DC) residual element of the
        A->B double plus A(ij;ab)[t_ia R^X_jb] there (the internal-singles
        products, zero in the CAS case; ``twod.residual_so``)."""
        if self._W is None:
            i, j, a, b = self.fr.q_ab()
            t1 = self.t1
            w = self.r2x(i, j, a, b)
            for (p, q, r, u, sg) in ((i, a, j, b, 1.0), (j, b, i, a, 1.0), (j, a, i, b, -1.0), (i, b, j, a, -1.0)):
                if t1[p, q] != 0.0:
                    w += sg * t1[p, q] * self.r1x(r, u)
            self._W = w
        return self._W

    # --- the 2D residual -----------------------------------------------------------
    def r1(self, i, a):
        """R1_ia = R^X_ia - W c_ia (Eqs. 3-4)."""
        return self.r1x(i, a) - self.W() * self.c([i], [a])

    def r2(self, i, j, a, b):
        """R2_ijab = R^X_ijab - W (c_ijab - A(ij;ab)[t_ia c_jb]); 0 at the A->B
        double and its permutations (Eqs. 3-4 and the text after Eq. 4)."""
        qi, qj, qa, qb = self.fr.q_ab()
        if {i, j} == {qi, qj} and {a, b} == {qa, qb}:
            return 0.0
        if i == j or a == b:
            return 0.0
        t1 = self.t1
        c1 = lambda p, r: self.c([p], [r])  # noqa: E731
        tc = t1[i, a] * c1(j, b) - t1[j, a] * c1(i, b) - t1[i, b] * c1(j, a) + t1[j, b] * c1(i, a)
        return self.r2x(i, j, a, b) - self.W() * (self.c([i, j], [a, b]) - tc)


def abi_to_so(o, v, block, idx):
    """Spin-orbital position of an ABI element: block 0..4 = T1a, T1b, T2aa,
    T2bb, T2ab; idx its (i, a) or (i, j, a, b)."""
    if block == 0:
        return (idx[0], idx[1])
    if block == 1:
        return (o + idx[0], v + idx[1])
    i, j, a, b = idx
    if block == 2:
        return (i, j, a, b)
    if block == 3:
        return (o + i, o + j, v + a, v + b)
    return (i, o + j, a, v + b)


def residual_element(eo: ElementOracle, block, idx):
    """One element of the ABI residual (R1a, R1b, R2aa, R2bb, R2ab)."""
    so = abi_to_so(eo.o, eo.v, block, idx)
    return eo.r1(*so) if block < 2 else eo.r2(*so)
