"""Two-determinant (2D-CCSD / 2D-DCSD) residual layer (oracle; test
infrastructure only).

Section II, Eqs. 2-4.  With the Jeziorski-Monkhorst wave operator
exp(T_A)|A><A| + exp(T_B)|B><B| and intermediate normalisation, projecting
the Bloch equation onto an excited determinant <A_q| gives

  Omega_q = <A_q| H_N exp(T_A) |A> - c^A_q dE_A - c^B_q W = 0,
  c^X_q   = <A_q| exp(T_X) |X>,   W = <B| H_N exp(T_A) |A>.

Splitting off the single-reference connected part R^CC (first term of
Eqs. 3/4) this reads, for singles and doubles,

  R1_ia   = R^CC_ia   - W c^B_ia
  R2_ijab = R^CC_ijab - W ( c^B_ijab - A(ij;ab)[ t_ia c^B_jb ] ),

the M*W renormalisation terms of Eqs. 3-4 (R2 = Omega2 - A[t1 Omega1]).
The A->B doubles amplitude is fixed by the C-condition (``c_condition``:
zero in the CAS case, as the text after Eq. 4 states), W = <B|H_N e^{T_A}|A>
is the residual element of that excitation (plus the internal-singles
products of the IAS case) and the element itself is then zeroed.
T_B is T_A with alpha and beta exchanged (Section II).  The coefficients
c^B_q are evaluated exactly by cluster-to-CI algebra on determinants, so no
term with a spin-orbital occurring twice can arise (the omission the paper
makes explicit after Eq. 4).  DC changes only R^CC (Section II: the M terms
are not modified by DC); W is then the DC residual element.

Phase convention: Phi_B is the canonically ordered (alpha string, then beta
string, ascending orbitals) determinant, which equals E_{A->B} Phi_A; with it
the singlet is dE_A + W and the triplet dE_A - W (Eq. 2 and text after Eq.
4), checked by <S^2> in the brute-force tests.
"""
from __future__ import annotations

import numpy as np

from . import ccsd
from .spinorb import Frame, unpack, pack, flip_abi

CCSD, DCSD = 0, 1


# ----------------------------------------------------------------------------
# determinants as sorted gid tuples; gid = spin * n + spatial
# ----------------------------------------------------------------------------

def annihilate(det, p):
    if det is None or p not in det:
        return None, 0
    k = det.index(p)
    return det[:k] + det[k + 1:], (-1) ** k


def create(det, p):
    if det is None or p in det:
        return None, 0
    k = sum(1 for x in det if x < p)
    return det[:k] + (p,) + det[k:], (-1) ** k


def apply_excitation(det, holes, parts):
    """E = a+_{A1} ... a+_{Ak} a_{Ik} ... a_{I1} applied to det; returns
    (det', sign) or (None, 0)."""
    s = 1
    for p in holes:
        det, s1 = annihilate(det, p)
        s *= s1
    for p in reversed(parts):
        det, s1 = create(det, p)
        s *= s1
    return det, s


def frame_det(fr):
    n = fr.n
    return tuple(sorted(int(s * n + p) for p, s in zip(fr.occ_sp, fr.occ_spin)))


# ----------------------------------------------------------------------------
# cluster-to-CI coefficient, symbolic in the index tokens
# ----------------------------------------------------------------------------

def expand(I, A):
    """Coefficient of E_I^A |Phi> in exp(T1 + T2)|Phi> as a list of
    (sign, factors); factor = ('t1', i, a) or ('t2', i, j, a, b).

    The cluster holding the first hole I[0] is either a single I[0] -> A[p]
    or a double (I[0], I[q]) -> (A[p], A[r]), p < r; moving its operators to
    the front of E_I^A costs (-1)^p, resp. (-1)^(p+r+q) (0-based positions),
    and the remaining clusters give the coefficient of the rest."""
    if not I:
        return [(1, [])]
    i1, k = I[0], len(I)
    out = []
    for p in range(k):
        for s, f in expand(I[1:], A[:p] + A[p + 1:]):
            out.append(((-1) ** p * s, [("t1", i1, A[p])] + f))
    for q in range(1, k):
        for p in range(k):
            for r in range(p + 1, k):
                sg = (-1) ** (p + r + q)
                restI = I[1:q] + I[q + 1:]
                restA = [A[x] for x in range(k) if x not in (p, r)]
                for s, f in expand(restI, restA):
                    out.append((sg * s, [("t2", i1, I[q], A[p], A[r])] + f))
    return out


class _Tok:
    """Free index token: ranges over a domain of spin-orbitals."""

    def __init__(self, name, gids, spin):
        self.name, self.gids, self.spin = name, list(gids), spin

    def __repr__(self):
        return self.name


def c_other(fr: Frame, fro: Frame, t1o, t2o):
    """c1[o,v], c2[o,o,v,v] (dense spin-orbital, this frame) with
    c_q = <Phi_q^this| exp(T_other) |Phi_other>."""
    n, o, v = fr.n, fr.o, fr.v
    no, nv_ = 2 * o, 2 * v
    gid_occ = [int(s * n + p) for p, s in zip(fr.occ_sp, fr.occ_spin)]
    gid_vir = [int(s * n + p) for p, s in zip(fr.vir_sp, fr.vir_spin)]
    pos_o_other = {int(s * n + p): k for k, (p, s) in enumerate(zip(fro.occ_sp, fro.occ_spin))}
    pos_v_other = {int(s * n + p): k for k, (p, s) in enumerate(zip(fro.vir_sp, fro.vir_spin))}
    pos_o_this = {g: k for k, g in enumerate(gid_occ)}
    pos_v_this = {g: k for k, g in enumerate(gid_vir)}
    det_this, det_other = frame_det(fr), frame_det(fro)
    active = {fr.n_c, fr.n_c + 1}
    spin_of = lambda g: g // n  # noqa: E731

    def choices(gids):
        fixed = [("fix", g) for g in gids if g % n in active]
        free = []
        for s in (0, 1):
            dom = [g for g in gids if g % n not in active and spin_of(g) == s]
            if dom:
                free.append(("free", tuple(dom), s))
        return fixed + free

    occ_ch, vir_ch = choices(gid_occ), choices(gid_vir)
    c1 = np.zeros((no, nv_))
    c2 = np.zeros((no, no, nv_, nv_))

    def chspin(c):
        return spin_of(c[1]) if c[0] == "fix" else c[2]

    def build_class(chs, names):
        # free tokens with representatives (two representative sets)
        used = {}
        toks, reps1, reps2 = [], [], []
        for c, nm in zip(chs, names):
            if c[0] == "fix":
                toks.append(c[1])
                reps1.append(c[1])
                reps2.append(c[1])
                continue
            dom = c[1]
            k = used.get(dom, 0)
            used[dom] = k + 1
            if k >= len(dom):
                return None
            tk = _Tok(nm, dom, c[2])
            toks.append(tk)
            reps1.append(dom[k])
            reps2.append(dom[min(len(dom) - 1, k + 1)] if len(dom) > k + 1 else None)
        return toks, reps1, reps2

    def excitation_tokens(toks, reps, nocc_q):
        holes, parts = reps[:nocc_q], reps[nocc_q:]
        D, s1 = apply_excitation(det_this, holes, parts)
        if D is None:
            return None
        I = [g for g in det_other if g not in D]
        A = [g for g in D if g not in det_other]
        D2, s2 = apply_excitation(det_other, I, A)
        assert D2 == D
        rmap = {}
        for tk, r in zip(toks, reps):
            if isinstance(tk, _Tok):
                rmap[r] = tk
        It = [rmap.get(g, g) for g in I]
        At = [rmap.get(g, g) for g in A]
        return s1 * s2, It, At

    def check_sign(toks, reps2, nocc_q, s, It, At):
        if any(r is None for r in reps2):
            return
        holes, parts = reps2[:nocc_q], reps2[nocc_q:]
        D, s1 = apply_excitation(det_this, holes, parts)
        rmap = {tk.name: r for tk, r in zip(toks, reps2) if isinstance(tk, _Tok)}
        conc = lambda x: rmap[x.name] if isinstance(x, _Tok) else x  # noqa: E731
        D2, s2 = apply_excitation(det_other, [conc(x) for x in It], [conc(x) for x in At])
        assert D2 == D and s1 * s2 == s, "class sign depends on index values"

    def tok_spin(x):
        return x.spin if isinstance(x, _Tok) else spin_of(x)

    def factor_array(f):
        kind, idx = f[0], f[1:]
        arr = t1o if kind == "t1" else t2o
        nh = 1 if kind == "t1" else 2
        sel, labels = [], []
        for k, x in enumerate(idx):
            pos = pos_o_other if k < nh else pos_v_other
            if isinstance(x, _Tok):
                sel.append(np.array([pos[g] for g in x.gids]))
                labels.append(x.name)
            else:
                sel.append(np.array([pos[x]]))
        val = arr[np.ix_(*sel)]
        keep = [k for k, x in enumerate(idx) if isinstance(x, _Tok)]
        val = val.reshape([val.shape[k] for k in keep])
        return val, labels

    def spin_ok(f):
        idx = f[1:]
        if f[0] == "t1":
            return tok_spin(idx[0]) == tok_spin(idx[1])
        return sorted([tok_spin(idx[0]), tok_spin(idx[1])]) == sorted([tok_spin(idx[2]), tok_spin(idx[3])])

    def evaluate(toks, s, It, At):
        free = [t for t in toks if isinstance(t, _Tok)]
        shape = [len(t.gids) for t in free]
        out_lbl = "".join(t.name for t in free)
        total = np.zeros(shape)
        for sg, facs in expand(It, At):
            if not all(spin_ok(f) for f in facs):
                continue
            ops, subs = [], []
            for f in facs:
                val, lbl = factor_array(f)
                ops.append(val)
                subs.append("".join(lbl))
            total += sg * np.einsum(",".join(subs) + "->" + out_lbl, *ops) if ops else sg
        return s * total

    def scatter_index(toks, kinds):
        sel = []
        for tk, k in zip(toks, kinds):
            pos = pos_o_this if k == "o" else pos_v_this
            if isinstance(tk, _Tok):
                sel.append(np.array([pos[g] for g in tk.gids]))
            else:
                sel.append(np.array([pos[tk]]))
        return np.ix_(*sel)

    # singles
    for ci in occ_ch:
        for ca in vir_ch:
            if chspin(ci) != chspin(ca):
                continue
            r = build_class([ci, ca], ["i", "a"])
            if r is None:
                continue
            toks, reps1, reps2 = r
            ex = excitation_tokens(toks, reps1, 1)
            if ex is None:
                continue
            s, It, At = ex
            check_sign(toks, reps2, 1, s, It, At)
            val = evaluate(toks, s, It, At)
            shape = [len(t.gids) if isinstance(t, _Tok) else 1 for t in toks]
            c1[scatter_index(toks, "ov")] = val.reshape(shape)

    # doubles
    for ci in occ_ch:
        for cj in occ_ch:
            if ci[0] == "fix" and ci == cj:
                continue
            for ca in vir_ch:
                for cb in vir_ch:
                    if ca[0] == "fix" and ca == cb:
                        continue
                    if sorted([chspin(ci), chspin(cj)]) != sorted([chspin(ca), chspin(cb)]):
                        continue
                    r = build_class([ci, cj, ca, cb], ["i", "j", "a", "b"])
                    if r is None:
                        continue
                    toks, reps1, reps2 = r
                    ex = excitation_tokens(toks, reps1, 2)
                    if ex is None:
                        continue
                    s, It, At = ex
                    check_sign(toks, reps2, 2, s, It, At)
                    val = evaluate(toks, s, It, At)
                    shape = [len(t.gids) if isinstance(t, _Tok) else 1 for t in toks]
                    c2[scatter_index(toks, "oovv")] = val.reshape(shape)
    # repeated spin-orbitals are not determinants
    ii = np.arange(no)
    c2[ii, ii, :, :] = 0.0
    aa = np.arange(nv_)
    c2[:, :, aa, aa] = 0.0
    return c1, c2


# ----------------------------------------------------------------------------
# the two-determinant residual
# ----------------------------------------------------------------------------

def frames(sys, ref):
    eri = getattr(sys, "eri", None)
    fr = Frame(sys.n_c, sys.n_v, sys.B, sys.fock_a, sys.fock_b, ref, eri=eri)
    fro = Frame(sys.n_c, sys.n_v, sys.B, sys.fock_a, sys.fock_b, 1 - ref, eri=eri)
    return fr, fro


def c_condition(T):
    """ABI amplitudes with the A->B doubles element fixed by the C-condition.

    Intermediate normalisation of the Jeziorski-Monkhorst wave operator
    requires <other| exp(T) |this> = 0.  That coefficient is the A->B doubles
    amplitude plus the product of the two internal singles t alpha -> u
    alpha and u beta -> t beta (sign +1 in both frames, checked with CI
    vectors), so the element equals -T1a[o-1,0] T1b[o-1,0].  In the CAS case
    of Section II the internal singles vanish by symmetry and the element is
    zero, as the paper states; in the IAS case they do not (Section II: the
    terms with the all-internal singles have to be included)."""
    T = tuple(np.array(x, dtype=float) for x in T)
    o = T[0].shape[0]
    T[4][o - 1, o - 1, 0, 0] = -T[0][o - 1, 0] * T[1][o - 1, 0]
    return T


def _c_condition_so(fr, t1, t2):
    i, j, a, b = fr.q_ab()
    t2 = t2.copy()
    val = -t1[i, a] * t1[j, b]
    t2[i, j, a, b], t2[j, i, a, b], t2[i, j, b, a], t2[j, i, b, a] = val, -val, -val, val
    return t2


def residual_so(fr, fro, method, t1, t2, t1o, t2o):
    """Spin-orbital 2D residual; returns (R1, R2, W, dE_A, R1cc, R2cc).  The
    A->B element of t2 and t2o is set by the C-condition first.

    W = <B| H_N exp(T_A) |A> = R^X_AB + A(ij;ab)[t_ia R^X_jb] at the A->B
    double (and + c^A_AB dE_A, zero by the C-condition): the residual element
    of the text after Eq. 4, plus the internal-singles products that the IAS
    case adds (zero in the CAS case)."""
    t2 = _c_condition_so(fr, t1, t2)
    t2o = _c_condition_so(fro, t1o, t2o)
    R1x, R2x = ccsd.ccsd_residual(fr, t1, t2)
    if method == DCSD:
        R2x = R2x + ccsd.dc_delta(fr, t2)
    i, j, a, b = fr.q_ab()
    W = (R2x[i, j, a, b] + t1[i, a] * R1x[j, b] - t1[j, a] * R1x[i, b] - t1[i, b] * R1x[j, a]
         + t1[j, b] * R1x[i, a])
    c1, c2 = c_other(fr, fro, t1o, t2o)
    tc = np.einsum("ia,jb->ijab", t1, c1)
    tc = ccsd.P_ij(ccsd.P_ab(tc))
    R1 = R1x - W * c1
    R2 = R2x - W * (c2 - tc)
    for (p, q, r, s, sg) in ((i, j, a, b, 1), (j, i, a, b, -1), (i, j, b, a, -1), (j, i, b, a, 1)):
        R2[p, q, r, s] = 0.0
    dE = ccsd.energy(fr, t1, t2)
    return R1, R2, W, dE, R1x, R2x


def residual(sys, ref, method, T):
    """ABI-level oracle call: T = (T1a, T1b, T2aa, T2bb, T2ab) normal-ordered
    to Phi_A (ref 0) or Phi_B (ref 1).  Returns (R, W, dE_A) with R in the
    same layout."""
    fr, fro = frames(sys, ref)
    T = c_condition(T)
    t1, t2 = unpack(fr.o, fr.v, T)
    t1o, t2o = unpack(fr.o, fr.v, flip_abi(T))
    R1, R2, W, dE, _, _ = residual_so(fr, fro, method, t1, t2, t1o, t2o)
    return pack(fr.o, fr.v, R1, R2), W, dE
