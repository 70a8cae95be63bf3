"""Single-reference spin-orbital CCSD residual, energy and the DC modification
(oracle; test infrastructure only).

R^CC_q = <Phi_q| exp(-T) H_N exp(T) |Phi>, the connected single-reference
residual that opens Eqs. 3 and 4 of the paper (Section II), written with the
textbook spin-orbital intermediates of Stanton, Gauss, Watts and Bartlett
(J. Chem. Phys. 94, 4334 (1991)), valid for a non-diagonal Fock matrix (ROHF
and 2D-SCF orbitals, Section III).  The residual keeps the diagonal Fock
terms, so that R = 0 is the amplitude equation itself.

Notation: i,j,m,n occupied; a,b,e,f virtual spin-orbitals; P(pq) X = X -
X(p<->q); <pq||rs> antisymmetrised integrals.
"""
from __future__ import annotations

import numpy as np

E = lambda s, *a: np.einsum(s, *a, optimize=True)  # noqa: E731


def P_ij(x):
    return x - x.transpose(1, 0, 2, 3)


def P_ab(x):
    return x - x.transpose(0, 1, 3, 2)


def taus(t1, t2):
    tt = E("ia,jb->ijab", t1, t1)
    tt = tt - tt.transpose(0, 1, 3, 2)
    return t2 + 0.5 * tt, t2 + tt  # tau-tilde, tau


def energy(fr, t1, t2):
    """Delta E_A = <Phi|H_N exp(T)|Phi> = sum f_ia t_ia + 1/4 <ij||ab> t_ijab
    + 1/2 <ij||ab> t_ia t_jb (first term of Eq. 2)."""
    g = fr.g("oovv")
    return (E("ia,ia->", fr.f("ov"), t1) + 0.25 * E("ijab,ijab->", g, t2)
            + 0.5 * E("ijab,ia,jb->", g, t1, t1))


def ccsd_residual(fr, t1, t2, a_chunk=16):
    """(R1[o,v], R2[o,o,v,v]) spin-orbital CCSD residual for frame fr."""
    f_oo, f_ov, f_vv, f_vo = fr.f("oo"), fr.f("ov"), fr.f("vv"), fr.f("vo")
    g_oooo, g_ooov, g_oovo = fr.g("oooo"), fr.g("ooov"), fr.g("oovo")
    g_oovv, g_ovov, g_ovvo = fr.g("oovv"), fr.g("ovov"), fr.g("ovvo")
    g_ovvv, g_vovv, g_ovoo, g_vvvo = fr.g("ovvv"), fr.g("vovv"), fr.g("ovoo"), fr.g("vvvo")
    tau_t, tau = taus(t1, t2)

    # one-particle intermediates (diagonal Fock kept)
    Fae = (f_vv - 0.5 * E("me,ma->ae", f_ov, t1) + E("mf,mafe->ae", t1, g_ovvv)
           - 0.5 * E("mnaf,mnef->ae", tau_t, g_oovv))
    Fmi = (f_oo + 0.5 * E("ie,me->mi", t1, f_ov) + E("ne,mnie->mi", t1, g_ooov)
           + 0.5 * E("inef,mnef->mi", tau_t, g_oovv))
    Fme = f_ov + E("nf,mnef->me", t1, g_oovv)

    # two-particle intermediates
    x = E("je,mnie->mnij", t1, g_ooov)
    Wmnij = g_oooo + (x - x.transpose(0, 1, 3, 2)) + 0.25 * E("ijef,mnef->mnij", tau, g_oovv)
    Wmbej = (g_ovvo + E("jf,mbef->mbej", t1, g_ovvv) - E("nb,mnej->mbej", t1, g_oovo)
             - E("jnfb,mnef->mbej", 0.5 * t2 + E("jf,nb->jnfb", t1, t1), g_oovv))

    # singles
    R1 = (f_vo.T + E("ie,ae->ia", t1, Fae) - E("ma,mi->ia", t1, Fmi)
          + E("imae,me->ia", t2, Fme) - E("nf,naif->ia", t1, g_ovov)
          - 0.5 * E("imef,maef->ia", t2, g_ovvv) - 0.5 * E("mnae,nmei->ia", t2, g_oovo))

    # doubles
    R2 = g_oovv.copy()
    R2 += P_ab(E("ijae,be->ijab", t2, Fae - 0.5 * E("mb,me->be", t1, Fme)))
    R2 -= P_ij(E("imab,mj->ijab", t2, Fmi + 0.5 * E("je,me->mj", t1, Fme)))
    R2 += 0.5 * E("mnab,mnij->ijab", tau, Wmnij)
    # 1/2 sum_ef tau_ij^ef W_abef, W_abef = <ab||ef> - P(ab) t_m^b <am||ef>
    #   + 1/4 tau_mn^ab <mn||ef>; built for a few rows a at a time (memory only)
    nv = t1.shape[1]
    for a0 in range(0, nv, a_chunk):
        rows = np.arange(a0, min(nv, a0 + a_chunk))
        W = fr.g_vvvv_rows(rows)
        W -= E("mb,amef->abef", t1, g_vovv[rows])
        W += E("ma,bmef->abef", t1[:, rows], g_vovv)
        W += 0.25 * E("mnab,mnef->abef", tau[:, :, rows, :], g_oovv)
        R2[:, :, rows, :] += 0.5 * E("ijef,abef->ijab", tau, W)
    ring = E("imae,mbej->ijab", t2, Wmbej) - E("ie,ma,mbej->ijab", t1, t1, g_ovvo)
    R2 += P_ij(P_ab(ring))
    R2 += P_ij(E("ie,abej->ijab", t1, g_vvvo))
    R2 -= P_ab(E("ma,mbij->ijab", t1, g_ovoo))
    return R1, R2


def dc_delta(fr, t2):
    """Distinguishable-cluster modification of the doubles residual.

    Reading (Section II applies DC to the doubles as in single-reference DCSD and
    defers the term list to its DC reference): of the four T2*T2 terms of
    the CCD doubles residual -- the ladder 1/4 <mn||ef> t_ij^ef t_mn^ab, the
    ring 1/2 P(ij)P(ab) <mn||ef> t_im^ae t_jn^bf and the two Fock-like terms
    -1/2 P(ij) t_im^ab <mn||ef> t_jn^ef and -1/2 P(ab) t_ij^ae <mn||ef>
    t_mn^bf -- DC keeps the ladder, keeps only the direct (intra-cluster)
    Coulomb part <mn|ef> of the ring, and keeps only the direct part of the
    Fock-like terms, which for antisymmetric amplitudes is one half.  T1
    enters DCSD through the T1-similarity-transformed Hamiltonian, which
    leaves the occupied-virtual <mn||ef> unchanged, so the modification is a
    function of t2 alone.  Returns DCSD doubles - CCSD doubles:
      + 1/2 P(ij)P(ab) <mn|fe> t_im^ae t_jn^bf
      + 1/4 P(ij) t_im^ab t_jn^ef <mn||ef>
      + 1/4 P(ab) t_ij^ae t_mn^bf <mn||ef>.
    Parity unpinned against the DC literature.  Pinned: its switch-off
    limit, spin-flip symmetry and orbital-rotation invariance, equality with
    the closed-shell list, cancellation for two electrons, and covariance
    under the particle-hole relabeling (which requires the hole and the
    particle Fock-like terms to be treated alike)."""
    g = fr.g("oovv")
    gx = fr.g_direct("oovv").transpose(0, 1, 3, 2)  # gx[m,n,e,f] = <mn|fe>
    ring = E("imae,mnef,jnbf->ijab", t2, gx, t2)
    occ = E("imab,jnef,mnef->ijab", t2, t2, g)
    vir = E("ijae,mnbf,mnef->ijab", t2, t2, g)
    return 0.5 * P_ij(P_ab(ring)) + 0.25 * P_ij(occ) + 0.25 * P_ab(vir)
