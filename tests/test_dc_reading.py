"""The distinguishable-cluster (DC) modification of the oracle (ccsd.dc_delta)
against its closed-shell statement.

The paper applies DC to the single-reference doubles equations as that
method does and leaves the term list to the DC literature (Section II).  The reading transcribed in
ccsd.dc_delta is stated here in the closed-shell, spin-adapted form in
which the DC equations were first published: of the T2*T2 terms of the CCD
doubles, DC keeps

  * the ladder term       sum_kl T^kl_ab sum_cd (kc|ld) T^ij_cd,
  * the direct ring term  sum_{kc,ld} Tt^ik_ac (kc|ld) Tt^jl_bd,
  * half of the two Fock-like terms, built with the same Tt:
      - 1/2 sum_k (T^ik_ab x_kj + T^kj_ab x_ki),   x_kj = sum_lcd (kc|ld) Tt^jl_cd
      - 1/2 sum_c (T^ij_ac y_cb + T^ij_cb y_ca),   y_cb = sum_kld (kc|ld) Tt^kl_bd

with Tt^ij_ab = 2 T^ij_ab - T^ij_ba, and drops the exchange-type rings.
These tests check, on the CPU:

  D1  the spin-orbital oracle's T2*T2 terms with dc_delta, on closed-shell
      amplitudes, equal the closed-shell list above (written here
      independently, in closed-shell notation), element by element;
  D2  for two electrons (one doubly occupied orbital) the CCD T2*T2 terms
      equal -E_c T (CCD is then exact, a textbook fact), while the DC list
      above cancels exactly: a single electron pair has no second cluster
      to be distinguished from;
  D3  each of three alternative term sets -- exchange rings kept, Fock-like
      terms not halved, ladder halved -- planted here in the oracle's
      place, fails D1 or D2;
  D4  particle-hole relabeling.  Read with the roles of occupied and virtual
      spin orbitals exchanged, e^{-T} H_N e^{T} is the same operator and the
      projections are the same equations: with F' = -F^T, the same <pq|rs>,
      t1' = -t1^T, t2'[a,b,i,j] = t2[i,j,a,b], the CCSD residual maps to
      R1' = -R1^T, R2'[a,b,i,j] = R2[i,j,a,b] and the energy is unchanged
      (an exact identity, checked for the oracle's CCSD).  The relabeling
      exchanges the hole and the particle Fock-like terms and maps the
      ladder and the direct ring to themselves, so a T2*T2 modification
      keeps the identity only if it treats the two Fock-like terms alike:
      the DC list does; halving only one of them, planted here, does not.
      (Exchange rings kept and the ladder halved keep the identity: D4 does
      not decide those, D1-D3 do.)

What this does not do: compare the list with the published equations
themselves, which are not available offline (parity of the DC term set is
unpinned against the literature).
"""
import numpy as np
import pytest

from synth import make_system
from oracle import ccsd
from oracle.spinorb import ALPHA, BETA, Frame

E = lambda s, *a: np.einsum(s, *a, optimize=True)  # noqa: E731


def closed_frame(s, nocc):
    """Spin-orbital frame of the closed-shell determinant that doubly
    occupies spatial orbitals 0..nocc-1 (alpha and beta Fock = fock_a)."""
    fr = Frame(s.n_c, s.n_v, s.B, s.fock_a, s.fock_a, 0)
    occ, vir = list(range(nocc)), list(range(nocc, s.n))
    fr.occ_sp = np.array(occ + occ)
    fr.occ_spin = np.array([ALPHA] * nocc + [BETA] * nocc)
    fr.vir_sp = np.array(vir + vir)
    fr.vir_spin = np.array([ALPHA] * len(vir) + [BETA] * len(vir))
    return fr


def closed_amplitudes(rng, o, v, scale):
    """Spin-adapted T[i,j,a,b] = T^ij_ab with T^ij_ab = T^ji_ba, and its
    spin-orbital form: alpha-beta block T, same-spin blocks T - T(a<->b)."""
    T = rng.normal(0, scale, (o, o, v, v))
    T = 0.5 * (T + T.transpose(1, 0, 3, 2))
    t2 = np.zeros((2 * o, 2 * o, 2 * v, 2 * v))
    ss = T - T.transpose(0, 1, 3, 2)
    t2[:o, :o, :v, :v] = ss
    t2[o:, o:, v:, v:] = ss
    t2[:o, o:, :v, v:] = T
    t2[o:, :o, :v, v:] = -T.transpose(1, 0, 2, 3)
    t2[:o, o:, v:, :v] = -T.transpose(0, 1, 3, 2)
    t2[o:, :o, v:, :v] = T.transpose(1, 0, 3, 2)
    return T, t2


def quadratic_so(fr, t2, dc_fn):
    """The T2*T2 part of the spin-orbital doubles residual at t1 = 0:
    R(t) = R0 + L(t) + Q(t), so Q(t) = (R(t) + R(-t)) / 2 - R(0)."""
    z1 = np.zeros((t2.shape[0], t2.shape[2]))

    def R(x):
        r2 = ccsd.ccsd_residual(fr, z1, x)[1]
        return r2 + dc_fn(fr, x) if dc_fn is not None else r2
    return 0.5 * (R(t2) + R(-t2)) - R(np.zeros_like(t2))


def ovov(s, nocc):
    """(kc|ld) as K[k,c,l,d] for occupied k,l and virtual c,d (spatial)."""
    Bov = s.B[:, :nocc, nocc:]
    return E("Lkc,Lld->kcld", Bov, Bov)


def dc_closed(T, K):
    """The closed-shell DC T2*T2 list of the module docstring."""
    Tt = 2.0 * T - T.transpose(0, 1, 3, 2)
    lad = E("klab,kcld,ijcd->ijab", T, K, T)
    ring = E("ikac,kcld,jlbd->ijab", Tt, K, Tt)
    x = E("kcld,jlcd->kj", K, Tt)
    y = E("kcld,klbd->cb", K, Tt)
    hole = -0.5 * (E("ikab,kj->ijab", T, x) + E("kjab,ki->ijab", T, x))
    part = -0.5 * (E("ijac,cb->ijab", T, y) + E("ijcb,ca->ijab", T, y))
    return lad + ring + hole + part


def _setup(nocc, nv, X, seed):
    s = make_system((nocc - 1, nv, X), seed=seed)  # spatial orbitals only; the open-shell labels are unused
    s.n_c = nocc - 1
    fr = closed_frame(s, nocc)
    o, v = nocc, s.n - nocc
    T, t2 = closed_amplitudes(np.random.default_rng(seed), o, v, 0.05)
    return s, fr, T, t2, o, v


@pytest.mark.parametrize("nocc,nv,X,seed", [(2, 4, 10, 1), (3, 5, 12, 2), (4, 3, 9, 3)])
def test_d1_spin_orbital_dc_equals_closed_shell_list(nocc, nv, X, seed):
    s, fr, T, t2, o, v = _setup(nocc, nv, X, seed)
    Q = quadratic_so(fr, t2, ccsd.dc_delta)
    ref = dc_closed(T, ovov(s, o))
    assert np.abs(Q[:o, o:, :v, v:] - ref).max() < 1e-14
    assert np.abs(ref).max() > 1e-5
    # the same-spin blocks are the antisymmetrised closed-shell list
    ss = ref - ref.transpose(0, 1, 3, 2)
    assert np.abs(Q[:o, :o, :v, :v] - ss).max() < 1e-14


@pytest.mark.parametrize("nv,X,seed", [(4, 10, 4), (6, 12, 5)])
def test_d2_two_electrons(nv, X, seed):
    s, fr, T, t2, o, v = _setup(1, nv + 1, X, seed)
    K = ovov(s, 1)
    Ec = float(E("kcld,klcd->", K, 2.0 * T - T.transpose(0, 1, 3, 2)))
    q_ccd = quadratic_so(fr, t2, None)[:o, o:, :v, v:]
    assert np.abs(q_ccd + Ec * T).max() < 1e-15 + 1e-12 * np.abs(q_ccd).max()
    q_dc = quadratic_so(fr, t2, ccsd.dc_delta)[:o, o:, :v, v:]
    assert np.abs(q_dc).max() < 1e-15 + 1e-12 * np.abs(q_ccd).max()
    assert np.abs(dc_closed(T, K)).max() < 1e-15 + 1e-12 * np.abs(q_ccd).max()
    assert abs(Ec) > 1e-5


def _variants():
    def ring_exchange_kept(fr, t2):
        g = fr.g("oovv")
        occ = E("imab,jnef,mnef->ijab", t2, t2, g)
        vir = E("ijae,mnbf,mnef->ijab", t2, t2, g)
        return 0.25 * ccsd.P_ij(occ) + 0.25 * ccsd.P_ab(vir)

    def fock_not_halved(fr, t2):
        gx = fr.g_direct("oovv").transpose(0, 1, 3, 2)
        ring = E("imae,mnef,jnbf->ijab", t2, gx, t2)
        return 0.5 * ccsd.P_ij(ccsd.P_ab(ring))

    def ladder_halved(fr, t2):
        g = fr.g("oovv")
        return ccsd.dc_delta(fr, t2) - 0.125 * E("mnab,mnef,ijef->ijab", t2, g, t2)
    return {"ring exchange kept": ring_exchange_kept, "Fock-like terms not halved": fock_not_halved,
            "ladder halved": ladder_halved}


@pytest.mark.parametrize("name", list(_variants()))
def test_d3_alternative_term_sets_fail(name):
    fn = _variants()[name]
    s, fr, T, t2, o, v = _setup(3, 5, 12, 2)
    Q = quadratic_so(fr, t2, fn)[:o, o:, :v, v:]
    d1 = np.abs(Q - dc_closed(T, ovov(s, o))).max()
    s2, fr2, T2, t22, o2, v2 = _setup(1, 5, 10, 4)
    d2 = np.abs(quadratic_so(fr2, t22, fn)[:o2, o2:, :v2, v2:]).max()
    assert d1 > 1e-6 and d2 > 1e-6, (name, d1, d2)


# ---------------------------------------------------------------------------
# D4: particle-hole relabeling
# ---------------------------------------------------------------------------

class DenseFrame:
    """Explicit spin-orbital integrals F[p,q] and direct <pq|rs> over all
    spin orbitals, with the index lists of the occupied and the virtual ones:
    the blocks the oracle's residual functions read."""

    def __init__(self, F, Gd, occ, vir):
        self.F, self.Gd = F, Gd
        self.G = Gd - Gd.transpose(0, 1, 3, 2)
        self.ix = {"o": np.asarray(occ), "v": np.asarray(vir)}

    def f(self, kinds):
        return self.F[np.ix_(self.ix[kinds[0]], self.ix[kinds[1]])]

    def g_direct(self, kinds):
        return self.Gd[np.ix_(*(self.ix[k] for k in kinds))]

    def g(self, kinds):
        return self.G[np.ix_(*(self.ix[k] for k in kinds))]

    def g_vvvv_rows(self, rows):
        v = self.ix["v"]
        return self.G[np.ix_(v[rows], v, v, v)]


def spin_orbital_problem(seed, ns, X, occ_alpha, occ_beta, scale=0.1):
    """Real Hamiltonian on 2*ns spin orbitals (p = P + ns*spin): <pq|rs> =
    (PR|QS) with spin conservation, (PR|QS) = sum_L B_PR B_QS (B symmetric),
    spin-blocked symmetric Fock matrix; an open-shell occupation; random
    spin-conserving t1 and antisymmetric t2."""
    rng = np.random.default_rng(seed)
    B = rng.normal(0, 0.3, (X, ns, ns))
    B = 0.5 * (B + B.transpose(0, 2, 1))
    eri = E("Lpr,Lqs->prqs", B, B)
    n = 2 * ns
    sp, sg = np.arange(n) % ns, np.arange(n) // ns
    Gd = eri[np.ix_(sp, sp, sp, sp)].transpose(0, 2, 1, 3).copy()
    Gd *= (sg[:, None] == sg[None, :])[:, None, :, None]
    Gd *= (sg[:, None] == sg[None, :])[None, :, None, :]
    F = np.zeros((n, n))
    for s in (ALPHA, BETA):
        h = rng.normal(0, 0.05, (ns, ns))
        h = 0.5 * (h + h.T) + np.diag(np.linspace(-1.0, 2.0, ns))
        m = np.where(sg == s)[0]
        F[np.ix_(m, m)] = h
    occ = list(occ_alpha) + [ns + p for p in occ_beta]
    vir = [p for p in range(n) if p not in occ]
    so, sv = sg[occ], sg[vir]
    t1 = rng.normal(0, scale, (len(occ), len(vir))) * (so[:, None] == sv[None, :])
    t2 = rng.normal(0, scale, (len(occ), len(occ), len(vir), len(vir)))
    t2 = t2 - t2.transpose(1, 0, 2, 3)
    t2 = t2 - t2.transpose(0, 1, 3, 2)
    t2 *= (so[:, None, None, None] + so[None, :, None, None]) == (sv[None, None, :, None] + sv[None, None, None, :])
    return DenseFrame(F, Gd, occ, vir), DenseFrame(-F.T, Gd, vir, occ), t1, t2


PH_CASES = [(1, 5, 8, (0, 1, 2), (0, 1)), (2, 6, 9, (0, 1), (0, 1, 2)), (3, 6, 7, (0, 1, 2, 3), (0,))]


@pytest.mark.parametrize("seed,ns,X,occ_a,occ_b", PH_CASES)
def test_d4_ccsd_is_covariant_under_particle_hole_relabeling(seed, ns, X, occ_a, occ_b):
    fr, fp, t1, t2 = spin_orbital_problem(seed, ns, X, occ_a, occ_b)
    t1p, t2p = -t1.T, t2.transpose(2, 3, 0, 1)
    R1, R2 = ccsd.ccsd_residual(fr, t1, t2)
    R1p, R2p = ccsd.ccsd_residual(fp, t1p, t2p)
    assert np.abs(R1p + R1.T).max() < 1e-13 * np.abs(R1).max()
    assert np.abs(R2p - R2.transpose(2, 3, 0, 1)).max() < 1e-13 * np.abs(R2).max()
    e, ep = ccsd.energy(fr, t1, t2), ccsd.energy(fp, t1p, t2p)
    assert abs(e - ep) < 1e-13 * abs(e) and abs(e) > 1e-3


@pytest.mark.parametrize("seed,ns,X,occ_a,occ_b", PH_CASES)
def test_d4_dc_list_is_covariant_under_particle_hole_relabeling(seed, ns, X, occ_a, occ_b):
    fr, fp, t1, t2 = spin_orbital_problem(seed, ns, X, occ_a, occ_b)
    D = ccsd.dc_delta(fr, t2)
    Dp = ccsd.dc_delta(fp, t2.transpose(2, 3, 0, 1))
    assert np.abs(D).max() > 1e-3
    assert np.abs(Dp - D.transpose(2, 3, 0, 1)).max() < 1e-13 * np.abs(D).max()


def _one_fock_like_halved(which):
    def fn(fr, t2):
        g = fr.g("oovv")
        gx = fr.g_direct("oovv").transpose(0, 1, 3, 2)
        ring = 0.5 * ccsd.P_ij(ccsd.P_ab(E("imae,mnef,jnbf->ijab", t2, gx, t2)))
        if which == "hole":
            return ring + 0.25 * ccsd.P_ij(E("imab,jnef,mnef->ijab", t2, t2, g))
        return ring + 0.25 * ccsd.P_ab(E("ijae,mnbf,mnef->ijab", t2, t2, g))
    return fn


@pytest.mark.parametrize("which", ["hole", "particle"])
def test_d4_halving_one_fock_like_term_breaks_covariance(which):
    fn = _one_fock_like_halved(which)
    fr, fp, t1, t2 = spin_orbital_problem(*PH_CASES[0])
    D = fn(fr, t2)
    Dp = fn(fp, t2.transpose(2, 3, 0, 1))
    assert np.abs(Dp - D.transpose(2, 3, 0, 1)).max() > 1e-3 * np.abs(D).max()
