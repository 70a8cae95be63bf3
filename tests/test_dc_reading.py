"""The distinguishable-cluster (DC) modification of the oracle (ccsd.dc_delta)
against its closed-shell statement.

The paper applies DC to the doubles "in the usual way" and defers the term
list to the DC literature (Section II).  The reading transcribed in
ccsd.dc_delta is stated in DESIGN in the closed-shell, spin-adapted form in
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
      place, fails D1 or D2.

What this does not do: compare the list with the published equations
themselves, which are not available offline (parity of the DC term set is
unpinned against the literature; see DESIGN).
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
