"""FCIDUMP input (Section III: the paper's integrals come in FCIDUMP files)
on the CPU: the library's reader, Cholesky factorisation and preparation
(frozen core, Fock matrices of Phi_A, reference energy) against the oracle's
independent reader and four-index arithmetic, and the oracle's four-index
path against what fixes it.

  * the library reads back exactly what was written (17 significant
    digits), including Fortran D exponents and the "/" header terminator;
  * its Cholesky factors reproduce every (pq|rs) within the threshold;
  * its Fock matrices of Phi_A equal the oracle's; its reference energy
    equals <Phi_A|H|Phi_A> from brute-force CI vectors and does not change
    when core orbitals are frozen (the frozen-core folding is exact for the
    reference determinant);
  * the oracle's residual from four-index integrals equals its residual from
    the factors the integrals were made of;
  * frozen core: the residual of the correlated orbitals from the folded
    integrals equals the all-electron residual at the same elements when
    the frozen orbitals' amplitudes are zero.
"""
import numpy as np
import pytest

from synth import make_pin_system, make_system, random_amplitudes
from synth import fcidump as wfcidump
from oracle import brute, twod
from oracle import fcidump as ofcidump
from oracle.spinorb import fock_from_h


def _write(tmp_path, s, drop=0.0, exp_char="E", name="FCIDUMP"):
    eri = wfcidump.eri_from_factors(s.B)
    nelec = 2 * s.n_c + 2
    path = str(tmp_path / name)
    wfcidump.write(path, s.h, eri, nelec, 0, ecore=1.25, orbsym=[1 + int(p) for p in s.parity], drop=drop,
                   exp_char=exp_char)
    return path, eri


@pytest.fixture
def pin(tmp_path):
    s = make_pin_system(2, 4, 10, seed=3)
    path, eri = _write(tmp_path, s)
    return s, path, eri


def test_library_reads_back_the_file(pin, tmp_path):
    from paper_2401_11935_gb300 import _lib as L
    s, path, eri = pin
    assert L.dcsd_fcidump_header(path) == (s.n, 2 * s.n_c + 2, 0)
    h, e, ec = L.dcsd_fcidump_read(path)
    assert np.array_equal(h, s.h) and np.array_equal(e, eri) and ec == 1.25
    # Fortran exponents and the "/" terminator
    p2 = str(tmp_path / "FCIDUMP_D")
    import re
    txt = re.sub(r"(\d)E([+-])", r"\1D\2", open(path).read()).replace("&END", "/")
    assert "D-" in txt or "D+" in txt
    open(p2, "w").write(txt)
    h2, e2, ec2 = L.dcsd_fcidump_read(p2)
    assert np.array_equal(h2, s.h) and np.array_equal(e2, eri) and ec2 == 1.25
    # the oracle's own reader agrees
    n, nelec, ms2, ho, eo, eco = ofcidump.read(path)
    assert np.array_equal(ho, s.h) and np.array_equal(eo, eri) and eco == 1.25


def test_library_refuses_bad_files(tmp_path):
    from paper_2401_11935_gb300 import _lib as L
    p = tmp_path / "bad"
    p.write_text("no header here\n")
    with pytest.raises(L.DcsdError):
        L.dcsd_fcidump_header(str(p))
    p.write_text(" &FCI NORB=2,NELEC=2,MS2=0, &END\n 0.5 1 1 3 1\n")
    with pytest.raises(L.DcsdError):
        L.dcsd_fcidump_read(str(p))
    p.write_text(" &FCI NORB=3,NELEC=3,MS2=1, &END\n 0.5 1 1 1 1\n")
    with pytest.raises(L.DcsdError):
        L.dcsd_fcidump_prepare(str(p))
    with pytest.raises(L.DcsdError):
        L.dcsd_fcidump_header(str(tmp_path / "missing"))


_HDR = " &FCI NORB={n},NELEC={ne},MS2={ms},{extra} &END\n"
_BAD = [
    # (file text, call, keyword arguments, words of the error message)
    (" &FCI MS2=0, &END\n", "header", {}, "NORB or NELEC"),
    (_HDR.format(n=2, ne=2, ms=0, extra="") .replace("NELEC=2,", ""), "header", {}, "NORB or NELEC"),
    (_HDR.format(n=0, ne=2, ms=0, extra=""), "header", {}, "NORB out of range"),
    (_HDR.format(n=161, ne=2, ms=0, extra=""), "header", {}, "NORB out of range"),
    (_HDR.format(n=2, ne=2, ms=0, extra="IUHF=1,"), "header", {}, "unrestricted"),
    (_HDR.format(n=2, ne=2, ms=0, extra="") + " 0.5 1 x 1 1\n", "read", {}, "malformed integral line 1"),
    (_HDR.format(n=2, ne=2, ms=0, extra="") + " 0.5 1 1 1 1\n\n 0.25 2 2\n", "read", {}, "malformed integral line 3"),
    (_HDR.format(n=2, ne=2, ms=0, extra="") + " 0.5 -1 1 1 1\n", "read", {}, "out of range on integral line 1"),
    (_HDR.format(n=4, ne=4, ms=2, extra="") + " 0.5 1 1 1 1\n", "prepare", {}, "MS2 = 0"),
    (_HDR.format(n=4, ne=3, ms=0, extra="") + " 0.5 1 1 1 1\n", "prepare", {}, "MS2 = 0"),
    (_HDR.format(n=4, ne=4, ms=0, extra="") + " 0.5 1 1 1 1\n", "prepare", {"n_frozen": 2}, "frozen-core count"),
    (_HDR.format(n=3, ne=4, ms=0, extra="") + " 0.5 1 1 1 1\n", "prepare", {}, "at least one virtual"),
    (_HDR.format(n=4, ne=4, ms=0, extra="") + " 0.5 1 1 1 1\n", "prepare", {"chol_tol": 0.0}, "threshold must be positive"),
    (_HDR.format(n=4, ne=4, ms=0, extra="") + " -1.0 1 1 0 0\n 0.3 1 2 0 0\n", "prepare", {}, "zero to the Cholesky"),
]


@pytest.mark.parametrize("text,call,kw,words", _BAD)
def test_library_names_each_bad_input(tmp_path, text, call, kw, words):
    """Each refusal of the host-side reader and preparation comes back as
    INVALID_ARG with its own message (no file is read partially)."""
    from paper_2401_11935_gb300 import _lib as L
    p = tmp_path / "FCIDUMP"
    p.write_text(text)
    fn = {"header": L.dcsd_fcidump_header, "read": L.dcsd_fcidump_read, "prepare": L.dcsd_fcidump_prepare}[call]
    with pytest.raises(L.DcsdError) as ei:
        fn(str(p), **kw)
    assert ei.value.status == 1 and words in str(ei.value), str(ei.value)


def test_library_accepts_the_same_inputs_when_valid(tmp_path):
    """The valid counterparts of the refusals above are read: a header split
    over lines with ORBSYM, blank lines between integrals, D exponents."""
    from paper_2401_11935_gb300 import _lib as L
    p = tmp_path / "FCIDUMP"
    p.write_text(" &FCI NORB=4,NELEC=4,\n  ORBSYM=1,1,1,1,\n  ISYM=1, MS2=0,\n &END\n"
                 " 0.5D0 1 1 1 1\n\n 0.25 2 2 2 2\n 0.125 3 3 3 3\n 0.0625 4 4 4 4\n"
                 " -1.0 1 1 0 0\n -0.5 2 2 0 0\n 0.1 3 3 0 0\n 0.2 4 4 0 0\n 0.75 0 0 0 0\n")
    assert L.dcsd_fcidump_header(str(p)) == (4, 4, 0)
    h, eri, ec = L.dcsd_fcidump_read(str(p))
    assert eri[0, 0, 0, 0] == 0.5 and eri[1, 1, 1, 1] == 0.25 and h[0, 0] == -1.0 and ec == 0.75
    info, fa, fb, B = L.dcsd_fcidump_prepare(str(p), n_frozen=1)
    assert info.n_c == 0 and info.n_v == 1


@pytest.mark.parametrize("tol", [1e-8, 1e-12])
def test_cholesky_reproduces_integrals(pin, tol):
    from paper_2401_11935_gb300 import _lib as L
    s, path, eri = pin
    B, left = L.dcsd_cholesky_host(eri, tol)
    rec = np.einsum("Lpq,Lrs->pqrs", B, B)
    assert np.abs(rec - eri).max() <= max(left, 1e-15) and left <= tol
    assert np.abs(B - B.transpose(0, 2, 1)).max() < 1e-15
    assert B.shape[0] <= s.naux  # the integrals were made from naux factors


@pytest.mark.parametrize("n_frozen", [0, 1, 2])
def test_prepare_fock_and_reference_energy(pin, n_frozen):
    from paper_2401_11935_gb300 import _lib as L
    s, path, eri = pin
    info, fa, fb, B = L.dcsd_fcidump_prepare(path, n_frozen=n_frozen)
    so, eref = ofcidump.system(path, n_frozen=n_frozen)
    assert (info.n_c, info.n_v) == (so.n_c, so.n_v) == (s.n_c - n_frozen, s.n_v)
    assert np.abs(fa - so.fock_a).max() < 1e-13 and np.abs(fb - so.fock_b).max() < 1e-13
    assert abs(info.e_ref - eref) < 1e-12
    # <Phi_A|H|Phi_A> from CI vectors (all electrons, core energy 1.25)
    b = brute.Brute(s)
    fr, _ = twod.frames(s, 0)
    x0 = b.space.vec(twod.frame_det(fr))
    assert abs(info.e_ref - (1.25 + x0 @ b.H @ x0)) < 1e-12
    # the library's Fock matrices (all electrons) equal the textbook ones
    if n_frozen == 0:
        fa0, fb0, _ = fock_from_h(s.h, s.B, s.n_c)
        assert np.abs(fa - fa0).max() < 1e-13 and np.abs(fb - fb0).max() < 1e-13
    rec = np.einsum("Lpq,Lrs->pqrs", B, B)
    c = slice(n_frozen, s.n)
    assert np.abs(rec - eri[c, c, c, c]).max() <= info.chol_max_error + 1e-15


@pytest.mark.parametrize("ref,method", [(0, 0), (1, 1)])
def test_oracle_four_index_path_equals_factor_path(pin, ref, method):
    s, path, eri = pin
    fa, fb, _ = fock_from_h(s.h, s.B, s.n_c)
    s.fock_a, s.fock_b = fa, fb
    T = random_amplitudes(s, seed=5, ref=ref, scale1=0.05, scale2=0.05)
    R1, W1, E1 = twod.residual(s, ref, method, T)
    so, _ = ofcidump.system(path)
    R2, W2, E2 = twod.residual(so, ref, method, T)
    assert max(np.abs(a - b).max() for a, b in zip(R1, R2)) < 1e-14
    assert abs(W1 - W2) < 1e-14 and abs(E1 - E2) < 1e-14


@pytest.mark.parametrize("method", [0, 1])
def test_frozen_core_residual_equals_all_electron(pin, method):
    """The frozen-core Hamiltonian reproduces the all-electron residual of
    the correlated amplitudes when the frozen orbitals' amplitudes vanish."""
    s, path, eri = pin
    s_all, _ = ofcidump.system(path, n_frozen=0)
    s_fc, _ = ofcidump.system(path, n_frozen=1)
    Tfc = random_amplitudes(s_fc, seed=9, scale1=0.05, scale2=0.05, z2=False)
    o_fc, o_all = s_fc.o, s_all.o
    # embed: frozen orbital = occupied index 0 of each spin in the all-electron layout
    Tall = [np.zeros((o_all, s_all.v)), np.zeros((o_all, s_all.v))] + [np.zeros((o_all, o_all, s_all.v, s_all.v))
                                                                       for _ in range(3)]
    Tall[0][1:], Tall[1][1:] = Tfc[0], Tfc[1]
    for k in (2, 3, 4):
        Tall[k][1:, 1:] = Tfc[k]
    R_all, W_all, E_all = twod.residual(s_all, 0, method, tuple(Tall))
    R_fc, W_fc, E_fc = twod.residual(s_fc, 0, method, Tfc)
    assert abs(W_all - W_fc) < 1e-13 and abs(E_all - E_fc) < 1e-13
    assert np.abs(R_all[0][1:] - R_fc[0]).max() < 1e-13
    for k in (2, 3, 4):
        assert np.abs(R_all[k][1:, 1:] - R_fc[k]).max() < 1e-13
    assert max(np.abs(x).max() for x in R_fc) > 1e-3
