"""The library's two-determinant term tables (derived on the host by
excitation algebra on occupation strings, and used by the device kernels of
the M.W terms, Section II, Eqs. 3-4) evaluated on the host through the C ABI
(dcsd_coupling_host) against the oracle's coupling coefficients
c_q = <Phi_q| exp(T_other) |Phi_other>, which the brute-force CI pins fix.
No GPU needed."""
import numpy as np
import pytest

from oracle import twod
from oracle.spinorb import flip_abi, pack, unpack
from synth import make_system, random_amplitudes


def _oracle_c(s, ref, T):
    fr, fro = twod.frames(s, ref)
    t1o, t2o = unpack(fr.o, fr.v, flip_abi(T))
    c1, c2 = twod.c_other(fr, fro, t1o, t2o)
    return pack(fr.o, fr.v, c1, c2)


@pytest.mark.parametrize("dims,seed", [((0, 2, 4), 1), ((1, 2, 6), 2), ((2, 3, 8), 3), ((3, 2, 8), 4)])
@pytest.mark.parametrize("ref", [0, 1])
def test_host_tables_match_oracle_coefficients(dims, seed, ref):
    from paper_2401_11935_gb300 import _lib
    s = make_system(dims, seed=seed)
    # large amplitudes, so that every product order of the cluster-to-CI
    # expansion contributes well above rounding
    T = random_amplitudes(s, seed=seed + 40, ref=ref, scale1=0.3, scale2=0.3)
    got = _lib.dcsd_coupling_host(ref, s.n_c, s.n_v, T)
    want = _oracle_c(s, ref, T)
    o = s.n_c + 1
    for k, (g, w) in enumerate(zip(got, want)):
        w = np.array(w)
        if k == 4:
            w[o - 1, o - 1, 0, 0] = 0.0  # the A->B element (its coefficient is 1; not used)
        if k in (2, 3):  # same-spin diagonals carry no determinant
            for i in range(o):
                w[i, i] = 0.0
            for a in range(w.shape[2]):
                w[:, :, a, a] = 0.0
        scale = max(1.0, float(np.abs(w).max()))
        assert np.abs(g - w).max() < 1e-13 * scale, (k, float(np.abs(g - w).max()))
    assert max(float(np.abs(x).max()) for x in want) > 1e-2


def test_host_tables_reject_bad_arguments():
    from paper_2401_11935_gb300 import _lib
    T = [np.zeros((1, 2)), np.zeros((1, 2)), np.zeros((1, 1, 2, 2)), np.zeros((1, 1, 2, 2)),
         np.zeros((1, 1, 2, 2))]
    with pytest.raises(_lib.DcsdError):
        _lib.dcsd_coupling_host(2, 0, 1, T)
