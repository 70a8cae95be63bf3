"""Singlet-triplet gaps from one or two calculations (stgap.gaps, the
comparison of Table 4) on the GPU against the oracle's converged total
energies of the same FCIDUMP files (tests/test_stgap_oracle.py builds and
pins them): total energies to 1e-9 Eh; for two electrons the one-run and
two-run gaps agree (2D-CCSD is exact there)."""
import pytest

from tests.test_stgap_oracle import orbital_sets, totals, write_sets
from oracle import twod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


@pytest.mark.parametrize("nc,nv,X,seed,scale,method", [(0, 4, 10, 21, 0.1, 0), (2, 5, 12, 22, 0.05, 1)])
def test_gaps_match_oracle(P, tmp_path, nc, nv, X, seed, scale, method):
    from paper_2401_11935_gb300 import stgap
    s, sets = orbital_sets(nc, nv, X, seed, scale)
    paths = write_sets(tmp_path, s, sets)
    g = stgap.gaps(paths[0], singlet=paths[1], triplet=paths[2], method=method, tol=1e-10)
    E0 = totals(paths[0], method)
    E1 = totals(paths[1], method)
    E2 = totals(paths[2], method)
    assert abs(g["single"]["E_S"] - E0[0]) < 1e-9 and abs(g["single"]["E_T"] - E0[1]) < 1e-9
    assert abs(g["state_specific"]["E_S"] - E1[0]) < 1e-9 and abs(g["state_specific"]["E_T"] - E2[1]) < 1e-9
    assert abs(g["single"]["gap"] - 2 * g["single"]["W"]) < 1e-12
    if nc == 0:
        assert abs(g["single"]["gap"] - g["state_specific"]["gap"]) < 1e-9
