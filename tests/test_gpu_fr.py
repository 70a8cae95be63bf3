"""Fixed-reference FR-CCSD / FR-DCSD on the GPU (methods 2..5 of the C ABI)
against the FR oracle (oracle/fr.py, pinned in tests/test_fr_oracle.py).

Residuals at random amplitudes, both frames, both fixed values: FP64 to
1e-9 in max |R| and 1e-10 in the energy and the fixed element's residual;
tensor-core precisions within the tolerances of the 2D parity tests.
Converged energies of the smallest named workload (4 core + 2 open, 20
virtuals, naux 60) against tests/golden/c1_energies.json (written by
tests/golden/make_golden.py from the oracle) to 1e-10 Eh.
"""
import json
import os

import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import fr as ofr

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_R, TOL_E = 1e-9, 1e-10
SIGN = {2: 1.0, 3: 1.0, 4: -1.0, 5: -1.0}
BASE = {2: 0, 3: 1, 4: 0, 5: 1}   # CCSD / DCSD term set


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


@pytest.mark.parametrize("dims,seed", [((0, 3, 7), 1), ((2, 5, 12), 3), ((6, 13, 40), 5)])
@pytest.mark.parametrize("ref", [0, 1])
@pytest.mark.parametrize("method", [2, 3, 4, 5])
def test_fr_residual_fp64_matches_oracle(P, dims, seed, ref, method):
    s = make_system(dims, seed=seed)
    T = random_amplitudes(s, seed=seed + 100, ref=ref, scale1=0.03, scale2=0.03)
    eng = P.Engine.from_system(s)
    R, Rq, dE = eng.residual(eng.to_device(T), ref=ref, method=method)
    R = [x.cpu().numpy() for x in R]
    Ro, Rqo, dEo = ofr.residual(s, ref, BASE[method], T, SIGN[method])
    assert max(float(np.abs(r - ro).max()) for r, ro in zip(R, Ro)) < TOL_R
    assert abs(Rq - Rqo) < TOL_E and abs(dE - dEo) < TOL_E
    eng.close()


@pytest.mark.parametrize("prec,rtol", [(1, 2e-2), (4, 2e-5)])
@pytest.mark.parametrize("method", [3, 4])
def test_fr_residual_tensor_core_within_precision(P, prec, rtol, method):
    s = make_system((6, 40, 64), seed=5)
    T = random_amplitudes(s, seed=105, scale1=0.02, scale2=0.02)
    eng = P.Engine.from_system(s)
    R, Rq, dE = eng.residual(eng.to_device(T), method=method, precision=prec)
    R = [x.cpu().numpy() for x in R]
    Ro, Rqo, dEo = ofr.residual(s, 0, BASE[method], T, SIGN[method])
    rmax = max(np.abs(x).max() for x in Ro)
    assert max(float(np.abs(r - ro).max()) for r, ro in zip(R, Ro)) < rtol * rmax
    assert abs(dE - dEo) < 1e-12
    eng.close()


@pytest.mark.parametrize("method,key", [(2, "FR-CCSD S"), (3, "FR-DCSD S"), (4, "FR-CCSD T"), (5, "FR-DCSD T")])
@pytest.mark.parametrize("ref", [0, 1])
def test_fr_solve_c1_matches_oracle(P, method, key, ref):
    gold = json.load(open(os.path.join(HERE, "golden", "c1_energies.json")))["results"][key]
    s = make_system("c1")
    eng = P.Engine.from_system(s)
    T, res = eng.solve(method=method, ref=ref, tol=1e-10, maxiter=100)
    assert res.converged
    assert abs(res.dEA - gold["E"]) < TOL_E
    E_state = res.E_S if SIGN[method] > 0 else res.E_T
    other = res.E_T if SIGN[method] > 0 else res.E_S
    assert abs(E_state - gold["E"]) < TOL_E and np.isnan(other)
    # the fixed amplitude is returned, and the oracle residual vanishes
    Tn = [x.cpu().numpy() for x in T]
    assert Tn[4][s.o - 1, s.o - 1, 0, 0] == SIGN[method]
    Ro, _, _ = ofr.residual(s, ref, BASE[method], tuple(Tn), SIGN[method])
    assert max(np.abs(x).max() for x in Ro) < 1e-9
    eng.close()


def test_fr_methods_refused_by_reverse_mode(P):
    s = make_system((1, 2, 4), seed=1)
    eng = P.Engine.from_system(s)
    with pytest.raises(P.DcsdError) as e:
        eng.vjp(eng.zeros(), method=3)
    assert e.value.status == 1
    eng.close()
