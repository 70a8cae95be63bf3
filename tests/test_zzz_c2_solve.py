"""FP64 solve of the 10+2 occupied/open, 120 virtual, naux 360 workload on
the GPU against the oracle.  The full oracle takes minutes per residual at
this size, so instead of an independent oracle solve the element-wise oracle
(oracle/element.py, pinned element by element against the full oracle) is
evaluated at the GPU's converged amplitudes:
  * its Delta E_A and W (Eq. 2 and the A->B residual element), hence the
    singlet and triplet energies Delta E_A +- W, equal the GPU's to 1e-10 Eh;
  * its residual (Eqs. 3-4) vanishes at sampled, symmetry-allowed elements
    of every block (below 1e-9): the GPU converged to a solution of the
    oracle's equations.
Collected after the other GPU tests."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import element
from synth import make_system

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _positions():
    spec = importlib.util.spec_from_file_location("make_elements", os.path.join(HERE, "golden", "make_elements.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.positions


def check_against_element_oracle(s, method, T, dEA, W, tol_e=1e-10, tol_r=1e-9, per_block=3):
    """Oracle energies and sampled residual elements at amplitudes T (frame A)."""
    eo = element.ElementOracle(s, 0, method, T)
    assert abs(eo.energy() - dEA) < tol_e
    assert abs(eo.W() - W) < tol_e
    worst = 0.0
    for blk, idx, _ in _positions()(s, per_block, np.random.default_rng(5)):
        worst = max(worst, abs(element.residual_element(eo, blk, idx)))
    assert worst < tol_r, worst
    return worst


@pytest.mark.parametrize("method", [0, 1])
def test_c2_fp64_solve_matches_oracle(method):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    s = make_system("c2")
    eng = P.Engine.from_system(s)
    T, res = eng.solve(method=method, ref=0, precision=P.PREC_FP64, tol=1e-10, maxiter=150)
    Tn = tuple(x.cpu().numpy() for x in T)
    eng.close()
    assert res.converged and res.max_r < 1e-10
    assert abs(res.E_S - (res.dEA + res.W)) < 1e-12 and abs(res.E_T - (res.dEA - res.W)) < 1e-12
    check_against_element_oracle(s, method, Tn, res.dEA, res.W)


def test_c2_fp64_solve_matches_golden_oracle_solve():
    """The converged 2D-DCSD energies against an independent oracle solve of the
    same workload (tests/golden/c2_energies.json, written by
    tests/golden/make_golden.py: the full FP64 oracle with DIIS to max|R| <
    1e-10): singlet and triplet energies, Delta E_A and W to 1e-10 Eh."""
    import json
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    with open(os.path.join(HERE, "golden", "c2_energies.json")) as f:
        gold = json.load(f)
    assert gold["workload"] == "c2"
    ref = gold["results"]["2D-DCSD"]
    s = make_system("c2")
    eng = P.Engine.from_system(s)
    T, res = eng.solve(method=P.DCSD, ref=0, precision=P.PREC_FP64, tol=1e-11, maxiter=200)
    eng.close()
    assert res.converged
    for key in ("dEA", "W", "E_S", "E_T"):
        print(key, getattr(res, key) - ref[key])
        assert abs(getattr(res, key) - ref[key]) < 1e-10, key
