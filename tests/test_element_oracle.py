"""Pins of the element-wise oracle (oracle/element.py), which evaluates
single residual elements of Eqs. 3-4 for systems of any size through the DF
factors: every element, and W, must equal the full oracle (twod.residual,
itself pinned by two-electron FCI, brute-force CI and the invariances) on
small systems, for both references, CCSD and DCSD, CAS and non-CAS
amplitudes."""
import numpy as np
import pytest

from oracle import element, twod
from synth import make_system, random_amplitudes


@pytest.mark.parametrize("dims,seed,ref,method,z2", [
    ((0, 2, 6), 1, 0, 0, True),
    ((1, 3, 8), 2, 1, 1, True),
    ((2, 4, 12), 3, 0, 1, True),
    ((2, 3, 10), 4, 1, 0, True),
    ((3, 3, 10), 5, 0, 1, False),
    ((2, 4, 12), 6, 1, 1, False),
])
def test_every_element_matches_full_oracle(dims, seed, ref, method, z2):
    s = make_system(dims, seed=seed)
    T = random_amplitudes(s, seed=seed + 50, ref=ref, scale1=0.08, scale2=0.08, z2=z2)
    R, W, dE = twod.residual(s, ref, method, T)
    eo = element.ElementOracle(s, ref, method, T)
    scale = max(float(np.abs(x).max()) for x in R)
    assert abs(eo.W() - W) < 1e-13 * max(1.0, abs(W))
    assert abs(eo.energy() - dE) < 1e-14
    for blk, x in enumerate(R):
        for idx in np.ndindex(x.shape):
            assert abs(element.residual_element(eo, blk, idx) - x[idx]) < 1e-13 * scale, (blk, idx)
    assert scale > 1e-2


def test_amplitude_slices_match_dense_tensor():
    from oracle.spinorb import unpack
    s = make_system((2, 3, 10), seed=7)
    T = random_amplitudes(s, seed=8, ref=0, scale1=0.1, scale2=0.1, z2=False)
    eo = element.ElementOracle(s, 0, 1, T)
    _, t2 = unpack(eo.o, eo.v, twod.c_condition(T))
    rng = np.random.default_rng(1)
    for mask in np.ndindex(2, 2, 2, 2):
        for _ in range(4):
            sel = tuple(slice(None) if m else int(rng.integers(t2.shape[k])) for k, m in enumerate(mask))
            assert np.array_equal(eo.T.t2(*sel), t2[sel])


@pytest.mark.parametrize("ref,method", [(0, 1), (1, 0)])
def test_sampled_elements_match_full_oracle_c1(ref, method):
    """The smallest named workload (4 core + 2 open, 20 virtuals, naux 60):
    sampled elements of every block and W against the full oracle."""
    s = make_system("c1")
    T = random_amplitudes(s, seed=70 + ref, ref=ref, scale1=0.05, scale2=0.05)
    R, W, _ = twod.residual(s, ref, method, T)
    eo = element.ElementOracle(s, ref, method, T)
    scale = max(float(np.abs(x).max()) for x in R)
    assert abs(eo.W() - W) < 1e-13 * max(1.0, abs(W))
    rng = np.random.default_rng(ref)
    for blk, x in enumerate(R):
        for _ in range(8):
            idx = tuple(int(rng.integers(n)) for n in x.shape)
            assert abs(element.residual_element(eo, blk, idx) - x[idx]) < 1e-13 * scale, (blk, idx)
