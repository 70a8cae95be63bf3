"""Lambda equations and the response density (dcsd_lambda, through the C ABI).

By stationarity of the Lagrangian L = E + Lambda.R at converged T and Lambda,
the derivative of the converged state energy E = dE_A +- W with respect to a
Fock-matrix perturbation equals <gamma, df> with gamma = dL/df.  The test
re-converges the amplitudes at f + e df for several e and compares the
finite-difference derivative with <gamma, df>.  (The GPU FP64 solve itself
matches the oracle to 1e-10 Eh: test_gpu_parity.)
"""
import dataclasses

import numpy as np
import pytest

from synth import make_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


def _energy(P, s, method, state):
    eng = P.Engine.from_system(s)
    T, res = eng.solve(method=method, tol=1e-11, maxiter=200)
    eng.close()
    assert res.converged
    return res.dEA + state * res.W


@pytest.mark.parametrize("method,state", [(1, 1), (1, -1), (0, 1)])
def test_density_is_energy_derivative(P, method, state):
    s = make_system("c1")
    eng = P.Engine.from_system(s)
    T, res = eng.solve(method=method, tol=1e-11, maxiter=200)
    assert res.converged
    Lam, ga, gb, lres = eng.lambda_solve(T, state=state, method=method, tol=1e-10, maxiter=200)
    eng.close()
    assert lres.converged and lres.max_r <= 1e-10
    ga, gb = ga.cpu().numpy(), gb.cpu().numpy()
    # a uniform shift of all orbital energies leaves the correlation energy
    # unchanged (f enters the residual through commutators), so tr(gamma) = 0
    assert abs(np.trace(ga) + np.trace(gb)) < 1e-9
    rng = np.random.default_rng(17 + method + state)
    mask = (s.parity[:, None] == s.parity[None, :]).astype(float)
    def sym(x):
        return 0.5 * (x + x.T) * mask
    dfa, dfb = sym(rng.normal(0, 1e-2, ga.shape)), sym(rng.normal(0, 1e-2, gb.shape))
    pred = float((ga * dfa).sum() + (gb * dfb).sum())

    def E(e):
        sp = dataclasses.replace(s, fock_a=s.fock_a + e * dfa, fock_b=s.fock_b + e * dfb)
        return _energy(P, sp, method, state)

    h = 0.05
    fd = (8 * (E(h) - E(-h)) - (E(2 * h) - E(-2 * h))) / (12 * h)
    assert abs(pred - fd) < 1e-7 * max(1.0, abs(fd)) + 1e-9, (pred, fd)
    assert abs(fd) > 1e-5  # the check is not vacuous
