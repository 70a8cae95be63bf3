"""Pins of the oracle's derivative machinery (oracle/vjp.py), the reference
for the reverse mode of the residual.

  * along amplitude directions, the derivative of dE_A equals the closed
    form obtained by differentiating the energy of Eq. 2 term by term;
  * the residual is linear in the Fock matrix, so the stencil derivative
    along a Fock direction equals the plain difference phi(f+df) - phi(f);
  * the stencil has converged (steps h and h/2 agree);
  * the per-element gradient and the directional derivative agree.
"""
import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import twod
from oracle import vjp as ovjp
from oracle.spinorb import unpack


def _antisym_dir(rng, T):
    # the A->B element is not a free amplitude (the C-condition fixes it)
    d = [rng.normal(0, 1, t.shape) for t in T]
    d[2], d[3] = ovjp.antisym(d[2]), ovjp.antisym(d[3])
    o = d[0].shape[0]
    d[4][o - 1, o - 1, 0, 0] = 0.0
    return d


def _sym(x):
    return 0.5 * (x + np.swapaxes(x, -1, -2))


@pytest.mark.parametrize("ref", [0, 1])
def test_energy_derivative_closed_form(ref):
    s = make_system((1, 3, 8), seed=11)
    T = random_amplitudes(s, seed=5, ref=ref, scale1=0.05, scale2=0.05)
    rng = np.random.default_rng(3)
    dT = _antisym_dir(rng, T)
    got = ovjp.directional(s, ref, 1, T, None, Ebar=1.0, dT=dT)
    fr, _ = twod.frames(s, ref)
    t1, _ = unpack(fr.o, fr.v, T)
    d1, d2 = unpack(fr.o, fr.v, dT)
    g = fr.g("oovv")
    want = (np.einsum("ia,ia->", fr.f("ov"), d1) + 0.25 * np.einsum("ijab,ijab->", g, d2)
            + 0.5 * (np.einsum("ijab,ia,jb->", g, d1, t1) + np.einsum("ijab,ia,jb->", g, t1, d1)))
    assert abs(got - want) < 1e-10 * max(1.0, abs(want))
    assert abs(want) > 1e-3


@pytest.mark.parametrize("method", [0, 1])
def test_fock_direction_is_linear(method):
    s = make_system((1, 3, 8), seed=12)
    T = random_amplitudes(s, seed=6, scale1=0.05, scale2=0.05)
    rng = np.random.default_rng(4)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    dfa, dfb = _sym(rng.normal(0, 1e-2, s.fock_a.shape)), _sym(rng.normal(0, 1e-2, s.fock_b.shape))
    got = ovjp.directional(s, 0, method, T, Rb, 0.3, -0.7, dfa=dfa, dfb=dfb)
    import dataclasses
    sp = dataclasses.replace(s, fock_a=s.fock_a + dfa, fock_b=s.fock_b + dfb)
    want = (ovjp.objective(sp, 0, method, T, Rb, 0.3, -0.7) - ovjp.objective(s, 0, method, T, Rb, 0.3, -0.7))
    assert abs(got - want) < 1e-10 * max(1.0, abs(want))


def test_stencil_converged():
    s = make_system((1, 2, 6), seed=13)
    T = random_amplitudes(s, seed=7, scale1=0.05, scale2=0.05)
    rng = np.random.default_rng(5)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    dT = _antisym_dir(rng, T)
    a = ovjp.directional(s, 0, 1, T, Rb, 0.5, 0.25, dT=dT, h=1e-3)
    b = ovjp.directional(s, 0, 1, T, Rb, 0.5, 0.25, dT=dT, h=5e-4)
    assert abs(a - b) < 1e-9 * max(1.0, abs(a))


def test_gradient_matches_directional():
    s = make_system((0, 2, 5), seed=14)
    T = random_amplitudes(s, seed=8, scale1=0.05, scale2=0.05)
    rng = np.random.default_rng(6)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    G = ovjp.gradient_T(s, 1, 1, T, Rb, 0.2, 0.4)
    dT = [rng.normal(0, 1, t.shape) for t in T]
    lhs = sum(float((g * d).sum()) for g, d in zip(G, dT))
    rhs = ovjp.directional(s, 1, 1, T, Rb, 0.2, 0.4, dT=dT)
    assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(rhs))
