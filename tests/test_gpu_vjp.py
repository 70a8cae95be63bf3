"""Reverse mode of the FP64 residual (dcsd_vjp, through the C ABI) against
the oracle's derivatives and against finite differences of the GPU residual.

Gradients are compared along symmetry-respecting directions: same-spin
doubles antisymmetric, B and the Fock matrices symmetric (oracle/vjp.py
explains why only those are implementation-independent).
"""
import dataclasses

import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import vjp as ovjp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    return P


def _sym(x):
    return 0.5 * (x + np.swapaxes(x, -1, -2))


def _gpu_vjp(P, eng, T, Rb, Eb, Wb, ref, method, want_B=False, want_fock=False):
    import torch
    Td = eng.to_device(T)
    Rd = eng.to_device(Rb)
    Tb, Bb, Fa, Fb = eng.vjp(Td, Rbar=Rd, Ebar=Eb, Wbar=Wb, ref=ref, method=method, want_B=want_B,
                             want_fock=want_fock)
    torch.cuda.synchronize()
    cpu = lambda x: None if x is None else x.cpu().numpy()  # noqa: E731
    return tuple(cpu(x) for x in Tb), cpu(Bb), cpu(Fa), cpu(Fb)


@pytest.mark.parametrize("dims,seed", [((0, 2, 5), 1), ((1, 2, 6), 2)])
@pytest.mark.parametrize("ref", [0, 1])
@pytest.mark.parametrize("method", [0, 1])
def test_vjp_gradient_matches_oracle(P, dims, seed, ref, method):
    s = make_system(dims, seed=seed)
    T = random_amplitudes(s, seed=seed + 20, ref=ref, scale1=0.05, scale2=0.05)
    rng = np.random.default_rng(seed)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    Eb, Wb = 0.3, -0.8
    eng = P.Engine.from_system(s)
    G, _, _, _ = _gpu_vjp(P, eng, T, Rb, Eb, Wb, ref, method)
    eng.close()
    Go = ovjp.gradient_T(s, ref, method, T, Rb, Eb, Wb)
    scale = max(float(np.abs(g).max()) for g in Go)
    for g, go in zip(ovjp.project(G), ovjp.project(Go)):
        assert np.abs(g - go).max() < 1e-8 * scale
    assert scale > 1e-2


@pytest.mark.parametrize("dims,seed", [((2, 5, 12), 3), ((4, 20, 30), 4)])
@pytest.mark.parametrize("method", [0, 1])
def test_vjp_directions_match_oracle(P, dims, seed, method):
    s = make_system(dims, seed=seed)
    ref = seed % 2
    T = random_amplitudes(s, seed=seed + 30, ref=ref, scale1=0.02, scale2=0.02)
    rng = np.random.default_rng(seed + 1)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    Eb, Wb = -0.4, 1.1
    eng = P.Engine.from_system(s)
    G, Bb, Fa, Fb = _gpu_vjp(P, eng, T, Rb, Eb, Wb, ref, method, want_B=True, want_fock=True)
    eng.close()
    dT = [rng.normal(0, 1, t.shape) for t in T]
    dT[2], dT[3] = ovjp.antisym(dT[2]), ovjp.antisym(dT[3])
    dB = _sym(rng.normal(0, 1e-2, s.B.shape))
    dfa, dfb = _sym(rng.normal(0, 1e-2, s.fock_a.shape)), _sym(rng.normal(0, 1e-2, s.fock_b.shape))
    for kind in ("T", "B", "f"):
        if kind == "T":
            gpu = sum(float((g * d).sum()) for g, d in zip(G, dT))
            ora = ovjp.directional(s, ref, method, T, Rb, Eb, Wb, dT=dT)
        elif kind == "B":
            gpu = float((Bb * dB).sum())
            ora = ovjp.directional(s, ref, method, T, Rb, Eb, Wb, dB=dB)
        else:
            gpu = float((Fa * dfa).sum() + (Fb * dfb).sum())
            ora = ovjp.directional(s, ref, method, T, Rb, Eb, Wb, dfa=dfa, dfb=dfb)
        assert abs(gpu - ora) < 1e-8 * max(1.0, abs(ora)), (kind, gpu, ora)


def test_vjp_matches_gpu_finite_differences(P):
    import torch
    s = make_system((6, 40, 64), seed=5)
    T = random_amplitudes(s, seed=41, scale1=0.02, scale2=0.02)
    rng = np.random.default_rng(9)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    dT = [rng.normal(0, 1, t.shape) for t in T]
    dT[2], dT[3] = ovjp.antisym(dT[2]), ovjp.antisym(dT[3])
    eng = P.Engine.from_system(s)
    G, _, _, _ = _gpu_vjp(P, eng, T, Rb, 0.5, 0.5, 0, 1)

    def phi(e):
        R, W, dE = eng.residual(eng.to_device([t + e * d for t, d in zip(T, dT)]), method=1)
        torch.cuda.synchronize()
        return sum(float((r.cpu().numpy() * rb).sum()) for r, rb in zip(R, Rb)) + 0.5 * dE + 0.5 * W

    h = 1e-3
    fd = (8 * (phi(h) - phi(-h)) - (phi(2 * h) - phi(-2 * h))) / (12 * h)
    eng.close()
    gpu = sum(float((g * d).sum()) for g, d in zip(G, dT))
    assert abs(gpu - fd) < 1e-8 * max(1.0, abs(fd))


def test_autograd_function_matches_vjp(P):
    import torch
    s = make_system((2, 5, 12), seed=3)
    T = random_amplitudes(s, seed=51, scale1=0.02, scale2=0.02)
    rng = np.random.default_rng(10)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    eng = P.Engine.from_system(s)
    Tt = [x.clone().requires_grad_(True) for x in eng.to_device(T)]
    out = eng.residual_autograd(Tt, ref=0, method=1)
    Rbt = eng.to_device(Rb)
    loss = sum((o * r).sum() for o, r in zip(out[:5], Rbt)) + 0.7 * out[5] - 0.2 * out[6]
    loss.backward()
    G, _, _, _ = _gpu_vjp(P, eng, T, Rb, -0.2, 0.7, 0, 1)
    eng.close()
    for t, g in zip(Tt, G):
        assert np.abs(t.grad.cpu().numpy() - g).max() < 1e-12 * max(1.0, float(np.abs(g).max()))


def test_vjp_c4_matches_gpu_finite_differences(P):
    """The adjoint workload (12 core + 2 open, 160 virtuals, naux 480), FP64:
    <T_bar, dT> and <B_bar, dB> against central differences of the GPU
    residual (fourth-order stencil, step 1e-5 along unit-scale directions)."""
    import torch
    s = make_system("c4")
    T = random_amplitudes(s, seed=61, scale1=0.02, scale2=0.02)
    rng = np.random.default_rng(12)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    dT = [rng.normal(0, 1, t.shape) for t in T]
    dT[2], dT[3] = ovjp.antisym(dT[2]), ovjp.antisym(dT[3])
    dB = _sym(rng.normal(0, 1, s.B.shape))
    eng = P.Engine.from_system(s)
    G, Bb, _, _ = _gpu_vjp(P, eng, T, Rb, 0.3, -0.6, 0, 1, want_B=True)
    eng.close()

    def phi(eT, eB):
        sp = dataclasses.replace(s, B=s.B + eB * dB)
        e2 = P.Engine.from_system(sp)
        R, W, dE = e2.residual(e2.to_device([t + eT * d for t, d in zip(T, dT)]), method=1)
        torch.cuda.synchronize()
        v = sum(float((r.cpu().numpy() * rb).sum()) for r, rb in zip(R, Rb)) + 0.3 * dE - 0.6 * W
        e2.close()
        return v

    h = 1e-5
    for kind, gpu in (("T", sum(float((g * d).sum()) for g, d in zip(G, dT))), ("B", float((Bb * dB).sum()))):
        f = (lambda e: phi(e, 0.0)) if kind == "T" else (lambda e: phi(0.0, e))
        fd = (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)
        assert abs(gpu - fd) < 1e-6 * max(1.0, abs(fd)), (kind, gpu, fd)


@pytest.mark.parametrize("prec,rtol", [(4, 2e-4), (2, 2e-3), (1, 5e-2)])
def test_tensor_core_vjp_matches_fp64(P, prec, rtol):
    """Reverse mode with the ladder and G-pass contractions of both sweeps on
    the tensor cores (BF16X6, BF16X3, BF16) against the FP64 reverse mode:
    projected amplitude gradients and B_bar within rtol of their largest
    element (the tensor-core products carry the operand-split error of the
    forward residual, about 1e-5 relative for BF16X6)."""
    s = make_system((6, 60, 120), seed=7)
    T = random_amplitudes(s, seed=71, scale1=0.02, scale2=0.02)
    rng = np.random.default_rng(13)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    eng = P.Engine.from_system(s)
    import torch
    Td, Rd = eng.to_device(T), eng.to_device(Rb)
    out = {}
    for pr in (0, prec):
        Tb, Bb, Fa, _ = eng.vjp(Td, Rbar=Rd, Ebar=0.4, Wbar=-0.7, ref=0, method=1, want_B=True, want_fock=True,
                                precision=pr)
        torch.cuda.synchronize()
        out[pr] = ([x.cpu().numpy() for x in Tb], _sym(Bb.cpu().numpy()), _sym(Fa.cpu().numpy()))
    eng.close()
    G64, B64, F64 = out[0]
    G, Bt, Ft = out[prec]
    scale = max(float(np.abs(g).max()) for g in ovjp.project(G64))
    for g, g64 in zip(ovjp.project(G), ovjp.project(G64)):
        assert np.abs(g - g64).max() <= rtol * scale
    assert np.abs(Bt - B64).max() <= rtol * float(np.abs(B64).max())
    assert np.abs(Ft - F64).max() <= rtol * float(np.abs(F64).max())
    assert scale > 1e-2
