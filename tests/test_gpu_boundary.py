"""The C ABI's contracts beyond parity (GPU; every call goes through the ABI):

* failure paths in the forms that fault nothing: a NaN in the amplitudes
  gives DCSD_ERR_NUMERIC; a solve that reaches maxiter gives
  DCSD_ERR_NOT_CONVERGED with the amplitudes of the last update returned;
* memory: after dcsd_reserve, residuals and solves of the reserved
  precision allocate no device memory (cudaMemGetInfo unchanged), while
  without a reservation the first tensor-core residual does allocate;
* the torch.autograd.Function returns the DF-factor and Fock-matrix
  gradients of dcsd_vjp, checked against the oracle's derivatives.
"""
import ctypes

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


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_amplitude_gives_numeric_status(P, prec):
    s = make_system((2, 5, 12), seed=3)
    T = [np.array(x) for x in random_amplitudes(s, seed=4)]
    T[4][0, 0, 1, 2] = np.nan
    eng = P.Engine.from_system(s)
    with pytest.raises(P.DcsdError) as e:
        eng.residual(eng.to_device(T), precision=prec)
    assert e.value.status == 6
    with pytest.raises(P.DcsdError) as e:
        eng.residual_host(T)
    assert e.value.status == 6
    # the context stays usable
    R, W, dE = eng.residual(eng.to_device(random_amplitudes(s, seed=4)))
    assert np.isfinite(W) and np.isfinite(dE)
    eng.close()


def _raw_solve(P, eng, T, maxiter, use_guess, diis_n=0):
    from paper_2401_11935_gb300 import _lib as L
    opts = L.dcsd_solve_opts(1, 0, 0, maxiter, diis_n, 1e-12, 1e-5, use_guess, 0.0)
    res = L.dcsd_result()
    st = L.load().dcsd_solve(eng.ctx, ctypes.byref(opts), L.MEM_DEVICE, *[x.data_ptr() for x in T],
                             ctypes.byref(res))
    return st, res


def test_maxiter_gives_not_converged_with_last_iterate(P):
    import torch
    s = make_system((2, 5, 12), seed=3)
    eng = P.Engine.from_system(s)
    T2 = eng.zeros()
    st, res = _raw_solve(P, eng, T2, 2, 0)
    assert st == 4 and res.iters == 2 and res.converged == 0
    # two Jacobi updates then one more from there equal three updates
    st1, _ = _raw_solve(P, eng, T2, 1, 1)
    T3 = eng.zeros()
    st3, _ = _raw_solve(P, eng, T3, 3, 0)
    torch.cuda.synchronize()
    assert st1 == 4 and st3 == 4
    nz = max(float(x.abs().max()) for x in T3)
    assert nz > 1e-4
    for a, b in zip(T2, T3):
        assert float((a - b).abs().max()) <= 1e-14 * nz
    eng.close()


def _pointers(eng):
    import torch
    T = tuple(torch.zeros(s, dtype=torch.float64, device="cuda") for s in eng.shapes())
    R = tuple(torch.empty_like(x) for x in T)
    return T, R


def _bf16_work(P, eng, T, R):
    """One BF16 residual and a three-iteration BF16 solve with DIIS, through
    the raw ABI (no torch allocation in between)."""
    from paper_2401_11935_gb300 import _lib as L
    L.dcsd_residual(eng.ctx, 0, 1, 1, L.MEM_DEVICE, [x.data_ptr() for x in T], [x.data_ptr() for x in R])
    opts = L.dcsd_solve_opts(1, 0, 1, 3, 8, 1e-12, 1e-5, 0, 0.0)
    L.dcsd_solve(eng.ctx, opts, L.MEM_DEVICE, [x.data_ptr() for x in T])


def test_reserve_then_no_device_allocation(P):
    import torch
    s = make_system((6, 40, 64), seed=5)
    # without a reservation the first tensor-core residual allocates (this
    # run also loads every kernel of the path, so that module loading does
    # not show up in the measurement below)
    e0 = P.Engine.from_system(s)
    T, R = _pointers(e0)
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    _bf16_work(P, e0, T, R)
    torch.cuda.synchronize()
    f1 = torch.cuda.mem_get_info()[0]
    assert f1 < f0
    e0.close()
    del T, R
    # with a reservation nothing is allocated by residuals and solves
    e1 = P.Engine.from_system(s)
    e1.reserve(P.PREC_BF16, diis_n=8)
    T, R = _pointers(e1)
    torch.cuda.synchronize()
    g0 = torch.cuda.mem_get_info()[0]
    _bf16_work(P, e1, T, R)
    _bf16_work(P, e1, T, R)
    torch.cuda.synchronize()
    g1 = torch.cuda.mem_get_info()[0]
    assert g1 == g0, (g0, g1)
    e1.close()


def test_reserve_rejects_bad_arguments(P):
    s = make_system((1, 2, 4), seed=1)
    eng = P.Engine.from_system(s)
    from paper_2401_11935_gb300 import _lib as L
    for args in ((9, 8, 0), (0, 17, 0), (0, 8, 2), (0, -1, 0)):
        with pytest.raises(P.DcsdError) as e:
            L.dcsd_reserve(eng.ctx, *args)
        assert e.value.status == 1
    eng.close()


@pytest.mark.parametrize("method", [0, 1])
def test_autograd_gives_B_and_fock_gradients(P, method):
    import torch
    s = make_system((2, 5, 12), seed=3)
    T = random_amplitudes(s, seed=52, ref=1, scale1=0.03, scale2=0.03)
    rng = np.random.default_rng(14)
    Rb = [rng.normal(0, 1, t.shape) for t in T]
    eng = P.Engine.from_system(s)
    Tt = [x.clone().requires_grad_(True) for x in eng.to_device(T)]
    fa, fb, Bt = eng.inputs()
    out = eng.residual_autograd(Tt, ref=1, method=method, inputs=(fa, fb, Bt))
    Rbt = eng.to_device(Rb)
    loss = sum((o * r).sum() for o, r in zip(out[:5], Rbt)) - 0.4 * out[5] + 0.9 * out[6]
    loss.backward()
    torch.cuda.synchronize()
    dB = _sym(rng.normal(0, 1e-2, s.B.shape))
    dfa, dfb = _sym(rng.normal(0, 1e-2, s.fock_a.shape)), _sym(rng.normal(0, 1e-2, s.fock_b.shape))
    gB = float((Bt.grad.cpu().numpy() * dB).sum())
    gf = float((fa.grad.cpu().numpy() * dfa).sum() + (fb.grad.cpu().numpy() * dfb).sum())
    oB = ovjp.directional(s, 1, method, T, Rb, 0.9, -0.4, dB=dB)
    of = ovjp.directional(s, 1, method, T, Rb, 0.9, -0.4, dfa=dfa, dfb=dfb)
    assert abs(gB - oB) < 1e-8 * max(1.0, abs(oB)), (gB, oB)
    assert abs(gf - of) < 1e-8 * max(1.0, abs(of)), (gf, of)
    with pytest.raises(ValueError):
        eng.residual_autograd(Tt, inputs=(fa.detach().clone(), fb, Bt))
    eng.close()
