"""GB300-native two-determinant CCSD / DCSD residual engine (arXiv 2401.11935).

PyTorch supplies device memory and the CUDA stream; every step of the
residual, the energy, the DIIS solve and the effective Hamiltonian runs in
the CUDA kernels of libdcsd.so, reached through the C ABI of
include/dcsd.h (ctypes binding in ``_lib``).
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from ._lib import (CCSD, DCSD, FR_CCSD_S, FR_CCSD_T, FR_DCSD_S, FR_DCSD_T, MEM_DEVICE,  # noqa: F401
                   MEM_HOST, PREC_BF16, PREC_BF16X3, PREC_BF16X6, PREC_FP64, PREC_MIXED, DcsdError, dcsd_heff)

__all__ = ["Engine", "CCSD", "DCSD", "FR_CCSD_S", "FR_DCSD_S", "FR_CCSD_T", "FR_DCSD_T", "PREC_FP64", "PREC_BF16", "PREC_BF16X3", "PREC_BF16X6", "PREC_MIXED",
           "dcsd_heff", "DcsdError"]


def _ptr(x):
    if hasattr(x, "data_ptr"):
        if x.dtype.__str__() != "torch.float64" or not x.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous float64")
        return x.ctypes.data
    raise TypeError(type(x))


class Engine:
    """One context of the C library bound to a torch CUDA stream.

    Inputs (Fock matrices of Phi_A and DF factors) are copied to the device
    once; amplitudes/residuals are torch float64 CUDA tensors (device calls)
    or numpy arrays (host calls, copies inside the library call)."""

    def __init__(self, n_c, n_v, naux, fock_a, fock_b, B, eps=None, stream=None):
        import torch
        self.torch = torch
        self.n_c, self.n_v, self.naux = n_c, n_v, naux
        self.o, self.v = n_c + 1, n_v + 1
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        as_t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).to(dev)  # noqa: E731
        with torch.cuda.stream(self.stream):
            fa, fb, Bt = as_t(fock_a), as_t(fock_b), as_t(B)
            self.stream.synchronize()
            self.ctx = L.dcsd_init(n_c, n_v, naux, None, fa.data_ptr(), fb.data_ptr(), Bt.data_ptr(),
                                   MEM_DEVICE, self.stream.cuda_stream)
        # the library holds its own copy; these tensors are kept only as the
        # differentiable handles of residual_autograd (see inputs())
        self._inputs = (fa, fb, Bt)

    @classmethod
    def from_system(cls, s, **kw):
        return cls(s.n_c, s.n_v, s.naux, s.fock_a, s.fock_b, s.B, **kw)

    @classmethod
    def from_fcidump(cls, path, n_frozen=0, chol_tol=1e-12, stored_ladder=False, stream=None):
        """Context from an FCIDUMP file (dcsd_init_fcidump): frozen-core
        folding, Fock matrices of Phi_A and Cholesky factors are prepared by
        the library; .fcidump holds its dcsd_fcidump_info (dimensions,
        reference energy e_ref for total energies)."""
        import torch
        self = cls.__new__(cls)
        self.torch = torch
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.ctx, info = L.dcsd_init_fcidump(path, n_frozen, chol_tol, stored_ladder, self.stream.cuda_stream)
        self.fcidump = info
        self.n_c, self.n_v, self.naux = info.n_c, info.n_v, info.naux
        self.o, self.v = self.n_c + 1, self.n_v + 1
        self._inputs = None
        return self

    # -- layout helpers --------------------------------------------------
    def shapes(self):
        o, v = self.o, self.v
        return [(o, v), (o, v), (o, o, v, v), (o, o, v, v), (o, o, v, v)]

    def zeros(self):
        t = self.torch
        return tuple(t.zeros(s, dtype=t.float64, device="cuda") for s in self.shapes())

    def to_device(self, T):
        t = self.torch
        return tuple(t.as_tensor(np.ascontiguousarray(x), dtype=t.float64).cuda() for x in T)

    # -- C ABI calls -----------------------------------------------------
    def reserve(self, precision=PREC_FP64, diis_n=8, host_staging=False):
        """Allocate up front the device memory of residuals at `precision`,
        a solve with diis_n DIIS vectors and (optionally) host-memory calls."""
        L.dcsd_reserve(self.ctx, precision, diis_n, 1 if host_staging else 0)

    def residual(self, T, ref=0, method=DCSD, precision=PREC_FP64, out=None):
        """Device call: T are CUDA tensors; returns (R tuple, W, dE_A)."""
        R = out if out is not None else tuple(self.torch.empty_like(x) for x in T)
        W, dE = L.dcsd_residual(self.ctx, ref, method, precision, MEM_DEVICE,
                                [_ptr(x) for x in T], [_ptr(x) for x in R])
        return R, W, dE

    def residual_host(self, T, ref=0, method=DCSD, precision=PREC_FP64):
        """Host call: T are numpy arrays; copies happen inside the library."""
        T = [np.ascontiguousarray(x, dtype=np.float64) for x in T]
        R = [np.empty_like(x) for x in T]
        W, dE = L.dcsd_residual(self.ctx, ref, method, precision, MEM_HOST,
                                [_ptr(x) for x in T], [_ptr(x) for x in R])
        return tuple(R), W, dE

    def energy(self, T, ref=0, method=DCSD):
        return L.dcsd_energy(self.ctx, ref, method, MEM_DEVICE, [_ptr(x) for x in T])

    def solve(self, method=DCSD, ref=0, precision=PREC_FP64, tol=1e-10, maxiter=100, diis_n=8,
              switch_tol=1e-5, T0=None, polish_tol=1e-7):
        """Converge the amplitudes on the device; returns (T, dcsd_result).
        MIXED: BF16 until max|R| < switch_tol, BF16X6 until max|R| <
        polish_tol, then defect correction (FP64 residuals on outer steps,
        BF16X6 inner steps); polish_tol = 0 keeps plain BF16X6."""
        T = tuple(x.clone() for x in T0) if T0 is not None else self.zeros()
        opts = L.dcsd_solve_opts(method, ref, precision, maxiter, diis_n, tol, switch_tol,
                                 1 if T0 is not None else 0, polish_tol)
        res = L.dcsd_solve(self.ctx, opts, MEM_DEVICE, [_ptr(x) for x in T])
        return T, res

    def vjp(self, T, Rbar=None, Ebar=0.0, Wbar=0.0, ref=0, method=DCSD, want_B=False, want_fock=False,
            precision=PREC_FP64):
        """Reverse mode of the residual (device call).  Returns the gradients
        of <Rbar, R(T)> + Ebar * dE_A(T) + Wbar * W(T) with respect to the
        five amplitude arrays, and optionally to the DF factors B [naux, n, n]
        and the two Fock matrices [n, n]: (Tbar, Bbar, fa_bar, fb_bar), absent
        ones None.  precision PREC_FP64 differentiates on the FP64 CUDA cores;
        a tensor-core precision runs the ladder and G-pass contractions of
        both sweeps on the tensor cores with that operand split."""
        t = self.torch
        n = self.n_c + 2 + self.n_v
        Tb = tuple(t.zeros_like(x) for x in T)
        dev = T[0].device
        Bb = t.zeros((self.naux, n, n), dtype=t.float64, device=dev) if want_B else None
        Fa = t.zeros((n, n), dtype=t.float64, device=dev) if want_fock else None
        Fb = t.zeros((n, n), dtype=t.float64, device=dev) if want_fock else None
        L.dcsd_vjp(self.ctx, ref, method, precision, MEM_DEVICE, [_ptr(x) for x in T],
                   [_ptr(x) for x in Rbar] if Rbar is not None else None, Ebar, Wbar,
                   [_ptr(x) for x in Tb], _ptr(Bb) if Bb is not None else None,
                   _ptr(Fa) if Fa is not None else None, _ptr(Fb) if Fb is not None else None)
        return Tb, Bb, Fa, Fb

    def lambda_solve(self, T, state=1, method=DCSD, ref=0, tol=1e-9, maxiter=100, diis_n=8, L0=None,
                     want_rdm=True):
        """Lambda equations for E = dE_A + state * W at converged amplitudes T
        (CUDA tensors); returns (Lambda tuple, gamma_a, gamma_b, dcsd_result)."""
        t = self.torch
        n = self.n_c + 2 + self.n_v
        Lam = tuple(x.clone() for x in L0) if L0 is not None else tuple(t.zeros_like(x) for x in T)
        ga = t.zeros((n, n), dtype=t.float64, device=T[0].device) if want_rdm else None
        gb = t.zeros((n, n), dtype=t.float64, device=T[0].device) if want_rdm else None
        opts = L.dcsd_solve_opts(method, ref, PREC_FP64, maxiter, diis_n, tol, 0.0, 1 if L0 is not None else 0,
                                 0.0)
        res = L.dcsd_lambda(self.ctx, opts, state, MEM_DEVICE, [_ptr(x) for x in T], [_ptr(x) for x in Lam],
                            _ptr(ga) if ga is not None else None, _ptr(gb) if gb is not None else None)
        return Lam, ga, gb, res

    def inputs(self, requires_grad=True):
        """(fock_a, fock_b, B): device tensors holding the values this engine
        was created with, as leaves for residual_autograd (their gradients
        are the Fock-matrix and DF-factor parts of dcsd_vjp).  Modifying them
        does not change the engine: the library keeps its own copy."""
        if self._inputs is None:
            raise ValueError("this engine was not created from in-memory inputs")
        for x in self._inputs:
            x.requires_grad_(requires_grad)
        return self._inputs

    def residual_autograd(self, T, ref=0, method=DCSD, inputs=None):
        """FP64 residual as a differentiable torch function: returns (R1a,
        R1b, R2aa, R2bb, R2ab, W, dE_A) as tensors whose backward pass calls
        dcsd_vjp.  Differentiable with respect to the five amplitude tensors
        T and, when inputs = self.inputs() is passed, to the Fock matrices and
        the DF factors as well."""
        if inputs is None:
            return _residual_function().apply(self, ref, method, *T)
        if len(inputs) != 3 or any(x is not y for x, y in zip(inputs, self._inputs)):
            raise ValueError("inputs must be the tensors returned by this engine's inputs()")
        return _residual_function().apply(self, ref, method, *T, *inputs)

    def launches(self):
        return L.dcsd_kernel_launches(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            L.dcsd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_RESIDUAL_FN = None


def _residual_function():
    """torch.autograd.Function over the C ABI residual (built on first use so
    that importing the package does not import torch)."""
    global _RESIDUAL_FN
    if _RESIDUAL_FN is not None:
        return _RESIDUAL_FN
    import torch

    class ResidualFunction(torch.autograd.Function):
        @staticmethod
        def forward(ctx, engine, ref, method, *args):
            # args: the five amplitude tensors, then optionally (fock_a,
            # fock_b, B), whose values the engine already holds
            T = tuple(x.detach().contiguous() for x in args[:5])
            R, W, dE = engine.residual(T, ref=ref, method=method, precision=PREC_FP64)
            ctx.engine, ctx.ref, ctx.method = engine, ref, method
            ctx.n_inputs = len(args) - 5
            ctx.save_for_backward(*T)
            dev = T[0].device
            return (*R, torch.tensor(W, dtype=torch.float64, device=dev),
                    torch.tensor(dE, dtype=torch.float64, device=dev))

        @staticmethod
        def backward(ctx, *g):
            T = ctx.saved_tensors
            Rb = [gi.contiguous() if gi is not None else torch.zeros_like(x) for gi, x in zip(g[:5], T)]
            Wb = float(g[5]) if g[5] is not None else 0.0
            Eb = float(g[6]) if g[6] is not None else 0.0
            need = ctx.needs_input_grad[3 + 5:] if ctx.n_inputs else ()
            want_fock = any(need[:2]) if need else False
            want_B = bool(need[2]) if need else False
            Tb, Bb, Fa, Fb = ctx.engine.vjp(T, Rbar=Rb, Ebar=Eb, Wbar=Wb, ref=ctx.ref, method=ctx.method,
                                            want_B=want_B, want_fock=want_fock)
            extra = (Fa, Fb, Bb) if ctx.n_inputs else ()
            return (None, None, None, *Tb, *extra)

    _RESIDUAL_FN = ResidualFunction
    return _RESIDUAL_FN
