"""GB300-native two-determinant CCSD / DCSD residual engine (arXiv 2401.11935).

PyTorch supplies device memory and the CUDA stream; every step of the
residual, the energy, the DIIS solve and the effective Hamiltonian runs in
the CUDA kernels of libdcsd.so, reached through the C ABI of
include/dcsd.h (ctypes binding in ``_lib``).
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from ._lib import (CCSD, DCSD, MEM_DEVICE, MEM_HOST, PREC_BF16, PREC_BF16X3, PREC_BF16X6,  # noqa: F401
                   PREC_FP64, PREC_MIXED, DcsdError, dcsd_heff)

__all__ = ["Engine", "CCSD", "DCSD", "PREC_FP64", "PREC_BF16", "PREC_BF16X3", "PREC_BF16X6", "PREC_MIXED",
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
        del fa, fb, Bt

    @classmethod
    def from_system(cls, s, **kw):
        return cls(s.n_c, s.n_v, s.naux, s.fock_a, s.fock_b, s.B, **kw)

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
              switch_tol=1e-5, T0=None):
        """Converge the amplitudes on the device; returns (T, dcsd_result)."""
        T = tuple(x.clone() for x in T0) if T0 is not None else self.zeros()
        opts = L.dcsd_solve_opts(method, ref, precision, maxiter, diis_n, tol, switch_tol,
                                 1 if T0 is not None else 0)
        res = L.dcsd_solve(self.ctx, opts, MEM_DEVICE, [_ptr(x) for x in T])
        return T, res

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
