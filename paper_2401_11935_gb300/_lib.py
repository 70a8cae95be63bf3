"""ctypes binding of include/dcsd.h (argument marshalling only).

The functions below carry the C names and forward their arguments to
libdcsd.so; every step of the method runs in the library's CUDA kernels.
Loading fails loudly if the library has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdcsd.so")

DCSD_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "TIMEOUT",
          6: "NUMERIC", 7: "NO_DEVICE"}
CCSD, DCSD = 0, 1
FR_CCSD_S, FR_DCSD_S, FR_CCSD_T, FR_DCSD_T = 2, 3, 4, 5
MEM_HOST, MEM_DEVICE = 0, 1
PREC_FP64, PREC_BF16, PREC_BF16X3, PREC_MIXED, PREC_BF16X6 = 0, 1, 2, 3, 4

EXPORTS = ["dcsd_init", "dcsd_residual", "dcsd_energy", "dcsd_solve", "dcsd_heff",
           "dcsd_destroy", "dcsd_last_error", "dcsd_kernel_launches", "dcsd_profile",
           "dcsd_energy_noalloc", "dcsd_selftest_conversions", "dcsd_vjp", "dcsd_lambda",
           "dcsd_coupling_host", "dcsd_einsum_host", "dcsd_reserve", "dcsd_fcidump_header",
           "dcsd_fcidump_read", "dcsd_cholesky_host", "dcsd_fcidump_prepare", "dcsd_init_fcidump",
           "dcsd_fcidump_error"]
PROF_CLASSES = ["ladder_tc", "tc_other", "pack", "fp64", "c4", "c5", "c6", "c7"]


class dcsd_dims(C.Structure):
    _fields_ = [("n_c", C.c_int), ("n_v", C.c_int), ("naux", C.c_int)]


class dcsd_solve_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("ref", C.c_int), ("precision", C.c_int),
                ("maxiter", C.c_int), ("diis_n", C.c_int), ("tol", C.c_double),
                ("switch_tol", C.c_double), ("use_guess", C.c_int), ("polish_tol", C.c_double)]


class dcsd_result(C.Structure):
    _fields_ = [("dEA", C.c_double), ("W", C.c_double), ("E_S", C.c_double),
                ("E_T", C.c_double), ("max_r", C.c_double), ("iters", C.c_int),
                ("converged", C.c_int), ("seconds", C.c_double), ("switched_at", C.c_int),
                ("polished_at", C.c_int)]


class dcsd_fcidump_info(C.Structure):
    _fields_ = [("norb", C.c_int), ("nelec", C.c_int), ("ms2", C.c_int), ("n_frozen", C.c_int),
                ("n_c", C.c_int), ("n_v", C.c_int), ("naux", C.c_int), ("e_core", C.c_double),
                ("e_ref", C.c_double), ("chol_max_error", C.c_double)]


class DcsdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dcsd status {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2401_11935_gb300.build` (no CPU fallback exists)")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    D = C.POINTER(C.c_double)
    lib.dcsd_init.argtypes = [C.POINTER(P), C.POINTER(dcsd_dims), P, P, P, P, C.c_int, P]
    lib.dcsd_residual.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int] + [P] * 10 + [D, D]
    lib.dcsd_energy.argtypes = [P, C.c_int, C.c_int, C.c_int] + [P] * 5 + [D, D]
    lib.dcsd_solve.argtypes = [P, C.POINTER(dcsd_solve_opts), C.c_int] + [P] * 5 + [C.POINTER(dcsd_result)]
    lib.dcsd_heff.argtypes = [C.c_double, C.c_double, D, D, C.POINTER(C.c_int)]
    lib.dcsd_destroy.argtypes = [P]
    lib.dcsd_last_error.argtypes = [P]
    lib.dcsd_last_error.restype = C.c_char_p
    lib.dcsd_kernel_launches.argtypes = [P]
    lib.dcsd_kernel_launches.restype = C.c_longlong
    lib.dcsd_profile.argtypes = [P, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    lib.dcsd_profile.restype = C.c_int
    lib.dcsd_energy_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int] + [P] * 10
    lib.dcsd_energy_noalloc.restype = C.c_int
    lib.dcsd_vjp.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int] + [P] * 10 + [C.c_double, C.c_double] + [P] * 8
    lib.dcsd_vjp.restype = C.c_int
    lib.dcsd_lambda.argtypes = [P, C.POINTER(dcsd_solve_opts), C.c_int, C.c_int] + [P] * 12 + \
        [C.POINTER(dcsd_result)]
    lib.dcsd_lambda.restype = C.c_int
    lib.dcsd_selftest_conversions.argtypes = [P, C.POINTER(C.c_longlong)]
    lib.dcsd_selftest_conversions.restype = C.c_int
    lib.dcsd_coupling_host.argtypes = [C.c_int, C.c_int, C.c_int] + [P] * 10
    lib.dcsd_coupling_host.restype = C.c_int
    view = [P, C.c_int, P, P]
    lib.dcsd_einsum_host.argtypes = [C.c_char_p, C.c_double] + view + view + [C.c_double] + view
    lib.dcsd_einsum_host.restype = C.c_int
    lib.dcsd_reserve.argtypes = [P, C.c_int, C.c_int, C.c_int]
    lib.dcsd_reserve.restype = C.c_int
    lib.dcsd_fcidump_header.argtypes = [C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.dcsd_fcidump_read.argtypes = [C.c_char_p, C.c_int, P, P, D]
    lib.dcsd_cholesky_host.argtypes = [C.c_int, P, C.c_double, C.c_int, P, C.POINTER(C.c_int), D]
    lib.dcsd_fcidump_prepare.argtypes = [C.c_char_p, C.c_int, C.c_double, C.POINTER(dcsd_fcidump_info), P, P, P]
    lib.dcsd_init_fcidump.argtypes = [C.POINTER(P), C.c_char_p, C.c_int, C.c_double, C.c_int, P,
                                      C.POINTER(dcsd_fcidump_info)]
    lib.dcsd_fcidump_error.argtypes = []
    lib.dcsd_fcidump_error.restype = C.c_char_p
    for name in ("dcsd_fcidump_header", "dcsd_fcidump_read", "dcsd_cholesky_host", "dcsd_fcidump_prepare",
                 "dcsd_init_fcidump"):
        getattr(lib, name).restype = C.c_int
    for name in ("dcsd_init", "dcsd_residual", "dcsd_energy", "dcsd_solve", "dcsd_heff", "dcsd_destroy"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != DCSD_OK:
        msg = load().dcsd_last_error(ctx).decode(errors="replace")
        raise DcsdError(status, msg)


def dcsd_init(n_c, n_v, naux, eps, fock_a, fock_b, B, mem_kind, stream):
    """Create a context; pointers are ints (host or device addresses)."""
    lib = load()
    ctx = C.c_void_p()
    d = dcsd_dims(n_c, n_v, naux)
    st = lib.dcsd_init(C.byref(ctx), C.byref(d), eps, fock_a, fock_b, B, mem_kind, stream)
    _check(st, None)
    return ctx


def dcsd_residual(ctx, ref, method, precision, mem_kind, T, R):
    lib = load()
    W, dE = C.c_double(), C.c_double()
    st = lib.dcsd_residual(ctx, ref, method, precision, mem_kind, *T, *R, C.byref(W), C.byref(dE))
    _check(st, ctx)
    return W.value, dE.value


def dcsd_energy(ctx, ref, method, mem_kind, T):
    lib = load()
    W, dE = C.c_double(), C.c_double()
    st = lib.dcsd_energy(ctx, ref, method, mem_kind, *T, C.byref(dE), C.byref(W))
    _check(st, ctx)
    return dE.value, W.value


def dcsd_solve(ctx, opts, mem_kind, T, allow_not_converged=True):
    lib = load()
    res = dcsd_result()
    st = lib.dcsd_solve(ctx, C.byref(opts), mem_kind, *T, C.byref(res))
    if not (allow_not_converged and st == 4):
        _check(st, ctx)
    return res


def dcsd_reserve(ctx, precision, diis_n=8, host_staging=0):
    """Allocate ahead of time what residuals of `precision`, a solve with
    diis_n DIIS vectors and (host_staging=1) host-memory calls need."""
    _check(load().dcsd_reserve(ctx, precision, diis_n, host_staging), ctx)


def dcsd_heff(dEA, W):
    lib = load()
    H = (C.c_double * 4)()
    ev = (C.c_double * 2)()
    si = C.c_int()
    _check(lib.dcsd_heff(dEA, W, H, ev, C.byref(si)))
    return [H[0], H[1], H[2], H[3]], [ev[0], ev[1]], si.value


def dcsd_destroy(ctx):
    _check(load().dcsd_destroy(ctx))


def dcsd_kernel_launches(ctx):
    return load().dcsd_kernel_launches(ctx)


def dcsd_profile(ctx, enable, reset, read=True):
    """Returns {class: (ms, launches)} when read is True."""
    lib = load()
    ms = (C.c_double * 8)()
    ln = (C.c_longlong * 8)()
    _check(lib.dcsd_profile(ctx, enable, reset, ms if read else None, ln if read else None), ctx)
    if not read:
        return None
    return {PROF_CLASSES[k]: (ms[k], ln[k]) for k in range(8)}


def dcsd_energy_noalloc(n_c, n_v, naux, ref, fock_a, fock_b, B, T, dEA, stream):
    """Allocation-free Delta E_A; all pointers are device addresses (ints)."""
    st = load().dcsd_energy_noalloc(n_c, n_v, naux, ref, fock_a, fock_b, B, *T, dEA, stream)
    if st != DCSD_OK:
        raise DcsdError(st, "dcsd_energy_noalloc failed")


def dcsd_selftest_conversions(stream=None):
    """Number of mismatches between the library's integer-unit FP64<->FP32
    conversions and the hardware conversions on the current device."""
    n = C.c_longlong(-1)
    st = load().dcsd_selftest_conversions(stream, C.byref(n))
    if st != 0:
        raise DcsdError(st, "dcsd_selftest_conversions failed")
    return n.value


def dcsd_coupling_host(ref, n_c, n_v, T):
    """Coupling coefficients c_q of frame `ref` (host evaluation from the
    library's term tables); T: five C-contiguous float64 numpy arrays in the
    amplitude layout.  Returns five arrays in the same layout."""
    import numpy as np
    T = [np.ascontiguousarray(x, dtype=np.float64) for x in T]
    out = [np.zeros_like(x) for x in T]
    st = load().dcsd_coupling_host(ref, n_c, n_v, *[x.ctypes.data for x in T], *[x.ctypes.data for x in out])
    if st != 0:
        raise DcsdError(st, "dcsd_coupling_host failed")
    return tuple(out)


def dcsd_einsum_host(spec, alpha, a, b, beta, c):
    """c = beta c + alpha einsum(spec)(a, b) executed on the host from the
    library's contraction plan; a, b, c: float64 numpy arrays or strided
    views of them (c written in place)."""
    import numpy as np

    keep = []

    def view(x):
        if x.dtype != np.float64:
            raise TypeError("float64 arrays only")
        n = max(1, x.ndim)
        sz = (C.c_long * n)(*x.shape)
        st = (C.c_long * n)(*[s // 8 for s in x.strides])
        keep.append((sz, st))
        return [x.__array_interface__["data"][0], x.ndim, C.cast(sz, C.c_void_p), C.cast(st, C.c_void_p)]

    st = load().dcsd_einsum_host(spec.encode(), float(alpha), *view(a), *view(b), float(beta), *view(c))
    if st != 0:
        raise DcsdError(st, "dcsd_einsum_host failed for " + spec)


def dcsd_vjp(ctx, ref, method, precision, mem_kind, T, Rbar, Ebar, Wbar, Tbar, Bbar=None, Fa=None, Fb=None):
    """Raw call; T, Rbar (or None), Tbar: 5 pointers each."""
    Rb = list(Rbar) if Rbar is not None else [None] * 5
    st = load().dcsd_vjp(ctx, ref, method, precision, mem_kind, *T, *Rb, float(Ebar), float(Wbar), *Tbar, Bbar, Fa, Fb)
    _check(st, ctx)


def dcsd_lambda(ctx, opts, state, mem_kind, T, Lam, rdm_a=None, rdm_b=None):
    """Raw call; returns the dcsd_result (raises unless converged)."""
    res = dcsd_result()
    st = load().dcsd_lambda(ctx, C.byref(opts), state, mem_kind, *T, *Lam, rdm_a, rdm_b, C.byref(res))
    if st not in (0, 4):
        _check(st, ctx)
    return res


def _fcidump_check(st):
    if st != DCSD_OK:
        raise DcsdError(st, load().dcsd_fcidump_error().decode(errors="replace"))


def dcsd_fcidump_header(path):
    """(norb, nelec, ms2) of an FCIDUMP file."""
    n, ne, ms = C.c_int(), C.c_int(), C.c_int()
    _fcidump_check(load().dcsd_fcidump_header(os.fsencode(path), C.byref(n), C.byref(ne), C.byref(ms)))
    return n.value, ne.value, ms.value


def dcsd_fcidump_read(path):
    """(h [n,n], eri [n,n,n,n], ecore) as numpy arrays, read by the library."""
    import numpy as np
    n, _, _ = dcsd_fcidump_header(path)
    h = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    ec = C.c_double()
    _fcidump_check(load().dcsd_fcidump_read(os.fsencode(path), n, h.ctypes.data, eri.ctypes.data, C.byref(ec)))
    return h, eri, ec.value


def dcsd_cholesky_host(eri, tol=1e-12):
    """Pivoted Cholesky factors B [rank, n, n] of (pq|rs) and the bound on the
    remaining error."""
    import numpy as np
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    n = eri.shape[0]
    cap = n * (n + 1) // 2
    B = np.zeros((cap, n, n))
    r, left = C.c_int(), C.c_double()
    st = load().dcsd_cholesky_host(n, eri.ctypes.data, tol, cap, B.ctypes.data, C.byref(r), C.byref(left))
    if st != DCSD_OK:
        raise DcsdError(st, "dcsd_cholesky_host failed")
    return B[:r.value].copy(), left.value


def dcsd_fcidump_prepare(path, n_frozen=0, chol_tol=1e-12):
    """(info, fock_a, fock_b, B) as prepared by the library for dcsd_init."""
    import numpy as np
    info = dcsd_fcidump_info()
    p = os.fsencode(path)
    _fcidump_check(load().dcsd_fcidump_prepare(p, n_frozen, chol_tol, C.byref(info), None, None, None))
    n = info.n_c + 2 + info.n_v
    fa, fb = np.zeros((n, n)), np.zeros((n, n))
    B = np.zeros((info.naux, n, n))
    _fcidump_check(load().dcsd_fcidump_prepare(p, n_frozen, chol_tol, C.byref(info), fa.ctypes.data,
                                               fb.ctypes.data, B.ctypes.data))
    return info, fa, fb, B


def dcsd_init_fcidump(path, n_frozen, chol_tol, stored_ladder, stream):
    """Create a context from an FCIDUMP file; returns (ctx, info)."""
    ctx = C.c_void_p()
    info = dcsd_fcidump_info()
    _fcidump_check(load().dcsd_init_fcidump(C.byref(ctx), os.fsencode(path), n_frozen, chol_tol,
                                            1 if stored_ladder else 0, stream, C.byref(info)))
    return ctx, info
