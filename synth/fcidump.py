"""Writes integrals in the FCIDUMP text format (input generation only: the
file layout, no method arithmetic).

Header "&FCI NORB=n,NELEC=N,MS2=m, ORBSYM=..., ISYM=1, &END", then
(ij|kl) for i >= j, k >= l, (ij) >= (kl) (1-based, chemists' notation),
h_ij for i >= j with k = l = 0, and the core energy with all indices 0.
Values below `drop` in magnitude are omitted, as integral programs do.
"""
from __future__ import annotations

import numpy as np


def write(path, h, eri, nelec, ms2=0, ecore=0.0, orbsym=None, drop=0.0, exp_char="E"):
    n = h.shape[0]
    orbsym = [1] * n if orbsym is None else list(orbsym)
    fmt = lambda v: ("%.17E" % v).replace("E", exp_char)  # noqa: E731
    with open(path, "w") as f:
        f.write(f" &FCI NORB={n},NELEC={nelec},MS2={ms2},\n")
        f.write("  ORBSYM=" + ",".join(str(x) for x in orbsym) + ",\n")
        f.write("  ISYM=1,\n &END\n")
        for i in range(n):
            for j in range(i + 1):
                ij = i * (i + 1) // 2 + j
                for k in range(n):
                    for l in range(k + 1):
                        if k * (k + 1) // 2 + l > ij:
                            continue
                        v = eri[i, j, k, l]
                        if abs(v) > drop:
                            f.write(f"{fmt(v)} {i + 1} {j + 1} {k + 1} {l + 1}\n")
        for i in range(n):
            for j in range(i + 1):
                if abs(h[i, j]) > drop:
                    f.write(f"{fmt(h[i, j])} {i + 1} {j + 1} 0 0\n")
        f.write(f"{fmt(ecore)} 0 0 0 0\n")


def eri_from_factors(B):
    """(pq|rs) = sum_L B[L,p,q] B[L,r,s] -- the four-index array a DF
    factor set stands for (layout conversion of the synthetic inputs)."""
    return np.einsum("Lpq,Lrs->pqrs", B, B, optimize=True)


def random_ov_rotation(parity, n_occ, scale, seed):
    """A seeded orthogonal orbital rotation U = exp(K) that mixes the first
    n_occ orbitals (occupied in the reference) with the rest, only within
    the same symmetry label: K antisymmetric, K[p, q] ~ N(0, scale^2) for p
    occupied, q virtual, parity[p] == parity[q].  Stands in for the orbital
    relaxation between two orbital sets of one molecule (state-averaged vs
    state-specific orbitals)."""
    from scipy.linalg import expm
    n = len(parity)
    rng = np.random.default_rng(seed)
    K = np.zeros((n, n))
    for p in range(n_occ):
        for q in range(n_occ, n):
            if parity[p] == parity[q]:
                K[p, q] = rng.normal(0.0, scale)
    K = K - K.T
    return expm(K)


def rotate(h, eri, U):
    """Integrals in the rotated orbitals phi'_p = sum_q phi_q U[q, p]:
    h' = U^T h U, (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd) (a basis change
    of the inputs)."""
    h2 = U.T @ h @ U
    e = np.einsum("abcd,ap->pbcd", eri, U, optimize=True)
    e = np.einsum("pbcd,bq->pqcd", e, U, optimize=True)
    e = np.einsum("pqcd,cr->pqrd", e, U, optimize=True)
    e = np.einsum("pqrd,ds->pqrs", e, U, optimize=True)
    return h2, e
