"""Singlet-triplet gaps from one or from two calculations (the comparison of
the paper's Table 4, Section IV.B).

A two-determinant calculation is state-universal: one solve with one set of
orbitals (for instance state-averaged 2D-SCF orbitals) gives both the
open-shell singlet dE_A + W and the M_s = 0 triplet dE_A - W, so the gap is
2W.  The state-specific alternative solves twice, with orbitals optimised
for each state, and subtracts total energies.  Both run here on FCIDUMP
files (dcsd_init_fcidump), and each total energy is the file's reference
energy <Phi_A|H|Phi_A> plus the correlation energy; every solve runs in the
library's kernels.  The orbital optimisations themselves (2D-SCF, ROHF,
state averaging) are outside this library: the files carry their result.
"""
from __future__ import annotations

import time

from . import DCSD, PREC_FP64, Engine


def _solve(path, method, n_frozen, tol, precision, maxiter):
    eng = Engine.from_fcidump(path, n_frozen=n_frozen)
    try:
        t0 = time.perf_counter()
        _, res = eng.solve(method=method, precision=precision, tol=tol, maxiter=maxiter)
        dt = time.perf_counter() - t0
        if not res.converged:
            raise RuntimeError(f"solve of {path} did not converge (max|R| {res.max_r:.2e})")
        e_ref = eng.fcidump.e_ref
    finally:
        eng.close()
    return {"E_S": e_ref + res.E_S, "E_T": e_ref + res.E_T, "e_ref": e_ref, "W": res.W, "dEA": res.dEA,
            "iters": res.iters, "seconds": dt}


def gaps(single, singlet=None, triplet=None, method=DCSD, n_frozen=0, tol=1e-8, precision=PREC_FP64,
         maxiter=100):
    """Total singlet and triplet energies and S-T gaps (E_S - E_T, in Eh).

    single  : FCIDUMP of the orbitals for the single calculation (e.g.
              state-averaged); gives 'single' = both states from one solve.
    singlet, triplet : FCIDUMPs of the state-specific orbitals; when given,
              'state_specific' holds E_S from the singlet orbitals, E_T from
              the triplet orbitals (the M_s = 0 root of each solve) and their
              difference."""
    out = {"method": method}
    one = _solve(single, method, n_frozen, tol, precision, maxiter)
    out["single"] = dict(one, gap=one["E_S"] - one["E_T"])
    if singlet is not None and triplet is not None:
        s = _solve(singlet, method, n_frozen, tol, precision, maxiter)
        t = _solve(triplet, method, n_frozen, tol, precision, maxiter)
        out["state_specific"] = {"E_S": s["E_S"], "E_T": t["E_T"], "gap": s["E_S"] - t["E_T"],
                                 "seconds": s["seconds"] + t["seconds"], "iters": s["iters"] + t["iters"]}
    return out
