"""Command-line runs of the engine on seeded synthetic inputs (for timing and
for profiler captures of single kernels).

    python -m paper_2401_11935_gb300 residual --dims 30,500,1500 --precision bf16 --repeat 1
    python -m paper_2401_11935_gb300 solve --dims 10,120,360 --precision mixed --maxiter 40
    python -m paper_2401_11935_gb300 compare --dims c3 --tol 1e-8
    python -m paper_2401_11935_gb300 vjp --dims c4 --repeat 2
    python -m paper_2401_11935_gb300 vjp --dims c5 --precision bf16x6
    python -m paper_2401_11935_gb300 lambda --dims c4
    python -m paper_2401_11935_gb300 stgap --fcidump SA --singlet S --triplet T
    python -m paper_2401_11935_gb300 stgap --dims 4,20,60 --rotate 0.05

compare converges the FP64 and the mixed-precision solves from the same
guess and prints their energies (Delta E_A, W, singlet and triplet energies,
gap 2W), the differences and the wall time of each converged solve.

--dims is n_c,n_v,naux (core orbitals, external virtuals, DF functions) or
one of the named workloads c1..c5.  --precision defaults to bf16, except
for vjp and lambda, which default to fp64.  The inputs come from the seeded
generator in ``synth``; the residual is evaluated at seeded random
amplitudes of magnitude 1e-3.  Prints one line per call with the device
time.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

PREC = {"fp64": 0, "bf16": 1, "bf16x3": 2, "mixed": 3, "bf16x6": 4}


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2401_11935_gb300")
    ap.add_argument("what", choices=["residual", "solve", "compare", "vjp", "lambda", "stgap"])
    ap.add_argument("--fcidump", default=None, help="stgap: FCIDUMP of the single calculation")
    ap.add_argument("--singlet", default=None, help="stgap: FCIDUMP of the singlet's own orbitals")
    ap.add_argument("--triplet", default=None, help="stgap: FCIDUMP of the triplet's own orbitals")
    ap.add_argument("--rotate", type=float, default=0.05,
                    help="stgap without files: size of the orbital rotations of the synthetic sets")
    ap.add_argument("--frozen", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--switch-tol", type=float, default=1e-5)
    ap.add_argument("--polish-tol", type=float, default=1e-7)
    ap.add_argument("--dims", default="c3")
    ap.add_argument("--precision", default=None, choices=sorted(PREC))
    ap.add_argument("--method", default="dcsd", choices=["ccsd", "dcsd"])
    ap.add_argument("--ref", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--maxiter", type=int, default=60)
    ap.add_argument("--seed", type=int, default=3)
    a = ap.parse_args(argv)
    if a.precision is None:
        a.precision = "fp64" if a.what in ("vjp", "lambda") else "bf16"

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    from synth import CONFIGS, make_system, random_amplitudes
    import paper_2401_11935_gb300 as P

    if a.what == "stgap":
        return stgap_main(a, P)
    if a.dims in CONFIGS:
        s = make_system(a.dims)
    else:
        s = make_system(tuple(int(x) for x in a.dims.split(",")), seed=a.seed)
    method = P.DCSD if a.method == "dcsd" else P.CCSD
    eng = P.Engine.from_system(s)
    try:
        if a.what == "residual":
            Td = eng.to_device(random_amplitudes(s, seed=a.seed, ref=a.ref, scale1=1e-3, scale2=1e-3))
            for k in range(a.repeat):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, W, dE = eng.residual(Td, ref=a.ref, method=method, precision=PREC[a.precision])
                torch.cuda.synchronize()
                print(f"residual {k} dims=({s.n_c},{s.n_v},{s.naux}) precision={a.precision} "
                      f"{time.perf_counter() - t0:.4f} s  W={W:.12g} dEA={dE:.12g}", flush=True)
        elif a.what == "vjp":
            Td = eng.to_device(random_amplitudes(s, seed=a.seed, ref=a.ref, scale1=1e-3, scale2=1e-3))
            Rb = eng.to_device(random_amplitudes(s, seed=a.seed + 1, ref=a.ref))
            for k in range(a.repeat):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                eng.vjp(Td, Rbar=Rb, Ebar=1.0, Wbar=1.0, ref=a.ref, method=method, want_B=True, want_fock=True,
                        precision=PREC[a.precision])
                torch.cuda.synchronize()
                print(f"vjp {k} dims=({s.n_c},{s.n_v},{s.naux}) precision={a.precision} "
                      f"{time.perf_counter() - t0:.4f} s", flush=True)
        elif a.what == "lambda":
            T, res = eng.solve(ref=a.ref, method=method, precision=0, maxiter=a.maxiter, tol=a.tol)
            for state in (1, -1):
                _, ga, gb, lr = eng.lambda_solve(T, state=state, method=method, ref=a.ref, tol=a.tol,
                                                 maxiter=a.maxiter)
                tr = float(ga.diagonal().sum() + gb.diagonal().sum())
                print(f"lambda state={state:+d} dims=({s.n_c},{s.n_v},{s.naux}) iters={lr.iters} "
                      f"converged={lr.converged} max|dL/dT|={lr.max_r:.2e} seconds={lr.seconds:.3f} "
                      f"trace(gamma)={tr:+.6e}", flush=True)
        elif a.what == "solve":
            _, res = eng.solve(ref=a.ref, method=method, precision=PREC[a.precision], maxiter=a.maxiter,
                               tol=a.tol, switch_tol=a.switch_tol, polish_tol=a.polish_tol)
            print(f"solve dims=({s.n_c},{s.n_v},{s.naux}) precision={a.precision} iters={res.iters} "
                  f"converged={res.converged} switched_at={res.switched_at} polished_at={res.polished_at} "
                  f"seconds={res.seconds:.3f} max|R|={res.max_r:.2e} dEA={res.dEA:.12f} W={res.W:.12f} "
                  f"E_S={res.E_S:.12f} E_T={res.E_T:.12f}", flush=True)
        else:
            out = {}
            for name in ("fp64", "mixed"):
                _, res = eng.solve(ref=a.ref, method=method, precision=PREC[name], maxiter=a.maxiter,
                                   tol=a.tol, switch_tol=a.switch_tol, polish_tol=a.polish_tol)
                out[name] = res
                print(f"{name:5s} iters={res.iters} converged={res.converged} switched_at={res.switched_at} "
                      f"polished_at={res.polished_at} "
                      f"seconds={res.seconds:.3f} max|R|={res.max_r:.2e} dEA={res.dEA:.12f} W={res.W:.12f} "
                      f"E_S={res.E_S:.12f} E_T={res.E_T:.12f}", flush=True)
            f, m = out["fp64"], out["mixed"]
            print(f"mixed - fp64: dEA {m.dEA - f.dEA:+.3e}  W {m.W - f.W:+.3e}  E_S {m.E_S - f.E_S:+.3e}  "
                  f"E_T {m.E_T - f.E_T:+.3e}  gap {2 * (m.W - f.W):+.3e} Eh;  time ratio fp64/mixed "
                  f"{f.seconds / m.seconds:.2f}", flush=True)
    finally:
        eng.close()


def stgap_main(a, P):
    """Singlet-triplet gaps from one calculation (the first file) and from
    two (singlet and triplet files).  Without files, three orbital sets of a
    synthetic system (core Hamiltonian and four-index integrals) are written
    to a temporary directory: the generated orbitals and two sets rotated by
    occupied-virtual mixing of size --rotate."""
    import tempfile
    from paper_2401_11935_gb300 import stgap
    method = P.DCSD if a.method == "dcsd" else P.CCSD
    paths = [a.fcidump, a.singlet, a.triplet]
    tmp = None
    if a.fcidump is None:
        from synth import make_pin_system
        from synth import fcidump as wf
        dims = tuple(int(x) for x in a.dims.split(",")) if "," in a.dims else (4, 20, 60)
        s = make_pin_system(*dims, seed=a.seed, b_sigma=0.08)
        eri = wf.eri_from_factors(s.B)
        tmp = tempfile.TemporaryDirectory()
        sets = [(s.h, eri)] + [wf.rotate(s.h, eri, wf.random_ov_rotation(s.parity, s.n_c + 2, a.rotate, a.seed + k))
                               for k in (1, 2)]
        paths = []
        for k, (h, e) in enumerate(sets):
            p = os.path.join(tmp.name, f"FCIDUMP.{k}")
            wf.write(p, h, e, 2 * s.n_c + 2, 0, orbsym=[1 + int(x) for x in s.parity])
            paths.append(p)
    g = stgap.gaps(paths[0], singlet=paths[1], triplet=paths[2], method=method, n_frozen=a.frozen, tol=a.tol,
                   precision=PREC[a.precision or "fp64"], maxiter=a.maxiter)
    one = g["single"]
    print(f"one calculation:  E_S {one['E_S']:.10f}  E_T {one['E_T']:.10f}  gap {one['gap']:.10f} Eh "
          f"({one['gap'] * 27.211386:.4f} eV)  {one['iters']} iterations, {one['seconds']:.3f} s", flush=True)
    if "state_specific" in g:
        ss = g["state_specific"]
        print(f"two calculations: E_S {ss['E_S']:.10f}  E_T {ss['E_T']:.10f}  gap {ss['gap']:.10f} Eh "
              f"({ss['gap'] * 27.211386:.4f} eV)  {ss['iters']} iterations, {ss['seconds']:.3f} s", flush=True)
        print(f"difference (one - two): {(one['gap'] - ss['gap']) * 27211.386:+.3f} meV", flush=True)
    if tmp is not None:
        tmp.cleanup()
    return 0


if __name__ == "__main__":
    main()
