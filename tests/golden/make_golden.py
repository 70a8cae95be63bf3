"""Write oracle energies of the named workloads to tests/golden/*.json.

Calls only the CPU oracle (oracle/) and the seeded generator (synth/).
Usage: python tests/golden/make_golden.py c1 [c2 ...] [--only 2D-DCSD]
The GPU tests compare the library's converged energies with these files:
2D-CCSD and 2D-DCSD (Section II), and the fixed-reference FR-CCSD and
FR-DCSD (Section I) for the singlet (fixed amplitude +1) and the M_s = 0
triplet (-1).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import dataclasses  # noqa: E402

import numpy as np  # noqa: E402

from synth import CONFIGS, CONFIG_SEED, b_sigma_for, make_system  # noqa: E402
from oracle import solve  # noqa: E402

TOL = {"c1": 1e-10, "c2": 1e-10, "c3": 1e-9, "c4": 1e-10}


def response_direction(s, method):
    """Seeded symmetric Fock perturbation (df_alpha, df_beta), N(0, 0.01^2)
    entries, zero where the orbital Z2 labels differ (the perturbed system
    keeps the symmetry of the unperturbed one)."""
    rng = np.random.default_rng(17 + method)
    mask = (s.parity[:, None] == s.parity[None, :]).astype(float)

    def sym(x):
        return 0.5 * (x + x.T) * mask
    return sym(rng.normal(0, 1e-2, s.fock_a.shape)), sym(rng.normal(0, 1e-2, s.fock_b.shape))


def response(s, method, tol, h=0.05):
    """d E_S / de and d E_T / de of the converged 2D energies along
    f -> f + e df (fourth-order central stencil of four oracle solves)."""
    dfa, dfb = response_direction(s, method)
    E = {}
    for e in (-2 * h, -h, h, 2 * h):
        sp = dataclasses.replace(s, fock_a=s.fock_a + e * dfa, fock_b=s.fock_b + e * dfb)
        _, info = solve.solve(sp, method, ref=0, tol=tol, maxiter=300)
        assert info["converged"]
        E[e] = (info["E_S"], info["E_T"])
    d = [(8 * (E[h][k] - E[-h][k]) - (E[2 * h][k] - E[-2 * h][k])) / (12 * h) for k in (0, 1)]
    return {"h": h, "direction_seed": 17 + method, "direction_abs_sum": float(np.abs(dfa).sum() + np.abs(dfb).sum()),
            "dE_S": d[0], "dE_T": d[1]}


def main(names, only=None):
    """only: restrict to one entry of the results (e.g. "2D-DCSD") -- the
    second workload's oracle solve takes hours per method."""
    for name in names:
        s = make_system(name)
        out = {"workload": name, "dims": CONFIGS[name][:3], "seed": CONFIG_SEED[name],
               "b_sigma": b_sigma_for(s.naux, s.v), "generator": "synth.make_system", "results": {}}
        for method, mname in ((0, "2D-CCSD"), (1, "2D-DCSD")):
            if only and mname != only:
                continue
            t0 = time.time()
            _, info = solve.solve(s, method, ref=0, tol=TOL[name], maxiter=300, verbose=True)
            out["results"][mname] = {k: float(info[k]) for k in ("dEA", "W", "E_S", "E_T", "max_r")}
            out["results"][mname]["iters"] = int(info["iters"])
            out["results"][mname]["converged"] = bool(info["converged"])
            out["results"][mname]["oracle_seconds"] = time.time() - t0
            print(name, mname, out["results"][mname], flush=True)
        for method, mname in ((0, "FR-CCSD"), (1, "FR-DCSD")):
            for sign, st in ((1.0, "S"), (-1.0, "T")):
                if only and f"{mname} {st}" != only:
                    continue
                t0 = time.time()
                _, info = solve.solve(s, method, ref=0, tol=TOL[name], maxiter=300, fixed=sign)
                key = f"{mname} {st}"
                out["results"][key] = {k: float(info[k]) for k in ("E", "W", "max_r")}
                out["results"][key]["iters"] = int(info["iters"])
                out["results"][key]["converged"] = bool(info["converged"])
                out["results"][key]["oracle_seconds"] = time.time() - t0
                print(name, key, out["results"][key], flush=True)
        if name == "c1":
            out["response"] = {}
            for method, mname in ((0, "2D-CCSD"), (1, "2D-DCSD")):
                out["response"][mname] = response(s, method, 1e-12)
                print(name, "response", mname, out["response"][mname], flush=True)
        with open(os.path.join(HERE, f"{name}_energies.json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    args = sys.argv[1:]
    only = None
    if "--only" in args:
        k = args.index("--only")
        only = args[k + 1]
        del args[k:k + 2]
    main(args or ["c1"], only)
