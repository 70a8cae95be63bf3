"""Write oracle values of single residual elements of a full-size workload
to tests/golden/<name>_elements.json.

Calls only the element-wise CPU oracle (oracle/element.py) and the seeded
generator (synth/).  The amplitudes are the ones the command-line residual
run uses (``python -m paper_2401_11935_gb300 residual --dims <name>``:
synth.random_amplitudes with seed 3, magnitude 1e-3, reference A), the
method 2D-DCSD.  Stored: Delta E_A (first term of Eq. 2), W (the A->B
residual element) and sampled elements of R1a, R1b, R2aa, R2bb, R2ab
(Eqs. 3-4), at fixed pseudo-random positions.

Usage: python tests/golden/make_elements.py c5 [n_samples]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from synth import CONFIGS, frame_orbitals, make_system, random_amplitudes  # noqa: E402
from oracle import element  # noqa: E402

SEED, SCALE, REF, METHOD = 3, 1e-3, 0, 1


def positions(s, n, rng):
    """n element positions per block: same-spin diagonals excluded, and only
    excitations whose orbital Z2 labels add up to even (the others vanish by
    the symmetry of the synthetic Hamiltonian)."""
    o, v = s.n_c + 1, s.n_v + 1
    oa, ob, va, vb = frame_orbitals(s.n_c, s.n_v, REF)
    par = s.parity
    occ = (oa, ob, oa)   # spins of i (and j) per block: R1a, R1b / R2aa, R2bb, R2ab
    vir = (va, vb, va)
    occ2 = (oa, ob, ob)
    vir2 = (va, vb, vb)
    out = []
    for blk in range(5):
        k = 0
        while k < n:
            if blk < 2:
                i, a = int(rng.integers(o)), int(rng.integers(v))
                if par[occ[blk][i]] ^ par[vir[blk][a]]:
                    continue
                idx = (i, a)
            else:
                b3 = blk - 2
                i, j, a, b = (int(x) for x in (rng.integers(o), rng.integers(o), rng.integers(v), rng.integers(v)))
                if b3 < 2 and (i == j or a == b):
                    continue
                if par[occ[b3][i]] ^ par[occ2[b3][j]] ^ par[vir[b3][a]] ^ par[vir2[b3][b]]:
                    continue
                idx = (i, j, a, b)
            out.append((blk, idx))
            k += 1
    return out


def main(name, n):
    t0 = time.time()
    s = make_system(name)
    T = random_amplitudes(s, seed=SEED, ref=REF, scale1=SCALE, scale2=SCALE)
    eo = element.ElementOracle(s, REF, METHOD, T)
    res = {"workload": name, "dims": CONFIGS[name][:3], "amplitudes": {"seed": SEED, "scale": SCALE},
           "ref": REF, "method": "2D-DCSD", "generator": "synth.make_system + synth.random_amplitudes",
           "oracle": "oracle/element.py", "W": eo.W(), "dEA": eo.energy(), "elements": []}
    print(name, "W", res["W"], "dEA", res["dEA"], flush=True)
    for blk, idx in positions(s, n, np.random.default_rng(11)):
        val = element.residual_element(eo, blk, idx)
        res["elements"].append({"block": blk, "index": list(idx), "value": val})
        print(blk, idx, val, flush=True)
    res["oracle_seconds"] = time.time() - t0
    with open(os.path.join(HERE, f"{name}_elements.json"), "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "c5", int(sys.argv[2]) if len(sys.argv) > 2 else 2)
