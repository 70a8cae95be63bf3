"""Write oracle values of single residual elements of a full-size workload
to tests/golden/<name>_elements.json.

Calls only the element-wise CPU oracle (oracle/element.py) and the seeded
generator (synth/).  The amplitudes are the ones the command-line residual
run uses (``python -m paper_2401_11935_gb300 residual --dims <name>``:
synth.random_amplitudes with seed 3, magnitude 1e-3, reference A), the
method 2D-DCSD.  Stored: Delta E_A (first term of Eq. 2), W (the A->B
residual element) and sampled elements of R1a, R1b, R2aa, R2bb, R2ab
(Eqs. 3-4), at fixed pseudo-random positions; and, for the reverse mode, the
derivative of one R2ab element along a seeded direction d (fourth-order
central stencil of the element-wise oracle).  Checksums of the generated
inputs let a consumer detect inputs that differ from these (another numpy
random stream).

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
from oracle.vjp import antisym  # noqa: E402

SEED, SCALE, REF, METHOD = 3, 1e-3, 0, 1
DIR_SEED, H = 91, 1e-3


def direction(T, seed=DIR_SEED):
    """Random direction over the five amplitude arrays, antisymmetric in the
    same-spin doubles."""
    rng = np.random.default_rng(seed)
    d = [rng.normal(0.0, 1.0, t.shape) for t in T]
    d[2], d[3] = antisym(d[2]), antisym(d[3])
    return d


def checksums(s, T, d=None):
    """Sums of absolute values (no cancellation: the same-spin doubles are
    antisymmetric and sum to zero)."""
    a = lambda x: float(np.abs(x).sum())  # noqa: E731
    out = {"B": a(s.B), "fock_a": a(s.fock_a), "fock_b": a(s.fock_b), "T": [a(x) for x in T]}
    if d is not None:
        out["d"] = [a(x) for x in d]
    return out


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
    # reverse mode: d/de R_q(T + e d) for the first sampled R2ab element
    q = next(e for e in res["elements"] if e["block"] == 4)
    d = direction(T)

    def r(e):
        Te = tuple(t + e * x for t, x in zip(T, d))
        return element.residual_element(element.ElementOracle(s, REF, METHOD, Te), 4, tuple(q["index"]))
    deriv = (8.0 * (r(H) - r(-H)) - (r(2 * H) - r(-2 * H))) / (12.0 * H)
    res["vjp"] = {"block": 4, "index": q["index"], "direction_seed": DIR_SEED, "h": H, "value": deriv}
    print("vjp directional derivative", deriv, flush=True)
    res["checksums"] = checksums(s, T, d)
    res["oracle_seconds"] = time.time() - t0
    with open(os.path.join(HERE, f"{name}_elements.json"), "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "c5", int(sys.argv[2]) if len(sys.argv) > 2 else 2)
