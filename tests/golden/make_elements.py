"""Write oracle values of single residual elements of a full-size workload
to tests/golden/<name>_elements.json.

Calls only the element-wise CPU oracle (oracle/element.py) and the seeded
generator (synth/).  The amplitudes are the ones the command-line residual
run uses (``python -m paper_2401_11935_gb300 residual --dims <name>``:
synth.random_amplitudes with seed 3, magnitude 1e-3, reference A), the
method 2D-DCSD.  Stored: Delta E_A (first term of Eq. 2), W (the A->B
residual element) and sampled elements of R1a, R1b, R2aa, R2bb, R2ab
(Eqs. 3-4); for each doubles element also its particle-particle ladder
piece 1/2 sum_ef tau_ijef <ab||ef>, so that a consumer can check that its
tolerance is far below what a missing or misplaced ladder contribution
would change.  The doubles positions are stratified: per block, random
positions plus positions whose first virtual index lies in the first or in
the last rows of the virtual range (the first and last integral chunks of a
ladder that is built row block by row block), with the second virtual index
on either side of the first, and, for the same-spin blocks, rows with i > j
as well as i < j.  For the reverse mode: the derivative of one R2ab element
along a seeded direction d (fourth-order central stencil of the
element-wise oracle).  Checksums of the generated inputs let a consumer
detect inputs that differ from these (another numpy random stream).

Usage: python tests/golden/make_elements.py c5 [n_random_per_block]
       python tests/golden/make_elements.py c5 --vjp-only   (recompute the derivative only)
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


def _allowed(s, blk, idx):
    """Excitations whose orbital Z2 labels add up to even (the others vanish
    by the symmetry of the synthetic Hamiltonian); same-spin diagonals
    excluded."""
    oa, ob, va, vb = frame_orbitals(s.n_c, s.n_v, REF)
    par = s.parity
    if blk < 2:
        occ, vir = (oa, ob)[blk], (va, vb)[blk]
        i, a = idx
        return not (par[occ[i]] ^ par[vir[a]])
    b3 = blk - 2
    i, j, a, b = idx
    if b3 < 2 and (i == j or a == b):
        return False
    o1, o2 = ((oa, oa), (ob, ob), (oa, ob))[b3]
    v1, v2 = ((va, va), (vb, vb), (va, vb))[b3]
    return not (par[o1[i]] ^ par[o2[j]] ^ par[v1[a]] ^ par[v2[b]])


def positions(s, n_random, rng, edge=7):
    """Per block: n_random random positions (singles: 2 n_random); for the
    doubles also 8 targeted ones: a in the first or last `edge` virtual
    rows, b < a or b > a, and (same-spin blocks) i < j or i > j."""
    o, v = s.n_c + 1, s.n_v + 1
    out = []

    def draw(blk, make):
        while True:
            idx = make()
            if _allowed(s, blk, idx):
                return idx
    for blk in range(5):
        if blk < 2:
            for _ in range(2 * n_random):
                idx = draw(blk, lambda: (int(rng.integers(o)), int(rng.integers(v))))
                out.append((blk, idx, "random"))
            continue
        for _ in range(n_random):
            idx = draw(blk, lambda: tuple(int(x) for x in (rng.integers(o), rng.integers(o),
                                                            rng.integers(v), rng.integers(v))))
            out.append((blk, idx, "random"))
        for region in ("first", "last"):
            for side in ("b<a", "b>a"):
                for rows in ("i<j", "i>j"):
                    def make():
                        a = int(rng.integers(1, edge)) if region == "first" else int(rng.integers(v - edge, v - 1))
                        b = int(rng.integers(0, a)) if side == "b<a" else int(rng.integers(a + 1, v))
                        i, j = sorted(int(x) for x in rng.choice(o, 2, replace=False))
                        if rows == "i>j":
                            i, j = j, i
                        return (i, j, a, b)
                    out.append((blk, draw(blk, make), f"{region} {side} {rows}"))
    return out


def vjp_entry(s, T, q_index):
    """Derivative of the R2ab element q along the seeded direction d (the
    C-condition fixes the A->B element, so d's component there does not
    enter)."""
    d = direction(T)

    def r(e):
        Te = tuple(t + e * x for t, x in zip(T, d))
        return element.residual_element(element.ElementOracle(s, REF, METHOD, Te), 4, tuple(q_index))
    deriv = (8.0 * (r(H) - r(-H)) - (r(2 * H) - r(-2 * H))) / (12.0 * H)
    return {"block": 4, "index": list(q_index), "direction_seed": DIR_SEED, "h": H, "value": deriv}, d


def vjp_only(name):
    """Recompute only the stored reverse-mode derivative of an existing file."""
    path = os.path.join(HERE, f"{name}_elements.json")
    res = json.load(open(path))
    s = make_system(name)
    T = random_amplitudes(s, seed=SEED, ref=REF, scale1=SCALE, scale2=SCALE)
    res["vjp"], d = vjp_entry(s, T, res["vjp"]["index"])
    res["checksums"] = checksums(s, T, d)
    print("vjp directional derivative", res["vjp"]["value"], flush=True)
    with open(path, "w") as f:
        json.dump(res, f, indent=1)


def main(name, n):
    t0 = time.time()
    s = make_system(name)
    T = random_amplitudes(s, seed=SEED, ref=REF, scale1=SCALE, scale2=SCALE)
    eo = element.ElementOracle(s, REF, METHOD, T)
    res = {"workload": name, "dims": CONFIGS[name][:3], "amplitudes": {"seed": SEED, "scale": SCALE},
           "ref": REF, "method": "2D-DCSD", "generator": "synth.make_system + synth.random_amplitudes",
           "oracle": "oracle/element.py", "W": eo.W(), "dEA": eo.energy(), "elements": []}
    print(name, "W", res["W"], "dEA", res["dEA"], flush=True)
    for blk, idx, kind in positions(s, n, np.random.default_rng(11)):
        val = element.residual_element(eo, blk, idx)
        rec = {"block": blk, "index": list(idx), "kind": kind, "value": val}
        if blk >= 2:
            rec["ladder"] = eo.ladder(*element.abi_to_so(eo.o, eo.v, blk, idx))
        res["elements"].append(rec)
        print(blk, idx, kind, val, rec.get("ladder"), flush=True)
    # reverse mode: d/de R_q(T + e d) for the first sampled R2ab element
    q = next(e for e in res["elements"] if e["block"] == 4)
    res["vjp"], d = vjp_entry(s, T, q["index"])
    print("vjp directional derivative", res["vjp"]["value"], flush=True)
    res["checksums"] = checksums(s, T, d)
    res["oracle_seconds"] = time.time() - t0
    with open(os.path.join(HERE, f"{name}_elements.json"), "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    if "--vjp-only" in sys.argv:
        vjp_only(sys.argv[1])
    else:
        main(sys.argv[1] if len(sys.argv) > 1 else "c5", int(sys.argv[2]) if len(sys.argv) > 2 else 4)
