"""FCIDUMP input for the oracle (test infrastructure only): an independent
reader of the integral file format the paper's calculations use (Section
III), frozen-core folding, and the Fock matrices of Phi_A from four-index
integrals.  The spin-orbital frames (spinorb.Frame) take the four-index
integrals directly when a system carries them (System.eri), so oracle
residuals of FCIDUMP inputs use no factorisation at all.
"""
from __future__ import annotations

import dataclasses
import re

import numpy as np

from synth import System


def orbsym(path):
    """ORBSYM of the header (irrep labels 1..8), or all 1 when absent."""
    text = open(path).read()
    head = re.search(r"&FCI(.*?)(&END|/)", text, re.S | re.I).group(1).upper()
    n = int(re.search(r"NORB\s*=\s*(\d+)", head).group(1))
    m = re.search(r"ORBSYM\s*=\s*([\d,\s]+)", head)
    if not m:
        return [1] * n
    return [int(x) for x in re.findall(r"\d+", m.group(1))][:n]


def read(path):
    """(norb, nelec, ms2, h [n,n], eri [n,n,n,n] (pq|rs), ecore)."""
    text = open(path).read()
    m = re.search(r"&FCI(.*?)(&END|/)", text, re.S | re.I)
    head = m.group(1).upper()
    key = lambda k, d=None: int(re.search(k + r"\s*=\s*(-?\d+)", head).group(1)) if re.search(k + r"\s*=", head) else d  # noqa: E731,E501
    n, nelec, ms2 = key("NORB"), key("NELEC"), key("MS2", 0)
    h = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    ecore = 0.0
    for line in text[m.end():].splitlines():
        parts = line.replace("D", "E").replace("d", "e").split()
        if len(parts) < 5:
            continue
        v = float(parts[0])
        i, j, k, l = (int(x) for x in parts[1:5])
        if i and j and k and l:
            i, j, k, l = i - 1, j - 1, k - 1, l - 1
            for p, q, r, s in ((i, j, k, l), (j, i, k, l), (i, j, l, k), (j, i, l, k),
                               (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)):
                eri[p, q, r, s] = v
        elif i and j:
            h[i - 1, j - 1] = h[j - 1, i - 1] = v
        elif not (i or j or k or l):
            ecore = v
    return n, nelec, ms2, h, eri, ecore


def fock(h, eri, occ_a, occ_b):
    """f^sigma_pq = h_pq + sum_{k in occ} (pq|kk) - sum_{k in occ_sigma} (pk|kq)."""
    J = sum(eri[:, :, k, k] for k in list(occ_a) + list(occ_b))
    Ka = sum((eri[:, k, k, :] for k in occ_a), np.zeros_like(h))
    Kb = sum((eri[:, k, k, :] for k in occ_b), np.zeros_like(h))
    return h + J - Ka, h + J - Kb


def system(path, n_frozen=0):
    """System of the correlated orbitals of an FCIDUMP file (frozen core
    folded into h and the core energy) and the total reference energy
    <Phi_A|H|Phi_A>.  Phi_A doubly occupies the first (NELEC-2)/2 orbitals,
    then t alpha and u beta."""
    n, nelec, ms2, h, eri, ecore = read(path)
    nd = (nelec - 2) // 2
    f = list(range(n_frozen))
    hf = h + sum((2.0 * eri[:, :, k, k] - eri[:, k, k, :] for k in f), np.zeros_like(h))
    ec = ecore + sum(2.0 * h[k, k] for k in f) + sum(2.0 * eri[k, k, l, l] - eri[k, l, l, k] for k in f for l in f)
    c = slice(n_frozen, n)
    hc, ec4 = hf[c, c], eri[c, c, c, c]
    nc = nd - n_frozen
    occ_a, occ_b = list(range(nc)) + [nc], list(range(nc)) + [nc + 1]
    fa, fb = fock(hc, ec4, occ_a, occ_b)
    eref = ec + sum(hc[k, k] for k in occ_a + occ_b)
    for sa, A in ((0, occ_a), (1, occ_b)):
        for sb, Bo in ((0, occ_a), (1, occ_b)):
            for k in A:
                for l in Bo:
                    eref += 0.5 * (ec4[k, k, l, l] - (ec4[k, l, l, k] if sa == sb else 0.0))
    nv = n - n_frozen - nc - 2
    # irrep labels as XOR-able bits (the product of irreps i and j of the
    # D2h subgroups in this numbering is ((i-1) xor (j-1)) + 1)
    par = (np.array(orbsym(path)) - 1).astype(np.int8)[n_frozen:]
    s = System(nc, nv, 0, np.diag(fa).copy(), par, np.zeros(0, dtype=np.int8),
               np.zeros((0, n - n_frozen, n - n_frozen)), fa, fb, hc)
    s = dataclasses.replace(s, eri=ec4)
    return s, eref
