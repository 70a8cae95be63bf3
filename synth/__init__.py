"""Seeded synthetic inputs for the two-determinant CC residual (shared by the
oracle tests, the GPU tests and the benchmark).

This module draws random numbers and lays them out; it contains none of the
method's arithmetic (no Fock build, no integral transformation, no residual
terms).  Everything here is a deterministic function of (sizes, seed).

Orbital order (spatial, used by every array):  core 0..n_c-1, t = n_c,
u = n_c+1, external virtuals V = n_c+2..n-1.  Phi_A occupies core(alpha,beta),
t(alpha), u(beta); Phi_B is its spin flip (core, u(alpha), t(beta)) -- the two
determinants of the paper's Fig. 1 (Section II).

Recipe (stand-in for the paper's molecules, which are not available):
  * orbital energies: core ~ U[-1.5,-0.3] (sorted), eps_t, eps_u fixed
    (-0.2/-0.1, or -0.15/-0.14 for the near-degenerate diradical-like case),
    external virtuals ~ U[0.2,3.0] (sorted);
  * a Z2 "symmetry" label per orbital (t even, u odd, others random) and per
    auxiliary function, so t and u lie in different irreps (the CAS case of
    Section II) and active-active singles vanish exactly; with ias=True t
    and u are both even (the IAS case: the internal singles do not vanish);
  * DF factors B[L,p,q] ~ N(0, sigma^2), drawn for p<=q and mirrored, zeroed
    unless parity(p) xor parity(q) == parity(L).  sigma = 0.05 for the
    smallest workload (naux = 60, 21 virtuals per spin) and
    sigma = 0.05 * (60 * 21^2 / (naux * v^2))^(1/4) when that is smaller, so
    that a pair's second-order correlation, sum_ab (ia|jb)^2 / D ~
    v^2 * naux * sigma^4, keeps the size it has there.  With a fixed sigma the
    exchange integrals (pq|pq) = sum_L B_pq^2 grow like naux (1.9 Eh at
    naux = 1500) and the pair correlation like v^2 naux: the amplitude
    equations then diverge even in FP64;
  * Fock matrices f^alpha, f^beta = diag(eps) + symmetric off-diagonal noise
    N(0, 0.005^2), independent per spin, zeroed where parities differ.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# (n_c, n_v, naux, eps_t, eps_u) of the five workloads
CONFIGS = {
    "c1": (4, 20, 60, -0.2, -0.1),
    "c2": (10, 120, 360, -0.2, -0.1),
    "c3": (20, 300, 900, -0.2, -0.1),
    "c4": (12, 160, 480, -0.2, -0.1),
    "c5": (30, 500, 1500, -0.15, -0.14),
}
CONFIG_SEED = {"c1": 1, "c2": 2, "c3": 3, "c4": 4, "c5": 5}


@dataclasses.dataclass
class System:
    n_c: int
    n_v: int
    naux: int
    eps: np.ndarray        # [n]
    parity: np.ndarray     # [n] int8 Z2 label per orbital
    parity_aux: np.ndarray  # [naux]
    B: np.ndarray          # [naux, n, n] symmetric in (p,q)
    fock_a: np.ndarray     # [n, n] Fock matrix of alpha spin w.r.t. Phi_A
    fock_b: np.ndarray     # [n, n] Fock matrix of beta spin w.r.t. Phi_A
    h: np.ndarray | None = None  # [n, n] core Hamiltonian (pin systems only)
    eri: np.ndarray | None = None  # [n, n, n, n] four-index (pq|rs), when given instead of factors

    @property
    def n(self):
        return self.n_c + 2 + self.n_v

    @property
    def o(self):
        return self.n_c + 1

    @property
    def v(self):
        return self.n_v + 1


def _parities(rng, n_c, n_v, naux, ias=False):
    par = np.empty(n_c + 2 + n_v, dtype=np.int8)
    par[:n_c] = rng.integers(0, 2, n_c)
    par[n_c] = 0
    par[n_c + 1] = 0 if ias else 1
    par[n_c + 2:] = rng.integers(0, 2, n_v)
    par_aux = rng.integers(0, 2, naux).astype(np.int8)
    return par, par_aux


def _sym_noise(rng, n, sigma, mask):
    x = rng.normal(0.0, sigma, (n, n))
    x = np.triu(x, 1)
    x = x + x.T
    return x * mask


def make_B(rng, n, naux, par, par_aux, sigma=0.05):
    """DF factors, symmetric in (p,q), Z2-masked."""
    B = np.empty((naux, n, n))
    pq = (par[:, None] ^ par[None, :]).astype(np.int8)
    iu = np.triu_indices(n)
    for L in range(naux):
        x = np.zeros((n, n))
        x[iu] = rng.normal(0.0, sigma, iu[0].size)
        x = x + np.triu(x, 1).T
        B[L] = x * (pq == par_aux[L])
    return B


def b_sigma_for(naux, v):
    """DF factor spread: 0.05 * min(1, (60 * 21^2 / (naux * v^2))^(1/4))."""
    return 0.05 * min(1.0, (60.0 * 21.0 ** 2 / (naux * float(v) ** 2)) ** 0.25)


def make_system(name_or_dims, seed=None, eps_t=None, eps_u=None,
                fock_noise=0.005, b_sigma=None, ias=False) -> System:
    """Synthetic DF Hamiltonian for a named workload ('c1'..'c5') or for
    explicit (n_c, n_v, naux).  ias=True gives t and u the same Z2 label
    (the incomplete-active-space case of Section II: the internal singles
    t -> u no longer vanish by symmetry)."""
    if isinstance(name_or_dims, str):
        n_c, n_v, naux, et, eu = CONFIGS[name_or_dims]
        if seed is None:
            seed = CONFIG_SEED[name_or_dims]
    else:
        n_c, n_v, naux = name_or_dims
        et, eu = -0.2, -0.1
    if eps_t is not None:
        et = eps_t
    if eps_u is not None:
        eu = eps_u
    rng = np.random.Generator(np.random.PCG64(seed if seed is not None else 0))
    n = n_c + 2 + n_v
    par, par_aux = _parities(rng, n_c, n_v, naux, ias)
    eps = np.empty(n)
    eps[:n_c] = np.sort(rng.uniform(-1.5, -0.3, n_c))
    eps[n_c] = et
    eps[n_c + 1] = eu
    eps[n_c + 2:] = np.sort(rng.uniform(0.2, 3.0, n_v))
    mask = (par[:, None] == par[None, :]).astype(float)
    fa = np.diag(eps) + _sym_noise(rng, n, fock_noise, mask)
    fb = np.diag(eps) + _sym_noise(rng, n, fock_noise, mask)
    B = make_B(rng, n, naux, par, par_aux, b_sigma if b_sigma is not None else b_sigma_for(naux, n_v + 1))
    return System(n_c, n_v, naux, eps, par, par_aux, B, fa, fb)


def make_pin_system(n_c, n_v, naux, seed, eps_t=-0.2, eps_u=-0.1,
                    h_noise=0.02, b_sigma=0.15, z2=True, ias=False) -> System:
    """Small system defined by a spin-free core Hamiltonian h and DF factors
    B (for brute-force / FCI pins).  fock_a/fock_b are left as None-like
    zeros: the Fock matrices are built from h by the code under test."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_c + 2 + n_v
    if z2:
        par, par_aux = _parities(rng, n_c, n_v, naux, ias)
    else:
        par = np.zeros(n, dtype=np.int8)
        par_aux = np.zeros(naux, dtype=np.int8)
    eps = np.empty(n)
    eps[:n_c] = np.sort(rng.uniform(-1.5, -0.3, n_c))
    eps[n_c] = eps_t
    eps[n_c + 1] = eps_u
    eps[n_c + 2:] = np.sort(rng.uniform(0.2, 3.0, n_v))
    mask = (par[:, None] == par[None, :]).astype(float)
    h = np.diag(eps) + _sym_noise(rng, n, h_noise, mask)
    B = make_B(rng, n, naux, par, par_aux, b_sigma)
    z = np.zeros((n, n))
    return System(n_c, n_v, naux, eps, par, par_aux, B, z, z.copy(), h)


# ----------------------------------------------------------------------------
# amplitude layout (the C ABI layout) and random amplitudes
# ----------------------------------------------------------------------------

def frame_orbitals(n_c, n_v, ref):
    """Spatial orbital lists (occ_alpha, occ_beta, vir_alpha, vir_beta) of the
    determinant the amplitudes are normal-ordered to (ref 0 = Phi_A,
    1 = Phi_B).  This is the index convention of the C ABI."""
    core = list(range(n_c))
    t, u = n_c, n_c + 1
    V = list(range(n_c + 2, n_c + 2 + n_v))
    if ref == 0:
        return core + [t], core + [u], [u] + V, [t] + V
    return core + [u], core + [t], [t] + V, [u] + V


def random_amplitudes(sys: System, seed, ref=0, scale1=0.02, scale2=0.02,
                      z2=True):
    """Random T1/T2 in the ABI layout: T1a,T1b [o][v]; T2aa,T2bb [o][o][v][v]
    antisymmetric; T2ab [o][o][v][v] (alpha-occ, beta-occ, alpha-vir,
    beta-vir).  The A->B doubles element T2ab[o-1][o-1][0][0] is zero.  With
    z2=True amplitudes whose orbitals do not conserve the Z2 label are zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    o, v = sys.o, sys.v
    oa, ob, va, vb = (np.array(x) for x in frame_orbitals(sys.n_c, sys.n_v, ref))
    p = sys.parity.astype(int)
    T1a = rng.normal(0, scale1, (o, v))
    T1b = rng.normal(0, scale1, (o, v))
    T2aa = rng.normal(0, scale2, (o, o, v, v))
    T2bb = rng.normal(0, scale2, (o, o, v, v))
    T2ab = rng.normal(0, scale2, (o, o, v, v))
    T2aa = T2aa - T2aa.transpose(1, 0, 2, 3)
    T2aa = T2aa - T2aa.transpose(0, 1, 3, 2)
    T2bb = T2bb - T2bb.transpose(1, 0, 2, 3)
    T2bb = T2bb - T2bb.transpose(0, 1, 3, 2)
    if z2:
        T1a *= (p[oa][:, None] == p[va][None, :])
        T1b *= (p[ob][:, None] == p[vb][None, :])

        def m2(oi, oj, va_, vb_):
            s = (p[oi][:, None, None, None] ^ p[oj][None, :, None, None]
                 ^ p[va_][None, None, :, None] ^ p[vb_][None, None, None, :])
            return s == 0
        T2aa *= m2(oa, oa, va, va)
        T2bb *= m2(ob, ob, vb, vb)
        T2ab *= m2(oa, ob, va, vb)
    T2ab[o - 1, o - 1, 0, 0] = 0.0
    return T1a, T1b, T2aa, T2bb, T2ab
