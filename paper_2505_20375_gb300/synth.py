"""Seeded synthetic inputs shared by the CUDA path's callers and by the oracle's tests.

This module draws random numbers and assembles integral tensors from them. It holds
none of the configuration-interaction arithmetic (no strings, no excitation lists, no
Hamiltonian matrix elements, no sigma build), so both sides can take their inputs from
it without sharing any of the method.

Random numbers come from a counter-based generator: ``u64 = splitmix64(key + i)`` for a
64-bit ``key`` derived from (seed, stream tag) and a running counter ``i``.  splitmix64
is Steele, Lea and Flood's mixing function (2014, "Fast splittable pseudorandom number
generators"); the constants below are the published ones.  Uniforms take the top 53
bits; normals use the Box-Muller transform.  Everything is vectorised numpy on uint64,
so the same seed gives the same bits on x86 and Arm.

The workloads imitate the active spaces of the paper's benchmarks (the Hamiltonian
operator of the "Methods" section; real spin-free integrals and complex Hermitian
two-spinor-like integrals, since molecular X2C integrals are not available here).
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to uint64 counters (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (x + _GOLDEN) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


class Stream:
    """A counter-based stream of uniforms/normals keyed by (seed, tag)."""

    def __init__(self, seed: int, tag: int = 0):
        k = _splitmix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64))
        k = _splitmix64(k ^ np.uint64(tag & 0xFFFFFFFFFFFFFFFF))
        self.key = k[0]
        self.counter = 0

    def bits(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter, self.counter + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _splitmix64((idx * _GOLDEN + self.key) & _M64)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1)."""
        return (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller (cosine branch only)."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def _sym_from_upper(n: int, vals_upper: np.ndarray, diag: np.ndarray) -> np.ndarray:
    m = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    m[iu] = vals_upper
    m = m + m.T
    m[np.diag_indices(n)] = diag
    return m


def real_integrals(n: int, n_chol: int, seed: int):
    """Real spin-free integrals for n spatial orbitals.

    h_pp: sorted uniform in [-2, 1]; h_pq (p<q): N(0, 0.05), mirrored.
    (pq|rs) = sum_P L^P_pq L^P_rs with L^P symmetric, entries (p<=q) N(0, 0.1).
    Returns (h[n,n], g[n,n,n,n]) in chemists' notation, row-major float64.
    Draw order: h diagonal, h upper triangle (row-major), then L^0, L^1, ... each as
    its diagonal followed by its upper triangle.
    """
    st = Stream(seed, tag=0x5EA1)
    diag = np.sort(st.uniform(n) * 3.0 - 2.0)
    off = st.normal(n * (n - 1) // 2) * 0.05
    h = _sym_from_upper(n, off, diag)
    L = np.empty((n_chol, n, n))
    for P in range(n_chol):
        d = st.normal(n) * 0.1
        u = st.normal(n * (n - 1) // 2) * 0.1
        L[P] = _sym_from_upper(n, u, d)
    g = np.einsum("Ppq,Prs->pqrs", L, L)
    return np.ascontiguousarray(h), np.ascontiguousarray(g)


def complex_integrals(n: int, n_chol: int, seed: int):
    """Complex Hermitian integrals for n spinors.

    h Hermitian: real diagonal sorted uniform in [-2, 1]; off-diagonal real and
    imaginary parts each N(0, 0.05/sqrt2).
    (pq|rs) = sum_P L^P_pq conj(L^P_sr) with L^P Hermitian (real diagonal N(0, 0.1),
    off-diagonal parts N(0, 0.1/sqrt2)), so (pq|rs) = (rs|pq) and conj((pq|rs)) = (qp|sr).
    Returns (h[n,n], g[n,n,n,n]) complex128, chemists' notation.
    """
    st = Stream(seed, tag=0xC0C0)
    diag = np.sort(st.uniform(n) * 3.0 - 2.0)
    m = n * (n - 1) // 2
    re = st.normal(m) * (0.05 / np.sqrt(2.0))
    im = st.normal(m) * (0.05 / np.sqrt(2.0))
    h = np.zeros((n, n), dtype=np.complex128)
    iu = np.triu_indices(n, 1)
    h[iu] = re + 1j * im
    h = h + h.conj().T
    h[np.diag_indices(n)] = diag
    L = np.zeros((n_chol, n, n), dtype=np.complex128)
    for P in range(n_chol):
        d = st.normal(n) * 0.1
        r = st.normal(m) * (0.1 / np.sqrt(2.0))
        i = st.normal(m) * (0.1 / np.sqrt(2.0))
        lp = np.zeros((n, n), dtype=np.complex128)
        lp[iu] = r + 1j * i
        lp = lp + lp.conj().T
        lp[np.diag_indices(n)] = d
        L[P] = lp
    # conj(L_sr) = L_rs for Hermitian L
    g = np.einsum("Ppq,Prs->pqrs", L, L)
    return np.ascontiguousarray(h), np.ascontiguousarray(g)


def random_vector(n: int, seed: int, complex_: bool = False, normalise: bool = True) -> np.ndarray:
    """N(0,1) entries (real, or real+imag parts each N(0, 1/sqrt2)), optionally unit norm."""
    st = Stream(seed, tag=0x7EC7)
    if complex_:
        v = (st.normal(n) + 1j * st.normal(n)) / np.sqrt(2.0)
    else:
        v = st.normal(n)
    if normalise:
        v = v / np.linalg.norm(v)
    return v


def hubbard_dimer(t: float, U: float):
    """Two-site Hubbard model as (h, g): h = [[0,-t],[-t,0]], (pp|pp) = U, all other g = 0."""
    h = np.array([[0.0, -t], [-t, 0.0]])
    g = np.zeros((2, 2, 2, 2))
    g[0, 0, 0, 0] = U
    g[1, 1, 1, 1] = U
    return h, g


# Workload shapes (orbitals, electrons per spin, Cholesky rank, seed) used by the tests
# and the benchmark.  Sizes follow the active spaces of the paper's workloads.
WORKLOADS = {
    "fci_8e8o": dict(n=8, na=4, nb=4, n_chol=16, seed=1),
    "fci_14e14o": dict(n=14, na=7, nb=7, n_chol=28, seed=2),
    "fci_12e12o": dict(n=12, na=6, nb=6, n_chol=24, seed=2),
    "das_24o_4x6": dict(n=24, spaces=[6, 6, 6, 6], ref=[3, 3, 3, 3], max_transfer=2, n_chol=48, seed=3),
    "das_16o_4x4": dict(n=16, spaces=[4, 4, 4, 4], ref=[2, 2, 2, 2], max_transfer=2, n_chol=48, seed=3),
    "das_16o_4x4_8e": dict(n=16, spaces=[4, 4, 4, 4], ref=[1, 1, 1, 1], max_transfer=1, n_chol=48, seed=5),
    "spinor_24s12e": dict(n=24, ne=12, n_chol=48, seed=4),
    # a smaller spinor problem of the same shape family (profiling captures)
    "spinor_20s10e": dict(n=20, ne=10, n_chol=40, seed=4),
}
