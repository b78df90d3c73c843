"""Oracle: a plain, slow, obviously correct CPU configuration-interaction code.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this package.
The product path (``paper_2505_20375_gb300``) never imports it, and it never imports the
product path: the two share no code.  Inputs reach both from
``paper_2505_20375_gb300.synth`` (random numbers and integral assembly only).

What it computes, and where the paper defines it:
  * sigma = H C for H = sum h_pq E_pq + 1/2 sum (pq|rs)(E_pq E_rs - delta_qr E_ps)
    ("Methods", Eqs. sigmaL, sigmaL1e, sigmaL2e; the operator being the one whose
    one-electron excitation lists the Introduction sizes at n_e (n_h + 1) N),
    determinant by determinant with Slater-Condon rules (fci_oracle.c);
  * the single-replacement list of every string (Introduction, excitation-list size);
  * dense H for tiny spaces, diagonalised by LAPACK (numpy.linalg.eigh);
  * the Davidson iteration and its preconditioners ("Results", Eq. davidsonPreconditioner
    and Eq. sparsePreconditioner) in ``oracle.davidson``;
  * STP-DAS categories (occupation patterns per distributed active space) in
    ``oracle.das``;
  * Algorithm 1's sigma on a categorically compressed vector (per-category nonzero values
    and local addresses, exponential search, a table keyed by target address), and the
    Davidson iteration on compressed vectors (H_ii on the fly, Eq. sparsePreconditioner) in
    ``oracle.alg1``.

Every function here is pinned by the ``-m "not gpu"`` tests in tests/test_oracle_*.py
against closed forms, brute force and invariants that the paper states.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        L.orc_enumerate_strings.argtypes = [i32, i32, vp]
        L.orc_enumerate_strings.restype = i64
        L.orc_replacement_table.argtypes = [i32, i32, vp, i64, vp, vp, vp, vp]
        L.orc_replacement_table.restype = i32
        L.orc_diag.argtypes = [i32, vp, vp, i64, vp, vp]
        L.orc_hij.argtypes = [i32, vp, vp, ctypes.c_uint64, ctypes.c_uint64, vp]
        L.orc_dense_h.argtypes = [i32, vp, vp, i64, vp, vp]
        L.orc_sigma.argtypes = [i32, vp, vp, dbl, i64, vp, vp, vp, i64, vp]
        L.orc_sigma.restype = i32
        L.orc_table_new.argtypes = [i64, vp]
        L.orc_table_new.restype = vp
        L.orc_table_free.argtypes = [vp]
        L.orc_table_free.restype = None
        L.orc_sigma_table.argtypes = [vp, i32, vp, vp, dbl, i64, vp, vp, vp, i64, vp]
        L.orc_sigma_table.restype = i32
        L.orc_num_threads.restype = i32
        _LIB = L
    return _LIB


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ------------------------------------------------------------------ strings

def enumerate_strings(m: int, ne: int) -> np.ndarray:
    """All m-orbital occupation strings with ne electrons, ascending as integers."""
    n = lib().orc_enumerate_strings(m, ne, None)
    if n < 0:
        raise ValueError("bad string shape")
    out = np.empty(n, dtype=np.uint64)
    lib().orc_enumerate_strings(m, ne, _ptr(out))
    return out


def replacement_table(m: int, ne: int):
    """Single-replacement list of every string: arrays (n_str, n_ent) of target index,
    created orbital a, annihilated orbital b and sign <S|a+_a a_b|T>."""
    s = enumerate_strings(m, ne)
    n_ent = ne * (m - ne + 1)
    shp = (len(s), n_ent)
    tgt = np.empty(shp, np.int32)
    a = np.empty(shp, np.int32)
    b = np.empty(shp, np.int32)
    sg = np.empty(shp, np.int8)
    rc = lib().orc_replacement_table(m, ne, _ptr(s), len(s), _ptr(tgt), _ptr(a), _ptr(b), _ptr(sg))
    if rc != n_ent:
        raise RuntimeError("replacement table failed")
    return dict(strings=s, target=tgt, a=a, b=b, sign=sg)


# --------------------------------------------------------------- integrals

def spin_orbital_integrals(h: np.ndarray, g: np.ndarray):
    """Spatial spin-free (h, (pq|rs)) -> spin-orbital (complex) arrays.
    Spin orbital P = p (alpha) or p + n (beta): all alpha spin orbitals precede beta."""
    n = h.shape[0]
    hso = np.zeros((2 * n, 2 * n), np.complex128)
    gso = np.zeros((2 * n,) * 4, np.complex128)
    for s in (0, 1):
        hso[s * n:(s + 1) * n, s * n:(s + 1) * n] = h
        for t in (0, 1):
            gso[s * n:(s + 1) * n, s * n:(s + 1) * n, t * n:(t + 1) * n, t * n:(t + 1) * n] = g
    return hso, gso


def spinor_integrals(h: np.ndarray, g: np.ndarray):
    return np.ascontiguousarray(h, np.complex128), np.ascontiguousarray(g, np.complex128)


# ------------------------------------------------------------ determinants

def fci_dets(n: int, na: int, nb: int) -> np.ndarray:
    """Spin-orbital masks of FCI(na alpha, nb beta in n orbitals), in the address order
    I = I_alpha * N_beta + I_beta (both string lists ascending)."""
    sa = enumerate_strings(n, na)
    sb = enumerate_strings(n, nb)
    return (sa[:, None] | (sb[None, :] << np.uint64(n))).reshape(-1)


def spinor_dets(n: int, ne: int) -> np.ndarray:
    return enumerate_strings(n, ne)


# ------------------------------------------------------------- hamiltonian

def _cplx(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def sigma(hso, gso, dets, C, e_core: float = 0.0, rows=None):
    """sigma = (H + e_core) C over the determinant list (rows: optional subset)."""
    nso = hso.shape[0]
    h, g, c = _cplx(hso), _cplx(gso), _cplx(C)
    dets = np.ascontiguousarray(dets, np.uint64)
    if rows is None:
        nrows, rp = len(dets), None
    else:
        rows = np.ascontiguousarray(rows, np.int64)
        nrows, rp = len(rows), _ptr(rows)
    out = np.empty(nrows, np.complex128)
    rc = lib().orc_sigma(nso, _ptr(h), _ptr(g), float(e_core), len(dets), _ptr(dets), _ptr(c),
                         rp, nrows, _ptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_sigma failed ({rc})")
    real_in = (not np.iscomplexobj(C)) and np.all(np.imag(hso) == 0) and np.all(np.imag(gso) == 0)
    return out.real.copy() if real_in else out


class SigmaTable:
    """The determinant lookup table of one list, built once and reused by many sigma
    calls over that list (the arithmetic is ``sigma``'s)."""

    def __init__(self, dets):
        self.dets = np.ascontiguousarray(dets, np.uint64)
        self._t = lib().orc_table_new(len(self.dets), _ptr(self.dets))
        if not self._t:
            raise RuntimeError("orc_table_new failed (allocation or duplicate determinants)")

    def close(self):
        if getattr(self, "_t", None):
            lib().orc_table_free(self._t)
            self._t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sigma(self, hso, gso, C, e_core: float = 0.0, rows=None):
        nso = hso.shape[0]
        h, g, c = _cplx(hso), _cplx(gso), _cplx(C)
        if rows is None:
            nrows, rp = len(self.dets), None
        else:
            rows = np.ascontiguousarray(rows, np.int64)
            nrows, rp = len(rows), _ptr(rows)
        out = np.empty(nrows, np.complex128)
        rc = lib().orc_sigma_table(self._t, nso, _ptr(h), _ptr(g), float(e_core), len(self.dets), _ptr(self.dets),
                                   _ptr(c), rp, nrows, _ptr(out))
        if rc != 0:
            raise RuntimeError(f"orc_sigma_table failed ({rc})")
        real_in = (not np.iscomplexobj(C)) and np.all(np.imag(hso) == 0) and np.all(np.imag(gso) == 0)
        return out.real.copy() if real_in else out


def diag(hso, gso, dets):
    h, g = _cplx(hso), _cplx(gso)
    dets = np.ascontiguousarray(dets, np.uint64)
    out = np.empty(len(dets), np.complex128)
    lib().orc_diag(hso.shape[0], _ptr(h), _ptr(g), len(dets), _ptr(dets), _ptr(out))
    return out.real.copy()


def hij(hso, gso, I: int, J: int) -> complex:
    h, g = _cplx(hso), _cplx(gso)
    out = np.empty(1, np.complex128)
    lib().orc_hij(hso.shape[0], _ptr(h), _ptr(g), int(I), int(J), _ptr(out))
    return complex(out[0])


def dense_h(hso, gso, dets):
    h, g = _cplx(hso), _cplx(gso)
    dets = np.ascontiguousarray(dets, np.uint64)
    out = np.empty((len(dets), len(dets)), np.complex128)
    lib().orc_dense_h(hso.shape[0], _ptr(h), _ptr(g), len(dets), _ptr(dets), _ptr(out))
    return out


def eigh_lowest(H: np.ndarray, k: int = 1):
    """Lowest k eigenpairs of a dense Hermitian matrix (LAPACK via numpy)."""
    if np.all(H.imag == 0):
        H = H.real
    w, v = np.linalg.eigh(H)
    return w[:k], v[:, :k]
