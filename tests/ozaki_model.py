"""Exact-integer numpy model of the split-precision (Ozaki) sigma, for tests only.

It states the scheme from its definition (Ozaki, Ogita, Oishi and Rump, "Error-free
transformations of matrix multiplication by using fast routines of matrix
multiplication", 2012: split both operands into slices whose products are exact, then
sum the slice products) in the fixed-point, signed base-256 form the CUDA kernel
documents, and evaluates every product in exact int64 arithmetic.  The CUDA kernel
forms the same slice products on tensor cores with FP32 accumulation; if that
accumulation were not exact, the two would differ by about 2^-24 of a level sum.
The replacement lists come from the oracle.
"""
from __future__ import annotations

import numpy as np

import oracle


def packed_contraction_matrix(h, g, n_el):
    """1/2 g' over unordered pairs, g' = (pq|rs) + (h'_pq d_rs + d_pq h'_rs)/N_e."""
    n = h.shape[0]
    hp = h - 0.5 * np.einsum("prrq->pq", g)
    pairs = [(p, q) for p in range(n) for q in range(p + 1)]
    idx = {pq: i for i, pq in enumerate(pairs)}
    np_ = len(pairs)
    G = np.zeros((np_, np_))
    for (p, q), i in idx.items():
        for (r, s), j in idx.items():
            v = g[p, q, r, s]
            if r == s:
                v += hp[p, q] / n_el
            if p == q:
                v += hp[r, s] / n_el
            G[i, j] = 0.5 * v
    return G, idx


def balanced_digits(X: np.ndarray, s: int):
    bias = 0
    for j in range(s):
        bias |= 0x80 << (8 * j)
    Y = X.astype(np.int64).astype(np.uint64) + np.uint64(bias)
    return [((Y >> np.uint64(8 * j)) & np.uint64(0xFF)).astype(np.int64) - 128 for j in range(s)]


def sigma_model(h, g, n, na, nb, C, s, e_core=0.0, e_fp32=False):
    """Split sigma of the FCI vector C.  e_fp32: store every E_int rounded to FP32 (round
    to nearest even, as the DAS kernel does) and sum the stored integers."""
    G, idx = packed_contraction_matrix(h, g, na + nb)
    np_ = G.shape[0]
    gmax = np.max(np.abs(G))
    eG = np.frexp(gmax)[1] if gmax > 0 else 0
    shG = 8 * s - 2 - int(eG)
    Gint = np.rint(np.ldexp(G, shG)).astype(np.int64)
    cmax = np.max(np.abs(C))
    eC = int(np.frexp(cmax)[1]) if cmax > 0 else 0
    shC = 8 * s - 3 - eC
    Cint = np.rint(np.ldexp(C, shC)).astype(np.int64)
    ta = oracle.replacement_table(n, na) if na > 0 else None
    tb = oracle.replacement_table(n, nb) if nb > 0 else None
    from math import comb

    nsa, nsb = comb(n, na), comb(n, nb)
    Cm = Cint.reshape(nsa, nsb)
    D = np.zeros((np_, nsa, nsb), np.int64)
    for t, spin in ((ta, 0), (tb, 1)):
        if t is None:
            continue
        for S in range(t["target"].shape[0]):
            for e in range(t["target"].shape[1]):
                T, a, b, sg = t["target"][S, e], t["a"][S, e], t["b"][S, e], int(t["sign"][S, e])
                pp = idx[(max(a, b), min(a, b))]
                if spin == 0:
                    D[pp, S, :] += sg * Cm[T, :]
                else:
                    D[pp, :, S] += sg * Cm[:, T]
    D = D.reshape(np_, -1)
    gd = balanced_digits(Gint, s)
    dd = balanced_digits(D, s)
    L0 = max(s - 1, 2 * s - 6)
    lo = np.zeros_like(D)
    hi = np.zeros_like(D)
    for L in range(s - 1, 2 * s - 1):
        SL = np.zeros_like(D)
        for i in range(s):
            j = L - i
            if 0 <= j < s:
                SL += gd[i] @ dd[j]
        assert np.max(np.abs(SL)) < 2 ** 24
        if L < L0:
            lo += SL << (8 * (L - (s - 1)))
        else:
            hi += SL << (8 * (L - L0))
    k = 8 * (L0 - (s - 1))
    E = hi + (((lo + (1 << (k - 1))) >> k) if k > 0 else 0)
    if e_fp32:
        assert np.max(np.abs(E)) < 2 ** 53
        E = E.astype(np.float32).astype(np.int64)
    # scatter: sigma_I = sum <I|E_pq|K> E[pq, K] (exact integers), then one conversion
    Em = E.reshape(np_, nsa, nsb)
    acc = np.zeros((nsa, nsb), np.int64)
    for t, spin in ((ta, 0), (tb, 1)):
        if t is None:
            continue
        for S in range(t["target"].shape[0]):
            for e in range(t["target"].shape[1]):
                T, a, b, sg = t["target"][S, e], t["a"][S, e], t["b"][S, e], int(t["sign"][S, e])
                pp = idx[(max(a, b), min(a, b))]
                if spin == 0:
                    acc[S, :] += sg * Em[pp, T, :]
                else:
                    acc[:, S] += sg * Em[pp, :, T]
    u = 8 * L0 - shG - shC
    return np.ldexp(acc.reshape(-1).astype(np.float64), u) + e_core * C


def das_sigma_model(h, g, spaces, ref, nel, max_transfer, C, s, e_core=0.0):
    """Split sigma on the DAS layout: the fused form (s <= 3) stores E rounded to FP32,
    the two-pass form (s >= 4) keeps E_int exact in int64.  The DAS sigma is the FCI sigma
    of the zero-padded vector restricted to the DAS determinants (every determinant one
    replacement away from a target one lies in the intermediate space), so the model
    embeds C, applies sigma_model and restricts."""
    from oracle import das as odas

    n = sum(spaces)
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, max_transfer)
    sa = oracle.enumerate_strings(n, nel)
    pos = {int(x): i for i, x in enumerate(sa)}
    mask = (1 << n) - 1
    addr = np.array([pos[int(d) & mask] * len(sa) + pos[int(d) >> n] for d in dets], dtype=np.int64)
    Cf = np.zeros(len(sa) ** 2)
    Cf[addr] = C
    return sigma_model(h, g, n, nel, nel, Cf, s, e_core=0.0, e_fp32=s <= 3)[addr] + e_core * C


def complex_contraction_matrix(h, g, n_el):
    """1/2 g' over ordered spinor pairs x = p n + q (complex integrals, no packing)."""
    n = h.shape[0]
    hp = h - 0.5 * np.einsum("prrq->pq", g)
    G = 0.5 * g.reshape(n * n, n * n).astype(complex)
    for p in range(n):
        for q in range(n):
            for r in range(n):
                G[p * n + q, r * n + r] += 0.5 * hp[p, q] / n_el
                G[r * n + r, p * n + q] += 0.5 * hp[p, q] / n_el
    return G


def balanced_digits7(X: np.ndarray, s: int):
    bias = 0
    for j in range(s):
        bias |= 64 << (7 * j)
    Y = X.astype(np.int64).astype(np.uint64) + np.uint64(bias)
    return [((Y >> np.uint64(7 * j)) & np.uint64(0x7F)).astype(np.int64) - 64 for j in range(s)]


def spinor_sigma_model(h, g, n, ne, C, s, e_core=0.0):
    """Split sigma for spinor strings with complex integrals: the complex contraction as
    one real product on the real embedding [[G_re, -G_im], [G_im, G_re]] (index 2x real,
    2x + 1 imaginary part of pair x), balanced base-128 digits, top s levels, exact int64."""
    G = complex_contraction_matrix(h, g, ne)
    n2 = n * n
    Gre = np.zeros((2 * n2, 2 * n2))
    Gre[0::2, 0::2] = G.real
    Gre[0::2, 1::2] = -G.imag
    Gre[1::2, 0::2] = G.imag
    Gre[1::2, 1::2] = G.real
    eG = int(np.frexp(np.max(np.abs(Gre)))[1])
    shG = 7 * s - 2 - eG
    Gint = np.rint(np.ldexp(Gre, shG)).astype(np.int64)
    cmax = max(np.max(np.abs(C.real)), np.max(np.abs(C.imag)))
    eC = int(np.frexp(cmax)[1]) if cmax > 0 else 0
    shC = 7 * s - 3 - eC
    Cr = np.rint(np.ldexp(C.real, shC)).astype(np.int64)
    Ci = np.rint(np.ldexp(C.imag, shC)).astype(np.int64)
    t = oracle.replacement_table(n, ne)
    N = len(C)
    D = np.zeros((2 * n2, N), np.int64)
    for S in range(t["target"].shape[0]):
        for e in range(t["target"].shape[1]):
            T, a, b, sg = t["target"][S, e], t["a"][S, e], t["b"][S, e], int(t["sign"][S, e])
            x = a * n + b
            D[2 * x, S] += sg * Cr[T]
            D[2 * x + 1, S] += sg * Ci[T]
    gd = balanced_digits7(Gint, s)
    dd = balanced_digits7(D, s)
    L0 = max(s - 1, 2 * s - 7)
    lo = np.zeros_like(D)
    hi = np.zeros_like(D)
    for L in range(s - 1, 2 * s - 1):
        SL = np.zeros_like(D)
        for i in range(s):
            j = L - i
            if 0 <= j < s:
                SL += gd[i] @ dd[j]
        assert np.max(np.abs(SL)) < 2 ** 24
        if L < L0:
            lo += SL << (7 * (L - (s - 1)))
        else:
            hi += SL << (7 * (L - L0))
    k = 7 * (L0 - (s - 1))
    E = hi + (((lo + (1 << (k - 1))) >> k) if k > 0 else 0)
    ar = np.zeros(N, np.int64)
    ai = np.zeros(N, np.int64)
    for S in range(t["target"].shape[0]):
        for e in range(t["target"].shape[1]):
            T, a, b, sg = t["target"][S, e], t["a"][S, e], t["b"][S, e], int(t["sign"][S, e])
            x = a * n + b
            ar[S] += sg * E[2 * x, T]
            ai[S] += sg * E[2 * x + 1, T]
    u = 7 * L0 - shG - shC
    return np.ldexp(ar.astype(np.float64), u) + 1j * np.ldexp(ai.astype(np.float64), u) + e_core * C
