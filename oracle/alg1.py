"""Algorithm 1 (Methods): the sigma build on a categorically compressed CI vector, written
out step by step as test infrastructure (oracle).  Only ``tests/`` may import it; it
shares nothing with the product path.

The CI vector is held as the paper's direct sum over categories (Results, categorical
compression): for every target category B with nonzero coefficients, V^B (the nonzero
values) and A^B (their local addresses inside the category block, ascending).  Categories
without nonzeros are simply absent (the categorical skip).

Sigma (Methods, Eqs. sigmaL, sigmaL2e, with the one-electron term folded into the
two-electron one through sum_r E_rr = N_e):

    H = 1/2 sum_pqrs g'_pqrs E_pq E_rs,
    g'_pqrs = (pq|rs) + (h'_pq delta_rs + delta_pq h'_rs) / N_e,
    h'_pq = h_pq - 1/2 sum_r (pr|rq),

evaluated through the intermediate determinants J (target and one-more-transfer
categories, the range that makes the product P H P exact):

    D[rs, J] = sum_K <J|E_rs|K> C_K            (Alg. 1: J's excitation list intersected
                                                with A^B by exponential search)
    E[pq, J] = 1/2 sum_rs g'_pqrs D[rs, J]     (the dense contraction)
    sigma_L += <L|E_pq|J> E[pq, J]             (accumulated into a table keyed by L,
                                                the paper's per-category hash table)

and sigma_L += e_core C_L.  Strings are orbital bit masks; a determinant is the alpha
string's creation operators followed by the beta string's, so a beta excitation carries
the sign of its own string only.
"""
from __future__ import annotations

import numpy as np

from . import das as odas


def exponential_search(A, key, lo: int = 0) -> int:
    """First index i >= lo with A[i] >= key (len(A) if none), A ascending: steps of
    1, 2, 4, ... from lo until A[lo + step] >= key brackets it, then a binary search
    between the last two probes (the paper's exponentialSearch subroutine)."""
    n = len(A)
    if lo >= n or A[lo] >= key:
        return lo
    step = 1
    while lo + step < n and A[lo + step] < key:
        step *= 2
    left, right = lo + step // 2 + 1, min(lo + step, n)  # A[lo + step // 2] < key
    while left < right:
        mid = (left + right) // 2
        if A[mid] < key:
            left = mid + 1
        else:
            right = mid
    return left


def excite(s: int, p: int, q: int):
    """a+_p a_q applied to the string s: (string, sign), or None if the result vanishes."""
    if not (s >> q) & 1:
        return None
    sign = -1 if bin(s & ((1 << q) - 1)).count("1") & 1 else 1
    s1 = s & ~(1 << q)
    if (s1 >> p) & 1:
        return None
    if bin(s1 & ((1 << p) - 1)).count("1") & 1:
        sign = -sign
    return s1 | (1 << p), sign


def pattern_of(s: int, spaces) -> tuple:
    out, o = [], 0
    for m in spaces:
        out.append(bin((s >> o) & ((1 << m) - 1)).count("1"))
        o += m
    return tuple(out)


def compress(c, spaces, ref_a, ref_b, n_a, n_b, max_transfer, tol: float = 0.0):
    """Dense DAS vector -> {category index: (A ascending local addresses, V values)} for the
    target categories holding a coefficient with |c| > tol."""
    cats, _ = odas.categories(spaces, ref_a, ref_b, n_a, n_b, max_transfer)
    out = {}
    for k, (_, _, na, nb, off) in enumerate(cats):
        blk = np.asarray(c[off:off + na * nb])
        A = np.flatnonzero(np.abs(blk) > tol)
        if len(A):
            out[k] = (A.astype(np.int64), blk[A].copy())
    return out


def folded_operator(h, g, n_el: int):
    """1/2 g' as an (n^2 x n^2) matrix over ordered pairs (pq), (rs)."""
    n = h.shape[0]
    hp = h - 0.5 * np.einsum("prrq->pq", g)
    eye = np.eye(n)
    gp = g + (hp[:, :, None, None] * eye[None, None, :, :] + eye[:, :, None, None] * hp[None, None, :, :]) / n_el
    return 0.5 * gp.reshape(n * n, n * n)


def sigma_alg1(h, g, e_core, spaces, ref_a, ref_b, n_a, n_b, max_transfer, csc):
    """Compressed sigma: {target address L: sigma_L} over every L one excitation from an
    intermediate determinant J with D[:, J] != 0 (the structural support)."""
    n = sum(spaces)
    tcats, _ = odas.categories(spaces, ref_a, ref_b, n_a, n_b, max_transfer)
    icats, _ = odas.categories(spaces, ref_a, ref_b, n_a, n_b, max_transfer + 1)
    tindex = {(pa, pb): k for k, (pa, pb, _, _, _) in enumerate(tcats)}
    strings = {}  # pattern -> (list of strings in local order, {string: local index})

    def strs(p):
        if p not in strings:
            lst = odas.pattern_strings(spaces, p)
            strings[p] = (lst, {s: i for i, s in enumerate(lst)})
        return strings[p]

    def coefficient(KA: int, KB: int):
        """C_K of the determinant (KA, KB) from the compressed vector, or None."""
        pa, pb = pattern_of(KA, spaces), pattern_of(KB, spaces)
        k = tindex.get((pa, pb))
        if k is None or k not in csc:  # outside the target space, or an empty category
            return None
        A, V = csc[k]
        local = strs(pa)[1][KA] * tcats[k][3] + strs(pb)[1][KB]
        i = exponential_search(A, local)
        return V[i] if i < len(A) and A[i] == local else None

    def target_address(LA: int, LB: int):
        pa, pb = pattern_of(LA, spaces), pattern_of(LB, spaces)
        k = tindex.get((pa, pb))
        if k is None:
            return None
        return tcats[k][4] + strs(pa)[1][LA] * tcats[k][3] + strs(pb)[1][LB]

    G = folded_operator(h, g, n_a + n_b)
    sigma = {}
    for pa, pb, na, nb, _ in icats:  # intermediate categories
        sa, sb = strs(pa)[0], strs(pb)[0]
        cols, D = [], []
        for JA in sa:
            for JB in sb:
                d = np.zeros(n * n)
                hit = False
                for r in range(n):
                    for s in range(n):
                        for spin in (0, 1):  # K = E_sr J, <J|E_rs|K> = the sign of that move
                            m = excite(JA if spin == 0 else JB, s, r)
                            if m is None:
                                continue
                            K, sg = m
                            v = coefficient(K, JB) if spin == 0 else coefficient(JA, K)
                            if v is not None:
                                d[r * n + s] += sg * v
                                hit = True
                if hit:
                    cols.append((JA, JB))
                    D.append(d)
        if not cols:
            continue
        E = G @ np.array(D).T  # [pq, column]
        for j, (JA, JB) in enumerate(cols):
            for p in range(n):
                for q in range(n):
                    e = E[p * n + q, j]
                    for spin in (0, 1):  # L = E_pq J
                        m = excite(JA if spin == 0 else JB, p, q)
                        if m is None:
                            continue
                        L, sg = m
                        addr = target_address(L, JB) if spin == 0 else target_address(JA, L)
                        if addr is not None:
                            sigma[addr] = sigma.get(addr, 0.0) + sg * e
    for k, (A, V) in csc.items():  # the constant term
        off = tcats[k][4]
        for a, v in zip(A, V):
            sigma[int(off + a)] = sigma.get(int(off + a), 0.0) + e_core * v
    return sigma
