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

``davidson_compressed`` runs the Davidson iteration with every vector kept compressed
(nonzero entries only), sigma by Algorithm 1 and the preconditioner of Eq.
sparsePreconditioner with H_ii evaluated on the fly.
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


# ----------------------------------------------------------- Davidson on compressed vectors

def _dot(u: dict, v: dict) -> float:
    if len(u) > len(v):
        u, v = v, u
    return sum(x * v[k] for k, x in u.items() if k in v)


def _comb(terms) -> dict:
    """sum_i a_i v_i over sparse vectors given as (a_i, v_i) pairs."""
    out = {}
    for a, v in terms:
        for k, x in v.items():
            out[k] = out.get(k, 0.0) + a * x
    return out


def _norm(v: dict) -> float:
    return float(np.sqrt(sum(x * x for x in v.values())))


def to_csc(v: dict, spaces, ref_a, ref_b, n_a, n_b, max_transfer):
    """Sparse vector {target address: value} -> the per-category (A, V) arrays of
    ``compress`` (nonzero entries only)."""
    cats, _ = odas.categories(spaces, ref_a, ref_b, n_a, n_b, max_transfer)
    offs = [c[4] for c in cats]
    import bisect

    per = {}
    for addr in sorted(k for k, x in v.items() if x != 0.0):
        c = bisect.bisect_right(offs, addr) - 1
        per.setdefault(c, []).append(addr)
    return {c: (np.array([a - offs[c] for a in lst], np.int64), np.array([v[a] for a in lst]))
            for c, lst in per.items()}


def davidson_compressed(h, g, e_core, spaces, ref_a, ref_b, n_a, n_b, max_transfer, guess: dict,
                        eps=0.0, tol_r=1e-6, tol_e=1e-10, max_iter=200, max_sub=32, guard=1e-12):
    """Lowest eigenpair of H on the DAS target space with every vector kept compressed
    (Results: the Davidson iteration with the compression-compatible preconditioner of
    Eq. sparsePreconditioner, and categorical compression of the CI vectors).

    Vectors are {target address: value} holding nonzero entries only; sigma of a vector
    is Algorithm 1 on its per-category compressed form (``sigma_alg1``), so only nonzero
    coefficients are ever touched.  H_ii is evaluated on the fly, for the addresses where
    the residual is nonzero, from the determinant's strings (the paper avoids storing the
    dense diagonal).  The preconditioner is Eq. sparsePreconditioner: s_i = r_i /
    (lambda - H_ii) where |lambda - H_ii| >= guard, else 0; t_i = s_i where
    |s_i| >= eps ||s||, else 0 (entries dropped are exact zeros of the next vector).
    Every other step follows oracle.davidson with the same readings (one new vector per
    iteration, collapse to the current and previous Ritz vectors at max_sub, two rounds
    of classical Gram-Schmidt, a new direction below 1e-10 dropped, convergence on ||r||
    and |dE|), so with the same guess the two agree up to rounding.
    Returns (E, c, log, converged); log entries add nnz_s and nnz_t, the nonzeros of the
    preconditioned residual before and after the eps threshold."""
    from . import diag as _diag, spin_orbital_integrals

    hso, gso = spin_orbital_integrals(h, g)
    hii = {}

    def h_diag(addrs):
        new = [a for a in addrs if a not in hii]
        if new:
            dets = odas.dets_of_addresses(spaces, ref_a, ref_b, n_a, n_b, max_transfer, new)
            for a, d in zip(new, _diag(hso, gso, dets)):
                hii[a] = float(d) + e_core
        return np.array([hii[a] for a in addrs])

    def matvec(v):
        csc = to_csc(v, spaces, ref_a, ref_b, n_a, n_b, max_transfer)
        s = sigma_alg1(h, g, e_core, spaces, ref_a, ref_b, n_a, n_b, max_transfer, csc)
        return {k: x for k, x in s.items() if x != 0.0}

    def scale(v, a):
        return {k: a * x for k, x in v.items()}

    def orth(t, V):
        for _ in range(2):
            for v in V:
                t = _comb([(1.0, t), (-_dot(v, t), v)])
        return t

    nv = _norm(guess)
    v = {k: x / nv for k, x in guess.items() if x != 0.0}
    V, S = [v], [matvec(v)]
    log, E_prev, c_prev, sc_prev, converged = [], None, None, None, False
    lam, c = None, v
    for it in range(max_iter):
        k = len(V)
        Hs = np.array([[_dot(V[i], S[j]) for j in range(k)] for i in range(k)])
        Hs = 0.5 * (Hs + Hs.T)
        w, y = np.linalg.eigh(Hs)
        lam, y0 = float(w[0]), y[:, 0]
        c = _comb([(float(y0[i]), V[i]) for i in range(k)])
        sc = _comb([(float(y0[i]), S[i]) for i in range(k)])
        if c_prev is not None:
            ph = _dot(c_prev, c)
            if ph < 0:
                c, sc = scale(c, -1.0), scale(sc, -1.0)
        r = _comb([(1.0, sc), (-lam, c)])
        rn = _norm(r)
        dE = None if E_prev is None else lam - E_prev
        dC = None
        if c_prev is not None:
            diff = _comb([(1.0, c), (-1.0, c_prev)])
            dC = max((abs(x) for x in diff.values()), default=0.0)
        entry = dict(iteration=it + 1, energy=lam, dE=dE, max_dC=dC, rnorm=rn, nnz_c=len(c))
        log.append(entry)
        if rn <= tol_r and dE is not None and abs(dE) <= tol_e:
            converged = True
            break
        addrs = [a for a, x in r.items() if x != 0.0]
        den = lam - h_diag(addrs)
        rv = np.array([r[a] for a in addrs])
        sv = np.where(np.abs(den) >= guard, rv / np.where(den == 0, 1.0, den), 0.0)
        if eps > 0.0:
            tv = np.where(np.abs(sv) >= eps * np.linalg.norm(sv), sv, 0.0)
        else:
            tv = sv
        entry["nnz_s"], entry["nnz_t"] = int(np.count_nonzero(sv)), int(np.count_nonzero(tv))
        t = {a: float(x) for a, x in zip(addrs, tv) if x != 0.0}
        if k >= max_sub:
            newV, newS = [c], [sc]
            if c_prev is not None:
                ov = _dot(c, c_prev)
                p = _comb([(1.0, c_prev), (-ov, c)])
                pn = _norm(p)
                if pn > 1e-10:
                    newV.append(scale(p, 1.0 / pn))
                    newS.append(scale(_comb([(1.0, sc_prev), (-ov, sc)]), 1.0 / pn))
            V, S = newV, newS
        t = orth(t, V)
        tn = _norm(t)
        E_prev, c_prev, sc_prev = lam, c, sc
        if tn < 1e-10:
            break
        t = scale(t, 1.0 / tn)
        V.append(t)
        S.append(matvec(t))
    return lam, c, log, converged
