"""STP-DAS categories from their definition (oracle; test infrastructure only).

The active space is split into distributed active spaces (DAS), each owning a
contiguous range of orbitals.  A category is one electron-occupation pattern over the
spaces ("Results", the categorical decomposition and the direct sum C = (+)_B C^B; the
Fig. 2A caption describes the split).  Per spin, a pattern is a tuple (n_1, ..., n_S);
a category is a pair (alpha pattern, beta pattern).  The paper's "at most T electrons
transferred" is read spin-resolved: the number of electrons a pattern holds above the
reference occupation, summed over spaces and over both spins, is at most T.

Canonical order (needed so that tables compare bit for bit):
  * per-spin patterns in ascending lexicographic order;
  * categories (a, b) in lexicographic order of (a, b);
  * inside a category, determinants row-major [alpha-local][beta-local];
  * a local string index is a mixed-radix number over the spaces, space 1 most
    significant, each digit the rank of that space's sub-string among the space's
    strings in ascending integer order.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np


def patterns(spaces, n_el):
    """All occupation tuples with 0 <= n_s <= spaces[s] and sum n_el, lexicographic."""
    out = []
    for p in itertools.product(*[range(m + 1) for m in spaces]):
        if sum(p) == n_el:
            out.append(tuple(p))
    return out


def excess(p, ref):
    return sum(max(0, a - r) for a, r in zip(p, ref))


def block_strings(spaces, p):
    return int(np.prod([comb(m, k) for m, k in zip(spaces, p)], dtype=object))


def categories(spaces, ref_a, ref_b, n_a, n_b, max_transfer):
    """[(alpha pattern, beta pattern, n_alpha_strings, n_beta_strings, offset)]."""
    pa = patterns(spaces, n_a)
    pb = patterns(spaces, n_b)
    cats = []
    off = 0
    for a in pa:
        for b in pb:
            if excess(a, ref_a) + excess(b, ref_b) <= max_transfer:
                na, nb = block_strings(spaces, a), block_strings(spaces, b)
                cats.append((a, b, na, nb, off))
                off += na * nb
    return cats, off


def _space_strings(m, k):
    return [x for x in range(1 << m) if bin(x).count("1") == k]


def pattern_strings(spaces, p):
    """Global masks of all strings with pattern p, in local (mixed-radix) order."""
    offs = np.cumsum([0] + list(spaces[:-1]))
    per = [[s << int(o) for s in _space_strings(m, k)] for m, k, o in zip(spaces, p, offs)]
    out = []
    for combo in itertools.product(*per):
        v = 0
        for s in combo:
            v |= s
        out.append(v)
    return out


def das_dets(spaces, ref_a, ref_b, n_a, n_b, max_transfer):
    """Spin-orbital masks (alpha in the low n bits, beta above) in DAS order."""
    n = sum(spaces)
    cats, total = categories(spaces, ref_a, ref_b, n_a, n_b, max_transfer)
    out = np.empty(total, np.uint64)
    k = 0
    for a, b, na, nb, off in cats:
        sa = np.array(pattern_strings(spaces, a), np.uint64)
        sb = np.array(pattern_strings(spaces, b), np.uint64)
        blk = (sa[:, None] | (sb[None, :] << np.uint64(n))).reshape(-1)
        out[off:off + len(blk)] = blk
        k += len(blk)
    assert k == total
    return out, cats


def dets_of_addresses(spaces, ref_a, ref_b, n_a, n_b, max_transfer, addrs):
    """Spin-orbital masks of the DAS determinants at the given addresses, decoded from the
    definition of the canonical order above (category by offset, then row-major
    [alpha-local][beta-local], each local index a mixed-radix number over the spaces, space
    1 most significant, digits the ranks of the spaces' sub-strings); for spaces too large
    to enumerate whole."""
    n = sum(spaces)
    cats, total = categories(spaces, ref_a, ref_b, n_a, n_b, max_transfer)
    offs = [c[4] for c in cats]
    space_off = np.cumsum([0] + list(spaces[:-1]))
    sub = {}

    def substrings(m, k):
        if (m, k) not in sub:
            sub[(m, k)] = _space_strings(m, k)
        return sub[(m, k)]

    def string_of(p, local):
        digits = []
        for m, k in reversed(list(zip(spaces, p))):
            r = comb(m, k)
            digits.append(local % r)
            local //= r
        digits.reverse()
        v = 0
        for (m, k), d, o in zip(zip(spaces, p), digits, space_off):
            v |= substrings(m, k)[d] << int(o)
        return v

    import bisect

    out = np.empty(len(addrs), np.uint64)
    for i, x in enumerate(addrs):
        x = int(x)
        if not 0 <= x < total:
            raise ValueError("address outside the DAS space")
        c = bisect.bisect_right(offs, x) - 1
        a, b, na, nb, off = cats[c]
        la, lb = divmod(x - off, nb)
        out[i] = string_of(a, la) | (string_of(b, lb) << n)
    return out
