"""Pins of the oracle against things other than itself (CPU only).

Each test would fail for a plausible slip in oracle/fci_oracle.c or oracle/*.py: a
dropped exchange term, a wrong fermion sign, a transposed integral index, a missing
1/2, a wrong determinant order.
"""
import itertools
import json
import os
from math import comb

import numpy as np
import pytest

import oracle
from oracle import das as odas
from oracle import davidson as odav
from paper_2505_20375_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- strings

@pytest.mark.parametrize("m,ne", [(1, 0), (1, 1), (4, 2), (8, 4), (10, 3), (14, 7), (16, 8)])
def test_strings_closed_form_count_and_order(m, ne):
    s = oracle.enumerate_strings(m, ne)
    assert len(s) == comb(m, ne)
    assert np.all(np.diff(s.astype(np.int64)) > 0)
    assert all(bin(int(x)).count("1") == ne for x in s[:2000])


def test_paper_printed_determinant_counts():
    """The determinant counts the paper prints equal C(n, n_e) (spinor strings)."""
    gold = json.load(open(os.path.join(GOLD, "paper_det_counts.json")))
    for c in gold["cases"]:
        N = comb(c["n"], c["ne"])
        assert abs(N - c["printed"]) <= c["rel_tol"] * c["printed"], c["name"]
    # and the oracle's string enumeration agrees with the count where it can run
    assert len(oracle.enumerate_strings(24, 12)) == comb(24, 12)


def _apply_by_position(occ, ops):
    """Apply operators right to left to a sorted occupation tuple, sign by position.
    ops: list of ('c'|'a', orbital) written left to right."""
    occ = list(occ)
    sign = 1
    for kind, p in reversed(ops):
        if kind == "a":
            if p not in occ:
                return None, 0
            k = occ.index(p)
            sign *= (-1) ** k
            occ.pop(k)
        else:
            if p in occ:
                return None, 0
            k = sum(1 for q in occ if q < p)
            sign *= (-1) ** k
            occ.insert(k, p)
    return tuple(occ), sign


@pytest.mark.parametrize("m,ne", [(5, 2), (6, 3), (8, 4), (9, 2)])
def test_replacement_table_against_position_parity(m, ne):
    t = oracle.replacement_table(m, ne)
    s = t["strings"]
    n_ent = ne * (m - ne + 1)  # n_e (n_h + 1) per string (Introduction)
    assert t["target"].shape == (len(s), n_ent)
    index = {int(x): i for i, x in enumerate(s)}
    for i, S in enumerate(s):
        occS = tuple(p for p in range(m) if (int(S) >> p) & 1)
        seen = set()
        for e in range(n_ent):
            a, b = int(t["a"][i, e]), int(t["b"][i, e])
            T = int(s[t["target"][i, e]])
            occT = tuple(p for p in range(m) if (T >> p) & 1)
            res, sg = _apply_by_position(occT, [("c", a), ("a", b)])
            assert res == occS and sg == int(t["sign"][i, e])
            assert a in occS and (b == a or b not in occS)
            seen.add((a, b))
        assert len(seen) == n_ent
        # order: a ascending, then b ascending
        pairs = [(int(t["a"][i, e]), int(t["b"][i, e])) for e in range(n_ent)]
        assert pairs == sorted(pairs)


# ------------------------------------------------------------------ Hamiltonian

def _jw_hamiltonian(hso, gso):
    """Dense Fock-space H from Jordan-Wigner matrices (independent of bit counting).
    Basis state index = occupation mask; a_P = Z x ... x Z x sigma^- x 1 ... with the
    Z string on the modes below P (creation operators in ascending order)."""
    nso = hso.shape[0]
    dim = 1 << nso
    A = []
    for P in range(nso):
        op = np.zeros((dim, dim))
        for x in range(dim):
            if (x >> P) & 1:
                parity = bin(x & ((1 << P) - 1)).count("1") & 1
                op[x ^ (1 << P), x] = -1.0 if parity else 1.0
        A.append(op)
    Ad = [a.T for a in A]
    H = np.zeros((dim, dim), np.complex128)
    for P in range(nso):
        for Q in range(nso):
            if hso[P, Q] != 0:
                H += hso[P, Q] * (Ad[P] @ A[Q])
    one = [[Ad[P] @ A[Q] for Q in range(nso)] for P in range(nso)]
    for P, Q, R, S in itertools.product(range(nso), repeat=4):
        v = gso[P, Q, R, S]
        if v != 0:
            # a+_P a+_R a_S a_Q = E_PQ E_RS - delta_QR E_PS
            term = one[P][Q] @ one[R][S]
            if Q == R:
                term = term - one[P][S]
            H += 0.5 * v * term
    return H


@pytest.mark.parametrize("kind", ["real_2o", "real_3o", "spinor_5", "spinor_6"])
def test_slater_condon_matches_jordan_wigner(kind):
    if kind.startswith("real"):
        n = int(kind[5])
        h, g = synth.real_integrals(n, 4, seed=11 + n)
        hso, gso = oracle.spin_orbital_integrals(h, g)
        dets = oracle.fci_dets(n, 1, 2) if n == 3 else oracle.fci_dets(n, 1, 1)
    else:
        n = int(kind[-1])
        h, g = synth.complex_integrals(n, 4, seed=21 + n)
        hso, gso = oracle.spinor_integrals(h, g)
        dets = oracle.spinor_dets(n, 3 if n == 6 else 2)
    Hjw = _jw_hamiltonian(hso, gso)
    idx = dets.astype(np.int64)
    Hsub = Hjw[np.ix_(idx, idx)]
    Hsc = oracle.dense_h(hso, gso, dets)
    assert np.max(np.abs(Hsc - Hsub)) < 1e-12
    # the determinant space is closed under H: nothing leaks out of it
    mask = np.ones(Hjw.shape[0], bool)
    mask[idx] = False
    assert np.max(np.abs(Hjw[np.ix_(mask, idx)])) < 1e-14


def test_position_parity_brute_force_4o():
    """FCI(2a,2b in 4 orbitals): every element vs an operator-string brute force over
    all (h, g) terms with signs from list positions (a third independent route)."""
    n = 4
    h, g = synth.real_integrals(n, 6, seed=5)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets = oracle.fci_dets(n, 2, 2)
    occ = [tuple(p for p in range(2 * n) if (int(d) >> p) & 1) for d in dets]
    pos = {o: i for i, o in enumerate(occ)}
    N = len(dets)
    Hb = np.zeros((N, N))
    nso = 2 * n
    for j, oJ in enumerate(occ):
        for P in range(nso):
            for Q in range(nso):
                if hso[P, Q] == 0:
                    continue
                r, s = _apply_by_position(oJ, [("c", P), ("a", Q)])
                if s and r in pos:
                    Hb[pos[r], j] += hso[P, Q].real * s
        for P, Q, R, S in itertools.product(range(nso), repeat=4):
            v = gso[P, Q, R, S].real
            if v == 0:
                continue
            r, s = _apply_by_position(oJ, [("c", P), ("c", R), ("a", S), ("a", Q)])
            if s and r in pos:
                Hb[pos[r], j] += 0.5 * v * s
    Hsc = oracle.dense_h(hso, gso, dets).real
    assert np.max(np.abs(Hsc - Hb)) < 1e-12


def test_hermiticity_real_and_complex():
    for cplx in (False, True):
        if cplx:
            h, g = synth.complex_integrals(8, 8, seed=3)
            hso, gso = oracle.spinor_integrals(h, g)
            dets = oracle.spinor_dets(8, 4)
        else:
            h, g = synth.real_integrals(6, 8, seed=3)
            hso, gso = oracle.spin_orbital_integrals(h, g)
            dets = oracle.fci_dets(6, 3, 3)
        x = synth.random_vector(len(dets), 1, complex_=cplx)
        y = synth.random_vector(len(dets), 2, complex_=cplx)
        Hx = oracle.sigma(hso, gso, dets, x)
        Hy = oracle.sigma(hso, gso, dets, y)
        lhs = np.vdot(x, Hy)
        rhs = np.vdot(Hx, y)
        assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


def test_sigma_equals_dense_h_times_c():
    h, g = synth.real_integrals(5, 6, seed=9)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets = oracle.fci_dets(5, 3, 2)
    H = oracle.dense_h(hso, gso, dets).real
    c = synth.random_vector(len(dets), 4)
    s = oracle.sigma(hso, gso, dets, c, e_core=0.75)
    assert np.max(np.abs(s - (H @ c + 0.75 * c))) < 1e-12


def test_one_electron_only_sum_of_orbital_energies():
    """g = 0: E0 = sum of the lowest n_alpha plus lowest n_beta eigenvalues of h."""
    n, na, nb = 6, 3, 2
    h, _ = synth.real_integrals(n, 2, seed=17)
    g = np.zeros((n,) * 4)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets = oracle.fci_dets(n, na, nb)
    E, _ = oracle.eigh_lowest(oracle.dense_h(hso, gso, dets))
    eps = np.linalg.eigvalsh(h)
    assert abs(E[0] - (eps[:na].sum() + eps[:nb].sum())) < 1e-12
    # spinor (complex Hermitian h): lowest n_e eigenvalues
    hc, _ = synth.complex_integrals(7, 2, seed=5)
    hs, gs = oracle.spinor_integrals(hc, np.zeros((7,) * 4))
    E2, _ = oracle.eigh_lowest(oracle.dense_h(hs, gs, oracle.spinor_dets(7, 3)))
    assert abs(E2[0] - np.linalg.eigvalsh(hc)[:3].sum()) < 1e-12


@pytest.mark.parametrize("t,U", [(1.0, 0.0), (1.0, 4.0), (0.3, 2.5), (2.0, 1.0)])
def test_hubbard_dimer_closed_form(t, U):
    h, g = synth.hubbard_dimer(t, U)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    E, _ = oracle.eigh_lowest(oracle.dense_h(hso, gso, oracle.fci_dets(2, 1, 1)))
    assert abs(E[0] - (U / 2 - np.sqrt(U * U / 4 + 4 * t * t))) < 1e-12


def test_two_electron_closed_forms():
    h, g = synth.real_integrals(2, 3, seed=8)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    # one doubly occupied orbital: 2 h_11 + (11|11)
    h1 = h[:1, :1].copy()
    g1 = g[:1, :1, :1, :1].copy()
    a, b = oracle.spin_orbital_integrals(h1, g1)
    E1 = oracle.dense_h(a, b, oracle.fci_dets(1, 1, 1)).real[0, 0]
    assert abs(E1 - (2 * h[0, 0] + g[0, 0, 0, 0])) < 1e-14
    # triplet of 2e in 2 orbitals: h11 + h22 + (11|22) - (12|21), present in the
    # Ms=0 spectrum and the single Ms=1 determinant
    trip = h[0, 0] + h[1, 1] + g[0, 0, 1, 1] - g[0, 1, 1, 0]
    w = np.linalg.eigvalsh(oracle.dense_h(hso, gso, oracle.fci_dets(2, 1, 1)).real)
    assert np.min(np.abs(w - trip)) < 1e-12
    Ems1 = oracle.dense_h(hso, gso, oracle.fci_dets(2, 2, 0)).real[0, 0]
    assert abs(Ems1 - trip) < 1e-12


def test_ms0_transpose_symmetry():
    """Spin-free integrals, n_alpha = n_beta: sigma(C^T) = sigma(C)^T."""
    n, ne = 6, 3
    h, g = synth.real_integrals(n, 6, seed=12)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets = oracle.fci_dets(n, ne, ne)
    ns = comb(n, ne)
    C = synth.random_vector(ns * ns, 5).reshape(ns, ns)
    s1 = oracle.sigma(hso, gso, dets, C.reshape(-1)).reshape(ns, ns)
    s2 = oracle.sigma(hso, gso, dets, C.T.reshape(-1)).reshape(ns, ns)
    assert np.max(np.abs(s1.T - s2)) < 1e-13


def test_sigma_row_subset_matches_full():
    h, g = synth.real_integrals(6, 6, seed=13)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets = oracle.fci_dets(6, 3, 3)
    c = synth.random_vector(len(dets), 6)
    full = oracle.sigma(hso, gso, dets, c)
    rows = np.array([0, 7, 100, len(dets) - 1])
    assert np.array_equal(oracle.sigma(hso, gso, dets, c, rows=rows), full[rows])


# --------------------------------------------------------------------------- DAS

def _brute_das_count(spaces, ref, n_el, T):
    """Count determinants by scanning every alpha and beta string of the full space."""
    n = sum(spaces)
    s = oracle.enumerate_strings(n, n_el).astype(np.int64)
    offs = np.cumsum([0] + list(spaces[:-1]))
    ex = np.zeros(len(s), np.int64)
    for m, o, r in zip(spaces, offs, ref):
        occ = np.zeros(len(s), np.int64)
        for p in range(o, o + m):
            occ += (s >> p) & 1
        ex += np.maximum(0, occ - r)
    hist = np.bincount(ex, minlength=T + 1)[: T + 1]
    return sum(int(hist[i]) * int(hist[: T + 1 - i].sum()) for i in range(T + 1))


@pytest.mark.parametrize("spaces,ref,nel,T", [
    ([4, 4, 4, 4], [2, 2, 2, 2], 8, 2),
    ([4, 4, 4, 4], [1, 1, 1, 1], 4, 1),
    ([4, 4, 4, 4], [2, 2, 2, 2], 8, 3),
    ([3, 3, 2], [1, 2, 1], 4, 1),
])
def test_das_counts_against_brute_force(spaces, ref, nel, T):
    cats, total = odas.categories(spaces, ref, ref, nel, nel, T)
    assert total == _brute_das_count(spaces, ref, nel, T)
    assert all(na * nb > 0 for _, _, na, nb, _ in cats)


def test_das_literal_24_orbital_space_count():
    """4 spaces x 6 orbitals, 12 alpha + 12 beta, reference 3/3 per space, <= 2 transfers."""
    cats, total = odas.categories([6] * 4, [3] * 4, [3] * 4, 12, 12, 2)
    # brute force over the 2,704,156 strings of 24 orbitals per spin
    assert total == _brute_das_count([6] * 4, [3] * 4, 12, 2)
    assert len(cats) == 253
    # the reference category alone: C(6,3)^8
    ref_cat = [c for c in cats if c[0] == (3, 3, 3, 3) and c[1] == (3, 3, 3, 3)][0]
    assert ref_cat[2] * ref_cat[3] == comb(6, 3) ** 8


def test_das_dets_are_the_pattern_restricted_fci_space():
    spaces, ref = [2, 2, 2], [1, 1, 1]
    dets, cats = odas.das_dets(spaces, ref, ref, 3, 3, 1)
    full = oracle.fci_dets(6, 3, 3)
    # every DAS determinant is an FCI determinant, each exactly once
    assert len(set(dets.tolist())) == len(dets)
    assert set(dets.tolist()) <= set(full.tolist())
    # local order inside a category: mixed radix, space 1 most significant
    a, b, na, nb, off = cats[0]
    sa = odas.pattern_strings(spaces, a)
    assert [int(x) & 0x3F for x in dets[off:off + na * nb:nb]] == sa


def test_das_sigma_is_projected_fci_sigma_and_compression_is_lossless():
    """DAS sigma = FCI sigma of the zero-padded C restricted to the DAS space (P H P),
    and dropping all-zero categories from the vector changes no sigma value
    (lossless categorical compression, Results; compression preservation, Methods)."""
    spaces, ref = [2, 2, 2], [1, 1, 1]
    n = 6
    h, g = synth.real_integrals(n, 8, seed=31)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets, cats = odas.das_dets(spaces, ref, ref, 3, 3, 1)
    c = synth.random_vector(len(dets), 8)
    s_das = oracle.sigma(hso, gso, dets, c)
    full = oracle.fci_dets(n, 3, 3)
    pos = {int(d): i for i, d in enumerate(full)}
    cf = np.zeros(len(full))
    idx = np.array([pos[int(d)] for d in dets])
    cf[idx] = c
    s_full = oracle.sigma(hso, gso, full, cf)
    assert np.max(np.abs(s_full[idx] - s_das)) < 1e-13
    # zero half of the categories, then drop them from the determinant list
    keep = np.zeros(len(dets), bool)
    for k, (_, _, na, nb, off) in enumerate(cats):
        if k % 2 == 0:
            keep[off:off + na * nb] = True
    cz = np.where(keep, c, 0.0)
    s_unc = oracle.sigma(hso, gso, dets, cz)
    # compressed: only nonzero categories as sources, all categories as outputs
    rows = np.arange(len(dets))
    s_cmp = np.array([0.0] * len(dets))
    src = dets[keep]
    for r in rows:
        sub = np.concatenate([[dets[r]], src[src != dets[r]]])
        csub = np.concatenate([[cz[r]], cz[keep][src != dets[r]]])
        s_cmp[r] = oracle.sigma(hso, gso, sub, csub, rows=np.array([0]))[0]
    assert np.array_equal(s_cmp, s_unc)


# ---------------------------------------------------------------------- Davidson

def _small_problem(n=6, ne=3, seed=41):
    h, g = synth.real_integrals(n, 8, seed=seed)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets = oracle.fci_dets(n, ne, ne)
    return hso, gso, dets


def test_davidson_matches_eigh_and_gap_bound():
    hso, gso, dets = _small_problem()
    H = oracle.dense_h(hso, gso, dets).real
    w = np.linalg.eigvalsh(H)
    hd = oracle.diag(hso, gso, dets)
    E, c, log, conv = odav.davidson(lambda v: H @ v, hd, tol_r=1e-7, tol_e=1e-12)
    assert conv
    assert abs(E - w[0]) < 1e-10
    # gap theorem (Methods, eigenvalue bound): |dE| <= ||r||^2 / gamma0
    r = log[-1]["rnorm"]
    assert abs(E - w[0]) <= r * r / (w[1] - w[0]) + 1e-14
    # eigenvector residual
    assert np.linalg.norm(H @ c - E * c) < 1e-6


def test_davidson_with_small_subspace_collapses_and_converges():
    hso, gso, dets = _small_problem(seed=43)
    H = oracle.dense_h(hso, gso, dets).real
    hd = oracle.diag(hso, gso, dets)
    E, c, log, conv = odav.davidson(lambda v: H @ v, hd, tol_r=1e-7, tol_e=1e-12, max_sub=4)
    assert conv and abs(E - np.linalg.eigvalsh(H)[0]) < 1e-10


def test_preconditioner_eps_zero_is_traditional_and_threshold_drops():
    rng = synth.Stream(3)
    r = rng.normal(50)
    hd = rng.normal(50)
    lam = -0.5
    hd[7] = lam  # guarded entry: |lambda - H_ii| < 1e-12
    t0 = odav.precondition(r, lam, hd, eps=0.0)
    trad = np.array([0.0 if abs(lam - h) < 1e-12 else ri / (lam - h) for ri, h in zip(r, hd)])
    assert np.array_equal(t0, trad)
    eps = 0.2
    t1 = odav.precondition(r, lam, hd, eps=eps)
    ns = np.linalg.norm(trad)
    assert np.array_equal(t1, np.where(np.abs(trad) >= eps * ns, trad, 0.0))
    assert np.count_nonzero(t1) < np.count_nonzero(t0)


def test_davidson_compression_compatible_preconditioner_converges():
    """eps > 0 still converges to the exact energy (Results: the preconditioner only
    changes the subspace expansion; sigma and ||r|| stay exact)."""
    hso, gso, dets = _small_problem(n=7, ne=3, seed=47)
    H = oracle.dense_h(hso, gso, dets).real
    hd = oracle.diag(hso, gso, dets)
    eps = 10.0 / np.sqrt(len(dets)) * 0.1
    E, c, log, conv = odav.davidson(lambda v: H @ v, hd, tol_r=1e-7, tol_e=1e-12, eps=eps,
                                    max_iter=400)
    assert conv and abs(E - np.linalg.eigvalsh(H)[0]) < 1e-9


def test_oracle_sigma_with_a_prebuilt_table_is_the_same_sigma():
    """The lookup table built once (oracle.SigmaTable, reused across calls, as the benchmark's
    CPU legs use it) gives the bits of the one-call sigma, on all rows and on a subset."""
    n, na, nb = 7, 3, 4
    h, g = synth.real_integrals(n, 9, 23)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets = oracle.fci_dets(n, na, nb)
    c = synth.random_vector(len(dets), seed=3)
    t = oracle.SigmaTable(dets)
    full = oracle.sigma(hso, gso, dets, c, e_core=0.7)
    assert np.array_equal(t.sigma(hso, gso, c, e_core=0.7), full)
    rows = np.array([len(dets) - 1, 0, 17, 17, 400])
    assert np.array_equal(t.sigma(hso, gso, c, e_core=0.7, rows=rows), full[rows])
    t.close()


@pytest.mark.parametrize("spaces,ref,nel,T", [([2, 2, 2], [1, 1, 1], 3, 1), ([3, 3, 2], [1, 2, 1], 4, 1),
                                              ([2, 3, 3], [1, 1, 2], 4, 2), ([4, 4, 4, 4], [1, 1, 1, 1], 4, 1)])
def test_das_address_decoding_matches_the_enumeration(spaces, ref, nel, T):
    """Decoding an address from the order's definition gives the determinant that the
    enumeration of the whole space puts there (so it can stand in for the enumeration of
    spaces too large to list, such as 24 orbitals in 4 x 6)."""
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    idx = np.arange(len(dets)) if len(dets) < 20000 else np.unique(synth.Stream(3).bits(4000) % len(dets))
    assert np.array_equal(odas.dets_of_addresses(spaces, ref, ref, nel, nel, T, idx), dets[idx])
