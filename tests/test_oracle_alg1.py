"""CPU pins of the oracle's Algorithm 1 (compressed sigma, oracle/alg1.py): its
exponential search is a lower-bound search, its fermion signs are those of the C oracle's
replacement table, and the compressed sigma equals the Slater-Condon sigma of the same
vector on the structural support and leaves nothing nonzero outside it (the lossless
compression and compression preservation of Results and Methods)."""
import numpy as np
import pytest

import oracle
from oracle import alg1
from oracle import das as odas
from paper_2505_20375_gb300 import synth


def test_exponential_search_is_the_lower_bound():
    rng = np.random.default_rng(0)
    for _ in range(3000):
        A = np.unique(rng.integers(0, 200, int(rng.integers(0, 60))))
        key = int(rng.integers(-5, 210))
        lo = int(rng.integers(0, len(A) + 1))
        assert alg1.exponential_search(A, key, lo) == lo + int(np.searchsorted(A[lo:], key, side="left"))
    assert alg1.exponential_search(np.array([], np.int64), 3) == 0


def test_excitation_signs_match_the_replacement_table():
    """a+_a a_b T = sign S for every entry (S, T, a, b, sign) of the C oracle's table."""
    for m, ne in ((6, 3), (7, 2), (5, 5)):
        t = oracle.replacement_table(m, ne)
        s = t["strings"]
        for i in range(len(s)):
            for e in range(t["target"].shape[1]):
                T = int(s[t["target"][i, e]])
                got = alg1.excite(T, int(t["a"][i, e]), int(t["b"][i, e]))
                assert got == (int(s[i]), int(t["sign"][i, e]))


def _case(spaces, ref, nel, T, frac, seed=5):
    n = sum(spaces)
    h, g = synth.real_integrals(n, 9, seed=31)
    dets, cats = odas.das_dets(spaces, ref, ref, nel, nel, T)
    c = synth.random_vector(len(dets), seed)
    u = synth.Stream(seed, tag=3).uniform(len(dets))
    c[u >= frac] = 0.0
    return h, g, dets, cats, c


@pytest.mark.parametrize("spaces,ref,nel,T,frac", [([3, 3, 2], [1, 2, 1], 4, 1, 0.02),
                                                   ([2, 3, 3], [1, 1, 2], 4, 2, 0.01),
                                                   ([2, 2, 2], [1, 1, 1], 3, 1, 1.0)])
def test_compressed_sigma_is_the_slater_condon_sigma_on_its_support(spaces, ref, nel, T, frac):
    h, g, dets, cats, c = _case(spaces, ref, nel, T, frac)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    csc = alg1.compress(c, spaces, ref, ref, nel, nel, T)
    assert sum(len(A) for A, _ in csc.values()) == np.count_nonzero(c)
    sg = alg1.sigma_alg1(h, g, 0.4, spaces, ref, ref, nel, nel, T, csc)
    ref_s = oracle.sigma(hso, gso, dets, c, e_core=0.4).real
    addr = np.array(sorted(sg))
    val = np.array([sg[a] for a in addr])
    assert np.max(np.abs(val - ref_s[addr])) <= 1e-13 * np.max(np.abs(ref_s))
    off = np.ones(len(dets), bool)
    off[addr] = False
    assert np.all(ref_s[off] == 0.0)
    if frac >= 1.0:  # a dense vector: the support is the whole space
        assert len(addr) == len(dets)
    else:
        assert set(np.flatnonzero(c).tolist()) <= set(addr.tolist()) and len(addr) < len(dets)



def _dense_reference(spaces, ref, nel, T, e_core, seed):
    h, g = synth.real_integrals(sum(spaces), 9, seed=seed)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    hd = oracle.diag(hso, gso, dets) + e_core
    H = oracle.dense_h(hso, gso, dets).real + e_core * np.eye(len(dets))
    return h, g, hso, gso, dets, hd, H


@pytest.mark.parametrize("eps_scale,seed,e_core", [(0.0, 61, 0.3), (1.0, 62, -0.2)])
def test_compressed_davidson_is_the_dense_davidson(eps_scale, seed, e_core):
    """The Davidson iteration on compressed vectors (Algorithm 1 sigma of the nonzero
    entries only, H_ii evaluated on the fly where the residual is nonzero) follows the dense
    oracle Davidson step for step from the same guess, with the traditional preconditioner
    (eps = 0) and with the compression-compatible one (Eq. sparsePreconditioner,
    eps = 1/sqrt(N)); both reach the lowest eigenvalue of the dense DAS Hamiltonian.  With
    eps > 0 the thresholded corrections drop entries and the early vectors stay sparse:
    the preconditioner changes only the expansion, sigma and ||r|| stay exact (Results)."""
    from oracle import davidson as odav

    spaces, ref, nel, T = [2, 2, 2], [1, 1, 1], 3, 1
    h, g, hso, gso, dets, hd, H = _dense_reference(spaces, ref, nel, T, e_core, seed)
    N = len(dets)
    eps = eps_scale / np.sqrt(N)
    i0 = int(np.argmin(hd))
    E_d, c_d, log_d, conv_d = odav.davidson(lambda v: oracle.sigma(hso, gso, dets, v, e_core=e_core), hd,
                                            tol_r=1e-6, tol_e=1e-10, eps=eps, max_iter=400)
    E_c, c_c, log_c, conv_c = alg1.davidson_compressed(h, g, e_core, spaces, ref, ref, nel, nel, T, {i0: 1.0},
                                                       eps=eps, tol_r=1e-6, tol_e=1e-10, max_iter=400)
    assert conv_d and conv_c and len(log_c) == len(log_d)
    # the two sum in different orders; with eps > 0 a rounding difference can move an entry
    # across the threshold, so the residual norms agree to 1e-4 there (1e-6 without)
    rtol = 1e-4 if eps > 0 else 1e-6
    for a, b in zip(log_c, log_d):
        assert abs(a["energy"] - b["energy"]) <= 1e-10
        assert abs(a["rnorm"] - b["rnorm"]) <= rtol * b["rnorm"] + 1e-12
    w0 = np.linalg.eigvalsh(H)[0]
    assert abs(E_c - w0) <= 1e-10 and abs(E_d - w0) <= 1e-10
    dense_c = np.zeros(N)
    for k, x in c_c.items():
        dense_c[k] = x
    assert np.max(np.abs(dense_c - c_d)) <= 1e-7
    if eps > 0:
        assert all(e["nnz_t"] <= e["nnz_s"] for e in log_c if "nnz_t" in e)
        assert any(e["nnz_t"] < e["nnz_s"] for e in log_c if "nnz_t" in e)
        assert log_c[2]["nnz_c"] < N // 4  # the third Ritz vector is still compressed
