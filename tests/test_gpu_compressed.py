"""GPU tests of the categorically compressed sigma (fci_sigma_compressed) on the DAS layout:
a sparse C in, sigma on its structural support out, against the dense FP64 DAS sigma of
the same vector (bit for bit) and against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import alg1
from oracle import das as odas
from paper_2505_20375_gb300 import fci, synth

from helpers import SIGMA_RTOL, gpu_fci, rel_inf

pytestmark = pytest.mark.gpu


def das_gpu(spaces, ref, nel, T, n_chol=9, seed=31, e_core=0.0):
    n = sum(spaces)
    h, g = synth.real_integrals(n, n_chol, seed)
    f = gpu_fci(dict(h=h, g=g, e_core=e_core, n=n, na=nel, nb=nel))
    f.build_das(spaces, ref, ref, T)
    return h, g, f


def sparse_vector(f, spaces, seed, keep_frac):
    """A unit vector with whole categories zero (every third) and, in the others, a random
    fraction of the coefficients kept."""
    cats = f.table("das_categories").cpu().numpy().reshape(-1, 2 * len(spaces) + 3)
    c = synth.random_vector(f.n_det, seed=seed)
    u = synth.Stream(seed, tag=3).uniform(f.n_det)
    c[u >= keep_frac] = 0.0
    for k, r in enumerate(cats):
        if k % 3 == 1:
            off, ln = int(r[-1]), int(r[-3] * r[-2])
            c[off:off + ln] = 0.0
    return c / np.linalg.norm(c)


@pytest.mark.parametrize("spaces,ref,nel,T,frac", [([3, 3, 2], [1, 2, 1], 4, 1, 0.05), ([2, 3, 3], [1, 1, 2], 4, 2, 0.2),
                                                   ([4, 4, 4, 4], [1, 1, 1, 1], 4, 1, 0.002)])
def test_compressed_sigma_equals_dense_sigma_on_its_support(fci_lib, spaces, ref, nel, T, frac):
    """Lossless categorical compression (Results; Methods, compression preservation): the
    compressed sigma holds exactly the dense FP64 sigma of the same vector on its support,
    bit for bit, the dense sigma is zero everywhere else, and both match the oracle."""
    h, g, f = das_gpu(spaces, ref, nel, T, e_core=0.4)
    c = sparse_vector(f, spaces, seed=5, keep_frac=frac)
    nz = np.flatnonzero(c)
    assert 0 < len(nz) < f.n_det
    addr, val = f.sigma_compressed(torch.from_numpy(nz), torch.from_numpy(c[nz]))
    addr, val = addr.cpu().numpy(), val.cpu().numpy()
    assert np.all(np.diff(addr) > 0) and addr[0] >= 0 and addr[-1] < f.n_det
    assert set(nz.tolist()) <= set(addr.tolist())  # the diagonal keeps every nonzero C_K
    dense = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    assert np.array_equal(val, dense[addr])
    off = np.ones(f.n_det, bool)
    off[addr] = False
    assert np.all(dense[off] == 0.0)
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    assert rel_inf(dense, oracle.sigma(hso, gso, dets, c, e_core=0.4)) <= SIGMA_RTOL


@pytest.mark.parametrize("spaces,ref,nel,T,frac", [([3, 3, 2], [1, 2, 1], 4, 1, 0.02), ([2, 3, 3], [1, 1, 2], 4, 2, 0.01)])
def test_compressed_sigma_against_the_oracles_algorithm_1(fci_lib, spaces, ref, nel, T, frac):
    """The oracle's Algorithm 1 (compressed C as per-category V/A arrays, exponential
    search, a table keyed by target address) gives the same support, address for address,
    and the same values to the FP64 tolerance."""
    h, g, f = das_gpu(spaces, ref, nel, T, e_core=0.4)
    c = synth.random_vector(f.n_det, seed=5)
    c[synth.Stream(5, tag=3).uniform(f.n_det) >= frac] = 0.0
    nz = np.flatnonzero(c)
    addr, val = f.sigma_compressed(torch.from_numpy(nz), torch.from_numpy(c[nz]))
    addr, val = addr.cpu().numpy(), val.cpu().numpy()
    ref_s = alg1.sigma_alg1(h, g, 0.4, spaces, ref, ref, nel, nel, T, alg1.compress(c, spaces, ref, ref, nel, nel, T))
    ref_addr = np.array(sorted(ref_s))
    assert np.array_equal(addr, ref_addr)
    ref_val = np.array([ref_s[a] for a in ref_addr])
    assert rel_inf(val, ref_val) <= SIGMA_RTOL


def test_compressed_sigma_edge_cases(fci_lib):
    h, g, f = das_gpu([3, 3, 2], [1, 2, 1], 4, 1)
    a, v = f.sigma_compressed(torch.zeros(0, dtype=torch.int64), torch.zeros(0, dtype=torch.float64))
    assert a.numel() == 0 and v.numel() == 0
    # one coefficient
    c = np.zeros(f.n_det)
    c[7] = 1.0
    a, v = f.sigma_compressed(torch.tensor([7]), torch.tensor([1.0]))
    dense = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    assert np.array_equal(v.cpu().numpy(), dense[a.cpu().numpy()])
    assert np.count_nonzero(dense) <= a.numel()
    # addresses must be ascending target addresses
    with pytest.raises(fci.FCIError) as e:
        f.sigma_compressed(torch.tensor([9, 7]), torch.tensor([1.0, 2.0]))
    assert e.value.code == fci.FCI_ERR_ARG
    with pytest.raises(fci.FCIError):
        f.sigma_compressed(torch.tensor([f.n_det]), torch.tensor([1.0]))
    # too small an output: the size needed is reported with FCI_ERR_ARG
    with pytest.raises(fci.FCIError) as e:
        f.sigma_compressed(torch.tensor([7]), torch.tensor([1.0]), capacity=1)
    assert e.value.code == fci.FCI_ERR_ARG


def test_compressed_sigma_24_orbitals_4x6(fci_lib):
    """The literal 4 x 6 space: 24 orbitals, 12 alpha + 12 beta electrons, <= 2 transfers
    (253 categories, 1,897,456,000,000 determinants; a dense vector would take 15 TB).  A C
    with 400 nonzero coefficients (a stated sparsity of 2.1e-10, spread over the categories
    by a seeded draw of addresses) gives sigma on its support; sampled entries of it match the
    oracle's Slater-Condon sigma of the same sparse vector."""
    spaces, ref, nel, T = [6, 6, 6, 6], [3, 3, 3, 3], 12, 2
    w = synth.WORKLOADS["das_24o_4x6"]
    h, g = synth.real_integrals(24, w["n_chol"], w["seed"])
    f = fci.FCI(0).setup_integrals(h, g).build_strings(nel, nel).build_das(spaces, ref, ref, T)
    N = f.n_det
    assert N == 1897456000000
    st = synth.Stream(17)
    nz = np.unique((st.uniform(400) * N).astype(np.int64))
    cv = st.normal(len(nz))
    cv /= np.linalg.norm(cv)
    addr, val = f.sigma_compressed(torch.from_numpy(nz), torch.from_numpy(cv))
    addr, val = addr.cpu().numpy(), val.cpu().numpy()
    f.close()
    assert np.all(np.diff(addr) > 0) and set(nz.tolist()) <= set(addr.tolist())
    # oracle: sigma_L = sum over the nonzero K of H_LK C_K for sampled L of the support
    pick = np.unique(np.concatenate([(synth.Stream(19).uniform(48) * len(addr)).astype(np.int64),
                                     np.searchsorted(addr, nz[:16])]))
    rows_addr = addr[pick]
    both = np.union1d(nz, rows_addr)
    dets = odas.dets_of_addresses(spaces, ref, ref, nel, nel, T, both)
    cfull = np.zeros(len(both))
    cfull[np.searchsorted(both, nz)] = cv
    hso, gso = oracle.spin_orbital_integrals(h, g)
    ref_rows = oracle.sigma(hso, gso, dets, cfull, rows=np.searchsorted(both, rows_addr))
    scale = np.max(np.abs(val))
    assert np.max(np.abs(val[pick] - ref_rows)) / scale <= SIGMA_RTOL
