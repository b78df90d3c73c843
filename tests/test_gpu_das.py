"""GPU tests of the STP-DAS categorical layout and sigma (FP64 path) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import das as odas
from paper_2505_20375_gb300 import synth

from helpers import ENERGY_TOL, SIGMA_RTOL, gpu_fci, rel_inf

pytestmark = pytest.mark.gpu


def das_problem(spaces, ref, nel, T, n_chol=8, seed=3, e_core=0.0):
    n = sum(spaces)
    h, g = synth.real_integrals(n, n_chol, seed)
    p = dict(h=h, g=g, e_core=e_core, n=n, na=nel, nb=nel)
    f = gpu_fci(p)
    f.build_das(spaces, ref, ref, T)
    return p, f


def _cat_table(f, S):
    t = f.table("das_categories").cpu().numpy().reshape(-1, 2 * S + 3)
    return [(tuple(r[:S]), tuple(r[S:2 * S]), int(r[2 * S]), int(r[2 * S + 1]), int(r[2 * S + 2])) for r in t]


@pytest.mark.parametrize("spaces,ref,nel,T", [
    ([2, 2, 2], [1, 1, 1], 3, 1),
    ([4, 4, 4, 4], [2, 2, 2, 2], 8, 2),     # 16-orbital stand-in of the 24-orbital case
    ([4, 4, 4, 4], [1, 1, 1, 1], 4, 1),     # 16-orbital, 8-electron serving problem
    ([6, 6, 6, 6], [3, 3, 3, 3], 12, 2),    # 24 orbitals in 4 x 6, 24 electrons, <= 2 transfers
    ([3, 3, 2], [1, 2, 1], 4, 1),
])
def test_das_categories_match_oracle(fci_lib, spaces, ref, nel, T):
    p, f = das_problem(spaces, ref, nel, T, n_chol=2)
    cats, total = odas.categories(spaces, ref, ref, nel, nel, T)
    got = _cat_table(f, len(spaces))
    assert got == [(tuple(a), tuple(b), na, nb, off) for a, b, na, nb, off in cats]
    assert f.info["n_det"] == total
    if spaces == [6, 6, 6, 6]:
        assert len(cats) == 253 and total > 10 ** 12


@pytest.mark.parametrize("spaces,ref,nel,T", [([2, 2, 2], [1, 1, 1], 3, 1), ([3, 3, 2], [1, 2, 1], 4, 1),
                                              ([4, 4, 4, 4], [1, 1, 1, 1], 4, 1)])
def test_das_addresses_match_oracle_order(fci_lib, spaces, ref, nel, T):
    p, f = das_problem(spaces, ref, nel, T, n_chol=2)
    n = sum(spaces)
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    sa = oracle.enumerate_strings(n, nel)
    pos = {int(x): i for i, x in enumerate(sa)}
    mask = (1 << n) - 1
    ref_addr = np.array([pos[int(d) & mask] * len(sa) + pos[int(d) >> n] for d in dets])
    got = f.table("das_address").cpu().numpy()
    assert np.array_equal(got, ref_addr)


@pytest.mark.parametrize("spaces,ref,nel,T,seed", [([2, 2, 2], [1, 1, 1], 3, 1, 31), ([3, 3, 2], [1, 2, 1], 4, 1, 32),
                                                   ([2, 3, 3], [1, 1, 2], 4, 2, 33), ([4, 4, 4], [2, 1, 1], 4, 0, 34)])
def test_das_sigma_fp64_parity(fci_lib, spaces, ref, nel, T, seed):
    p, f = das_problem(spaces, ref, nel, T, n_chol=9, seed=seed, e_core=0.3)
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    hso, gso = oracle.spin_orbital_integrals(p["h"], p["g"])
    c = synth.random_vector(len(dets), seed=7)
    s = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    refv = oracle.sigma(hso, gso, dets, c, e_core=0.3)
    assert rel_inf(s, refv) <= SIGMA_RTOL
    d = f.diagonal().cpu().numpy()
    assert np.max(np.abs(d - (oracle.diag(hso, gso, dets) + 0.3))) < 1e-12


def test_das_16o_8e_serving_problem_sampled_rows(fci_lib):
    """16 orbitals in 4 spaces, 4 alpha + 4 beta, <= 1 transfer (655,360 determinants)."""
    w = synth.WORKLOADS["das_16o_4x4_8e"]
    p, f = das_problem(w["spaces"], w["ref"], 4, w["max_transfer"], n_chol=w["n_chol"], seed=w["seed"])
    dets, _ = odas.das_dets(w["spaces"], w["ref"], w["ref"], 4, 4, w["max_transfer"])
    assert len(dets) == f.n_det == 655360
    hso, gso = oracle.spin_orbital_integrals(p["h"], p["g"])
    c = synth.random_vector(len(dets), seed=7)
    s = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    st = synth.Stream(5)
    rows = np.concatenate([np.unique((st.uniform(200) * len(dets)).astype(np.int64)), [0, len(dets) - 1]])
    refv = oracle.sigma(hso, gso, dets, c, rows=rows)
    assert np.max(np.abs(s[rows] - refv)) / np.max(np.abs(s)) <= SIGMA_RTOL


def test_das_sigma_is_fci_sigma_of_padded_vector_bit_for_bit(fci_lib):
    """Lossless categorical compression (Results; compression preservation, Methods):
    the DAS sigma equals, bit for bit, the FCI sigma of the zero-padded vector on the
    DAS determinants, also when whole categories of C are zero (skipped)."""
    spaces, ref, nel, T = [3, 3, 2], [1, 2, 1], 4, 1
    n = sum(spaces)
    h, g = synth.real_integrals(n, 8, 51)
    from paper_2505_20375_gb300 import fci

    fd = fci.FCI(0).setup_integrals(h, g).build_strings(nel, nel).build_das(spaces, ref, ref, T)
    ff = fci.FCI(0).setup_integrals(h, g).build_strings(nel, nel)
    addr = fd.table("das_address").cpu().numpy()
    cats = _cat_table(fd, len(spaces))
    c = synth.random_vector(fd.n_det, seed=7)
    for k, (_, _, na, nb, off) in enumerate(cats):
        if k % 3 == 1:
            c[off:off + na * nb] = 0.0
    sd = fd.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    cf = np.zeros(ff.n_det)
    cf[addr] = c
    sf = ff.sigma(torch.from_numpy(cf).cuda()).cpu().numpy()
    assert np.array_equal(sd, sf[addr])


def test_das_davidson_matches_dense_eigh(fci_lib):
    spaces, ref, nel, T = [3, 3, 2], [1, 2, 1], 4, 1
    p, f = das_problem(spaces, ref, nel, T, n_chol=9, seed=61, e_core=-1.0)
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    hso, gso = oracle.spin_orbital_integrals(p["h"], p["g"])
    H = oracle.dense_h(hso, gso, dets).real
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10)
    assert r.converged
    assert abs(r.energy - (np.linalg.eigvalsh(H)[0] - 1.0)) < ENERGY_TOL


def test_das_fp64_several_chunks_matches_oracle(fci_lib, monkeypatch):
    """The FP64 DAS sigma in several passes over the intermediate space (each pass adds
    its part of sigma): capped at a quarter of the intermediate determinants it takes at
    least three passes, and matches the oracle as the single pass does."""
    spaces, ref, nel, T = [3, 3, 2], [1, 2, 1], 4, 1
    p, f = das_problem(spaces, ref, nel, T, n_chol=9, seed=37, e_core=0.3)
    dets, cats = odas.das_dets(spaces, ref, ref, nel, nel, T)
    hso, gso = oracle.spin_orbital_integrals(p["h"], p["g"])
    c = synth.random_vector(len(dets), seed=7)
    refv = oracle.sigma(hso, gso, dets, c, e_core=0.3)
    cd = torch.from_numpy(c).cuda()
    one = f.sigma(cd).cpu().numpy()
    n_int = f.info["n_det_intermediate"]
    largest = max(na * nb for _, _, na, nb, _ in cats)
    cap = max(n_int // 4, largest)
    monkeypatch.setenv("FCI_DAS_FP64_CHUNK_DETS", str(cap))
    f.set_phase_timing(True)
    f.phase_times(reset=True)
    many = f.sigma(cd).cpu().numpy()
    passes = f.phase_times(reset=True)["contract"]["launches"]
    f.set_phase_timing(False)
    assert passes >= 3
    assert rel_inf(many, refv) <= SIGMA_RTOL
    assert rel_inf(one, refv) <= SIGMA_RTOL
    assert rel_inf(many, one) <= 1e-13


@pytest.fixture(scope="module")
def das_16e():
    """16 orbitals in 4 spaces of 4, 8 alpha + 8 beta electrons, <= 2 transfers: 253
    categories, 78,444,288 determinants (138,495,744 in the intermediate space)."""
    import oracle as _or

    w = synth.WORKLOADS["das_16o_4x4"]
    h, g = synth.real_integrals(w["n"], w["n_chol"], w["seed"])
    from paper_2505_20375_gb300 import fci

    f = fci.FCI(0).setup_integrals(h, g).build_strings(8, 8).build_das(w["spaces"], w["ref"], w["ref"],
                                                                        w["max_transfer"])
    dets, _ = odas.das_dets(w["spaces"], w["ref"], w["ref"], 8, 8, w["max_transfer"])
    hso, gso = _or.spin_orbital_integrals(h, g)
    c = synth.random_vector(len(dets), seed=7)
    st = synth.Stream(19)
    rows = np.concatenate([np.unique((st.uniform(120) * len(dets)).astype(np.int64)), [0, len(dets) - 1]])
    ref = _or.sigma(hso, gso, dets, c, rows=rows)
    del dets
    s64 = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    yield f, c, rows, ref, s64
    f.close()
    torch.cuda.empty_cache()


def test_das_16e_fp64_sampled_rows(fci_lib, das_16e):
    """The FP64 DAS sigma at 78 M determinants (several passes over the 138 M intermediate
    determinants, each pass within 16 GiB of D and E) on sampled rows the oracle computes."""
    f, c, rows, ref, s64 = das_16e
    assert f.n_det == 78444288
    assert np.max(np.abs(s64[rows] - ref)) / np.max(np.abs(s64)) <= SIGMA_RTOL


@pytest.mark.parametrize("s", [2, 3, 6])
def test_das_16e_split_sampled_rows(fci_lib, das_16e, s):
    """The split-precision DAS sigma at 78 M determinants, in the launch configuration the
    benchmark times, on the same sampled rows: within the per-slice tolerance (the fused
    form at 2 and 3 slices), within the FP64 bar (the two-pass form at 6 slices, E in two
    chunks of the intermediate space)."""
    from test_split_model import DZ_TOL

    DZ_TOL = {**DZ_TOL, 6: SIGMA_RTOL}
    f, c, rows, ref, s64 = das_16e
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    f.sync_status()
    scale = np.max(np.abs(s64))
    assert np.max(np.abs(sg[rows] - ref)) / scale <= DZ_TOL[s]
    assert np.max(np.abs(sg - s64)) / scale <= DZ_TOL[s]
