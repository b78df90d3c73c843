"""GPU tests of the split-precision (tcgen05) sigma on the STP-DAS layout."""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import das as odas
from paper_2505_20375_gb300 import fci, synth

from helpers import ENERGY_TOL, gpu_fci, rel_inf
from ozaki_model import das_sigma_model
from test_split_model import DZ_TOL

pytestmark = pytest.mark.gpu


def das_gpu(spaces, ref, nel, T, n_chol=9, seed=31, e_core=0.0):
    n = sum(spaces)
    h, g = synth.real_integrals(n, n_chol, seed)
    f = gpu_fci(dict(h=h, g=g, e_core=e_core, n=n, na=nel, nb=nel))
    f.build_das(spaces, ref, ref, T)
    return h, g, f


CASES = [([2, 2, 2], [1, 1, 1], 3, 1), ([3, 3, 2], [1, 2, 1], 4, 1), ([2, 3, 3], [1, 1, 2], 4, 2),
         ([4, 4, 4], [2, 1, 1], 4, 0),
         ([4, 4, 4, 4], [1, 1, 0, 0], 2, 1)]  # 16 orbitals: 136 pair rows, N = K = 144


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("spaces,ref,nel,T", CASES)
def test_das_split_equals_exact_integer_model(fci_lib, spaces, ref, nel, T, s):
    """Level sums exact in TMEM, E rounded to FP32 exactly as the model does, int64
    scatter: the GPU sigma equals the model to the rounding of the final scaling."""
    h, g, f = das_gpu(spaces, ref, nel, T, e_core=0.3)
    c = synth.random_vector(f.n_det, seed=7)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    f.sync_status()
    m = das_sigma_model(h, g, spaces, ref, nel, T, c, s, e_core=0.3)
    assert rel_inf(sg, m) <= 1e-14


@pytest.mark.parametrize("s", [2, 3])
def test_das_split_serving_problem_vs_oracle_sampled(fci_lib, s):
    """16 orbitals in 4 spaces, 4 alpha + 4 beta, <= 1 transfer: 655,360 determinants,
    2,191,360 in the intermediate space (17,120 tiles of 128, ragged last tile)."""
    w = synth.WORKLOADS["das_16o_4x4_8e"]
    h, g, f = das_gpu(w["spaces"], w["ref"], 4, w["max_transfer"], n_chol=w["n_chol"], seed=w["seed"])
    dets, _ = odas.das_dets(w["spaces"], w["ref"], w["ref"], 4, 4, w["max_transfer"])
    c = synth.random_vector(len(dets), seed=7)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    f.sync_status()
    hso, gso = oracle.spin_orbital_integrals(h, g)
    st = synth.Stream(5)
    rows = np.concatenate([np.unique((st.uniform(150) * len(dets)).astype(np.int64)), [0, len(dets) - 1]])
    ref = oracle.sigma(hso, gso, dets, c, rows=rows)
    s64 = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    assert np.max(np.abs(sg[rows] - ref)) / np.max(np.abs(s64)) <= DZ_TOL[s]
    assert rel_inf(sg, s64) <= DZ_TOL[s]


def test_das_split_chunked_equals_single_pass(fci_lib, monkeypatch):
    """Several intermediate chunks (int64 partial sums kept across chunks) give the same
    bits as one pass."""
    h, g, f = das_gpu([3, 3, 2], [1, 2, 1], 4, 1, e_core=-0.2)
    c = torch.from_numpy(synth.random_vector(f.n_det, seed=3)).cuda()
    one = f.sigma(c, precision="oz_bf16", n_slices=3).clone()
    monkeypatch.setenv("FCI_DAS_CHUNK_DETS", "700")
    assert f.sigma_workspace_bytes("oz_bf16", 3) > 0
    many = f.sigma(c, precision="oz_bf16", n_slices=3).clone()
    f.sync_status()
    assert torch.equal(one, many)


def test_das_split_grouped_equals_individual(fci_lib):
    """DAS split jobs share one contraction launch; alpha/beta split and FP64 jobs in the
    same call take their own paths; every result equals its own call bit for bit."""
    probs = [das_gpu([3, 3, 2], [1, 2, 1], 4, 1, seed=41), das_gpu([2, 3, 3], [1, 1, 2], 4, 2, seed=42),
             das_gpu([4, 4, 4, 4], [1, 1, 0, 0], 2, 1, seed=43)]
    fs = [p[2] for p in probs]
    h, g = synth.real_integrals(8, 9, 44)
    ff = fci.FCI(0).setup_integrals(h, g).build_strings(4, 4)
    fs.append(ff)
    precs = [("oz_bf16", 3), ("oz_bf16", 3), ("oz_bf16", 3), ("oz_bf16", 6)]
    Cs = [torch.from_numpy(synth.random_vector(f.n_det, seed=9 + i)).cuda() for i, f in enumerate(fs)]
    ref = [f.sigma(C, precision=pr, n_slices=sl).clone() for f, C, (pr, sl) in zip(fs, Cs, precs)]
    outs = [torch.full_like(C, float("nan")) for C in Cs]
    keep, jobs = [], []
    for f, C, o, (pr, sl) in zip(fs, Cs, outs, precs):
        nb = f.sigma_workspace_bytes(pr, sl)
        buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        keep.append(buf)
        jobs.append((f, C, o, pr, sl, (buf.data_ptr() + 255) & ~255, nb))
    fci.sigma_grouped(jobs)
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)


def test_das_split_rejects_unsupported_slices(fci_lib):
    """16 orbitals (136 pairs): 8 slices could push a level sum past 2^24 (8 x 136 > 1023)."""
    _, _, f = das_gpu([4, 4, 4, 4], [1, 1, 0, 0], 2, 1)
    c = torch.zeros(f.n_det, dtype=torch.float64, device="cuda")
    with pytest.raises(fci.FCIError, match="2\\^24"):
        f.sigma(c, precision="oz_bf16", n_slices=8)
    with pytest.raises(fci.FCIError, match="2\\^24"):
        f.davidson(precision="oz_bf16", n_slices=3, final_precision="oz_bf16", final_slices=8)


def test_das_mixed_davidson_matches_fp64_and_dense(fci_lib):
    """Split s=3 sigma until ||r|| < 1e-4, then the FP64 path: the same energy as the
    FP64 solve and as dense diagonalisation."""
    spaces, ref, nel, T = [3, 3, 2], [1, 2, 1], 4, 1
    n = sum(spaces)
    h, g, f = das_gpu(spaces, ref, nel, T, seed=61, e_core=-1.0)
    r64 = f.davidson(tol_residual=1e-6, tol_energy=1e-10)
    rmx = f.davidson(tol_residual=1e-6, tol_energy=1e-10, precision="oz_bf16", n_slices=3, switch_residual=1e-4,
                     final_precision="fp64")
    assert r64.converged and rmx.converged
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    H = oracle.dense_h(hso, gso, dets).real
    e0 = np.linalg.eigvalsh(H)[0] - 1.0
    assert abs(r64.energy - e0) < ENERGY_TOL
    assert abs(rmx.energy - e0) < ENERGY_TOL


@pytest.mark.parametrize("cfg", ["6,12", "6,8", "4,8", "2,8"])
def test_das_split_kernel_configs_agree(fci_lib, monkeypatch, cfg):
    """Every K-chunk width / producer-warp count gives the same bits (integer path)."""
    h, g, f = das_gpu([4, 4, 4, 4], [1, 1, 0, 0], 2, 1, seed=45)
    h2, g2, f2 = das_gpu([3, 3, 2], [1, 2, 1], 4, 1, seed=46)
    outs = []
    for env in (None, cfg):
        if env:
            monkeypatch.setenv("FCI_DZ_CONFIG", env)
        for ff in (f, f2):
            c = torch.from_numpy(synth.random_vector(ff.n_det, seed=5)).cuda()
            outs.append(ff.sigma(c, precision="oz_bf16", n_slices=3).clone())
    assert torch.equal(outs[0], outs[2]) and torch.equal(outs[1], outs[3])


# ------------------------------------------------ two-pass form (FP64-class slice counts)

@pytest.mark.parametrize("s", [4, 5, 6, 7])
@pytest.mark.parametrize("spaces,ref,nel,T", CASES)
def test_das_two_pass_split_equals_exact_integer_model(fci_lib, spaces, ref, nel, T, s):
    """4 to 7 slices on the DAS layout (digit image of D, bulk-copy GEMM with pair rows on
    M, exact int64 E, integer scatter): the GPU sigma equals the exact-integer model to the
    rounding of the inputs (1e-13, as for the alpha/beta two-pass form: at 6 and 7 slices
    the fixed-point G keeps 46 to 54 bits, so the last bit of the FP64 operator, which the
    library and the model assemble in different orders, reaches it)."""
    h, g, f = das_gpu(spaces, ref, nel, T, e_core=0.3)
    c = synth.random_vector(f.n_det, seed=7)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    f.sync_status()
    m = das_sigma_model(h, g, spaces, ref, nel, T, c, s, e_core=0.3)
    assert rel_inf(sg, m) <= (1e-14 if s <= 5 else 1e-13)


@pytest.mark.parametrize("s", [6, 7])
@pytest.mark.parametrize("spaces,ref,nel,T", [([3, 3, 2], [1, 2, 1], 4, 1), ([4, 4, 4, 4], [1, 1, 0, 0], 2, 1)])
def test_das_two_pass_split_reaches_the_fp64_bar(fci_lib, spaces, ref, nel, T, s):
    """6 and 7 slices: within 1e-11 of the oracle's sigma (the FP64 parity bar)."""
    from helpers import SIGMA_RTOL

    h, g, f = das_gpu(spaces, ref, nel, T, seed=71, e_core=-0.6)
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    c = synth.random_vector(len(dets), seed=7)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    f.sync_status()
    assert rel_inf(sg, oracle.sigma(hso, gso, dets, c, e_core=-0.6)) <= SIGMA_RTOL


def test_das_two_pass_chunks_and_pieces_equal_single_pass(fci_lib, monkeypatch):
    """E in several chunks (int64 partial sums kept across chunks) and the digit image in
    several pieces per chunk give the same bits as one pass."""
    h, g, f = das_gpu([3, 3, 2], [1, 2, 1], 4, 1, e_core=-0.2)
    c = torch.from_numpy(synth.random_vector(f.n_det, seed=3)).cuda()
    one = f.sigma(c, precision="oz_bf16", n_slices=6).clone()
    monkeypatch.setenv("FCI_DAS_CHUNK_DETS", "700")
    monkeypatch.setenv("FCI_DAS_IMAGE_DETS", "150")
    many = f.sigma(c, precision="oz_bf16", n_slices=6).clone()
    f.sync_status()
    assert f.info["n_det_intermediate"] > 2 * 704  # at least three E chunks
    assert torch.equal(one, many)


def test_das_mixed_davidson_with_split_correction_phase(fci_lib):
    """3-slice sigma until ||r|| < 1e-4, then the 6-slice two-pass form as the FP64-class
    correction phase: the energy of the lowest eigenvalue of the oracle's dense H, and of the
    FP64 solve."""
    spaces, ref, nel, T = [3, 3, 2], [1, 2, 1], 4, 1
    h, g, f = das_gpu(spaces, ref, nel, T, seed=61, e_core=-1.0)
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10, precision="oz_bf16", n_slices=3, switch_residual=1e-4,
                   final_precision="oz_bf16", final_slices=6)
    r64 = f.davidson(tol_residual=1e-6, tol_energy=1e-10)
    assert r.converged and r64.converged
    assert [it["precision"] for it in r.iterations][-1] == 1
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    e0 = np.linalg.eigvalsh(oracle.dense_h(hso, gso, dets).real)[0] - 1.0
    assert abs(r.energy - e0) < ENERGY_TOL and abs(r.energy - r64.energy) < ENERGY_TOL


def test_das_two_pass_grouped_call_equals_individual(fci_lib):
    """A DAS job with 6 slices in a grouped call (it runs on its own) beside fused DAS jobs
    gives the bits of its own call."""
    probs = [das_gpu([3, 3, 2], [1, 2, 1], 4, 1, seed=41), das_gpu([2, 3, 3], [1, 1, 2], 4, 2, seed=42)]
    fs = [p[2] for p in probs]
    precs = [("oz_bf16", 6), ("oz_bf16", 3)]
    Cs = [torch.from_numpy(synth.random_vector(f.n_det, seed=9 + i)).cuda() for i, f in enumerate(fs)]
    ref = [f.sigma(C, precision=pr, n_slices=sl).clone() for f, C, (pr, sl) in zip(fs, Cs, precs)]
    outs = [torch.full_like(C, float("nan")) for C in Cs]
    keep, jobs = [], []
    for f, C, o, (pr, sl) in zip(fs, Cs, outs, precs):
        nb = f.sigma_workspace_bytes(pr, sl)
        buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        keep.append(buf)
        jobs.append((f, C, o, pr, sl, (buf.data_ptr() + 255) & ~255, nb))
    fci.sigma_grouped(jobs)
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)
