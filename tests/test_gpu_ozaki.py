"""GPU tests of the split-precision (Ozaki, bf16 slices on tcgen05) sigma path."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2505_20375_gb300 import synth

from helpers import ENERGY_TOL, SIGMA_RTOL, fci_problem, gpu_fci, rel_inf
from ozaki_model import sigma_model

pytestmark = pytest.mark.gpu

# ||sigma_oz - sigma_exact||_inf / ||sigma_exact||_inf bounds per slice count: the
# triangular truncation leaves about 2^-8 per slice, measured by the exact-integer model
# against the oracle; s >= 6 meets the FP64 bar of 1e-11.
OZ_TOL = {2: 2e-3, 3: 2e-5, 4: 1e-7, 5: 5e-10, 6: SIGMA_RTOL, 7: SIGMA_RTOL}


@pytest.mark.parametrize("s", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (9, 4, 3)])
def test_oz_sigma_equals_exact_integer_model(fci_lib, n, na, nb, s):
    """The tensor-core slice products are summed exactly: the GPU result equals the
    exact-integer model of the same split to rounding of the inputs (1e-13), far below
    the 2^-24 a single inexact FP32 accumulation would leave."""
    p = fci_problem(n, na, nb, n_chol=n + 2, seed=3 + n, e_core=0.5)
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=7)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    f.sync_status()
    m = sigma_model(p["h"], p["g"], n, na, nb, c, s, e_core=0.5)
    assert rel_inf(sg, m) <= 1e-13


@pytest.mark.parametrize("s", [2, 3, 4, 5, 6, 7])
def test_oz_sigma_vs_oracle_tolerance(fci_lib, s):
    w = synth.WORKLOADS["fci_8e8o"]
    p = fci_problem(w["n"], w["na"], w["nb"], w["n_chol"], w["seed"])
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=7)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c)
    assert rel_inf(sg, ref) <= OZ_TOL[s]


@pytest.mark.parametrize("n,na,nb", [(1, 1, 1), (2, 1, 1), (5, 0, 3), (7, 7, 6), (10, 5, 5), (11, 6, 4)])
def test_oz_fp64_class_edge_shapes(fci_lib, n, na, nb):
    """Single determinant, empty alpha strings, ragged tiles (N not a multiple of 32)."""
    p = fci_problem(n, na, nb, n_chol=n + 1, seed=40 + n, e_core=-0.3)
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=9)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=7).cpu().numpy()
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c, e_core=-0.3)
    assert rel_inf(sg, ref) <= SIGMA_RTOL


def test_oz_zero_vector_gives_zero(fci_lib):
    p = fci_problem(6, 3, 3)
    f = gpu_fci(p)
    z = torch.zeros(len(p["dets"]), dtype=torch.float64, device="cuda")
    assert torch.count_nonzero(f.sigma(z, precision="oz_bf16", n_slices=6)).item() == 0


def test_oz_14e14o_full_size_sampled_rows(fci_lib):
    """Full 14e/14o workload (N = 11,778,624) with 6 and 7 slices in the benchmark's
    launch configuration, against oracle rows and against the FP64 GPU path."""
    w = synth.WORKLOADS["fci_14e14o"]
    p = fci_problem(w["n"], w["na"], w["nb"], w["n_chol"], w["seed"])
    f = gpu_fci(p)
    N = len(p["dets"])
    c = synth.random_vector(N, seed=7)
    cd = torch.from_numpy(c).cuda()
    s64 = f.sigma(cd).cpu().numpy()
    st = synth.Stream(12)
    rows = np.concatenate([np.unique((st.uniform(200) * N).astype(np.int64)), [0, N - 1]])
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c, rows=rows)
    scale = np.max(np.abs(s64))
    for s in (6, 7):
        so = f.sigma(cd, precision="oz_bf16", n_slices=s).cpu().numpy()
        f.sync_status()
        assert np.max(np.abs(so[rows] - ref)) / scale <= SIGMA_RTOL
        assert np.max(np.abs(so - s64)) / scale <= SIGMA_RTOL


def _stall_case(kind):
    """A small problem on each kernel that waits on mbarriers: the fused alpha/beta
    kernel, the two-pass bulk-copy GEMM (alpha/beta and complex spinor), the DAS kernel."""
    from helpers import spinor_problem

    if kind == "spinor":
        return gpu_fci(spinor_problem(8, 4, n_chol=6, seed=41)), 3, {}
    if kind == "das":
        h, g = synth.real_integrals(8, 9, 31)
        f = gpu_fci(dict(h=h, g=g, e_core=0.0, n=8, na=4, nb=4))
        return f.build_das([3, 3, 2], [1, 2, 1], [1, 2, 1], 1), 3, {}
    return gpu_fci(fci_problem(6, 3, 3)), 4, {"FCI_OZ_PATH": "fused" if kind == "fused" else "gemm"}


@pytest.mark.parametrize("kind", ["fused", "gemm", "spinor", "das"])
def test_oz_bounded_wait_reports_timeout_and_context_survives(fci_lib, monkeypatch, kind):
    """Failure detection without a GPU fault: one side of the pipeline never signals (a
    flag that nothing sets: producers that never mark a slot full, or an MMA thread that
    never consumes a stage), the other side's bounded wait expires, the kernel waits for
    the copies and MMAs it already issued, frees its tensor memory and returns; the host
    reads FCI_ERR_TIMEOUT, sigma is NaN, and the next call gives the same bits as a call
    made before the stall."""
    from paper_2505_20375_gb300 import fci

    f, s, env = _stall_case(kind)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    c = torch.from_numpy(synth.random_vector(f.n_det, seed=7, complex_=f.is_complex)).cuda()
    before = f.sigma(c, precision="oz_bf16", n_slices=s).cpu()
    f.sync_status()
    monkeypatch.setenv("FCI_TEST_STALL_PRODUCER", "1")
    monkeypatch.setenv("FCI_WAIT_TIMEOUT_MS", "50")
    out = f.sigma(c, precision="oz_bf16", n_slices=s)
    with pytest.raises(fci.FCIError) as e:
        f.sync_status()
    assert e.value.code == fci.FCI_ERR_TIMEOUT
    assert torch.isnan(torch.view_as_real(out) if out.is_complex() else out).all()
    f.sync_status()  # the status was cleared by the read
    monkeypatch.delenv("FCI_TEST_STALL_PRODUCER")
    monkeypatch.delenv("FCI_WAIT_TIMEOUT_MS")
    after = f.sigma(c, precision="oz_bf16", n_slices=s).cpu()
    f.sync_status()
    assert torch.equal(before, after)


def test_status_word_survives_workspace_reallocation(fci_lib, monkeypatch):
    """The timeout record lives in the handle, not in the caller's workspace: growing the
    workspace (the binding frees the old buffer) between the failed call and the status
    read neither loses the record nor touches freed memory."""
    from paper_2505_20375_gb300 import fci

    f = gpu_fci(fci_problem(6, 3, 3))
    c = torch.from_numpy(synth.random_vector(f.n_det, seed=7)).cuda()
    monkeypatch.setenv("FCI_OZ_PATH", "fused")
    monkeypatch.setenv("FCI_TEST_STALL_PRODUCER", "1")
    monkeypatch.setenv("FCI_WAIT_TIMEOUT_MS", "50")
    f.sigma(c, precision="oz_bf16", n_slices=2)
    monkeypatch.delenv("FCI_TEST_STALL_PRODUCER")
    monkeypatch.delenv("FCI_WAIT_TIMEOUT_MS")
    torch.cuda.synchronize()
    f._workspace(f._ws_bytes * 4)  # a new, larger buffer; the old one goes back to torch
    f.sigma(c)                     # FP64 sigma: leaves the record alone
    with pytest.raises(fci.FCIError) as e:
        f.sync_status()
    assert e.value.code == fci.FCI_ERR_TIMEOUT


@pytest.mark.parametrize("final", [("fp64", 0), ("oz_bf16", 7), ("oz_bf16", 6)])
def test_mixed_precision_davidson_reaches_fp64_energy(fci_lib, final):
    """3-slice sigma until ||r|| <= 1e-4, then the residual correction with an FP64-class
    sigma: the energy matches dense diagonalisation within 1e-8 Eh."""
    w = synth.WORKLOADS["fci_8e8o"]
    p = fci_problem(w["n"], w["na"], w["nb"], w["n_chol"], w["seed"])
    f = gpu_fci(p)
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10, precision="oz_bf16", n_slices=3, switch_residual=1e-4,
                   final_precision=final[0], final_slices=final[1])
    assert r.converged
    precs = [it["precision"] for it in r.iterations]
    assert precs[0] == 1 and precs[-1] == (0 if final[0] == "fp64" else 1)
    H = oracle.dense_h(p["hso"], p["gso"], p["dets"]).real
    assert abs(r.energy - np.linalg.eigvalsh(H)[0]) < ENERGY_TOL


@pytest.mark.parametrize("sl", [6, 7])
def test_oz_davidson_fp64_class_throughout(fci_lib, sl):
    p = fci_problem(9, 4, 4, n_chol=12, seed=77, e_core=1.5)
    f = gpu_fci(p)
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10, precision="oz_bf16", n_slices=sl, switch_residual=1e-30,
                   final_precision="oz_bf16", final_slices=sl, max_iter=60)
    r64 = f.davidson(tol_residual=1e-6, tol_energy=1e-10)
    assert r.converged and r64.converged
    assert abs(r.energy - r64.energy) < ENERGY_TOL
