"""Host-side failure paths of libfci (no GPU fault is involved): injected device
allocation failures and a Davidson solve that runs out of iterations."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_20375_gb300 import synth

from helpers import fci_problem, gpu_fci

pytestmark = pytest.mark.gpu


def _das_sequence(fci, h, g):
    """Every allocating call of a DAS problem: handle, strings, categories, FP64 and split
    sigma (the split path builds its operand tables on first use)."""
    f = fci.FCI(0)
    try:
        f.setup_integrals(h, g).build_strings(4, 4).build_das([3, 3, 2], [1, 2, 1], [1, 2, 1], 1)
        c = torch.from_numpy(synth.random_vector(f.n_det, seed=7)).cuda()
        s64 = f.sigma(c).cpu().numpy()
        s3 = f.sigma(c, precision="oz_bf16", n_slices=3).cpu().numpy()
        f.sync_status()
        return s64, s3
    finally:
        f.close()


def _free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failures_return_oom_and_leak_nothing(fci_lib, monkeypatch):
    """FCI_FAULT_ALLOC_AT=n fails the n-th device allocation: every call that allocates
    returns FCI_ERR_OOM (raised by the binding), the handle is still destroyed cleanly,
    the device's free memory does not shrink, and an uninjected run gives the same bits."""
    fci = fci_lib
    h, g = synth.real_integrals(8, 9, 31)
    ref64, ref3 = _das_sequence(fci, h, g)  # warm-up: kernel images, torch allocator
    free0 = _free_bytes()
    failed = 0
    for n in range(1, 200):
        monkeypatch.setenv("FCI_FAULT_ALLOC_AT", str(n))
        try:
            out = _das_sequence(fci, h, g)
        except fci.FCIError as e:
            assert e.code == fci.FCI_ERR_OOM, (n, str(e))
            assert "injected" in str(e)
            failed += 1
            continue
        finally:
            monkeypatch.delenv("FCI_FAULT_ALLOC_AT")
        # n is past the last allocation: the run completes and matches the reference
        assert np.array_equal(out[0], ref64) and np.array_equal(out[1], ref3)
        break
    else:
        pytest.fail("the sequence never completed")
    assert failed >= 10  # handle, strings, tables, categories and split operands all allocate
    free1 = _free_bytes()
    assert free1 >= free0 - (4 << 20), (free0, free1)
    # a second round of the same failures leaves the free memory where it was
    for n in range(1, failed + 1):
        monkeypatch.setenv("FCI_FAULT_ALLOC_AT", str(n))
        with pytest.raises(fci.FCIError):
            _das_sequence(fci, h, g)
        monkeypatch.delenv("FCI_FAULT_ALLOC_AT")
    assert _free_bytes() >= free1 - (4 << 20)


def test_davidson_out_of_iterations_returns_best_ritz_pair(fci_lib):
    """max_iter reached: FCI_ERR_NOT_CONVERGED (the binding reports converged = False), the
    log holds max_iter iterations, and the returned pair is the current Ritz pair: a unit
    vector whose Rayleigh quotient (oracle's dense H) is the returned energy, above the
    exact ground state, with the logged residual norm."""
    p = fci_problem(6, 3, 3, n_chol=8, seed=13, e_core=0.4)
    f = gpu_fci(p)
    r = f.davidson(max_iter=3, tol_residual=1e-12, tol_energy=1e-14)
    assert not r.converged
    assert len(r.iterations) == 3 and r.n_sigma >= 3
    H = oracle.dense_h(p["hso"], p["gso"], p["dets"]).real + 0.4 * np.eye(len(p["dets"]))
    c = r.vector.cpu().numpy()
    assert abs(np.linalg.norm(c) - 1.0) < 1e-12
    rq = float(c @ H @ c)
    assert abs(rq - r.energy) < 1e-10
    assert r.energy >= np.linalg.eigvalsh(H)[0] - 1e-12
    assert abs(r.energy - r.iterations[-1]["energy"]) < 1e-12
    assert abs(np.linalg.norm(H @ c - rq * c) - r.iterations[-1]["residual_norm"]) < 1e-8
