"""fci_sigma_noalloc: the FP64 sigma build for callers that cannot allocate device memory
when they need it (a framework that already reserved the memory pool, a host callback
on a stream, a loop that must not risk cudaMalloc's implicit synchronisation).

It is called here through the C ABI directly and compared with fci_sigma, which uses a
caller workspace, on two calls in a row with different vectors (the shared static
scratch keeps the previous call's contents, which must not leak into the next result).
This file is collected last so that a run stopping at the first failure has already
run every other test; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2505_20375_gb300 import synth

from helpers import SIGMA_RTOL, fci_problem, gpu_fci, rel_inf, spinor_problem

pytestmark = pytest.mark.gpu


def _noalloc(f, C, out):
    from paper_2505_20375_gb300 import fci

    fn = fci._lib.fci_sigma_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    rc = fn(f._h, ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


@pytest.mark.parametrize("kind", ["fci_8e8o", "spinor_10s5e"])
def test_noalloc_matches_workspace_sigma_twice(fci_lib, kind):
    if kind == "fci_8e8o":
        w = synth.WORKLOADS["fci_8e8o"]
        p = fci_problem(w["n"], w["na"], w["nb"], w["n_chol"], w["seed"], e_core=0.25)
        cplx = False
    else:
        p = spinor_problem(10, 5, n_chol=6, seed=17, e_core=0.25)
        cplx = True
    f = gpu_fci(p)
    N = len(p["dets"])
    for seed in (7, 8):  # two calls in a row through the shared scratch
        c = torch.from_numpy(synth.random_vector(N, seed=seed, complex_=cplx)).cuda()
        ref = f.sigma(c).cpu().numpy()
        out = torch.full_like(c, float("nan"))
        assert _noalloc(f, c, out) == 0, fci_lib.last_error(f._h)
        torch.cuda.synchronize()
        assert rel_inf(out.cpu().numpy(), ref) <= SIGMA_RTOL


def test_noalloc_rejects_sizes_above_its_static_maximum(fci_lib):
    """FCI(12e,12o) needs 2 x 78 x 853,776 x 8 bytes of scratch (about 1 GB) > 64 MiB."""
    p = fci_problem(12, 6, 6, n_chol=2, seed=1)
    f = gpu_fci(p)
    c = torch.zeros(len(p["dets"]), dtype=torch.float64, device="cuda")
    out = torch.empty_like(c)
    rc = _noalloc(f, c, out)
    assert rc == fci_lib.FCI_ERR_ARG
    assert "static maximum" in fci_lib.last_error(f._h)
