"""GPU tests of the split-precision (tcgen05, bulk-copy fed) sigma for complex spinor strings."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_20375_gb300 import fci, synth

from helpers import ENERGY_TOL, SIGMA_RTOL, gpu_fci, rel_inf, spinor_problem
from ozaki_model import spinor_sigma_model
from test_split_model import CZ_TOL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("s", [2, 3, 5, 8])
@pytest.mark.parametrize("n,ne", [(6, 3), (7, 3), (8, 4), (9, 2)])
def test_cplx_split_equals_exact_integer_model(fci_lib, n, ne, s):
    """Exact FP32 level sums in TMEM, int64 epilogue and scatter: the GPU sigma equals the
    integer model to the rounding of the final scaling (ragged M, K and N tiles)."""
    p = spinor_problem(n, ne, n_chol=n + 2, seed=80 + n, e_core=0.3)
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=7, complex_=True)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    f.sync_status()
    m = spinor_sigma_model(p["h"], p["g"], n, ne, c, s, e_core=0.3)
    assert rel_inf(sg, m) <= 1e-14


@pytest.mark.parametrize("s", [3, 6, 8])
def test_cplx_split_vs_oracle(fci_lib, s):
    p = spinor_problem(10, 5, n_chol=12, seed=91, e_core=-0.4)
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=7, complex_=True)
    sg = f.sigma(torch.from_numpy(c).cuda(), precision="oz_bf16", n_slices=s).cpu().numpy()
    f.sync_status()
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c, e_core=-0.4)
    assert rel_inf(sg, ref) <= CZ_TOL[s]


def test_cplx_split_24_spinors_12_electrons_sampled(fci_lib):
    """The complex configuration: 24 spinors, 12 electrons, 2,704,156 determinants,
    rank-48 complex integrals.  s = 8 meets the FP64 bar against the FP64 path over the
    whole vector and against the oracle on sampled rows."""
    w = synth.WORKLOADS["spinor_24s12e"]
    h, g = synth.complex_integrals(w["n"], w["n_chol"], w["seed"])
    f = fci.FCI(0).setup_integrals(h, g).build_strings(w["ne"], -1)
    N = f.n_det
    assert N == 2704156
    c = synth.random_vector(N, seed=7, complex_=True)
    cd = torch.from_numpy(c).cuda()
    s8 = f.sigma(cd, precision="oz_bf16", n_slices=8).cpu().numpy()
    f.sync_status()
    s64 = f.sigma(cd).cpu().numpy()
    assert rel_inf(s8, s64) <= SIGMA_RTOL
    hso, gso = oracle.spinor_integrals(h, g)
    dets = oracle.spinor_dets(w["n"], w["ne"])
    st = synth.Stream(5)
    rows = np.concatenate([np.unique((st.uniform(60) * N).astype(np.int64)), [0, N - 1]])
    ref = oracle.sigma(hso, gso, dets, c, rows=rows)
    assert np.max(np.abs(s8[rows] - ref)) / np.max(np.abs(s64)) <= SIGMA_RTOL


def test_cplx_mixed_davidson_matches_dense(fci_lib):
    """Split s = 3 until ||r|| < 1e-4, then s = 8 (FP64 class): the energy equals dense
    diagonalisation of the oracle's H."""
    p = spinor_problem(8, 4, n_chol=10, seed=95, e_core=0.7)
    f = gpu_fci(p)
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10, precision="oz_bf16", n_slices=3, switch_residual=1e-4,
                   final_precision="oz_bf16", final_slices=8)
    assert r.converged
    H = oracle.dense_h(p["hso"], p["gso"], p["dets"])
    assert abs(np.linalg.eigvalsh(H)[0] + 0.7 - r.energy) < ENERGY_TOL  # the lowest eigenvalue
    r64 = f.davidson(tol_residual=1e-6, tol_energy=1e-10)
    assert abs(r.energy - r64.energy) < ENERGY_TOL
