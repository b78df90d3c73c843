"""CPU checks of the exact-integer model of the split-precision sigma (the model the GPU
kernels are compared with bit for bit): against the oracle, its error falls by about
2^-8 per slice and stays inside the tolerances the GPU tests use."""
import numpy as np
import pytest

import oracle
from oracle import das as odas
from paper_2505_20375_gb300 import synth

from helpers import fci_problem, rel_inf
from ozaki_model import das_sigma_model, sigma_model, spinor_sigma_model

# ||sigma_split - sigma_exact||_inf / ||sigma_exact||_inf per slice count (alpha/beta strings)
OZ_TOL = {2: 2e-3, 3: 2e-5, 4: 1e-7, 5: 5e-10, 6: 1e-11, 7: 1e-11}
# DAS layout (16 orbitals: 136 pair terms per contraction, E stored in FP32)
DZ_TOL = {2: 5e-3, 3: 5e-5}
# complex spinor strings (balanced base-128 digits: 7 bits per slice)
CZ_TOL = {2: 1e-2, 3: 2e-4, 4: 2e-6, 5: 2e-8, 6: 2e-10, 7: 1e-11, 8: 1e-11}


def test_fci_model_error_falls_with_slices():
    p = fci_problem(6, 3, 3, n_chol=8, seed=11, e_core=0.2)
    c = synth.random_vector(len(p["dets"]), seed=7)
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c, e_core=0.2)
    errs = [rel_inf(sigma_model(p["h"], p["g"], 6, 3, 3, c, s, e_core=0.2), ref) for s in range(2, 8)]
    for s, e in zip(range(2, 8), errs):
        assert e <= OZ_TOL[s], (s, e)
    for a, b in zip(errs[:4], errs[1:5]):
        assert b < a / 30  # about 2^-8 per slice until FP64 rounding is reached


@pytest.mark.parametrize("spaces,ref,nel,T", [([3, 3, 2], [1, 2, 1], 4, 1), ([2, 3, 3], [1, 1, 2], 4, 2)])
@pytest.mark.parametrize("s", [2, 3])
def test_das_model_within_tolerance_of_oracle(spaces, ref, nel, T, s):
    n = sum(spaces)
    h, g = synth.real_integrals(n, 9, 31)
    dets, _ = odas.das_dets(spaces, ref, ref, nel, nel, T)
    c = synth.random_vector(len(dets), seed=7)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    exact = oracle.sigma(hso, gso, dets, c, e_core=-0.4)
    assert rel_inf(das_sigma_model(h, g, spaces, ref, nel, T, c, s, e_core=-0.4), exact) <= DZ_TOL[s]


def test_fp32_storage_of_E_is_below_the_split_error():
    """Rounding each exact E_int to 24 significant bits moves sigma by far less than the
    3-slice truncation does."""
    p = fci_problem(8, 4, 4, n_chol=10, seed=12)
    c = synth.random_vector(len(p["dets"]), seed=7)
    exact = oracle.sigma(p["hso"], p["gso"], p["dets"], c)
    a = sigma_model(p["h"], p["g"], 8, 4, 4, c, 3)
    b = sigma_model(p["h"], p["g"], 8, 4, 4, c, 3, e_fp32=True)
    assert 0 < rel_inf(b, a) < rel_inf(a, exact) / 20


def test_spinor_model_error_falls_with_slices():
    n, ne = 6, 3
    h, g = synth.complex_integrals(n, n + 2, 4)
    hso, gso = oracle.spinor_integrals(h, g)
    dets = oracle.spinor_dets(n, ne)
    c = synth.random_vector(len(dets), seed=7, complex_=True)
    exact = oracle.sigma(hso, gso, dets, c, e_core=0.2)
    errs = [rel_inf(spinor_sigma_model(h, g, n, ne, c, s, e_core=0.2), exact) for s in range(2, 9)]
    for s, e in zip(range(2, 9), errs):
        assert e <= CZ_TOL[s], (s, e)
    for a, b in zip(errs[:5], errs[1:6]):
        assert b < a / 30  # about 2^-7 per slice until FP64 rounding is reached
