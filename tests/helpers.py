"""Shared test set-up: the same seeded inputs handed to the oracle and to libfci."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2505_20375_gb300 import synth

SIGMA_RTOL = 1e-11  # ||sigma_gpu - sigma_oracle||_inf / ||sigma_oracle||_inf, FP64 path
ENERGY_TOL = 1e-8   # Eh


def rel_inf(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def fci_problem(n, na, nb, n_chol=8, seed=1, e_core=0.0):
    h, g = synth.real_integrals(n, n_chol, seed)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    dets = oracle.fci_dets(n, na, nb)
    return dict(h=h, g=g, hso=hso, gso=gso, dets=dets, e_core=e_core, n=n, na=na, nb=nb)


def spinor_problem(n, ne, n_chol=8, seed=4, e_core=0.0):
    h, g = synth.complex_integrals(n, n_chol, seed)
    hso, gso = oracle.spinor_integrals(h, g)
    dets = oracle.spinor_dets(n, ne)
    return dict(h=h, g=g, hso=hso, gso=gso, dets=dets, e_core=e_core, n=n, ne=ne)


def gpu_fci(p, device=0):
    from paper_2505_20375_gb300 import fci

    f = fci.FCI(device)
    f.setup_integrals(p["h"], p["g"], p["e_core"])
    if "ne" in p:
        f.build_strings(p["ne"], -1)
    else:
        f.build_strings(p["na"], p["nb"])
    return f
