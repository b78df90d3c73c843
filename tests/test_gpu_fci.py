"""GPU parity: libfci (through the C ABI) against the oracle on the same seeded inputs."""
from math import comb

import numpy as np
import pytest
import torch

import oracle
from oracle import davidson as odav
from paper_2505_20375_gb300 import synth

from helpers import ENERGY_TOL, SIGMA_RTOL, fci_problem, gpu_fci, rel_inf, spinor_problem

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------------- tables

@pytest.mark.parametrize("n,na,nb", [(1, 1, 0), (4, 2, 2), (8, 4, 4), (9, 4, 3), (12, 6, 5), (14, 7, 7), (16, 8, 8)])
def test_strings_and_replacement_tables_bit_exact(fci_lib, n, na, nb):
    p = fci_problem(n, na, nb, n_chol=2)
    f = gpu_fci(p)
    for spin, ne in (("alpha", na), ("beta", nb)):
        s = f.table("strings_" + spin).cpu().numpy().view(np.uint64)
        ref = oracle.enumerate_strings(n, ne)
        assert np.array_equal(s, ref)
        if ne == 0:
            continue
        t = f.table("repl_" + spin).cpu().numpy().reshape(len(ref), -1, 4)
        o = oracle.replacement_table(n, ne)
        assert t.shape[1] == ne * (n - ne + 1)
        assert np.array_equal(t[..., 0], o["target"])
        assert np.array_equal(t[..., 1], o["a"])
        assert np.array_equal(t[..., 2], o["b"])
        assert np.array_equal(t[..., 3], o["sign"].astype(np.int32))


def test_info_counts(fci_lib):
    f = gpu_fci(fci_problem(14, 7, 7, n_chol=2))
    inf = f.info
    assert inf["n_det"] == comb(14, 7) ** 2 == 11778624
    assert inf["n_pair"] == 105 and inf["n_ent_alpha"] == 7 * 8


# ------------------------------------------------------------------- diagonal

@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (8, 4, 4), (9, 5, 2)])
def test_diagonal(fci_lib, n, na, nb):
    p = fci_problem(n, na, nb, seed=7, e_core=-1.25)
    f = gpu_fci(p)
    d = f.diagonal().cpu().numpy()
    ref = oracle.diag(p["hso"], p["gso"], p["dets"]) + p["e_core"]
    assert np.max(np.abs(d - ref)) < 1e-12


def test_diagonal_alpha_beta_exchange_symmetric(fci_lib):
    """The spin-free H is invariant under exchanging the alpha and beta strings, so with
    n_alpha = n_beta H_(a,b),(a,b) = H_(b,a),(b,a); the diagonal kernel keeps this bit for
    bit (the start vector's tie-break between the two determinants depends on it)."""
    p = fci_problem(8, 4, 4, seed=17, e_core=0.3)
    f = gpu_fci(p)
    d = f.diagonal().cpu().numpy().reshape(70, 70)
    assert np.array_equal(d, d.T)
    ref = oracle.diag(p["hso"], p["gso"], p["dets"]) + p["e_core"]
    assert np.max(np.abs(d.reshape(-1) - ref)) < 1e-12


# ------------------------------------------------------------------- sigma

@pytest.mark.parametrize("n,na,nb", [(1, 1, 1), (2, 1, 1), (3, 2, 1), (5, 0, 3), (6, 3, 3), (8, 4, 4),
                                     (9, 4, 3), (10, 5, 5), (7, 7, 6)])
def test_sigma_fp64_full_parity(fci_lib, n, na, nb):
    p = fci_problem(n, na, nb, n_chol=n + 2, seed=3 + n, e_core=0.5)
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=7)
    s = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c, e_core=p["e_core"])
    assert rel_inf(s, ref) <= SIGMA_RTOL


def test_sigma_fp64_config_8e8o(fci_lib):
    """The 8e/8o workload: 70 x 70 strings, Cholesky rank 16, seed 1."""
    w = synth.WORKLOADS["fci_8e8o"]
    p = fci_problem(w["n"], w["na"], w["nb"], w["n_chol"], w["seed"])
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=7)
    s = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c)
    assert rel_inf(s, ref) <= SIGMA_RTOL


def test_sigma_fp64_batched_and_host_buffers(fci_lib):
    p = fci_problem(6, 3, 2, seed=9)
    f = gpu_fci(p)
    N = len(p["dets"])
    C = np.stack([synth.random_vector(N, seed=s) for s in (1, 2, 3)])
    S = f.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    Sh = f.sigma(torch.from_numpy(C).pin_memory()).numpy()  # host in, host out
    for i in range(3):
        ref = oracle.sigma(p["hso"], p["gso"], p["dets"], C[i])
        assert rel_inf(S[i], ref) <= SIGMA_RTOL
    assert np.array_equal(S, Sh)


def test_sigma_host_buffers_through_the_abi(fci_lib):
    """fci_sigma_host: C and sigma in host memory, pinned or pageable, with the copies
    inside the library call; the result equals the device call bit for bit, FP64 and
    split precision, and lands in the caller's output tensor."""
    p = fci_problem(8, 4, 4, seed=3)
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=4)
    for prec, sl in (("fp64", 0), ("oz_bf16", 6)):
        d = f.sigma(torch.from_numpy(c).cuda(), precision=prec, n_slices=sl).cpu().numpy()
        hp = f.sigma(torch.from_numpy(c).pin_memory(), precision=prec, n_slices=sl).numpy()
        hq = f.sigma(torch.from_numpy(c.copy()), precision=prec, n_slices=sl).numpy()
        assert np.array_equal(d, hp) and np.array_equal(d, hq)
    out = torch.empty(len(p["dets"]), dtype=torch.float64)
    r = f.sigma(torch.from_numpy(c), out=out)
    assert r.data_ptr() == out.data_ptr()
    assert np.array_equal(out.numpy(), f.sigma(torch.from_numpy(c).cuda()).cpu().numpy())
    with pytest.raises(ValueError):
        f.sigma(torch.from_numpy(c), out=torch.empty(3, dtype=torch.float64))
    # a device C takes a device output of its own shape and dtype, never a host one
    cd = torch.from_numpy(c).cuda()
    for bad in (torch.empty(3, dtype=torch.float64, device=cd.device), torch.empty_like(out),
                torch.empty(2 * len(c), dtype=torch.float64, device=cd.device)[::2]):
        with pytest.raises(ValueError):
            f.sigma(cd, out=bad)


def test_sigma_fp64_14e14o_sampled_rows(fci_lib):
    """Full-size 14e/14o (11,778,624 determinants, rank 28, seed 2) in the launch
    configuration the benchmark times, checked on sampled rows the oracle computes one
    by one, plus Hermiticity of the full product <x|Hy> = <Hx|y>."""
    w = synth.WORKLOADS["fci_14e14o"]
    p = fci_problem(w["n"], w["na"], w["nb"], w["n_chol"], w["seed"])
    f = gpu_fci(p)
    N = len(p["dets"])
    c = synth.random_vector(N, seed=7)
    cd = torch.from_numpy(c).cuda()
    s = f.sigma(cd).cpu().numpy()
    st = synth.Stream(11)
    rows = np.unique((st.uniform(300) * N).astype(np.int64))
    rows = np.concatenate([rows, [0, N - 1]])
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c, rows=rows)
    scale = np.max(np.abs(s))
    assert np.max(np.abs(s[rows] - ref)) / scale <= SIGMA_RTOL
    y = synth.random_vector(N, seed=8)
    yd = torch.from_numpy(y).cuda()
    hy = f.sigma(yd)
    lhs = torch.dot(cd, hy).item()
    rhs = float(np.dot(s, y))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_sigma_transpose_symmetry_gpu(fci_lib):
    n, ne = 8, 4
    p = fci_problem(n, ne, ne, seed=12)
    f = gpu_fci(p)
    ns = comb(n, ne)
    C = synth.random_vector(ns * ns, 5).reshape(ns, ns)
    s1 = f.sigma(torch.from_numpy(C.reshape(-1)).cuda()).cpu().numpy().reshape(ns, ns)
    s2 = f.sigma(torch.from_numpy(np.ascontiguousarray(C.T).reshape(-1)).cuda()).cpu().numpy().reshape(ns, ns)
    assert rel_inf(s1.T, s2) <= 1e-13


@pytest.mark.parametrize("n,ne", [(4, 2), (6, 3), (8, 4), (10, 3), (12, 6)])
def test_sigma_spinor_complex_parity(fci_lib, n, ne):
    p = spinor_problem(n, ne, n_chol=6, seed=20 + n, e_core=0.25)
    f = gpu_fci(p)
    c = synth.random_vector(len(p["dets"]), seed=7, complex_=True)
    s = f.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    ref = oracle.sigma(p["hso"], p["gso"], p["dets"], c, e_core=p["e_core"])
    assert rel_inf(s, ref) <= SIGMA_RTOL
    if ne <= 6:
        t = f.table("repl_alpha").cpu().numpy().reshape(len(p["dets"]), -1, 4)
        o = oracle.replacement_table(n, ne)
        assert np.array_equal(t[..., 0], o["target"]) and np.array_equal(t[..., 3], o["sign"].astype(np.int32))


def test_spinor_diagonal(fci_lib):
    p = spinor_problem(9, 4, seed=5)
    f = gpu_fci(p)
    assert np.max(np.abs(f.diagonal().cpu().numpy() - oracle.diag(p["hso"], p["gso"], p["dets"]))) < 1e-12


# ------------------------------------------------------------------- Davidson

def test_davidson_fp64_8e8o_matches_dense_eigh(fci_lib):
    w = synth.WORKLOADS["fci_8e8o"]
    p = fci_problem(w["n"], w["na"], w["nb"], w["n_chol"], w["seed"], e_core=0.0)
    f = gpu_fci(p)
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10)
    assert r.converged
    H = oracle.dense_h(p["hso"], p["gso"], p["dets"]).real
    wv = np.linalg.eigvalsh(H)
    assert abs(r.energy - wv[0]) < ENERGY_TOL
    # the returned vector is a unit Ritz vector with the logged residual
    c = r.vector.cpu().numpy()
    assert abs(np.linalg.norm(c) - 1) < 1e-12
    assert np.linalg.norm(H @ c - r.energy * c) < 2 * r.iterations[-1]["residual_norm"] + 1e-12
    # gap theorem bound (Methods): |dE| <= ||r||^2 / gamma0
    rn = r.iterations[-1]["residual_norm"]
    assert abs(r.energy - wv[0]) <= rn * rn / (wv[1] - wv[0]) + 1e-12


@pytest.mark.parametrize("n,ne,nch,seed", [(8, 4, 16, 3), (8, 4, 16, 7), (6, 3, 12, 2), (6, 2, 8, 10)])
def test_davidson_finds_the_lowest_root_outside_the_symmetric_sector(fci_lib, n, ne, nch, seed):
    """Seeded Hamiltonians whose ground state is antisymmetric under alpha <-> beta string
    exchange (C[a, b] = -C[b, a]).  The default start (unit vector at min H_II with a
    pseudo-random admixture) has a component in that sector and the solve returns the
    lowest eigenvalue of the oracle's dense H with an antisymmetric vector.  The bare
    closed-shell unit vector (start_mix = 0) is symmetric, so in exact arithmetic the
    iteration would stay in the symmetric sector; in floating point, rounding seeds the
    other sector and the solve still ends at an eigenvalue of H (measured: the ground
    state, for these four Hamiltonians)."""
    from math import comb

    p = fci_problem(n, ne, ne, n_chol=nch, seed=seed)
    H = oracle.dense_h(p["hso"], p["gso"], p["dets"]).real
    w, v = np.linalg.eigh(H)
    ns = comb(n, ne)
    v0 = v[:, 0].reshape(ns, ns)
    assert np.max(np.abs(v0 + v0.T)) < 1e-8  # the ground state is antisymmetric
    f = gpu_fci(p)
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10, max_iter=200)
    assert r.converged and abs(r.energy - w[0]) < ENERGY_TOL
    c = r.vector.cpu().numpy().reshape(ns, ns)
    assert np.max(np.abs(c + c.T)) < 1e-5
    r0 = f.davidson(tol_residual=1e-6, tol_energy=1e-10, max_iter=200, start_mix=0.0)
    assert r0.converged and np.min(np.abs(w - r0.energy)) < ENERGY_TOL


def test_davidson_gpu_follows_oracle_davidson(fci_lib):
    p = fci_problem(7, 4, 3, seed=21, e_core=-2.0)
    f = gpu_fci(p)
    r = f.davidson(tol_residual=1e-7, tol_energy=1e-12, max_subspace=6, start_mix=0.0)  # the oracle's start
    hd = oracle.diag(p["hso"], p["gso"], p["dets"])
    E, c, log, conv = odav.davidson(lambda v: oracle.sigma(p["hso"], p["gso"], p["dets"], v), hd,
                                    tol_r=1e-7, tol_e=1e-12, max_sub=6, e_shift=p["e_core"])
    assert conv and r.converged
    assert abs(r.energy - E) < ENERGY_TOL
    # the iteration tables agree while both are far from the rounding floor
    for a, b in zip(r.iterations[:4], log[:4]):
        assert abs(a["energy"] - b["energy"]) < 1e-9
        assert abs(a["residual_norm"] - b["rnorm"]) < 1e-7


def test_davidson_spinor_matches_dense_eigh(fci_lib):
    p = spinor_problem(10, 4, n_chol=6, seed=31)
    f = gpu_fci(p)
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10)
    assert r.converged
    w = np.linalg.eigvalsh(oracle.dense_h(p["hso"], p["gso"], p["dets"]))
    assert abs(r.energy - w[0]) < ENERGY_TOL


def test_davidson_compression_compatible_eps(fci_lib):
    p = fci_problem(8, 4, 4, seed=1, n_chol=16)
    f = gpu_fci(p)
    eps = 0.1 * 10.0 / np.sqrt(4900)
    r = f.davidson(tol_residual=1e-6, tol_energy=1e-10, eps=eps, max_iter=300)
    w = np.linalg.eigvalsh(oracle.dense_h(p["hso"], p["gso"], p["dets"]).real)
    assert r.converged and abs(r.energy - w[0]) < ENERGY_TOL


# ------------------------------------------------------------------- errors

def test_argument_errors_are_codes_not_faults(fci_lib):
    from paper_2505_20375_gb300 import fci

    f = fci.FCI(0)
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    rc = fci._sigma(f._h, z.data_ptr(), z.data_ptr() + 0, 1, 0, 0, ws.data_ptr(), 1024, None)
    assert rc == fci.FCI_ERR_STATE  # sigma before any strings
    h, g = synth.real_integrals(4, 2, 1)
    g_bad = g.copy()
    g_bad[0, 1, 2, 3] += 1e-3
    with pytest.raises(fci.FCIError) as e:
        f.setup_integrals(h, g_bad)
    assert e.value.code == fci.FCI_ERR_ARG
    f.setup_integrals(h, g)
    with pytest.raises(fci.FCIError):
        f.build_strings(5, 1)
    f.build_strings(2, 2)
    with pytest.raises(ValueError):
        f.sigma(torch.zeros(5, dtype=torch.float64, device="cuda"))
    with pytest.raises(fci.FCIError) as e:
        f.sigma(torch.zeros(36, dtype=torch.float64, device="cuda"), precision="oz_bf16", n_slices=1)
    assert e.value.code == fci.FCI_ERR_ARG
