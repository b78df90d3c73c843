"""Mutation check of the oracle's pins (CPU only).

Each case plants one plausible slip in a temporary copy of the oracle (a dropped term,
a wrong fermion sign, a transposed operand, an off-by-one in an enumeration or a search,
a wrong root) and runs the pin tests (test_oracle_pins.py, test_oracle_alg1.py) against
that copy in a subprocess: at least one pin must fail.  The unmutated copy must pass, so
that a failure means the pins caught the slip and not that the copy is broken.  The
oracle in the repository is never modified.

Mutants that are equivalent to the original are not listed, since no test can catch
them: a sign flip of a Davidson correction vector (it spans the same subspace); R == Q
kept in the single-replacement sum (its term is (PQ|QQ) - (PQ|QQ) = 0); and the
one-electron fold put on one side only, g' = g + 2 h' delta / N_e, which gives the same
H because sum_r E_rr = N_e commutes with every E_pq.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ("test_oracle_pins.py", "test_oracle_alg1.py")

# (what the slip is, file under oracle/, original text (must occur once), planted text)
MUTANTS = [
    # fci_oracle.c: Slater-Condon rules and the sigma loop ("Methods", Eqs. sigmaL*)
    ("diagonal_exchange_dropped", "fci_oracle.c",
     "cplx t = csub(G(H, P, P, R, R), G(H, P, R, R, P));",
     "cplx t = G(H, P, P, R, R);"),
    ("diagonal_half_missing", "fci_oracle.c",
     "e = cadd(e, cscale(t, 0.5));",
     "e = cadd(e, t);"),
    ("single_exchange_operand_transposed", "fci_oracle.c",
     "e = cadd(e, csub(G(H, P, Q, R, R), G(H, P, R, R, Q)));",
     "e = cadd(e, csub(G(H, P, Q, R, R), G(H, P, R, Q, R)));"),
    ("single_one_electron_operand_transposed", "fci_oracle.c",
     "cplx e = H->h[P * n + Q];",
     "cplx e = H->h[Q * n + P];"),
    ("single_sign_dropped", "fci_oracle.c",
     "        }\n        return cscale(e, (double)s);\n    }\n    if (nd == 4) {",
     "        }\n        return e;\n    }\n    if (nd == 4) {"),
    ("double_exchange_dropped", "fci_oracle.c",
     "cplx e = csub(G(H, P, Q, R, S), G(H, P, S, R, Q));",
     "cplx e = G(H, P, Q, R, S);"),
    ("double_creation_order_swapped", "fci_oracle.c",
     "s *= op_create(&w, R);\n        s *= op_create(&w, P);",
     "s *= op_create(&w, P);\n        s *= op_create(&w, R);"),
    ("double_operands_conjugate_order", "fci_oracle.c",
     "cplx e = csub(G(H, P, Q, R, S), G(H, P, S, R, Q));",
     "cplx e = csub(G(H, Q, P, S, R), G(H, P, S, R, Q));"),
    ("annihilation_parity_counts_above", "fci_oracle.c",
     "int below = popcount64(*m & (bit - 1));\n    *m &= ~bit;",
     "int below = popcount64(*m & ~(bit | (bit - 1)));\n    *m &= ~bit;"),
    ("sigma_core_energy_dropped", "fci_oracle.c",
     "cplx acc = cscale(C[i], e_core);",
     "cplx acc = cscale(C[i], 0.0);"),
    ("sigma_adjacent_pairs_skipped", "fci_oracle.c",
     "for (int b = a + 1; b < no; ++b) {",
     "for (int b = a + 2; b < no; ++b) {"),
    ("sigma_first_single_skipped", "fci_oracle.c",
     "for (int a = 0; a < no; ++a) {\n            for (int v = 0; v < nv; ++v) {\n"
     "                uint64_t J = (I & ~((uint64_t)1 << occ[a])) | ((uint64_t)1 << vir[v]);",
     "for (int a = 1; a < no; ++a) {\n            for (int v = 0; v < nv; ++v) {\n"
     "                uint64_t J = (I & ~((uint64_t)1 << occ[a])) | ((uint64_t)1 << vir[v]);"),
    ("replacement_sign_half", "fci_oracle.c",
     "sign[o] = (int8_t)(s1 * s2);",
     "sign[o] = (int8_t)(s2);"),
    ("replacement_orbitals_swapped", "fci_oracle.c",
     "a_out[o] = a;\n                b_out[o] = b;",
     "a_out[o] = b;\n                b_out[o] = a;"),
    ("strings_last_mask_dropped", "fci_oracle.c",
     "for (uint64_t x = 0; x < lim; ++x) {",
     "for (uint64_t x = 0; x + 1 < lim; ++x) {"),
    # das.py: categories ("Results", categorical decomposition)
    ("das_transfer_alpha_only", "das.py",
     "if excess(a, ref_a) + excess(b, ref_b) <= max_transfer:",
     "if excess(a, ref_a) <= max_transfer:"),
    ("das_transfer_off_by_one", "das.py",
     "if excess(a, ref_a) + excess(b, ref_b) <= max_transfer:",
     "if excess(a, ref_a) + excess(b, ref_b) < max_transfer:"),
    ("das_first_space_least_significant", "das.py",
     "for combo in itertools.product(*per):",
     "for combo in itertools.product(*per[::-1]):"),
    ("das_beta_block_transposed", "das.py",
     "blk = (sa[:, None] | (sb[None, :] << np.uint64(n))).reshape(-1)",
     "blk = (sa[None, :] | (sb[:, None] << np.uint64(n))).reshape(-1)"),
    # davidson.py ("Results", Eqs. davidsonPreconditioner, sparsePreconditioner)
    ("davidson_highest_root", "davidson.py",
     "lam, y0 = w[0], y[:, 0]",
     "lam, y0 = w[-1], y[:, -1]"),
    ("preconditioner_threshold_inverted", "davidson.py",
     "s = np.where(np.abs(s) >= eps * ns, s, 0.0)",
     "s = np.where(np.abs(s) < eps * ns, s, 0.0)"),
    ("preconditioner_guard_dropped", "davidson.py",
     "s = np.where(np.abs(den) >= guard, r / np.where(den == 0, 1.0, den), 0.0)",
     "s = r / np.where(den == 0, 1.0, den)"),
    # alg1.py (Methods, Algorithm 1 and its exponential search)
    ("exponential_search_upper_bound", "alg1.py",
     "        if A[mid] < key:\n            left = mid + 1",
     "        if A[mid] <= key:\n            left = mid + 1"),
    ("exponential_search_bracket_short", "alg1.py",
     "left, right = lo + step // 2 + 1, min(lo + step, n)",
     "left, right = lo + step // 2 + 1, min(lo + step - 1, n)"),
    ("excite_created_parity_dropped", "alg1.py",
     "    if bin(s1 & ((1 << p) - 1)).count(\"1\") & 1:\n        sign = -sign",
     "    if False:\n        sign = -sign"),
    ("fold_exchange_correction_dropped", "alg1.py",
     "hp = h - 0.5 * np.einsum(\"prrq->pq\", g)",
     "hp = h"),
    ("fold_electron_count_doubled", "alg1.py",
     "eye[:, :, None, None] * hp[None, None, :, :]) / n_el",
     "eye[:, :, None, None] * hp[None, None, :, :]) / (2 * n_el)"),
    ("fold_half_dropped", "alg1.py",
     "return 0.5 * gp.reshape(n * n, n * n)",
     "return gp.reshape(n * n, n * n)"),
    ("alg1_beta_move_uses_alpha_string", "alg1.py",
     "v = coefficient(K, JB) if spin == 0 else coefficient(JA, K)",
     "v = coefficient(K, JB) if spin == 0 else coefficient(K, JA)"),
    ("compressed_diagonal_without_core_energy", "alg1.py",
     "hii[a] = float(d) + e_core",
     "hii[a] = float(d)"),
    ("compressed_threshold_on_the_residual_norm", "alg1.py",
     "tv = np.where(np.abs(sv) >= eps * np.linalg.norm(sv), sv, 0.0)",
     "tv = np.where(np.abs(sv) >= eps * np.linalg.norm(rv), sv, 0.0)"),
    ("compressed_ritz_phase_not_aligned", "alg1.py",
     "            if ph < 0:\n                c, sc = scale(c, -1.0), scale(sc, -1.0)",
     "            if False:\n                c, sc = scale(c, -1.0), scale(sc, -1.0)"),
    ("alg1_constant_term_dropped", "alg1.py",
     "sigma[int(off + a)] = sigma.get(int(off + a), 0.0) + e_core * v",
     "sigma[int(off + a)] = sigma.get(int(off + a), 0.0) + 0.0 * v"),
]


def _sandbox(dst: str, mutant=None) -> None:
    """A copy of the oracle, the input generator and the pin tests, with one slip planted."""
    os.makedirs(os.path.join(dst, "oracle"))
    for f in ("__init__.py", "alg1.py", "build.py", "das.py", "davidson.py", "fci_oracle.c"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    os.makedirs(os.path.join(dst, "paper_2505_20375_gb300"))
    for f in ("__init__.py", "synth.py"):
        shutil.copy(os.path.join(ROOT, "paper_2505_20375_gb300", f),
                    os.path.join(dst, "paper_2505_20375_gb300", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    for f in ("conftest.py", "helpers.py") + PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    if mutant is not None:
        _, fname, old, new = mutant
        path = os.path.join(dst, "oracle", fname)
        text = open(path).read()
        assert text.count(old) == 1, f"{mutant[0]}: the original text must occur exactly once"
        open(path, "w").write(text.replace(old, new))


def _run_pins(dst: str):
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env.update(OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += [os.path.join("tests", f) for f in PIN_FILES]
    p = subprocess.run(cmd, cwd=dst, env=env, capture_output=True, text=True, timeout=900)
    tail = (p.stdout + p.stderr).strip().splitlines()
    return p.returncode, tail[-1] if tail else ""


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """(return code, pytest summary line) of the pin tests on the clean copy and on every
    mutant, run a few at a time."""
    base = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {"clean": None} | {m[0]: m for m in MUTANTS}
    dirs = {}
    for name, m in jobs.items():
        dirs[name] = str(base / name)
        _sandbox(dirs[name], m)
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        futs = {name: ex.submit(_run_pins, d) for name, d in dirs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_unmutated_copy_passes_the_pins(outcomes):
    rc, summary = outcomes["clean"]
    assert rc == 0, summary


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_the_planted_slip(outcomes, name):
    rc, summary = outcomes[name]
    # exit code 1 with failed tests: a pin caught it (not a collection or build error)
    assert rc == 1 and "failed" in summary and "error" not in summary, (name, rc, summary)
