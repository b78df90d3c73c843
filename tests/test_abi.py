"""The C-ABI library loads and exports every symbol include/fci.h declares (CPU only;
no compute call needs a GPU here)."""
import ctypes
import json
import os
import re
from math import comb

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fci.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2505_20375_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "sizeof")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fci_setup_integrals", "fci_build_strings", "das_build_categories", "fci_sigma",
                     "davidson_solve"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_count_determinants_host_only(lib):
    f = lib.fci_count_determinants
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    f.restype = ctypes.c_int64
    assert f(14, 7, 7) == comb(14, 7) ** 2
    assert f(8, 4, 4) == 4900
    assert f(24, 12, -1) == comb(24, 12)
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_det_counts.json")))
    for c in gold["cases"]:
        N = f(c["n"], c["ne"], -1)
        assert N == comb(c["n"], c["ne"])
        assert abs(N - c["printed"]) <= c["rel_tol"] * c["printed"]
    assert f(10, 11, 0) == -1 and f(-1, 0, 0) == -1


def test_create_reports_error_without_device(lib):
    """On a machine without a usable GPU fci_create returns an error code, not a crash."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib.fci_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    lib.fci_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    rc = lib.fci_create(ctypes.byref(h), 0)
    assert rc != 0 and not h.value
    assert lib.fci_last_error(None)


def test_binding_refuses_to_import_without_library(tmp_path, monkeypatch):
    """The product path has no CPU fallback: without libfci.so the binding raises."""
    import importlib.util

    src = os.path.join(ROOT, "paper_2505_20375_gb300", "fci.py")
    pkg = tmp_path / "pkg"
    pkg.mkdir()
    (pkg / "fci.py").write_text(open(src).read())
    spec = importlib.util.spec_from_file_location("fci_nolib", str(pkg / "fci.py"))
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


# Every entry point that takes a handle (or a Davidson state, or a job list), called with
# NULL for it and for every pointer: each must return FCI_ERR_ARG (fci_destroy: FCI_OK,
# "safe on NULL") without touching the device.  Arguments after the name, in order; "d"
# marks a double, "z" a size_t, "q" an int64_t, anything else an int or a NULL pointer.
NULL_CALLS = {
    "fci_destroy": [None],
    "fci_get_info": [None, None],
    "fci_setup_integrals": [None, 4, 0, None, None, "d", None],
    "fci_build_strings": [None, 2, 2, None],
    "das_build_categories": [None, 2, None, None, None, 1, None],
    "fci_diagonal": [None, None, None],
    "fci_sigma_workspace_bytes": [None, 1, 0, 0, None],
    "fci_sigma": [None, None, None, 1, 0, 0, None, "z", None],
    "fci_sigma_host_workspace_bytes": [None, 1, 0, 0, None],
    "fci_sigma_host": [None, None, None, 1, 0, 0, None, "z", None],
    "fci_davidson_workspace_bytes": [None, None, None],
    "davidson_solve": [None, None, None, None, None, None, "z", None],
    "fci_sigma_graph": [None, None, None, 0, 0, None, "z", None],
    "fci_clear_graphs": [None],
    "fci_tune_sigma": [None, 3, None, None, None, "z", 1, None, None],
    "fci_sigma_grouped": [None, 1, None],
    "fci_sigma_grouped_graph": [None, 1, None],
    "davidson_begin": [None, None, None, None, "z", None, None],
    "davidson_request": [None, None, None, None, None, None, None],
    "davidson_advance": [None, None],
    "davidson_finish": [None, None, None, None],
    "fci_table_bytes": [None, 0, None],
    "fci_copy_table": [None, 0, None, "z", None],
    "fci_sync_status": [None, None],
    "fci_set_phase_timing": [None, 1],
    "fci_get_phase_times": [None, None, None, 0],
    "fci_sigma_compressed_workspace_bytes": [None, "q", None],
    "fci_sigma_compressed": [None, None, None, "q", None, None, "q", None, None, "z", None],
    "fci_sigma_noalloc": [None, None, None, None],
}
# entry points without a handle argument (covered by the tests above and below)
HOST_ONLY = {"fci_create", "fci_last_error", "fci_count_determinants", "fci_davidson_default_opts",
             "fci_clear_grouped_graphs"}

_NULL_PROBE = r"""
import ctypes, json, sys
L = ctypes.CDLL(sys.argv[1])
conv = {"d": ctypes.c_double(0.0), "z": ctypes.c_size_t(0), "q": ctypes.c_int64(0)}
out = {}
for name, args in json.loads(sys.argv[2]).items():
    f = getattr(L, name)
    f.restype = ctypes.c_int
    out[name] = f(*[conv.get(a, a) if isinstance(a, str) else a for a in args])
print(json.dumps(out))
"""


def test_every_entry_point_rejects_a_null_handle(lib):
    import subprocess
    import sys

    from paper_2505_20375_gb300 import build

    assert set(NULL_CALLS) | HOST_ONLY == set(declared_functions())
    # in a child process, so that a NULL dereference shows as a failure, not a crash
    p = subprocess.run([sys.executable, "-c", _NULL_PROBE, build.build(), json.dumps(NULL_CALLS)],
                       capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    rc = json.loads(p.stdout.strip().splitlines()[-1])
    assert rc.pop("fci_destroy") == 0
    assert rc == {name: 1 for name in rc}  # FCI_ERR_ARG


def test_davidson_default_options_are_the_documented_ones():
    from paper_2505_20375_gb300 import fci

    o = fci.fci_davidson_opts()
    fci._lib.fci_davidson_default_opts(ctypes.byref(o))
    assert (o.max_iter, o.max_subspace, o.tol_residual, o.tol_energy, o.eps) == (100, 32, 1e-6, 1e-10, 0.0)
    assert (o.precision, o.switch_residual, o.use_guess, o.final_precision) == (fci.FCI_PREC_FP64, 1e-5, 0,
                                                                                   fci.FCI_PREC_FP64)
    assert (o.gap_bound, o.staged_sigma, o.start_mix) == (0, 0, 1e-2)
