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
