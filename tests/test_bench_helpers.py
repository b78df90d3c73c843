"""CPU tests of bench.py's host logic: the DRAM-traffic record is reported only for the
kernel sources it was measured on."""
import os

import bench


def _fake_tree(tmp_path, gemm_src=b"kernel v1"):
    csrc = tmp_path / "paper_2505_20375_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in bench._KERNEL_SOURCES["k_oz_gemm"] + bench._KERNEL_SOURCES["k_oz_contract"]:
        (csrc / fn).write_bytes(gemm_src if fn == "ozaki_gemm.cu" else b"shared " + fn.encode())
    (tmp_path / "profiles").mkdir()
    return tmp_path


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    root = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench._kernel_sources_sha("k_oz_gemm<6,8>")
    assert len(sha) == 16
    (root / "profiles" / "traffic.md").write_text(
        "| kernel | workload | sources sha | dram bytes per launch | read | write |\n"
        "|---|---|---|---|---|---|\n"
        f"| k_oz_gemm<6,8> | fci_14e14o | {sha} | 25726923008 | 15.88 GB | 9.85 GB |\n"
        f"| k_oz_gemm<6,8> | fci_12e12o | {sha} | 1308891904 | 0.82 GB | 0.49 GB |\n")
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o") == 25726923008.0
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_12e12o") == 1308891904.0
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_8e8o") is None  # no row for the workload
    assert bench._traffic_record("k_oz_gemm<7,8>", "fci_14e14o") is None  # no row for the form

    # a changed kernel source invalidates the record: the bench reports null, not a stale count
    (root / "paper_2505_20375_gb300" / "csrc" / "ozaki_gemm.cu").write_bytes(b"kernel v2")
    assert bench._kernel_sources_sha("k_oz_gemm<6,8>") != sha
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o") is None
    # the digest covers only the kernel's own sources
    assert bench._kernel_sources_sha("k_oz_contract<6,64>") == bench._kernel_sources_sha("k_oz_contract<6,32>")


def test_traffic_record_without_a_capture(tmp_path, monkeypatch):
    root = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert not os.path.exists(root / "profiles" / "traffic.md")
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o") is None
    (root / "profiles" / "traffic.md").write_text("| k_oz_gemm<6,8> | fci_14e14o | 0123456789abcdef | n/a |\n")
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o") is None
