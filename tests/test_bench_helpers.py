"""CPU tests of bench.py's host logic: the roofline follows the method's work, and the
DRAM-traffic record is reported only for the kernel sources it was measured on."""
import json
import os

import pytest

import bench


def _fake_tree(tmp_path, gemm_src=b"kernel v1"):
    csrc = tmp_path / "paper_2505_20375_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in bench._KERNEL_SOURCES["k_oz_gemm"] + bench._KERNEL_SOURCES["k_oz_contract"]:
        (csrc / fn).write_bytes(gemm_src if fn == "ozaki_gemm.cu" else b"shared " + fn.encode())
    (tmp_path / "profiles").mkdir()
    return tmp_path


def _write(root, recs):
    (root / "profiles" / "traffic.json").write_text(json.dumps({"records": recs}))


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    root = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench._kernel_sources_sha("k_oz_gemm<6,8>")
    assert len(sha) == 16
    _write(root, [{"kernel": "k_oz_gemm<6,8>", "workload": "fci_14e14o", "sources_sha": sha,
                   "dram_bytes_per_launch": 25726923008, "date": "2026-12-03", "scaled_from": "fci_12e12o"},
                  {"kernel": "k_oz_gemm<6,8>", "workload": "fci_12e12o", "sources_sha": sha,
                   "dram_bytes_per_launch": 1308891904}])
    r = bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o")
    assert r["bytes"] == 25726923008.0 and r["scaled_from"] == "fci_12e12o" and r["sources_sha"] == sha
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_12e12o")["bytes"] == 1308891904.0
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_8e8o") is None  # no record for the workload
    assert bench._traffic_record("k_oz_gemm<7,8>", "fci_14e14o") is None  # no record for the form

    # a changed kernel source invalidates the record: the bench reports null, not a stale count
    (root / "paper_2505_20375_gb300" / "csrc" / "ozaki_gemm.cu").write_bytes(b"kernel v2")
    assert bench._kernel_sources_sha("k_oz_gemm<6,8>") != sha
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o") is None
    # the digest covers only the kernel's own sources
    assert bench._kernel_sources_sha("k_oz_contract<6,64>") == bench._kernel_sources_sha("k_oz_contract<6,32>")


def test_traffic_record_without_a_capture(tmp_path, monkeypatch):
    root = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert not os.path.exists(root / "profiles" / "traffic.json")
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o") is None
    _write(root, [{"kernel": "k_oz_gemm<6,8>", "workload": "fci_14e14o", "sources_sha": "0123456789abcdef",
                   "dram_bytes_per_launch": 1}])
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o") is None
    (root / "profiles" / "traffic.json").write_text("not json")
    assert bench._traffic_record("k_oz_gemm<6,8>", "fci_14e14o") is None


def test_split_roofline_counts_the_methods_packed_work():
    """FCI(14e,14o), s = 6: 2 x 105^2 x 21 flop per determinant over 11,778,624
    determinants = 5.45e12 flop per launch; at 7.857 ms that is 694 TF/s, 0.359 of a
    1,933.5 TF/s peak.  The executed MMA shape (128 x 112, 64-determinant tiles) is 1.30x
    more and is reported apart; the whole step is compared with the 2.82 ms the work needs
    at the peak."""
    r = bench.split_roofline(105, 11778624, 6, 7.857, 14.65, 1933.5, two_pass=True)
    assert r["flops_per_launch"] == pytest.approx(2 * 105 ** 2 * 21 * 11778624)
    assert r["flops_per_launch"] == pytest.approx(5.4543e12, rel=1e-4)
    assert r["achieved"] == pytest.approx(694.2, rel=1e-3)
    assert r["frac"] == pytest.approx(0.359, abs=1e-3)
    ex = r["executed"]["flops_per_launch"] / r["flops_per_launch"]
    assert ex == pytest.approx(128 * 112 * (-(-11778624 // 64) * 64) / (105 * 105 * 11778624))
    assert 1.29 < ex < 1.31
    assert r["step"]["tensor_floor_ms"] == pytest.approx(5.4543e12 / 1933.5e12 * 1e3, rel=1e-4)
    assert r["step"]["frac"] == pytest.approx(r["step"]["tensor_floor_ms"] / 14.65)


def test_contraction_work_is_the_methods_dense_product():
    """E = G D per sigma: 2 n_pair^2 N_K flop (8 per complex multiply-add), times
    s(s+1)/2 slice products in split precision.  FCI(14e,14o) with 105 packed pairs:
    2.60e11 flop in FP64; 24 spinors, 12 electrons (576 ordered pairs, complex): 7.18e12."""
    fci = {"n_pair": 105, "n_det_intermediate": 11778624, "dtype": 0}
    assert bench.contraction_work(fci, 6, fp64=True) == pytest.approx(2.597e11, rel=1e-3)
    assert bench.contraction_work(fci, 6, fp64=False) == pytest.approx(21 * 2.597e11, rel=1e-3)
    sp = {"n_pair": 576, "n_det_intermediate": 2704156, "dtype": 1}
    assert bench.contraction_work(sp, 8, fp64=True) == pytest.approx(7.177e12, rel=1e-3)
    assert bench.contraction_work(sp, 8, fp64=False) == pytest.approx(36 * 7.177e12, rel=1e-3)


def test_clock_sampler_reads_median_clock_and_throttle_reasons(tmp_path, monkeypatch):
    """The sampler's parse of nvidia-smi's CSV (a stand-in script prints the samples): the
    median SM clock under load, the maximum, and every throttle reason seen Active."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!/bin/sh\n"
        "cat <<'END'\n"
        "0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, [N/A], 2070, 905.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1965, 2070, 1398.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2070, 2070, 1120.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "END\n"
        "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    s = bench.ClockSampler(0)
    s.start()
    rec = s.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(s.out.name)  # the sample file is removed

    # no nvidia-smi at all: the record says so instead of inventing clocks
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    assert not os.path.exists(s.out.name)


def test_oracle_leg_times_sigma_rows_of_a_fixed_table():
    """The CPU baseline: the determinant table is built once (its time reported apart), and
    the timed sample is whole sigma rows of the oracle, never more than the space holds."""
    import numpy as np

    import oracle
    from paper_2505_20375_gb300 import synth

    w = {"n": 6, "na": 3, "nb": 3}
    h, g = synth.real_integrals(6, 8, seed=1)
    leg = bench.OracleLeg(w, h, g)
    N = len(leg.dets)
    assert N == 400 and leg.setup_s >= 0.0 and leg.threads >= 1
    c = synth.random_vector(N, seed=7)
    rate, rows, secs = leg.rate(c, 0.05, rng_seed=3)
    assert 0 < rows <= N and secs > 0 and rate == pytest.approx(rows / secs)
    # the rows it times are the oracle's sigma rows (same table, same arithmetic)
    hso, gso = oracle.spin_orbital_integrals(h, g)
    perm = np.random.default_rng(3).permutation(N)[:50]
    assert np.array_equal(leg.table.sigma(leg.hso, leg.gso, c, rows=perm),
                          oracle.sigma(hso, gso, oracle.fci_dets(6, 3, 3), c, rows=perm))
