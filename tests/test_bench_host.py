"""Host arithmetic of bench.py's roofline object (no GPU): the algorithmic
operation counts, the peaks, the choice of the FP32 or FP64 pipe, and the
per-launch figures taken from a counter record (traffic, HBM and L2
throughput), checked against hand-computed values on a synthetic record."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_peaks_are_unit_counts_times_clock():
    assert bench.peak_fp32_ops() == pytest.approx(152 * 128 * 2.07e9)
    assert bench.peak_fp64_ops() == pytest.approx(152 * 2 * 2.07e9)


def test_force_pass_operation_model():
    # 12 nodes x (distance 2, switch 11, 3 per radial term for 3 + 2 terms,
    # G 3, force sums 6.25, width term 2) + static point + pair weights
    node = 2 + 11 + 3 * 5 + 3 + 4.25 + 2
    static = 2 + 11 + 4 * 2 + 1
    pair = 20 + 4 + 4 * 4 + 5 + 9 + 24
    assert bench.ops_per_pair("pair32_force", 3, 2, 2) == pytest.approx(12 * node + static + pair)
    assert bench.units_per_launch("pair32_force", 13824000) == 6912000    # unordered pairs
    assert bench.units_per_launch("gather32_force", 13824000) == 13824000


def _record(src_file, tmp_path, fp64_pct, fma_pct):
    text = "AAA kernel body BBB"
    (tmp_path / src_file).write_text(text)
    src = {"file": src_file, "from": "AAA", "to": "BBB"}
    return {"ncu_kernel": "k", "duration_ns": 1.0e5, "dram_read": 1.0e8, "dram_write": 5.0e7,
            "l2_bytes": 4.0e8, "fp64_lane_ops": 6.0e9, "fma_pipe_pct": fma_pct, "fp64_pipe_pct": fp64_pct,
            "source": src, "source_digest": None}


def test_roofline_from_a_counter_record(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec32 = _record("k32.cu", tmp_path, 0.0, 60.0)
    rec64 = _record("k64.cu", tmp_path, 88.0, 1.0)
    rec32["source_digest"] = bench.kernel_source_digest(rec32["source"])
    rec64["source_digest"] = bench.kernel_source_digest(rec64["source"])
    counters = tmp_path / "counters.json"
    counters.write_text(json.dumps({"kernels": {"pair32_force": rec32, "pair64_force": rec64}}))
    monkeypatch.setattr(bench, "COUNTERS", str(counters))

    shares = {"pair32_force": {"launches": 13, "total_ms": 1.95, "avg_ms": 0.15, "share": 0.2},
              "gather32_force": {"launches": 13, "total_ms": 0.65, "avg_ms": 0.05, "share": 0.1}}
    r = bench.roofline_of(shares, 13824000, 2, 3, 2, True)
    ops = 6912000 * bench.ops_per_pair("pair32_force", 3, 2, 2)
    assert r["kernel"] == "pair32_force" and r["unit"].startswith("Tops/s")
    assert r["achieved"] == pytest.approx(ops / 0.15e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / (bench.peak_fp32_ops() / 1e12))
    assert r["traffic"] == pytest.approx(1.5e8)
    assert r["hbm_gbs"] == pytest.approx(1.5e8 / 0.15e-3 / 1e9)
    assert r["l2_gbs"] == pytest.approx(4.0e8 / 0.15e-3 / 1e9)

    shares = {"pair64_force": {"launches": 13, "total_ms": 200.0, "avg_ms": 15.0, "share": 0.6}}
    r = bench.roofline_of(shares, 13824000, 2, 3, 2, True)
    assert r["unit"].startswith("T lane-ops/s")
    assert r["achieved"] == pytest.approx(6.0e9 / 15.0e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / (bench.peak_fp64_ops() / 1e12))


def test_a_changed_kernel_drops_its_record(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = _record("k.cu", tmp_path, 0.0, 60.0)
    rec["source_digest"] = bench.kernel_source_digest(rec["source"])
    counters = tmp_path / "counters.json"
    counters.write_text(json.dumps({"kernels": {"pair32_force": rec}}))
    monkeypatch.setattr(bench, "COUNTERS", str(counters))
    assert bench.ncu_traffic("pair32_force") == pytest.approx(1.5e8)
    (tmp_path / "k.cu").write_text("AAA kernel body, edited BBB")
    assert bench.ncu_traffic("pair32_force") is None
    shares = {"pair32_force": {"launches": 1, "total_ms": 0.15, "avg_ms": 0.15, "share": 1.0}}
    r = bench.roofline_of(shares, 13824000, 2, 3, 2, True)
    assert r["traffic"] is None and r["hbm_gbs"] is None
