"""Host-side logic of bench.py (no GPU): the default run's contract
(N = 1, W >= 3 warm-up steps), the roofline object, and the rule that the
committed ncu traffic record is reported only while the wavefront kernel's
sources are the ones it was captured on."""
import os
import shutil
import sys

import pytest

import bench


def test_default_run_is_one_gpu_with_three_warmup_steps(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.impl, a.N, a.mode) == (1, "ours", 1024, "bench")
    assert a.warmup >= 3 and a.steps >= 1


def test_roofline_object(monkeypatch):
    monkeypatch.setattr(bench, "ncu_traffic", lambda cls, pn: 1.5e6 if (cls, pn) == ("dts_gs", "fp64") else None)
    by_prec = {"mixed": {"dts_gs": {"GBps": 43.4, "ms": 100.0, "launches": 10, "bytes": 4.34e9, "chain_steps": 2e5},
                         "line_chain": {"GBps": 19.0, "ms": 50.0, "launches": 2, "bytes": 9.5e8}},
               "fp64": {"dts_gs": {"GBps": 30.0, "ms": 300.0, "launches": 10, "bytes": 9e9, "chain_steps": 2e5}}}
    peak, _ = bench.measured_peak()
    r = bench.roofline(by_prec, 2070.0)
    assert (r["kernel"], r["precision"]) == ("dts_gs", "fp64") and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == 30.0 and r["peak"] == peak and r["frac"] == round(30.0 / peak, 4)
    assert r["traffic"] == 1.5e6 and r["algorithmic_bytes_per_launch"] == 9e8
    floor_ms = 2e5 * bench.CHAIN_STEP_CYCLES["fp64"] / 2070e3
    assert r["chain_floor_ms"] == round(floor_ms, 3) and r["chain_floor_frac"] == round(floor_ms / 300.0, 4)
    assert bench.roofline({}, 2070.0) is None


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2108_13468_gb300", "csrc")
    dst = tmp_path / "paper_2108_13468_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("blp_common.cuh", "blp_dts.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    rec = tmp_path / "profiles" / "roofline_traffic.md"
    rec.write_text(f"source_hash: {h}\n\n| class | precision | bytes per launch |\n|---|---|---|\n"
                   "| dts_gs | fp64 | 1289372 |\n| dts_gs | mixed | 900000 |\n")
    assert bench.ncu_traffic("dts_gs", "fp64") == 1289372.0
    assert bench.ncu_traffic("dts_gs", "mixed") == 900000.0
    assert bench.ncu_traffic("line_chain", "fp64") is None
    with open(dst / "blp_dts.cuh", "a") as fh:                # the kernel changed since the capture
        fh.write("\n// edited\n")
    assert bench.kernel_source_hash() != h and bench.ncu_traffic("dts_gs", "fp64") is None
    rec.unlink()
    assert bench.ncu_traffic("dts_gs", "fp64") is None


def test_committed_record_parses():
    txt = open(os.path.join(bench.ROOT, "profiles", "roofline_traffic.md")).read()
    assert "source_hash:" in txt and "| dts_gs |" in txt
