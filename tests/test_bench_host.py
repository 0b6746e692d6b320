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
    monkeypatch.setattr(bench, "ncu_traffic", lambda cls: 1.5e6 if cls == "dts_gs" else None)
    classes = {"dts_gs": {"GBps": 43.4, "share": 0.46}, "line_chain": {"GBps": 19.0, "share": 0.2}}
    peak, _ = bench.measured_peak()
    r = bench.roofline(classes)
    assert r["kernel"] == "dts_gs" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == 43.4 and r["peak"] == peak and r["frac"] == round(43.4 / peak, 4)
    assert r["traffic"] == 1.5e6 and r["share"] == 0.46
    assert bench.roofline({}) is None


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
    rec.write_text(f"source_hash: {h}\n\n| class | bytes per launch |\n|---|---|\n| dts_gs | 1289372 |\n")
    assert bench.ncu_traffic("dts_gs") == 1289372.0
    assert bench.ncu_traffic("line_chain") is None
    with open(dst / "blp_dts.cuh", "a") as fh:                # the kernel changed since the capture
        fh.write("\n// edited\n")
    assert bench.kernel_source_hash() != h and bench.ncu_traffic("dts_gs") is None
    rec.unlink()
    assert bench.ncu_traffic("dts_gs") is None


def test_committed_record_parses():
    txt = open(os.path.join(bench.ROOT, "profiles", "roofline_traffic.md")).read()
    assert "source_hash:" in txt and "| dts_gs |" in txt
