#!/usr/bin/env python
"""Benchmark: time-to-solution and unknowns/s to relative residual 1e-10 of
the boundary-layer-preconditioned FGMRES solve, FP64 and mixed precision, on
one GB300, with the HBM roofline of the dominant kernel.

Workload (one "step"): N = 1024 intervals per axis (1 046 529 unknowns),
eps in {1e-2, 1e-4, 1e-6, 1e-8}; c1 = 1 + x^2, c2 = 1 + y^2, r = 1 + x y,
f = 16 seeded Fourier modes (seed 0); for each eps and each precision
(mixed FP32/FP64, plain FP64) one blp_setup + blp_solve to relative
residual 1e-10 of the row-normalised system.  The step's time is the sum of
those time-to-solutions (setup included, as in the paper's timings);
value = unknowns solved / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: independent replicas (one process per GPU, same workload each);
value = all ranks' unknowns / max-over-ranks time (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GMRES time-to-solution & unknowns/s to rel-res 1e-10, FP64 vs mixed; HBM roofline %"
UNIT = "unknowns/s"
EPS_LIST = (1e-2, 1e-4, 1e-6, 1e-8)
N_DEFAULT = 1024
TOL = 1e-10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=N_DEFAULT)
    ap.add_argument("--eps", default=",".join(str(e) for e in EPS_LIST))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the untimed-by-driver legs of configs 2-4 and "
                                                          "the paper mode")
    ap.add_argument("--mode", default="bench", choices=["bench", "precond", "solve"],
                    help="precond/solve: a short fixed run for profiling under ncu (no JSON line)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="for --mode precond/solve")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def build_inputs(N, eps_list):
    import numpy as np
    import paper_2108_13468_gb300 as blp
    from paper_2108_13468_gb300 import inputs
    probs = {}
    for eps in eps_list:
        x, _ = blp.mesh(N, eps)
        p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=0)
        probs[eps] = [np.ascontiguousarray(a) for a in (p.c1, p.c2, p.r, p.f)]
    return probs


def run_ours(args):
    import numpy as np
    import torch
    import paper_2108_13468_gb300 as blp
    from paper_2108_13468_gb300 import _native

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = args.N
    n = (N - 1) ** 2
    eps_list = [float(e) for e in args.eps.split(",")]
    precisions = ((blp.BLP_MIXED, "mixed"), (blp.BLP_FP64, "fp64"))
    host = build_inputs(N, eps_list)
    devin = {eps: [torch.from_numpy(a).to(dev) for a in arrs] for eps, arrs in host.items()}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)
    lib = _native.load()

    def one_step(record=None, profile=None):
        """All solves of the workload; returns launches and per-solve stats."""
        launches = 0
        stats = []
        for prec, pname in precisions:
            for eps in eps_list:
                c1, c2, r, f = devin[eps]
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(stream)
                s = blp.Solver(N, eps, c1, c2, r, precision=prec)
                if profile is not None:
                    lib.blp_profile(s.handle, 1)
                u, info = s.solve(f, tol=TOL)
                t1.record(stream)
                if profile is not None:
                    profile.append((pname, read_profile(lib, s)))
                launches += s.kernel_launches()
                s.close()
                stats.append((pname, eps, t0, t1, info.iters, info.relres, info.corner_cycles_max))
        return launches, stats

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        one_step()
        flush.zero_()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, launches, per = 0.0, 0, {}
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        l, stats = one_step()
        torch.cuda.synchronize(dev)
        launches += l
        for pname, eps, t0, t1, it, rr, cyc in stats:
            ms = t0.elapsed_time(t1)
            total_ms += ms
            d = per.setdefault((pname, eps), {"ms": [], "iters": it, "relres": rr, "corner_cycles_max": cyc})
            d["ms"].append(ms)
    barrier()
    clocks = sampler.stop()
    step_ms = max_over_ranks(total_ms / args.steps, dev)
    units = n * len(eps_list) * len(precisions)
    value = whole_job_value(units, world, step_ms)

    # e2e: host (pinned) inputs, host output, through the public API; the
    # same workload for --steps steps, mean time per step
    e2e = None
    if not args.no_e2e:
        pinned = {eps: [torch.from_numpy(a).pin_memory() for a in arrs] for eps, arrs in host.items()}
        uh = torch.zeros(n, dtype=torch.float64).pin_memory()
        ms_e2e = []
        for rep in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            for prec, _ in precisions:
                for eps in eps_list:
                    c1, c2, r, f = pinned[eps]
                    s = blp.Solver(N, eps, c1.numpy(), c2.numpy(), r.numpy(), precision=prec)
                    uh.zero_()
                    s.solve(f.numpy(), uh.numpy(), tol=TOL)
                    s.close()
            torch.cuda.synchronize(dev)
            ms_e2e.append((time.perf_counter() - t) * 1e3)
        nsolve = len(eps_list) * len(precisions)
        e2e_ms = max_over_ranks(statistics.mean(ms_e2e), dev)
        e2e = {"value": units * world / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
               "steps": len(ms_e2e), "h2d_bytes_per_step": 4 * n * 8 * nsolve, "d2h_bytes_per_step": n * 8 * nsolve}

    # instrumented replay of one step: per-kernel-class event timing
    prof = []
    flush.zero_()
    one_step(profile=prof)
    classes = merge_profiles([d for _, d in prof])
    by_prec = {pn: merge_profiles([d for q, d in prof if q == pn]) for _, pn in precisions}
    roof = roofline(by_prec, clocks.get("sm_mhz"))

    detail = {}
    for (pname, eps), d in per.items():
        ms = statistics.mean(d["ms"])
        detail.setdefault(pname, {})[f"{eps:g}"] = {"tts_ms": round(ms, 3), "iters": d["iters"],
                                                     "relres": d["relres"], "corner_cycles_max": d["corner_cycles_max"],
                                                     "unknowns_per_s": n / (ms * 1e-3)}
    for pname in detail:
        tot = sum(v["tts_ms"] for v in detail[pname].values())
        detail[pname]["all"] = {"tts_ms": round(tot, 3), "unknowns_per_s": n * len(eps_list) / (tot * 1e-3)}

    # the oracle's sample of the workload (eps = 1e-2 left out), timed on our
    # side from the same timed steps, so the CPU comparison is like for like
    matched = {"eps": list(CPU_SAMPLE_EPS), "note": "ours: mean time-to-solution of the timed steps over "
               "these eps only; cpu: the oracle on the same eps (FP64, setup + FGMRES(30) to 1e-10)"}
    for pname in [p for _, p in precisions]:
        ms = sum(statistics.mean(per[(pname, e)]["ms"]) for e in CPU_SAMPLE_EPS if (pname, e) in per)
        if ms > 0:
            matched[pname] = n * len(CPU_SAMPLE_EPS) / (ms * 1e-3)
    ms_both = sum(statistics.mean(per[(pn, e)]["ms"]) for pn in [p for _, p in precisions]
                  for e in CPU_SAMPLE_EPS if (pn, e) in per)
    if ms_both > 0:
        matched["value"] = n * len(CPU_SAMPLE_EPS) * len(precisions) / (ms_both * 1e-3)

    legs = None
    if not args.no_legs and rank == 0:
        legs = run_legs(blp, torch, dev)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": f"2D Shishkin N={N} ({n} unknowns), eps in {{{', '.join(f'{e:g}' for e in eps_list)}}}, "
                                  "c1=1+x^2, c2=1+y^2, r=1+xy, 16 seeded Fourier modes; setup+FGMRES(30) to rel-res 1e-10 "
                                  "in mixed and FP64 precision",
                      "N": N, "eps": eps_list, "precisions": [p for _, p in precisions], "tol": TOL,
                      "parallelism": f"replicas x{world}", "l2": "flushed between steps (256 MB write); working set > L2"},
           "gpu_launches": launches // args.steps, "clocks": clocks, "e2e": e2e, "roofline": roof,
           "detail": detail, "kernel_classes": classes,
           "kernel_classes_by_precision": {pn: {k: {kk: v[kk] for kk in ("launches", "ms", "share", "GBps")}
                                                for k, v in cl.items()} for pn, cl in by_prec.items()},
           "matched_sample": matched, "legs": legs}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(N)
        cpu = out["cpu_baseline"]["value"]
        for key in ("value", "mixed", "fp64"):
            if key in matched:
                matched[f"ratio_{key}_vs_cpu"] = round(matched[key] / cpu, 2)
        matched["cpu"] = cpu
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def max_over_ranks(step_ms, dev=None):
    """Replicas: the job's step time is the slowest rank's (max over ranks);
    a single process returns its own time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return step_ms
    t = torch.tensor([step_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, world, step_ms):
    """Unknowns solved by all ranks per second of the (max-over-ranks) step."""
    return units_per_rank * world / (step_ms * 1e-3)


def read_profile(lib, s):
    import ctypes
    from paper_2108_13468_gb300 import _native
    res = {}
    for c in range(lib.blp_kernel_class_count()):
        cnt, ms, by, st = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _native.check(lib.blp_profile_read(s.handle, c, ctypes.byref(cnt), ctypes.byref(ms), ctypes.byref(by)))
        _native.check(lib.blp_profile_chain_steps(s.handle, c, ctypes.byref(st)))
        res[lib.blp_kernel_class_name(c).decode()] = (cnt.value, ms.value, by.value, st.value)
    lib.blp_profile(s.handle, 0)
    return res


def merge_profiles(profs):
    tot = {}
    for p in profs:
        for k, vals in p.items():
            a = tot.setdefault(k, [0, 0.0, 0.0, 0.0])
            for i, v in enumerate(vals):
                a[i] += v
    all_ms = sum(v[1] for v in tot.values()) or 1.0
    out = {}
    for k, v in sorted(tot.items(), key=lambda kv: -kv[1][1]):
        if v[0] <= 0:
            continue
        out[k] = {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / all_ms, 4),
                  "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1) if v[1] > 0 else None, "bytes": v[2]}
        if v[3] > 0:
            out[k]["chain_steps"] = v[3]
    return out


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources that define the wavefront kernel (the dominant
    class) and the shared definitions it includes."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2108_13468_gb300", "csrc")
    for f in ("blp_common.cuh", "blp_dts.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class, precision):
    """Per-launch DRAM traffic of a kernel class in one precision from the
    committed ncu summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_hash:\s*(\w+)", txt)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(rf"^\|\s*{kernel_class}\s*\|\s*{precision}\s*\|\s*([0-9.eE+]+)\s*\|", txt, re.M)
    return float(m.group(1)) if m else None


# Latency of one step of a wavefront sweep's dependency chain (one shuffle and
# two dependent FMAs, one warp, no memory traffic), measured on GB300 with a
# development micro-benchmark: 34 cycles in FP32, 194 in FP64.
CHAIN_STEP_CYCLES = {"mixed": 34.0, "fp64": 194.0}


def roofline(by_prec, sm_mhz):
    """Roofline of the dominant (kernel class, precision) pair of the step:
    achieved = its algorithmic bytes / its CUDA-event device time against the
    measured HBM peak; for a wavefront class also the fraction of its
    dependency-chain floor (chain steps x step latency at the sampled clock)."""
    peak, src = measured_peak()
    pairs = [(c["ms"], pn, k, c) for pn, cl in by_prec.items() for k, c in cl.items()]
    if not pairs:
        return None
    _, pn, dom, c = max(pairs, key=lambda t: t[0])
    achieved = c["GBps"] or 0.0
    launches = c["launches"]
    out = {"bound": "hbm", "kernel": dom, "precision": pn, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": round(achieved / peak, 4),
           "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback (6.8 TB/s)",
           "traffic": ncu_traffic(dom, pn), "algorithmic_bytes_per_launch": round(c["bytes"] / launches),
           "launches": launches, "ms": c["ms"],
           "note": "achieved = algorithmic bytes / CUDA-event device time of every launch of the class, this "
                   "precision, in an instrumented replay of one step; traffic = ncu DRAM bytes per launch"}
    if c.get("chain_steps") and sm_mhz:
        floor_ms = c["chain_steps"] * CHAIN_STEP_CYCLES[pn] / (sm_mhz * 1e3)
        out["chain_floor_ms"] = round(floor_ms, 3)
        out["chain_floor_frac"] = round(floor_ms / c["ms"], 4)
        out["chain_note"] = (f"dependency chain: {c['chain_steps']:.0f} steps x {CHAIN_STEP_CYCLES[pn]:.0f} cycles at "
                             f"{sm_mhz:.0f} MHz = the latency floor of these sweeps; chain_floor_frac = floor / measured")
    return out


# ---------------------------------------------------------------------------
# legs: the other workloads, each timed once after the main timed region
# ---------------------------------------------------------------------------
# Table tab:exponential_times_iters (Sec. 3.3): the paper's seconds (setup
# included; serial C on one core of a 2.4 GHz Xeon) and FGMRES iterations for
# eq. (exponential_MMS), stop ||f - A u||_2 <= 10 ln(N) / N.
PAPER_EXP_TTS = {1e-4: ((128, 0.010, 3), (256, 0.041, 4), (512, 0.266, 6), (1024, 2.656, 14), (2048, 37.690, 40)),
                 1e-5: ((128, 0.010, 4), (256, 0.041, 4), (512, 0.178, 4), (1024, 1.103, 6), (2048, 7.625, 10)),
                 1e-6: ((128, 0.010, 4), (256, 0.041, 4), (512, 0.221, 5), (1024, 0.921, 5), (2048, 3.771, 5)),
                 1e-7: ((128, 0.010, 4), (256, 0.051, 5), (512, 0.221, 5), (1024, 0.923, 5), (2048, 4.519, 6))}


def _timed(torch, dev, fn):
    """Wall time of fn() with the device idle on both sides (ms), and its result."""
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    res = fn()
    torch.cuda.synchronize(dev)
    return (time.perf_counter() - t) * 1e3, res


def leg_large(blp, torch, dev):
    """N = 2048 and 4096, eps = 1e-6, trigonometric convection, r = 1, seed 2:
    setup + solve to rel-res 1e-10, mixed (both sizes) and FP64 (N = 2048)."""
    from paper_2108_13468_gb300 import inputs
    out = []
    for N, pname in ((2048, "mixed"), (2048, "fp64"), (4096, "mixed")):
        eps = 1e-6
        x, _ = blp.mesh(N, eps)
        p = inputs.problem_fourier_trig(x, x, N, eps, seed=2)
        c1, c2, r, f = (torch.from_numpy(a).to(dev) for a in (p.c1, p.c2, p.r, p.f))
        prec = blp.BLP_MIXED if pname == "mixed" else blp.BLP_FP64

        def run():
            s = blp.Solver(N, eps, c1, c2, r, precision=prec)
            u, info = s.solve(f, tol=TOL)
            s.close()
            return info
        run()   # warm-up
        ms, info = _timed(torch, dev, run)
        n = (N - 1) ** 2
        out.append({"N": N, "eps": eps, "precision": pname, "tts_ms": round(ms, 2), "iters": info.iters,
                    "relres": info.relres, "unknowns_per_s": n / (ms * 1e-3)})
        del c1, c2, r, f
    return out


def leg_batched(blp, torch, dev):
    """256 problems (seed 3): N in {64, 96, ..., 512}, log10 eps ~ U[-8, -2],
    c1 = 1 + a x^2, c2 = 1 + b y^2, own Fourier forcing.  The batched solver
    (mixed, concurrent streams, autotuned settings) against the same problems
    one at a time in FP64 on one stream, both to rel-res 1e-10, inputs on the
    device."""
    from paper_2108_13468_gb300 import inputs
    specs = inputs.batch_params(256, seed=3)
    probs = []
    for sp in specs:
        N, eps = sp["N"], sp["eps"]
        x, _ = blp.mesh(N, eps)
        p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=sp["seed"], a=sp["a"], b=sp["b"])
        probs.append(dict(N=N, eps=eps, **{k: torch.from_numpy(getattr(p, k)).to(dev) for k in ("c1", "c2", "r", "f")}))
    units = sum((q["N"] - 1) ** 2 for q in probs)

    def batched(tuned):
        items = [dict(q, precision=blp.BLP_MIXED, maxit=3000, u=torch.zeros_like(q["f"])) for q in probs]
        res = blp.solve_batched(items, tol=TOL, concurrency=16, autotune=tuned)
        return max(info.relres for _, info in res)

    def one_at_a_time():
        worst = 0.0
        for q in probs:
            s = blp.Solver(q["N"], q["eps"], q["c1"], q["c2"], q["r"], precision=blp.BLP_FP64, maxit=3000)
            u, info = s.solve(q["f"], tol=TOL)
            s.close()
            worst = max(worst, info.relres)
        return worst
    batched(True)   # warm-up; tunes each (N, precision) once and caches it
    ms_b, rr_b = _timed(torch, dev, lambda: batched(True))
    ms_s, rr_s = _timed(torch, dev, one_at_a_time)
    return {"problems": len(probs), "unknowns": units,
            "batched_mixed": {"ms": round(ms_b, 1), "unknowns_per_s": units / (ms_b * 1e-3), "max_relres": rr_b},
            "one_at_a_time_fp64": {"ms": round(ms_s, 1), "unknowns_per_s": units / (ms_s * 1e-3), "max_relres": rr_s},
            "speedup": round(ms_s / ms_b, 2)}


def leg_adjoint(blp, torch, dev):
    """N = 512, eps = 1e-5, 16 right-hand sides (seed 4): setup, 16 forward
    solves, 16 adjoint solves with M^T and 16 gradient assemblies, to rel-res
    1e-10, in FP64 and mixed precision."""
    from paper_2108_13468_gb300 import inputs
    N, eps, nrhs = 512, 1e-5, 16
    x, _ = blp.mesh(N, eps)
    c1, c2, r = (torch.from_numpy(a).to(dev) for a in inputs.fields_quadratic(x, x))
    coeffs, w = inputs.adjoint_batch(N, nrhs, seed=4)
    fs = [torch.from_numpy(inputs.fourier_rhs(x, x, a)).to(dev) for a in coeffs]
    wt = torch.from_numpy(w).to(dev)
    out = {}
    for prec, pname in ((blp.BLP_FP64, "fp64"), (blp.BLP_MIXED, "mixed")):
        def run():
            s = blp.Solver(N, eps, c1, c2, r, precision=prec)
            g = torch.zeros(3, (N - 1) ** 2, dtype=torch.float64, device=dev)
            for f in fs:
                u, _ = s.solve(f, tol=TOL)
                lam, _ = s.solve_adjoint(wt * u, tol=TOL)
                g1, g2, gr = s.grad(u, lam)
                g[0] += g1
                g[1] += g2
                g[2] += gr
            s.close()
            return g
        run()
        ms, _ = _timed(torch, dev, run)
        out[pname] = {"ms": round(ms, 1), "rhs_per_s": nrhs / (ms * 1e-3),
                      "unknowns_per_s": nrhs * (N - 1) ** 2 / (ms * 1e-3)}
    out["mixed_speedup"] = round(out["fp64"]["ms"] / out["mixed"]["ms"], 2)
    return out


def leg_paper(blp, torch, dev):
    """The paper's own experiment (Sec. 3.3, eq. exponential_MMS, sigma = 5/2,
    c1 = 2, c2 = 3, r = 1, stop ||f - A u||_2 <= 10 ln N / N, FP64 FGMRES on A):
    GPU time-to-solution (setup + solve) beside the paper's CPU seconds."""
    import numpy as np
    from paper_2108_13468_gb300 import inputs
    rows = []
    for eps, cells in PAPER_EXP_TTS.items():
        for N, paper_s, paper_it in cells:
            x, _ = blp.mesh(N, eps, 2.5, 2.0)
            y, _ = blp.mesh(N, eps, 2.5, 3.0)
            f, _ = inputs.mms_exponential(x, y, eps)
            one = np.ones_like(f)
            c1, c2, r, ft = (torch.from_numpy(a).to(dev) for a in (2.0 * one, 3.0 * one, one, f))
            tol = 10.0 * np.log(N) / N

            def run():
                # at eps = 1e-7, N = 2048 the unscaled residual's FP64 floor lies at the
                # paper's absolute target; the cap bounds that cell (its status is reported)
                s = blp.Solver(N, eps, c1, c2, r, sigma=2.5, beta_x=2.0, beta_y=3.0, maxit=100, restart=64,
                               precision=blp.BLP_FP64, stop_mode=blp.BLP_STOP_ABS2)
                u, info = s.solve(ft, tol=tol, raise_on_noconv=False)
                s.close()
                return info
            run()
            ms, info = _timed(torch, dev, run)
            rows.append({"eps": eps, "N": N, "gpu_ms": round(ms, 2), "iters": info.iters, "status": info.status,
                         "paper_s": paper_s, "paper_iters": paper_it, "speedup_vs_paper": round(paper_s * 1e3 / ms, 1)})
    return rows


def run_legs(blp, torch, dev):
    legs = {}
    for name, fn in (("config2_large", leg_large), ("config3_batched", leg_batched),
                     ("config4_adjoint", leg_adjoint), ("paper_mode", leg_paper)):
        try:
            legs[name] = fn(blp, torch, dev)
        except Exception as e:   # a failed leg is reported, the headline line still prints
            legs[name] = {"error": f"{type(e).__name__}: {e}"}
    return legs


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and --impl reference)
# ---------------------------------------------------------------------------
CPU_SAMPLE_EPS = (1e-4, 1e-6, 1e-8)


def cpu_oracle_solve(N, eps):
    import numpy as np
    import oracle
    from paper_2108_13468_gb300 import inputs
    x, _ = oracle.mesh(N, eps)
    p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=0)
    t = time.perf_counter()
    A = oracle.assemble(N, eps, x, x, p.c1, p.c2, p.r)
    P = oracle.Prec(N, eps, x, x, p.c1, p.c2, p.r)
    u, st, it, rr, mc = oracle.fgmres(N, A, p.f, P, tol=TOL)
    dt = time.perf_counter() - t
    assert st == 0 and np.isfinite(u).all()
    return dt


def host_cpu():
    """CPU model and the cores this process may use (the baseline uses one)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = {}
        for line in out.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                fields.setdefault(k.strip(), v.strip())
        if "Model name" in fields:
            model = fields["Model name"] + (f" ({fields['Vendor ID']})" if "Vendor ID" in fields else "")
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    import platform
    return {"model": model or platform.processor() or "unknown", "nproc": usable, "arch": platform.machine()}


def cpu_baseline(N):
    tot = 0.0
    for eps in CPU_SAMPLE_EPS:
        tot += cpu_oracle_solve(N, eps)
    n = (N - 1) ** 2
    return {"value": n * len(CPU_SAMPLE_EPS) / tot, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"oracle (plain C, FP64, 1 thread) setup + FGMRES(30) with the paper's preconditioner to "
                      f"rel-res 1e-10 at N={N}, eps in {{{', '.join(f'{e:g}' for e in CPU_SAMPLE_EPS)}}} "
                      f"({tot:.1f} s); the eps=1e-2 solve (hundreds of iterations) is left out to bound the run"}


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    N = args.N
    n = (N - 1) ** 2
    eps_s = CPU_SAMPLE_EPS
    step = lambda: sum(cpu_oracle_solve(N, e) for e in eps_s)   # noqa: E731
    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    step_s = sum(times) / len(times)
    value = n * len(eps_s) / step_s
    eps = eps_s
    sample = (f"oracle (plain C, FP64, 1 thread) setup + FGMRES(30) to rel-res 1e-10 at N={N}, "
              f"eps in {{{', '.join(f'{e:g}' for e in eps_s)}}} per step (eps=1e-2 left out: hundreds of iterations)")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic",
                      "config": {"workload": f"2D Shishkin N={N} ({n} unknowns), oracle sample of the workload",
                                 "N": N, "eps": list(eps), "tol": TOL},
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                                       "host": host_cpu()},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_profile_target(args):
    """Short fixed workload for ncu: setup on the first eps of --eps, then two
    preconditioner applications (--mode precond) or one solve (--mode solve)."""
    import numpy as np
    import torch
    import paper_2108_13468_gb300 as blp
    dev = torch.device("cuda", 0)
    N, eps = args.N, float(args.eps.split(",")[0])
    prec = blp.BLP_MIXED if args.precision == "mixed" else blp.BLP_FP64
    c1, c2, r, f = [torch.from_numpy(a).to(dev) for a in build_inputs(N, [eps])[eps]]
    s = blp.Solver(N, eps, c1, c2, r, precision=prec)
    lib = s.lib
    if args.mode == "precond":
        v = torch.from_numpy(np.random.default_rng(0).standard_normal((N - 1) ** 2)).to(dev)
        s.precond(v, precision=prec)
        lib.blp_profile(s.handle, 1)     # event-time the second application
        s.precond(v, precision=prec)
    else:
        lib.blp_profile(s.handle, 1)
        s.solve(f, tol=TOL)
    torch.cuda.synchronize()
    classes = merge_profiles([read_profile(lib, s)])
    print(f"profile target done: mode={args.mode} N={N} eps={eps:g} precision={args.precision}")
    print(json.dumps({"kernel_classes": classes}))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode != "bench":
        run_profile_target(a)
    else:
        run_ours(a)
