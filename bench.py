"""Benchmark: Pollock cell-steps/s on the 200x200x20 heterogeneous field.

Workload (one "step"): release 1e6 particles uniformly on the west face of
column 1 (Philox, on the device) and track every one of them to termination
with endpoint records plus timeseries records at 50 log-spaced times, on the
200x200x20 field of 5x5x1 m cells with ln K ~ N(-9.2, 1), exponential
covariance (10, 10, 2) cells, porosity 0.3, constant heads west/east.  The
headline value is the FP64 path; the mixed-precision path (FP32 in-cell,
FP64 time and position) is timed beside it on the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank tracks its own 1e6
particles (disjoint Philox counters) against its own copy of the field:
weak scaling, no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Pollock cell-steps/s (FP32+FP64-time vs FP64) at 1 GB300; request p50/p99 ms"
UNIT = "cell-steps/s"
WORKLOAD = ("200x200x20 cells (5x5x1 m), lnK N(-9.2,1) exp. cov. (10,10,2) cells, porosity 0.3, CH west/east, "
            "PCG head solve; 1e6 particles on the west face of column 1; endpoint + timeseries at 50 log times")
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
SEED_QUADTREE = 0x2302135906


# Algorithmic work per cell-step (one exit-time evaluation), FP64 form, as
# the plain statement of the method performs it (every axis evaluated;
# field-constant work - velocities, A, 1/A - excluded, it belongs to the
# cell, not the step).  Counting FP64 add/mul/compare as 1 flop, an FMA as
# 2 and an IEEE division as 10 (reciprocal seed, two Newton steps and a
# remainder correction):
#   log1p (bucket table, series to r^8): 8 add/mul + 10 FMA     =  28
#   expm1 (32-entry table, series to r^7): 1 mul + 11 FMA       =  23
#   exit time, 3 axes: (10 add/mul/compare + 1 div + log1p) x 3 = 144
#   smallest time, step end, stop test                          =   5
#   motion, 2 axes: (11 add/mul/compare + expm1) x 2            =  68
#   total                                                       = 217 flops.
FP64_FLOPS_PER_STEP = 217.0
# Bytes per cell-step an ideal gather needs: FP64 field 6 x 8 (face flows) +
# 8 (porosity) + 1 (neighbour ibound) = 57 B; FP32 field copy 6 x 4 + 4 + 1.
BYTES_PER_STEP = {"fp64": 57.0, "mixed": 29.0}
# DRAM traffic per full launch (dram__bytes_read.sum + dram__bytes_write.sum)
# of the two tracking kernels, from one ncu capture of the same kernels on
# 2e5 particles of this workload in their tuned launch configurations
# (profiles/k_track_cfg2_200k.md), scaled by
# 5 to the 1e6-particle launch: reads grow with the cell-steps, writes with
# the output records, both in proportion to the particle count.  Each figure
# holds only for the kernel sources it was taken from (the hash beside it,
# kernel_src_hash); otherwise the bench reports it as null.
MIXED_SRC = "d0b109deb9ab3b6a"   # mixed kernel at the capture (unchanged since)
FP64_SRC = "90bd096129eeb0ed"    # FP64 kernel at its capture
TRAFFIC = {"fp64": {"src": FP64_SRC, "value": 5 * (312.961792e6 + 306.072064e6)},
           "mixed": {"src": MIXED_SRC, "value": 5 * (43.280128e6 + 287.389184e6)}}
# From the same capture: the FP64 pipe's busy fraction in the FP64 kernel
# (sm__pipe_fp64_cycles_active, % of peak sustained active), the executed
# counterpart of the algorithmic fraction (which charges every axis's exit
# time while the kernel evaluates the exact one of about 1.1 axes a step).
FP64_PIPE_ACTIVE = {"src": FP64_SRC, "value": 0.7851}
# Warp-instructions per cell-step of the mixed kernel in the same capture
# (smsp__inst_executed.sum / cell-steps on 2e5 particles, static schedule,
# 256 threads: the tuned launch): the mixed kernel is issue-bound, and its
# issue view compares the implied issue rate with one warp-instruction per
# clock per SM sub-partition (152 SMs x 4 x 2.07 GHz).
MIXED_INST_PER_STEP = {"src": MIXED_SRC, "value": 1154103429.0 / 54832447.0}
ISSUE_PEAK_TINST = 152 * 4 * 2.07e9 / 1e12
# L2 read bytes per cell-step in the same capture (lts__t_sectors_srcunit_tex_op_read
# x 32 B / cell-steps): the record gather, cell sizes, output times.
L2_READ_PER_STEP = {"fp64": {"src": FP64_SRC, "value": 254077659.0 * 32 / 54832426.0},
                    "mixed": {"src": MIXED_SRC, "value": 61315161.0 * 32 / 54832447.0}}


# Sources of each tracking kernel's device code: its unit and every header
# it includes (mp_internal.h includes the public mp.h).
KERNEL_SOURCES = {
    "fp64": ("mp_fp64.cu", "mp_f64math.cuh", "mp_f64_tables.h", "mp_sched.cuh", "mp_internal.h", "mp.h"),
    "mixed": ("mp_mixed.cu", "mp_mixed.cuh", "mp_sched.cuh", "mp_internal.h", "mp.h"),
}


def kernel_src_hash(kind: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        d = "include" if name == "mp.h" else os.path.join("paper_2302_13590_gb300", "csrc")
        h.update(name.encode())
        h.update(open(os.path.join(ROOT, d, name), "rb").read())
    return h.hexdigest()[:16]


def ncu_figure(table: dict, kind: str):
    """A counter taken with ncu for one kernel, or None once its sources changed."""
    return table[kind]["value"] if kernel_src_hash(kind) == table[kind]["src"] else None


# GB300 FP64 rate, nominal: 152 SMs x 2.07 GHz x 4 flop/clk/SM = 1.26 TFLOP/s
# (1.25); the roofline uses the rate measured in the run (cuBLAS DGEMM) and
# reports this one beside it.
FP64_PEAK_TFLOPS = 1.25


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def l2_read_gbs(torch, dev) -> float:
    """L2-resident read bandwidth (64 MB buffer summed repeatedly)."""
    x = torch.ones(16 << 20, dtype=torch.float32, device=dev)
    for _ in range(3):
        x.sum()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(50):
        x.sum()
    b.record()
    torch.cuda.synchronize(dev)
    return 50 * x.numel() * 4 / (a.elapsed_time(b) / 1e3) / 1e9


def fp64_peak_tflops(torch, dev) -> float:
    """FP64 rate measured in this run: cuBLAS DGEMM through torch, 4096^3
    (2 N^3 flops), best of 3 after a warm-up (the analogue of the bf16 GEMM
    peak the pool measures; GB300 has no measured FP64 figure)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize(dev)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(w, seconds: float = 10.0, threads: int = 0, idx=None, keep: bool = False, repeats: int = 1):
    """The oracle as it stands (its plain arithmetic, the reference) on the
    host cores: particles handed out in chunks to `threads` threads (the
    paper's dynamic schedule) until `seconds` have passed, in a random
    order; or, with `idx`, exactly those particles, in full.  keep: also
    return the oracle's endpoints of the tracked particles (idx order).
    repeats: track the idx sample that many times over (a workload too small
    to time once)."""
    import oracle as O
    threads = threads or os.cpu_count() or 1
    n = w.release.n
    state = O.release_box(w.field, n, w.release.lo, w.release.hi, w.release.seed)
    of = O.as_oracle_field(w.field)
    if idx is None:
        order = np.random.default_rng(0).permutation(n)
    else:
        order = np.tile(np.asarray(idx, dtype=np.int64), max(1, repeats))
        seconds = float("inf")
    chunk = 512 if order.size >= 64 * threads else max(1, order.size // (4 * threads))
    lock = threading.Lock()
    nxt = [0]
    done = {"steps": 0, "particles": 0}
    parts = {}
    t_end = time.perf_counter() + seconds

    def worker():
        while time.perf_counter() < t_end:
            with lock:
                s = nxt[0]
                nxt[0] += chunk
            if s >= order.size:
                return
            sel = order[s:s + chunk]
            r = O.track(of, O.subset(state, sel), times=w.times)
            with lock:
                done["steps"] += int(r["steps"].astype(np.int64).sum())
                done["particles"] += sel.size
                if keep:
                    parts[s] = r

    t0 = time.perf_counter()
    ths = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    el = time.perf_counter() - t0
    what = ("random subset" if idx is None else
            "a fixed random sample, every one tracked" if repeats <= 1 else
            f"all {len(idx)} of them tracked {repeats} times over")
    out = {"value": done["steps"] / el, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{done['particles']} of the {n:.0e} particles ({what}), endpoint + {len(w.times)} output "
                     f"times, {el:.1f} s wall on {threads} host threads",
           "particles_per_s": done["particles"] / el, "seconds": el}
    if keep:
        ks = sorted(parts)
        out["endpoints"] = {k: np.concatenate([parts[s][k] for s in ks])
                            for k in ("hash", "t", "gx", "gy", "gz", "cell", "status", "steps")}
    return out


def cpu_baselines(args, w2, w1, w3, idx3):
    """The oracle timed on the host cores, 1 thread and all of them, on the
    50x50x1 workload in full, the 200x200x20 workload (all cores: every
    particle; 1 thread: a 3 s sample) and a 1e4-particle sample of the
    400x400x40 workload.  Returns the report and the oracle's endpoints on
    the last sample (used for the accuracy figures of that workload)."""
    cpu = cpu_baseline(w2, seconds=args.cpu_seconds)
    one = cpu_baseline(w2, seconds=min(args.cpu_seconds, 3.0), threads=1)
    cpu["single_thread"] = {"value": one["value"], "sample": one["sample"]}
    strip = lambda d: {k: v for k, v in d.items() if k not in ("endpoints", "unit", "kind")}
    wl = {"cfg2_200x200x20": {"all_cores": strip(cpu), "one_thread": strip(one)}}
    all1 = np.arange(w1.release.n)
    wl["cfg1_50x50x1"] = {"all_cores": strip(cpu_baseline(w1, idx=all1, repeats=1000)),
                          "one_thread": strip(cpu_baseline(w1, idx=all1, threads=1, repeats=100))}
    ref3 = None
    if w3 is not None:
        a3 = cpu_baseline(w3, idx=idx3, keep=True)
        ref3 = a3.pop("endpoints")
        wl["cfg3_400x400x40_1e4_sample"] = {"all_cores": strip(a3),
                                             "one_thread": strip(cpu_baseline(w3, idx=idx3, threads=1))}
    cpu["workloads"] = wl
    return cpu, ref3


def run_reference(args):
    """The oracle (plain single-threaded C per call) on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2302_13590_gb300 import inputs as I
    w = I.workload("cfg2")
    for _ in range(args.warmup):
        cpu_baseline(w, seconds=1.0)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, seconds=args.ref_seconds))
    value = float(np.mean([v["value"] for v in vals]))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean([v["seconds"] for v in vals])) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {**vals[-1], "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_quadtree(ctx, stream) -> dict:
    """The second grid shape (TC2's quadtree refinement): FP64 tracking on a
    rectangular unstructured grid, the same metric."""
    from paper_2302_13590_gb300 import mp
    from paper_2302_13590_gb300.inputs import usg as U
    tq = time.perf_counter()
    u = U.quadtree_field(10, 100, 100, seed=SEED_QUADTREE, n_wells=20, refine_frac=0.15, solver="cg")
    gen_s = time.perf_counter() - tq
    fu = ctx.field(u)
    nq = 1_000_000
    qc, qf = U.explicit_particles(u, nq, seed=SEED_QUADTREE + 1)
    ghq = mp.mp_release_group(ctx.h, fu, cell=qc, local=qf, stream=stream)
    # the launch configuration tuned on this grid, as the main line's
    tuned = mp.mp_autotune(ctx.h, ghq, mp.make_opts(precision=mp.PREC_FP64), sample=0, stream=stream)
    kms = []
    for rep in range(4):
        r = ctx.track(ghq, stream=stream, precision=mp.PREC_FP64, schedule=mp.SCHED_AUTO)
        st = r.stats()
        if rep > 0:
            kms.append(st["kernel_ms"])
        r.free()
    km = float(np.mean(kms))
    rate = st["cell_steps"] / (km / 1e3)
    achieved = FP64_FLOPS_PER_STEP * rate / 1e12
    quadtree = {"workload": f"quadtree: 10 x 100 x 100 base cells, 15 % of the columns and the 20 wells' "
                            f"neighbourhoods split 2 x 2 ({u.ncell} cells, {u.nsub} sub-faces), lnK variance 1, "
                            f"1e6 particles in the western fifth, endpoint mode, FP64",
                "cell_steps_per_s": rate, "particles_per_s": nq / (km / 1e3), "kernel_ms": km,
                "cell_steps": st["cell_steps"], "field_generation_s": gen_s, "tuning": tuned,
                "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": achieved / FP64_PEAK_TFLOPS, "flops_per_cell_step": FP64_FLOPS_PER_STEP,
                             "peak_source": "nominal GB300 FP64"}}
    mp.mp_group_free(ghq)
    mp.mp_field_free(fu)
    return quadtree


CFG3_WORKLOAD = ("400x400x40 cells (5x5x1 m), lnK variance 4, exp. cov. 8 cells, porosity U(0.2, 0.35) per cell, "
                 "20 seeded pumping wells (strong sinks), PCG head solve; 1e7 particles on a seeded plane x = x0; "
                 "endpoint + timeseries at 100 log times (32 GB of records); autotuned persistent launch")


def run_cfg3(ctx, stream, args):
    """The strongly heterogeneous workload the mixed form is quoted on: both
    precisions, each with its autotuned launch (tuned on a 2e6-particle
    prefix), two timed launches after an untimed one.  Returns the report,
    the workload, a 1e4-particle sample and the GPU endpoints on it."""
    from paper_2302_13590_gb300 import inputs as I
    from paper_2302_13590_gb300 import mp
    tg = time.perf_counter()
    w3 = I.workload("cfg3", n_particles=args.cfg3_particles or None)
    gen_s = time.perf_counter() - tg
    fh3 = ctx.field(w3.field)
    n3 = w3.release.n
    idx3 = np.sort(np.random.default_rng(4).choice(n3, min(10_000, n3), replace=False))
    rep3 = {"workload": CFG3_WORKLOAD, "particles": n3, "output_times": len(w3.times),
            "field_generation_s": gen_s, "field_bytes": mp.mp_field_bytes(fh3)}
    eps = {}
    mode = mp.MODE_ENDPOINT | mp.MODE_TIMESERIES
    for name, prec in (("mixed", mp.PREC_MIXED), ("fp64", mp.PREC_FP64)):
        gh = mp.mp_release_group(ctx.h, fh3, n=n3, lo=w3.release.lo, hi=w3.release.hi, seed=w3.release.seed,
                                 stream=stream)
        tuned = mp.mp_autotune(ctx.h, gh, mp.make_opts(mode=mode, precision=prec, times=w3.times),
                               sample=min(n3, 2_000_000), stream=stream)
        mp.mp_group_free(gh)
        kms, steps = [], 0
        for rep in range(3):
            gh = mp.mp_release_group(ctx.h, fh3, n=n3, lo=w3.release.lo, hi=w3.release.hi, seed=w3.release.seed,
                                     stream=stream)
            r = ctx.track(gh, stream=stream, mode=mode, precision=prec, schedule=mp.SCHED_AUTO, times=w3.times)
            st = r.stats()
            assert st["device_error"] == 0
            if rep > 0:
                kms.append(st["kernel_ms"])
                steps = st["cell_steps"]
            if rep == 2:
                ep = r.endpoints()
                eps[name] = {k: ep[k][idx3] for k in ("hash", "t", "x", "y", "z", "cell", "status")}
            r.free()
            mp.mp_group_free(gh)
        km = float(np.mean(kms))
        rep3[name] = {"cell_steps_per_s": steps / (km / 1e3), "particles_per_s": n3 / (km / 1e3), "kernel_ms": km,
                      "cell_steps": steps, "tuning": tuned}
    mp.mp_field_free(fh3)
    return rep3, w3, idx3, eps


def accuracy(field, ep, ref) -> dict:
    """GPU endpoints against the oracle's (both on the same particles):
    share of diverging cell sequences; on the others, relative travel-time
    error and endpoint error in cell widths (median, p99, max, share within
    the mixed form's stated 1e-5 and 1e-4)."""
    same = ep["hash"] == ref["hash"]
    fin = same & np.isfinite(ref["t"]) & (ref["t"] > 0)
    t_err = np.abs(ep["t"][fin] - ref["t"][fin]) / ref["t"][fin]
    c = ref["cell"][fin]
    j, i, k = c % field.ncol, (c // field.ncol) % field.nrow, c // (field.ncol * field.nrow)
    pos = np.maximum(np.abs(ep["x"][fin] - ref["gx"][fin]) / field.delr[j],
                     np.maximum(np.abs(ep["y"][fin] - ref["gy"][fin]) / field.delc[i],
                                np.abs(ep["z"][fin] - ref["gz"][fin]) / field.dz[k]))
    q = lambda a, v: float(np.quantile(a, v)) if a.size else 0.0
    return {"particles": int(same.size), "divergent_fraction": float(1.0 - same.mean()),
            "t_rel_err": {"median": q(t_err, 0.5), "p99": q(t_err, 0.99), "max": q(t_err, 1.0),
                          "within_1e-5": float(np.mean(t_err <= 1e-5)) if t_err.size else 1.0},
            "pos_err_cells": {"median": q(pos, 0.5), "p99": q(pos, 0.99), "max": q(pos, 1.0),
                              "within_1e-4": float(np.mean(pos <= 1e-4)) if pos.size else 1.0},
            "reference": "oracle, plain arithmetic (C library log1p/expm1, FP64)"}


def summary(line) -> dict:
    """The figures a reader needs first, last on the line (so a truncated
    log keeps them): both precisions on both heterogeneous workloads, their
    roofline fractions, batch and serving."""
    g = lambda d, *ks: (None if d is None else (g(d.get(ks[0]), *ks[1:]) if ks else d))
    r3 = lambda v: None if v is None else float(f"{v:.3g}")
    out = {"fp64_cfg2": r3(line["value"]), "fp64_cfg2_frac_alu": r3(g(line, "roofline", "frac")),
           "mixed_cfg2": r3(g(line, "mixed", "value")),
           "mixed_f64t_cfg2": r3(g(line, "mixed", "f64t_form", "cell_steps_per_s")),
           "mixed_cfg2_frac_hbm": r3(g(line, "mixed", "roofline", "frac")),
           "mixed_cfg2_frac_l2": r3(g(line, "mixed", "roofline", "l2_view", "frac")),
           "e2e_fp64": r3(g(line, "e2e", "value")), "e2e_mixed": r3(g(line, "e2e", "mixed"))}
    c3 = line.get("cfg3")
    if c3:
        for nm in ("mixed", "fp64"):
            out[f"{nm}_cfg3"] = r3(g(c3, nm, "cell_steps_per_s"))
            out[f"{nm}_cfg3_particles_per_s"] = r3(g(c3, nm, "particles_per_s"))
            out[f"{nm}_cfg3_frac"] = r3(g(c3, nm, "roofline", "frac"))
            acc = g(c3, nm, "accuracy")
            if acc:
                out[f"{nm}_cfg3_divergent"] = r3(acc["divergent_fraction"])
                out[f"{nm}_cfg3_t_err_p99"] = r3(acc["t_rel_err"]["p99"])
    b = line.get("batch")
    if b:
        out["batch_mixed"] = r3(g(b, "mixed", "cell_steps_per_s"))
        out["batch_fp64"] = r3(g(b, "fp64", "cell_steps_per_s"))
    sv = line.get("serving")
    if sv:
        for nm in ("mixed", "fp64"):
            out[f"serve_{nm}_p50_p99_ms"] = [r3(g(sv, nm, "p50_ms")), r3(g(sv, nm, "p99_ms"))]
            out[f"serve_{nm}_requests"] = g(sv, nm, "requests")
            out[f"serve_{nm}_particles_per_s"] = r3(g(sv, nm, "particles_per_s"))
            out[f"serve_{nm}_max_concurrent_batches"] = g(sv, nm, "max_concurrent_batches")
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2302_13590_gb300 import inputs as I
    from paper_2302_13590_gb300 import mp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2302_13590_gb300 import replicas
    w = I.workload("cfg2")
    n_part = args.particles or w.release.n
    rel = replicas.shard_release(I.Release(n_part, w.release.lo, w.release.hi, w.release.seed), rank)
    n = rel.n
    nt = len(w.times)
    ctx = mp.Context(local)
    fh = ctx.field(w.field)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def maxed(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def summed(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    def one_step(prec, sched):
        gh = mp.mp_release_group(ctx.h, fh, n=n, lo=rel.lo, hi=rel.hi, seed=rel.seed, id_offset=rel.id_offset,
                                 stream=stream)
        ts_mode = args.mode != "endpoint"
        opts = mp.make_opts(mode=mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if ts_mode else 0), precision=prec,
                            schedule=sched, times=w.times if ts_mode else None, block=args.block,
                            steps_per_fetch=args.spf)
        rid = mp.mp_track(ctx.h, gh, opts, stream)
        return gh, rid

    def timed(prec, sched, steps, warmup):
        for _ in range(warmup):
            gh, rid = one_step(prec, sched)
            mp.mp_wait(ctx.h, rid)
            mp.mp_req_free(ctx.h, rid)
            mp.mp_group_free(gh)
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        live = []
        clk = ClockSampler(local)
        clk.start()
        t_wall = time.perf_counter()
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            evs[k][0].record(stream)
            live.append(one_step(prec, sched))
            evs[k][1].record(stream)
        barrier()
        wall = time.perf_counter() - t_wall
        clocks = clk.stop()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        cell_steps = 0
        kern_ms = []
        counts = np.zeros(8, np.int64)
        for gh, rid in live:
            st = mp.mp_get_stats(ctx.h, rid)
            assert st["device_error"] == 0
            cell_steps += st["cell_steps"]
            kern_ms.append(st["kernel_ms"])
            counts += np.array(st["n_status"])
            mp.mp_req_free(ctx.h, rid)
            mp.mp_group_free(gh)
        return {"ms": ms, "wall_s": wall, "cell_steps": cell_steps, "kernel_ms": kern_ms, "clocks": clocks,
                "status_counts": counts.tolist()}

    # autotune the launch (block, schedule, steps per fetch) per precision on
    # the whole group, outside the timed region: tail and queue costs depend
    # on the particle count, so a smaller sample can rank the candidates wrongly
    tuning = {}
    if args.schedule == mp.SCHED_AUTO:
        for name, prec in (("fp64", mp.PREC_FP64), ("mixed", mp.PREC_MIXED)):
            if name not in args.precisions:
                continue
            gh = mp.mp_release_group(ctx.h, fh, n=n, lo=rel.lo, hi=rel.hi, seed=rel.seed, id_offset=rel.id_offset,
                                     stream=stream)
            o = mp.make_opts(mode=mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if args.mode != "endpoint" else 0),
                             precision=prec, times=w.times if args.mode != "endpoint" else None)
            tuning[name] = mp.mp_autotune(ctx.h, gh, o, sample=0, stream=stream)
            mp.mp_group_free(gh)

    results = {}
    precs = [(nm, pr) for nm, pr in (("fp64", mp.PREC_FP64), ("mixed", mp.PREC_MIXED)) if nm in args.precisions]
    for name, prec in precs:
        r = timed(prec, args.schedule, args.steps, args.warmup)
        steps_all, ms_max, value = replicas.job_rate(r["cell_steps"], r["ms"], world, dev)
        results[name] = dict(r, ms_max=ms_max, cell_steps_all=steps_all, value=value,
                             particles_per_s=summed(n * args.steps) / (ms_max / 1e3))

    # the mixed form with FP64 kept for the cumulative time and the near-zero
    # branch of the exit time (MP_PREC_MIXED_F64T), same workload: what those
    # two FP64 pieces cost on this GPU
    f64t = None
    if "mixed" in args.precisions and not args.particles and not args.no_f64t_form:
        gh = mp.mp_release_group(ctx.h, fh, n=n, lo=rel.lo, hi=rel.hi, seed=rel.seed, id_offset=rel.id_offset,
                                 stream=stream)
        kms = []
        for rep in range(3):
            r = ctx.track(gh, stream=stream, mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES,
                          precision=mp.PREC_MIXED_F64T, schedule=mp.SCHED_DYNAMIC, times=w.times)
            st = r.stats()
            if rep > 0:
                kms.append(st["kernel_ms"])
            r.free()
        mp.mp_group_free(gh)
        f64t = {"cell_steps_per_s": st["cell_steps"] / (np.mean(kms) / 1e3), "kernel_ms": float(np.mean(kms)),
                "what": "FP64 cumulative time and FP64 log1p(z)/z near z = 0; dynamic schedule, 128 threads"}

    # end to end through the C ABI with host buffers (mp_track_host): pinned host release
    # arrays in, endpoint and timeseries records out, every step
    e2e = None
    if not args.no_e2e:
        rng = np.random.default_rng(7)
        s0 = results  # noqa: F841
        ep_host = {k: torch.empty(n, dtype=getattr(torch, np.dtype(dt).name), pin_memory=True).numpy()
                   for k, dt in mp.ENDPOINT_DTYPES.items() if k != "hash"}
        ep_host["hash"] = torch.empty(n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        ts_host = torch.empty(nt * n * 32, dtype=torch.uint8, pin_memory=True).numpy().view(mp.TS_RECORD).reshape(nt, n)
        # explicit release arrays = the device release of this step's particles
        gh0 = mp.mp_release_group(ctx.h, fh, n=n, lo=rel.lo, hi=rel.hi, seed=rel.seed, id_offset=rel.id_offset)
        r0 = ctx.track(gh0, t_stop=0.0, schedule=mp.SCHED_STATIC)
        ep0 = r0.endpoints()
        r0.free()
        mp.mp_group_free(gh0)
        cells_h = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy()
        local_h = torch.empty(3 * n, dtype=torch.float64, pin_memory=True).numpy()
        cells_h[:] = ep0["cell"]
        c = ep0["cell"]
        j, i, k = c % w.field.ncol, (c // w.field.ncol) % w.field.nrow, c // (w.field.ncol * w.field.nrow)
        local_h[0::3] = ep0["px"] / w.field.delr[j]
        local_h[1::3] = ep0["py"] / w.field.delc[i]
        local_h[2::3] = ep0["pz"] / w.field.dz[k]
        h2d = cells_h.nbytes + local_h.nbytes
        d2h = sum(a.nbytes for a in ep_host.values()) + ts_host.nbytes
        e2e_vals = {}
        for name, prec in (("fp64", mp.PREC_FP64), ("mixed", mp.PREC_MIXED)):
            tot_steps = 0
            opts = mp.make_opts(mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, precision=prec,
                                schedule=args.schedule, times=w.times)
            for _ in range(args.warmup):   # untimed: memory pool growth, first launches
                mp.mp_track_host(ctx.h, fh, cells_h, local_h, opts, n_chunks=args.e2e_chunks, out=ep_host,
                                 ts_out=ts_host)
            barrier()
            t0 = time.perf_counter()
            calls = []
            # at least 10 calls: a host-side stall of one call (seen now and
            # then, 60-70 ms) then moves the mean by a few percent, not by a
            # quarter
            for _ in range(max(args.steps, 10)):
                # one call: chunked release + tracking on two streams, result
                # copies of one chunk overlapping the tracking of the next
                tc = time.perf_counter()
                _, _, st = mp.mp_track_host(ctx.h, fh, cells_h, local_h, opts, n_chunks=args.e2e_chunks,
                                            out=ep_host, ts_out=ts_host)
                calls.append(round((time.perf_counter() - tc) * 1e3, 2))
                tot_steps += st["cell_steps"]
            barrier()
            el = maxed(time.perf_counter() - t0)
            e2e_vals[name] = summed(tot_steps) / el
            e2e_vals[name + "_ms_per_call"] = calls
        e2e = {"value": e2e_vals["fp64"], "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "mixed": e2e_vals["mixed"], "calls": max(args.steps, 10),
               "ms_per_call": {"fp64": e2e_vals["fp64_ms_per_call"], "mixed": e2e_vals["mixed_ms_per_call"]},
               "call": "mp_track_host: pinned host arrays in and out; chunks on two streams, copies overlapped"}

    if rank != 0:
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return
    if args.precisions != "fp64,mixed" or args.mode != "endpoint+timeseries" or args.particles:
        # a partial run (profiling cases): report the timings only
        print(json.dumps({k: {"value": v["value"], "ms": v["ms_max"], "kernel_ms": v["kernel_ms"]}
                          for k, v in results.items()}), flush=True)
        ctx.close()
        return

    hbm, src = _peaks()
    l2 = l2_read_gbs(torch, dev)
    try:
        fp64_peak, fp64_src = fp64_peak_tflops(torch, dev), "measured in this run: cuBLAS DGEMM 4096^3, best of 3"
    except Exception as exc:   # keep the nominal figure when the probe cannot run
        fp64_peak, fp64_src = FP64_PEAK_TFLOPS, f"nominal GB300 FP64 (152 SMs x 2.07 GHz x 4 flop/clk); probe: {exc}"
    rf = {}
    for name in ("fp64", "mixed"):
        r = results[name]
        kms = float(np.mean(r["kernel_ms"]))
        steps_per_launch = r["cell_steps"] / len(r["kernel_ms"])
        rate = steps_per_launch / (kms / 1e3)
        gbs = BYTES_PER_STEP[name] * rate / 1e9
        traffic = args.traffic_fp64 if name == "fp64" else args.traffic_mixed
        if traffic is None:
            traffic = ncu_figure(TRAFFIC, name)
        l2_ncu = None
        l2b = ncu_figure(L2_READ_PER_STEP, name)
        if l2b is not None:
            l2_ncu = {"bytes_per_cell_step": l2b, "gbs": l2b * rate / 1e9, "peak_gbs": l2,
                      "frac": l2b * rate / 1e9 / l2}
        if name == "fp64":
            achieved = FP64_FLOPS_PER_STEP * rate / 1e12
            rf[name] = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                        "frac": achieved / fp64_peak, "traffic": traffic, "peak_source": fp64_src,
                        "nominal_peak": FP64_PEAK_TFLOPS, "frac_of_nominal": achieved / FP64_PEAK_TFLOPS,
                        "flops_per_cell_step": FP64_FLOPS_PER_STEP, "kernel_ms": kms,
                        "cell_steps_per_launch": steps_per_launch,
                        "fp64_pipe_active_ncu": (FP64_PIPE_ACTIVE["value"]
                                                 if kernel_src_hash("fp64") == FP64_PIPE_ACTIVE["src"] else None),
                        "hbm_view": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                                     "bytes_per_cell_step": BYTES_PER_STEP[name]},
                        "l2_read_ncu": l2_ncu}
        else:
            rf[name] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                        "traffic": traffic, "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)",
                        "bytes_per_cell_step": BYTES_PER_STEP[name], "kernel_ms": kms,
                        "cell_steps_per_launch": steps_per_launch,
                        "l2_view": {"achieved": gbs, "peak": l2, "unit": "GB/s", "frac": gbs / l2,
                                    "peak_source": "measured in this run: L2-resident 64 MB read"},
                        "l2_read_ncu": l2_ncu}
            if kernel_src_hash("mixed") == MIXED_INST_PER_STEP["src"]:
                ti = MIXED_INST_PER_STEP["value"] * rate / 1e12
                rf[name]["issue_view"] = {"achieved": ti, "peak": ISSUE_PEAK_TINST, "unit": "Twarp-inst/s",
                                          "frac": ti / ISSUE_PEAK_TINST,
                                          "warp_inst_per_cell_step": MIXED_INST_PER_STEP["value"],
                                          "peak_source": "nominal: 1 warp-instruction/clk per SMSP, 608 SMSPs, "
                                                         "2.07 GHz"}
    batch = None
    if not args.no_batch:
        try:
            specs = I.batch_workload()
            batch = {"workload": "256 requests on the 200x200x20 field, sizes log-uniform in 1e2..1e6 (3.0e7 particles), "
                                 "random boxes, half with 20 output times; one launch per precision, autotuned"}
            # autotune the batch's launch per precision and mode on its largest
            # request (the launch takes the tuned configuration of its first
            # request of that precision)
            big = max(specs, key=lambda x: x.release.n)
            ts_times = next(x.times for x in specs if x.timeseries)
            batch_tuning = {}
            for name, prec in (("mixed", mp.PREC_MIXED), ("fp64", mp.PREC_FP64)):
                for tsm in (False, True):
                    gh = mp.mp_release_group(ctx.h, fh, n=big.release.n, lo=big.release.lo, hi=big.release.hi,
                                             seed=big.release.seed, stream=stream)
                    o = mp.make_opts(mode=mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if tsm else 0), precision=prec,
                                     times=ts_times if tsm else None)
                    batch_tuning[f"{name}_{'timeseries' if tsm else 'endpoint'}"] = mp.mp_autotune(ctx.h, gh, o, sample=0,
                                                                                                 stream=stream)
                    mp.mp_group_free(gh)
            batch["tuning"] = batch_tuning
            for name, prec in (("mixed", mp.PREC_MIXED), ("fp64", mp.PREC_FP64)):
                best = None
                for rep in range(2):
                    groups = [mp.mp_release_group(ctx.h, fh, n=x.release.n, lo=x.release.lo, hi=x.release.hi,
                                                  seed=x.release.seed, stream=stream) for x in specs]
                    opts = [mp.make_opts(mode=mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if x.timeseries else 0),
                                         precision=prec, schedule=mp.SCHED_AUTO, times=x.times) for x in specs]
                    ids = mp.mp_track_batch(ctx.h, groups, opts, stream)
                    sts = [mp.mp_get_stats(ctx.h, i) for i in ids]
                    steps_b = sum(x["cell_steps"] for x in sts)
                    kms = sts[0]["kernel_ms"]
                    for i in ids:
                        mp.mp_req_free(ctx.h, i)
                    for g in groups:
                        mp.mp_group_free(g)
                    if rep == 1:
                        best = {"cell_steps_per_s": steps_b / (kms / 1e3), "kernel_ms": kms, "cell_steps": steps_b,
                                "particles": int(sum(x.release.n for x in specs))}
                batch[name] = best
            # the same kind of batch captured once as a CUDA graph (one batched
            # release, one tracking launch per precision) and replayed, against
            # the host-side sequence (a release per group, the batch table, the
            # tracking launch); wall time per batch, host included
            def wall_ms(fn, reps):
                fn()
                t0 = time.perf_counter()
                for _ in range(reps):
                    fn()
                return (time.perf_counter() - t0) / reps * 1e3

            rng = np.random.default_rng(7)
            Lx, Ly, Lz = w.field.extent
            small = []
            for i in range(256):
                nn = int(np.exp(rng.uniform(np.log(200), np.log(2000))))
                lo = np.array([rng.uniform(0, 0.5 * Lx), rng.uniform(0, 0.5 * Ly), 0.0])
                small.append(I.Release(nn, tuple(lo), tuple(lo + [0.1 * Lx, 0.1 * Ly, Lz]), seed=500 + i))
            graph = {}
            for key, rels, optf, reps in (
                    ("small", small, lambda x: mp.make_opts(precision=mp.PREC_MIXED), 20),
                    ("batch_workload_mixed", [x.release for x in specs],
                     lambda x: mp.make_opts(mode=mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if x.timeseries else 0),
                                            precision=mp.PREC_MIXED, times=x.times), 3)):
                opts = [optf(x) for x in (specs if key != "small" else rels)]

                def direct():
                    groups = [mp.mp_release_group(ctx.h, fh, n=r.n, lo=r.lo, hi=r.hi, seed=r.seed, stream=stream)
                              for r in rels]
                    ids = mp.mp_track_batch(ctx.h, groups, opts, stream)
                    stream.synchronize()
                    for i in ids:
                        mp.mp_req_free(ctx.h, i)
                    for g in groups:
                        mp.mp_group_free(g)

                gh, gids = mp.mp_graph_create(ctx.h, fh, rels, opts, stream=stream)

                def replay():
                    mp.mp_graph_launch(gh, stream=stream)
                    stream.synchronize()

                d_ms, g_ms = wall_ms(direct, reps), wall_ms(replay, reps)
                steps_g = sum(mp.mp_get_stats(ctx.h, i)["cell_steps"] for i in gids)
                mp.mp_graph_free(gh)
                graph[key] = {"requests": len(rels), "particles": int(sum(r.n for r in rels)), "direct_ms": d_ms,
                              "graph_ms": g_ms, "graph_cell_steps_per_s": steps_g / (g_ms / 1e3)}
            graph["small"]["workload"] = ("256 requests of 200..2000 particles (log-uniform) in random boxes, mixed "
                                          "precision, endpoint mode")
            batch["graph"] = graph
        except Exception as exc:   # an extra block must not cost the headline line
            batch = {"error": repr(exc)}

    quadtree = None
    if not args.no_quadtree:
        try:
            quadtree = run_quadtree(ctx, stream)
        except Exception as exc:   # an extra block must not cost the headline line
            quadtree = {"error": repr(exc)}
    if quadtree is not None and "roofline" in quadtree:
        qr = quadtree["roofline"]
        qr.update(peak=fp64_peak, frac=qr["achieved"] / fp64_peak, peak_source=fp64_src,
                  nominal_peak=FP64_PEAK_TFLOPS, frac_of_nominal=qr["achieved"] / FP64_PEAK_TFLOPS)

    serving = None
    if not args.no_serve:
        try:
            from paper_2302_13590_gb300 import serve as SV
            fields = {"cfg1": ctx.field(I.cfg1_field()), "cfg2": fh}
            serving = {}
            for name, prec, nreq in (("mixed", mp.PREC_MIXED, args.serve_requests),
                                     ("fp64", mp.PREC_FP64, args.serve_requests)):
                specs = I.serving_workload(n_req=nreq, rate_hz=200.0)
                srv = SV.Server(ctx, fields, precision=prec, schedule=mp.SCHED_STATIC)
                rep = srv.run(specs, realtime=True)
                sm = rep.summary()
                sm["offered_requests_per_s"] = 200.0
                sm["offered_particles_per_s"] = float(sum(x.release.n for x in specs)) / specs[-1].arrival_s
                serving[name] = sm
            serving["workload"] = ("Poisson arrivals at 200 requests/s on the 50x50x1 and 200x200x20 fields (p = 1/2), "
                                   "group sizes log-uniform in 1e3..1e6, endpoint or 20-time timeseries at random")
        except Exception as exc:   # an extra block must not cost the headline line
            serving = {"error": repr(exc)}
    cfg3 = w3 = idx3 = eps3 = None
    if not args.no_cfg3:
        try:
            cfg3, w3, idx3, eps3 = run_cfg3(ctx, stream, args)
            for name in ("mixed", "fp64"):
                rate = cfg3[name]["cell_steps_per_s"]
                gbs = BYTES_PER_STEP[name] * rate / 1e9
                if name == "fp64":
                    a = FP64_FLOPS_PER_STEP * rate / 1e12
                    cfg3[name]["roofline"] = {"bound": "alu", "achieved": a, "peak": fp64_peak, "unit": "TFLOP/s",
                                              "frac": a / fp64_peak, "peak_source": fp64_src,
                                              "hbm_view": {"achieved": gbs, "peak": hbm, "frac": gbs / hbm}}
                else:
                    cfg3[name]["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                              "frac": gbs / hbm, "bytes_per_cell_step": BYTES_PER_STEP[name],
                                              "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)",
                                              "l2_view": {"achieved": gbs, "peak": l2, "frac": gbs / l2}}
        except Exception as exc:   # an extra block must not cost the headline line
            cfg3 = {"error": repr(exc)}
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu, ref3 = cpu_baselines(args, w, I.workload("cfg1"), w3, idx3)
            if ref3 is not None:
                # the oracle's endpoints of the timed sample against the GPU's on
                # the same particles (numpy only)
                for name in ("mixed", "fp64"):
                    cfg3[name]["accuracy"] = accuracy(w3.field, eps3[name], ref3)
        except Exception as exc:   # an extra block must not cost the headline line
            cpu = {"error": repr(exc)}
    f64 = results["fp64"]
    line = {
        "metric": METRIC, "value": f64["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": f64["ms_max"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles_per_gpu": n, "output_times": nt,
                   "schedule": {0: "static", 1: "dynamic", 2: "autotuned"}[args.schedule],
                   "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{world}"},
        "particles_per_s": f64["particles_per_s"],
        "roofline": rf["fp64"],
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps * 2,
        "clocks": f64["clocks"],
        "mixed": {"value": results["mixed"]["value"], "ms_per_step": results["mixed"]["ms_max"] / args.steps,
                  "particles_per_s": results["mixed"]["particles_per_s"], "dtype": "f32+f64",
                  "roofline": rf["mixed"], "clocks": results["mixed"]["clocks"], "f64t_form": f64t},
        "status_counts": f64["status_counts"],
        "serving": serving,
        "batch": batch,
        "quadtree": quadtree,
        "cfg3": cfg3,
        "tuning": tuning or None,
    }
    line["summary"] = summary(line)
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--schedule", type=int, default=2, help="0 static, 1 dynamic, 2 autotuned (default)")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--spf", type=int, default=0)
    ap.add_argument("--particles", type=int, default=0, help="override the particle count (profiling cases)")
    ap.add_argument("--precisions", default="fp64,mixed")
    ap.add_argument("--mode", default="endpoint+timeseries", choices=["endpoint+timeseries", "endpoint"],
                    help="profiling cases only; the benchmark line uses endpoint+timeseries")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=0, help="chunks of the end-to-end call (0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-quadtree", action="store_true")
    ap.add_argument("--only-quadtree", action="store_true", help="run the quadtree line alone (profiling)")
    ap.add_argument("--serve-requests", type=int, default=5000)
    ap.add_argument("--no-cfg3", action="store_true")
    ap.add_argument("--no-f64t-form", action="store_true", help="skip timing the FP64-time mixed form (profiling)")
    ap.add_argument("--cfg3-particles", type=int, default=0, help="override cfg3's 1e7 particles (quick checks)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--traffic-fp64", type=float, default=None,
                    help="ncu dram bytes per full launch of the FP64 kernel (from profiles/)")
    ap.add_argument("--traffic-mixed", type=float, default=None,
                    help="ncu dram bytes per full launch of the mixed kernel (from profiles/)")
    args = ap.parse_args()
    if args.only_quadtree:
        import torch
        from paper_2302_13590_gb300 import mp
        torch.cuda.set_device(0)
        ctx = mp.Context(0)
        stream = torch.cuda.Stream()
        print(json.dumps({"quadtree": run_quadtree(ctx, stream)}), flush=True)
        ctx.close()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
