"""Benchmark of the MXE hot path on one GB300 (or N independent replicas).

Workload: the 256,000-site binary substitutional alloy (FCC 40^3 cells,
a = 3.6 A, x_A ~ U(0.85, 0.95), x_B = 0.999 - x_A, T = 1000 K), synthetic and
seeded.  One step = one pass of the whole hot path from the initial state:
neighbour/bond build, free energy + three gradients (excess chemical
potentials), one Euler step of the master equation, and a FIRE relaxation of
K iterations (K + 1 further free-energy/gradient evaluations).  The literal
potential of this workload has no free-energy minimum in sigma, so the
relaxation runs a fixed iteration count; every step restarts from the same
initial state so each timed step does identical work.

value = site free-energy+gradient evaluations per second over all ranks
(evaluations = n_sites x (K + 2) per step); diffusion steps/s is reported
beside it.  Timed with CUDA events on the library's stream, L2 flushed
(256 MB write) between steps outside the timed region.

--impl reference times the CPU oracle on the host cores (one neighbour build,
one free-energy/gradient evaluation and one Euler step of the same state per
step; value in the same unit).

--workload ensemble measures the batched ensemble instead: 512 independent
periodic single-species lattices (4..16 cells per side, 2.85 M sites in
all, T ~ U(300, 1200) K, vacancy fraction ~ U(1e-4, 1e-2) per system) in one
batched context, with the stable variant of the single-species potential
(pair exponent 5, density exponent 3: the literal one collapses the lattice
within ~40 steps of 10 FIRE iterations at fixed box, and its sigma has no
minimum), relax+diffuse loop replayed from one captured CUDA graph
(mxe_run_staggered), per-system Euler step = the system's stable step, pass
shape chosen by the autotuner.  The working set (~1 GB) exceeds L2, so no
flush is needed between steps.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1910_01235_gb300 import workloads as W  # noqa: E402

METRIC = "site free-energy+gradient evals/s and diffusion steps/s, FP32-mixed vs FP64"
WORKLOAD = "binary_alloy_fcc40_256k"
FIRE_ITERS = 10
DTYPES = {"fp64": "f64", "mixed": "f32 (f64 sums; mu from float-float node arithmetic)",
          "ff": "f32 (float-float sums and mu)"}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ---------------------------------------------------------------- replicas
# With N ranks every rank runs its own independent replica of the workload (its
# own seed): the path has no data exchange between systems, so there is no
# data-path collective; the ranks meet only at barriers and at the maximum of
# their step times.
def replica_workload(rank):
    return W.config_binary_alloy(seed=W.SEED + rank)


def max_over_ranks(value, dist, device=None):
    """Maximum of a float over all ranks (identity with one rank)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank_step, ms_per_step_max, world):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank_step / (ms_per_step_max / 1e3)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (clock, reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- algorithmic work
# FP32-pipe operations per (i, j) pair of each pass, counted from the algorithm
# as the kernels evaluate it (an FMA counts as one operation: one issue slot of
# the FP32 pipe).  n_phi, n_f: distinct pair and density terms; S species.
def ops_per_pair(kernel, n_phi, n_f, S):
    if kernel.startswith("density_fp32"):
        node = 2 + 7 + 2 * n_f                      # distance, switch, terms
        return 13 * node + 20 + 2 * S * S + 12 * S  # 12 nodes + static point, set-up, sums
    if kernel.startswith("gradient_fp32") and kernel.endswith("force_noe"):
        node = 2 + 11 + 3 * (n_phi + n_f) + 3 + 4.25   # distance, switch, factored terms, G, force sums
        static = 2 + 11 + 4 * n_f + 1
        pair = 20 + S * S + 4 * S * S + (n_phi + n_f) + 9 + 24
        return 12 * node + static + pair
    # float-float passes (csrc/ff.cuh): add 11, mul 7, exp 64 FP32 operations; per
    # radial term at a node: argument 18 + exp 64 + switch product 7 + sum 11
    # (the implementation's own count: quoted for these kernels only, never as
    # the step's roofline unless they are the largest share)
    term = 18 + 64 + 7 + 11
    node = 11 + 10 + 3                      # node distance, square root, switch test
    if kernel.startswith("density_ff"):
        return 13 * (node + term * n_f) + 300
    if kernel.startswith("gradient_ff"):
        return 12 * (node + term * (n_phi + n_f)) + (node + term * n_f) + 500
    if kernel == "pair_ff":                 # once per unordered pair: 12 nodes x all terms + static f
        return 12 * (node + term * (n_phi + n_f)) + (node + term * n_f) + 60
    if kernel == "pair32_density":          # the FP32 density terms of one unordered pair (13 points)
        return 13 * (2 + 7 + 2 * n_f) + 20
    if kernel == "pair32_force":            # the FP32 forces of one unordered pair, both width derivatives
        node = 2 + 11 + 3 * (n_phi + n_f) + 3 + 4.25 + 2
        return 12 * node + (2 + 11 + 4 * n_f + 1) + (20 + S * S + 4 * S * S + (n_phi + n_f) + 9 + 24)
    return None


def units_per_launch(kernel, entries):
    """Units the ops count applies to: the half-list kernels evaluate each
    unordered pair once, the full-list kernels each neighbour entry."""
    return entries // 2 if kernel.startswith("pair") else entries


def peak_fp32_ops(clock_mhz=2070.0):
    """FP32 pipe: 152 SMs x 128 lanes x clock (one FMA or add or multiply per lane per cycle)."""
    return 152 * 128 * clock_mhz * 1e6


def peak_fp64_ops(clock_mhz=2070.0):
    """FP64 pipe: the nominal 1.25 TFLOP/s of a GB300 (FMA = 2 flops) is 2
    FP64 instructions per SM per cycle: 152 SMs x 2 x clock."""
    return 152 * 2 * clock_mhz * 1e6


def kernel_shares(kern):
    """Per kernel class: launches, total and mean device time, share of the step."""
    shares = {}
    tot_k = sum(v[1] for v in kern.values()) if kern else 0.0
    for k_, (cnt, tms) in (kern or {}).items():
        shares[k_] = {"launches": cnt, "total_ms": tms, "avg_ms": tms / cnt, "share": tms / tot_k if tot_k else None}
    return shares


def roofline_of(shares, npairs, S, n_phi, n_f, with_traffic):
    """Roofline of the step's dominant kernel (largest share of the device
    time).  FP32-pipe kernels: algorithmic operations per pair (ops_per_pair)
    x pairs of one launch / mean launch time, against the FP32 lane count x
    clock.  FP64 kernels: FP64-pipe instructions of one launch (ncu count of
    the committed capture) / mean launch time, against the FP64 pipe's
    instruction rate -- the pipe utilisation."""
    if not shares:
        return None
    dom = max(shares, key=lambda k_: shares[k_]["total_ms"])
    avg_s = shares[dom]["avg_ms"] / 1e3
    fp64 = "64" in dom or dom.endswith("fp64") or dom.startswith("gradient_fp64") or dom.startswith("density_fp64")
    # a kernel whose capture shows the FP64 pipe busier than the FMA pipe (the
    # MIXED gathers: an FP64 conversion and add per record component) is
    # measured against the FP64 pipe
    rec = ncu_record(dom)
    if rec is not None and rec.get("fp64_pipe_pct", 0.0) > rec.get("fma_pipe_pct", 0.0):
        fp64 = True
    out = {"bound": "alu", "kernel": dom, "kernel_avg_ms": shares[dom]["avg_ms"], "share": shares[dom]["share"]}
    if fp64:
        ops = ncu_counter(dom, "fp64_lane_ops")
        peak = peak_fp64_ops()
        ach = ops / avg_s / 1e12 if ops else None
        out.update({"achieved": ach, "peak": peak / 1e12, "unit": "T lane-ops/s (FP64 pipe)",
                    "frac": ach / (peak / 1e12) if ach else None, "ops_per_launch": ops,
                    "ops_basis": ("FP64-pipe operations of one launch: 32 x smsp__inst_executed_pipe_fp64.sum "
                                  "from the committed ncu capture (the pipe's own count, FP64 exp, sqrt and "
                                  "division included)"),
                    "peak_note": "152 SMs x 2 FP64 lanes x 2070 MHz (nominal 1.25 TFLOP/s)"})
    else:
        opp = ops_per_pair(dom, n_phi, n_f, S)
        peak = peak_fp32_ops()
        ops_launch = units_per_launch(dom, npairs) * opp if opp else None
        ach = ops_launch / avg_s / 1e12 if ops_launch else None
        out.update({"achieved": ach, "peak": peak / 1e12, "unit": "Tops/s (FP32 pipe)",
                    "frac": ach / (peak / 1e12) if ach else None, "ops_per_launch": ops_launch,
                    "ops_basis": ("per unordered pair" if dom.startswith("pair") else
                                  "per neighbour entry (full list: each unordered pair evaluated from both ends)"),
                    "frac_half_list": ((ach / (peak / 1e12)) * (1.0 if dom.startswith("pair") else 0.5))
                                      if ach else None,
                    "peak_note": "152 SMs x 128 FP32 lanes x 2070 MHz (unit counts x max clock)"})
    out["traffic"] = ncu_traffic(dom) if with_traffic else None
    out["traffic_unit"] = "bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture)"
    # HBM and L2 throughput of the dominant kernel: the captured bytes of one
    # launch over its event-timed duration in this run
    rec = ncu_record(dom) if with_traffic else None
    out["hbm_gbs"] = (rec["dram_read"] + rec["dram_write"]) / avg_s / 1e9 if rec else None
    out["l2_gbs"] = rec["l2_bytes"] / avg_s / 1e9 if rec else None
    return out


COUNTERS = os.path.join(ROOT, "profiles", "counters_binary_alloy_256k.json")


def kernel_source_digest(src):
    """sha256 (first 16 hex digits) of one kernel's source text: the text of
    src["file"] from the marker src["from"] to the marker src["to"], followed
    by the whole text of every header in src["also"] (code the kernel inlines,
    e.g. the float-float arithmetic)."""
    import hashlib
    text = open(os.path.join(ROOT, src["file"])).read()
    a = text.find(src["from"])
    b = text.find(src["to"], a + 1) if a >= 0 else -1
    if a < 0 or b < 0:
        return None
    body = text[a:b]
    for extra in src.get("also", []):
        body += open(os.path.join(ROOT, extra)).read()
    return hashlib.sha256(body.encode()).hexdigest()[:16]


def ncu_record(kernel):
    """Per-launch counters of `kernel` (timing class name) from the committed
    ncu capture of the 256,000-site alloy, or None when the kernel's source
    text changed since the capture."""
    if not os.path.exists(COUNTERS):
        return None
    rec = json.load(open(COUNTERS))["kernels"].get(kernel)
    if rec is None or kernel_source_digest(rec["source"]) != rec["source_digest"]:
        return None
    return rec


def ncu_traffic(kernel):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    rec = ncu_record(kernel)
    return None if rec is None else rec["dram_read"] + rec["dram_write"]


def ncu_counter(kernel, name):
    rec = ncu_record(kernel)
    return None if rec is None else rec.get(name)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p))
    return {}


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1910_01235_gb300 import mxe as M

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sys0 = replica_workload(rank)
    n = sys0.n
    K = args.fire_iters
    fire = M.make_fire(check_every=K + 1)
    dt = sys0.dt_default()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def set_shape(g):
        """Pass shape: the autotuner's choice, or --pass-shape
        (lanes,threads[,pair_threads]); returns (lanes, threads, pair_threads)."""
        if args.pass_shape:
            v = [int(t) for t in args.pass_shape.split(",")]
            g.set_pass_shape(v[0], v[1], v[2] if len(v) > 2 else None)
        else:
            g.autotune()
        return g.pass_shape()

    def timed_arm(prec, steps, warmup, launches_out=None, kernel_events=False):
        stream = torch.cuda.Stream(dev)
        with torch.cuda.stream(stream):
            g = M.MxeSystem(sys0, prec, device=dev, stream=stream)
        q0, s0, x0 = g.q.clone(), g.sigma.clone(), g.x.clone()
        g.build_neighbors()
        shape = set_shape(g)
        total_ms = 0.0

        def one_step():
            g.build_neighbors()
            g.free_energy_grad(with_mu=False, asynchronous=True)
            g.diffuse_step(dt, mu_ex=g.mu_ex, asynchronous=True)
            st, it, fm = g.relax(0.0, K, fire)
            return it

        for i in range(warmup + steps):
            with torch.cuda.stream(stream):
                g.q.copy_(q0)
                g.sigma.copy_(s0)
                g.x.copy_(x0)
                flush.fill_(float(i))
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it = one_step()
            e1.record(stream)
            stream.synchronize()
            assert it == K
            if i >= warmup:
                total_ms += e0.elapsed_time(e1)
        g.sync_status()
        kern = None
        if kernel_events:
            # per-kernel-class device times of one more identical step, with
            # every launch of the library bracketed by CUDA events on its stream
            with torch.cuda.stream(stream):
                g.q.copy_(q0)
                g.sigma.copy_(s0)
                g.x.copy_(x0)
                flush.fill_(-1.0)
            stream.synchronize()
            M.mxe_timing_enable(g.ctx, True)
            one_step()
            st, kern = M.mxe_timing_read(g.ctx)
            M.mxe_timing_enable(g.ctx, False)
        npairs = g.n_pairs
        g.close()
        return total_ms, kern, npairs, shape

    main_prec = args.precision
    precs = [main_prec] + [p for p in ("fp64", "mixed", "ff") if p != main_prec and not args.quick]
    results = {}
    clocks = None
    for p in precs:
        steps = args.steps
        warm = args.warmup if p != "fp64" else 3
        sampler = ClockSampler(local) if p == main_prec else None
        if sampler:
            sampler.start()
        ms, kern, npairs, shape = timed_arm(p, steps, warm, kernel_events=True)
        if sampler:
            clocks = sampler.stop()
        results[p] = (max_over_ranks(ms / steps, dist, dev), steps, warm, npairs, kern, shape)

    # e2e through the public API with host buffers
    def e2e(prec, steps):
        stream = torch.cuda.Stream(dev)
        host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
                for k, v in (("q", sys0.q), ("sigma", sys0.sigma), ("x", sys0.x), ("T", sys0.T))}
        host_sub = torch.from_numpy(np.ascontiguousarray(sys0.sublattice)).pin_memory()
        out_x = torch.empty((sys0.S, n), dtype=torch.float64).pin_memory()
        out_F = torch.empty(4, dtype=torch.float64).pin_memory()
        with torch.cuda.stream(stream):
            g = M.MxeSystem(sys0, prec, device=dev, stream=stream)
        g.build_neighbors()
        set_shape(g)
        h2d = sum(t.numel() * t.element_size() for t in host.values()) + host_sub.numel()
        d2h = out_x.numel() * 8 + 32
        tot = 0.0
        for i in range(2 + steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                g.q.copy_(host["q"], non_blocking=True)
                g.sigma.copy_(host["sigma"], non_blocking=True)
                g.x.copy_(host["x"], non_blocking=True)
                g.T.copy_(host["T"], non_blocking=True)
                g.sub.copy_(host_sub, non_blocking=True)
            g.build_neighbors()
            g.free_energy_grad(with_mu=False, asynchronous=True)
            g.diffuse_step(dt, mu_ex=g.mu_ex, asynchronous=True)
            g.relax(0.0, K, fire)
            with torch.cuda.stream(stream):
                out_x.copy_(g.x, non_blocking=True)
                out_F.copy_(g.F4, non_blocking=True)
            e1.record(stream)
            stream.synchronize()
            if i >= 2:
                tot += e0.elapsed_time(e1)
        g.close()
        return tot / steps, h2d, d2h

    e2e_ms, h2d, d2h = e2e(main_prec, args.steps)
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)

    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    evals_per_step = n * (K + 2)
    ms, steps, warm, npairs, kern, shape = results[main_prec]
    value = aggregate_rate(evals_per_step, ms, world)
    dp = sys0.pot
    n_phi = 3 if dp.cross_geomean else 2
    n_f = 2
    shares = kernel_shares(kern)
    per_prec = {}
    for p, r in results.items():
        sh = kernel_shares(r[4])
        per_prec[p] = {"value": aggregate_rate(evals_per_step, r[0], world), "unit": "site-evals/s",
                       "ms_per_step": r[0], "steps": r[1], "warmup": r[2],
                       "diffusion_steps_per_s": world * 1e3 / r[0], "pass_shape": list(r[5]),
                       "dtype": DTYPES[p],
                       "roofline": roofline_of(sh, r[3], sys0.S, n_phi, n_f, with_traffic=(p == "ff"))}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "site-evals/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": warm,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPES[main_prec],
        "data": "synthetic (seeded FCC binary alloy, random-init composition)",
        "config": {"workload": WORKLOAD, "sites": n, "species": 2, "fire_iters_per_step": K,
                   "evals_per_step": K + 2, "neighbor_pairs": npairs, "parallelism": f"replicas{world}",
                   "l2": "flushed between steps (256 MB write)", "precision": main_prec,
                   "pass_shape": {"lanes_per_site": shape[0], "threads_per_block": shape[1],
                                  "pairs_per_block": shape[2],
                                  "chosen_by": "--pass-shape" if args.pass_shape else "autotuner"}},
        "diffusion_steps_per_s": world * 1e3 / ms,
        "kernels": shares,
        "e2e": {"value": aggregate_rate(evals_per_step, e2e_ms, world), "unit": "site-evals/s",
                "ms_per_step": e2e_ms, "steps": args.steps, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": per_prec[main_prec]["roofline"],
        "clocks": clocks,
        "gpu_launches": None,
    }
    # kernels per step, counted by the library's launch timing
    line["gpu_launches"] = steps * sum(v["launches"] for v in shares.values())
    # the metric's precision pair, one object per mode (FP32-mixed vs FP64)
    line.update(per_prec)
    if "fp64" in per_prec and main_prec != "fp64":
        line["speedup_vs_fp64"] = per_prec["fp64"]["ms_per_step"] / ms
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sys0)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(sys0, max_seconds=30.0):
    """The oracle as it stands on the host cores: one binned neighbour build and
    one free-energy/gradient evaluation of the full 256,000-site state."""
    import oracle as O
    t0 = time.perf_counter()
    rl = O.r_list_for(sys0)
    st, off, idx = O.neighbors(sys0.q, sys0.L, rl, binned=True)
    t1 = time.perf_counter()
    fe = O.free_energy(sys0, (off, idx))
    t2 = time.perf_counter()
    assert fe["status"] == O.OK
    return {"value": sys0.n / (t2 - t0), "unit": "site-evals/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"one neighbour build ({t1 - t0:.2f} s) + one free-energy/gradient evaluation "
                      f"({t2 - t1:.2f} s) of the full {sys0.n}-site state"}


# ---------------------------------------------------------------- batched ensemble
ENSEMBLE_STEPS = 50


def run_ensemble(args):
    import torch

    from paper_1910_01235_gb300 import mxe as M

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    systems = W.config_ensemble(seed=W.SEED + rank, pot=W.potential_variant_s())
    n = sum(t.n for t in systems)
    K = args.fire_iters
    steps_per_run = args.ensemble_steps
    prec = args.precision
    fire = M.make_fire(check_every=K + 1)
    dts = np.array([t.dt_default() for t in systems])
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        g = M.MxeBatch(systems, prec, device=dev, stream=stream)
    g.build_neighbors()
    g.set_dt_scale(list(dts))
    if args.pass_shape:
        v = [int(t) for t in args.pass_shape.split(",")]
        g.set_pass_shape(v[0], v[1], v[2] if len(v) > 2 else None)
    else:
        g.autotune()
    lanes, threads, pair_threads = g.pass_shape()
    q0, s0, x0 = g.q.clone(), g.sigma.clone(), g.x.clone()

    def restore():
        with torch.cuda.stream(stream):
            g.q.copy_(q0)
            g.sigma.copy_(s0)
            g.x.copy_(x0)
        stream.synchronize()
        g.build_neighbors()

    # warm-up: capture and replay
    for _ in range(args.warmup):
        restore()
        st, done = g.run_staggered(2, 1.0, 0.0, K, fire)
    times = []
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(max(1, args.steps // steps_per_run) if args.steps >= steps_per_run else 1):
        restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, done = g.run_staggered(steps_per_run, 1.0, 0.0, K, fire)
        e1.record(stream)
        stream.synchronize()
        assert st == M.OK and done == steps_per_run, (st, done)
        times.append(e0.elapsed_time(e1))
        launches, kernels_per_step = g.run_stats()
    clocks = sampler.stop()
    ms_run = float(np.median(times))
    ms_step = ms_run / steps_per_run
    moved = (g.x - x0).abs().max().item()
    g.close()
    evals_per_step = n * (K + 2)
    line = {
        "metric": METRIC, "value": aggregate_rate(evals_per_step, ms_step, world), "unit": "site-evals/s",
        "n_gpus": world, "steps": steps_per_run * len(times), "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[prec],
        "data": "synthetic (seeded ensemble of FCC single-species lattices with vacancies)",
        "config": {"workload": "ensemble_512_systems", "systems": len(systems), "sites": n,
                   "fire_iters_per_step": K, "evals_per_step": K + 2, "steps_per_graph_run": steps_per_run,
                   "pass_shape": {"lanes_per_site": lanes, "threads_per_block": threads,
                                  "pairs_per_block": pair_threads},
                   "potential": "single species, variant with pair exponent 5 and density exponent 3",
                   "precision": prec,
                   "l2": "working set ~1 GB > L2, not flushed", "parallelism": f"replicas{world}"},
        "diffusion_steps_per_s": world * 1e3 / ms_step,
        "graph_launches_per_run": launches, "kernels_per_step": kernels_per_step,
        "gpu_launches": kernels_per_step * steps_per_run * len(times),
        "max_abs_dx": moved,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- unrolled derivative
def run_unrolled_grad(args):
    """Gradient of the mean B fraction in the top sixth of the box (one bin of
    the z-profile) after 20 staggered steps with respect to the eight alloy
    parameters, on the 108,000-site binary alloy (30^3 cells, 1000 K), FP64,
    (q, sigma) checkpoints every 5 steps, relaxations to 1e-8 eV/A, conjugate
    gradients to 1e-8.  The exponent-swapped tables and a periodic box: the
    relaxations must reach a minimum, which neither the literal tables nor
    the free-surface slab have in this model."""
    import torch

    from paper_1910_01235_gb300 import mxe as M

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = W.config_binary_alloy(cells=30, seed=W.SEED + rank)
    s.pot = W.potential_binary_variant_s()
    n_steps, every, ftol = 20, 5, 1e-8
    g = M.MxeSystem(s, "fp64", device=dev)
    g.build_neighbors()
    # relax once so that the Euler step is sized at the relaxed state
    g.relax(ftol, 20000, allow=())
    g.free_energy_grad()
    x0 = g.x.clone()
    trial = s.dt_default() * 1e-9
    g.diffuse_step(trial, mu_ex=g.mu_ex)
    rate = (g.x - x0).abs().max().item() / trial
    g.x.copy_(x0)
    dt = 1e-4 / rate           # largest |dx| of a step ~1e-4 (x_v = 1e-3)
    zq = g.q[2].cpu().numpy()
    top = zq > s.L[2] * 5.0 / 6.0
    w = np.zeros_like(s.x)
    w[1, top] = 1.0 / top.sum()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    e0.record()
    dterm, dx0, info = g.unrolled_grad(n_steps, dt, w, ftol=ftol, max_iter=20000, every=every, cg_tol=1e-8,
                                       cg_max=20000)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    grad = M.element_param_grad(s.pot, dterm).reshape(-1)
    L = float((w * g.x.cpu().numpy()).sum())
    g.close()
    line = {"metric": "unrolled-gradient runs/s (20 staggered steps forward + reverse sweep)",
            "value": 1e3 / ms, "unit": "runs/s", "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded FCC binary alloy)",
            "config": {"workload": "binary_alloy_fcc30_108k_unrolled_grad", "sites": s.n, "steps": n_steps,
                       "checkpoint_every": every, "ftol": ftol, "cg_tol": 1e-8, "T": 1000.0,
                       "potential": "binary, exponent-swapped (pair 5, density 3)",
                       "objective": "mean x_B of the sites in the top sixth of the box (one z-profile bin)"},
            "L": L, "dL_dtheta": dict(zip(W.THETA_NAMES, grad.tolist())), "info": info, "dt": dt,
            "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- large slab
def run_slab(args):
    """The 4,000,000-site interstitial slab (100 x 100 x 50 cells: 2 M host
    sites, immobile, plus 2 M octahedral sites holding the solute in the top
    10 A; 20 A vacuum gap; T = 600 K).  A step is one diffusion step of the
    first kind: free energy with its gradients and chemical potentials, then
    the Euler step.  Reports the device-memory footprint of the context and
    its state (free device memory before and after set-up)."""
    import torch

    from paper_1910_01235_gb300 import mxe as M

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = W.config_interstitial_slab(seed=W.SEED + rank)
    prec = args.precision
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        g = M.MxeSystem(s, prec, device=dev, stream=stream)
    g.build_neighbors()
    g.free_energy_grad()
    torch.cuda.synchronize()
    footprint = free0 - torch.cuda.mem_get_info(dev)[0]
    # step size: a trial step scaled so that the largest |dx| is 1e-4 (the
    # free surface gives the solute large chemical-potential differences)
    x0 = g.x.clone()
    trial = s.dt_default() * 1e-9
    g.diffuse_step(trial, mu_ex=g.mu_ex)
    rate = (g.x - x0).abs().max().item() / trial
    g.x.copy_(x0)
    dt = 1e-4 / rate
    for _ in range(args.warmup):
        g.free_energy_grad(with_mu=False, asynchronous=True)
        g.diffuse_step(dt, mu_ex=g.mu_ex, asynchronous=True)
    g.sync_status()
    K = args.steps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    e0.record(stream)
    for _ in range(K):
        g.free_energy_grad(with_mu=False, asynchronous=True)
        g.diffuse_step(dt, mu_ex=g.mu_ex, asynchronous=True)
    e1.record(stream)
    stream.synchronize()
    clocks = sampler.stop()
    g.sync_status()
    ms = e0.elapsed_time(e1) / K
    npairs = g.n_pairs
    g.close()
    line = {"metric": "diffusion steps/s (free energy + gradients + chemical potentials, then the Euler step)",
            "value": world * 1e3 / ms, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[prec],
            "data": "synthetic (seeded FCC host + octahedral solute slab)",
            "config": {"workload": "interstitial_slab_100x100x50_4M", "sites": s.n, "neighbor_pairs": npairs,
                       "precision": prec, "l2": "working set > L2, not flushed"},
            "site_evals_per_s": world * s.n / (ms / 1e3), "dt": dt,
            "device_memory_bytes": int(footprint), "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- embedding average
def run_embedding(args):
    """The paper's Taylor form of the embedding average (Eq. F_taylor_mxe)
    against the exact third-degree rule over each site and its neighbours
    inside r_cut (App. B.2), both evaluated by the library in FP64 at the same
    state: the 500-site vacancy lattice and the 256,000-site binary alloy.
    Reports the differences in E_V, dF/dq, dF/dsigma and mu^ex, and the time
    of one free-energy evaluation in each form."""
    import torch

    from paper_1910_01235_gb300 import mxe as M

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = {}
    for name, sysf in (("vacancy_lattice_fcc5_500", W.config_vacancy_lattice),
                       ("binary_alloy_fcc40_256k", W.config_binary_alloy)):
        s = sysf()
        res = {}
        for mode in ("taylor", "exact"):
            g = M.MxeSystem(s, "fp64", device=dev)
            g.set_embedding(mode)
            g.build_neighbors()
            for _ in range(max(1, args.warmup)):
                g.free_energy_grad()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.free_energy_grad()
            e1.record()
            torch.cuda.synchronize()
            res[mode] = dict(F4=g.F4.cpu().numpy(), gq=g.gq.cpu().numpy(), gs=g.gs.cpu().numpy(),
                             mu=g.mu_ex.cpu().numpy(), ms=e0.elapsed_time(e1))
            g.close()
        t, e = res["taylor"], res["exact"]
        out[name] = {
            "sites": s.n,
            "E_V_per_site_taylor": t["F4"][0] / s.n, "E_V_per_site_exact": e["F4"][0] / s.n,
            "dE_V_per_site": (e["F4"][0] - t["F4"][0]) / s.n,
            "max_abs_d_dFdq": float(np.abs(e["gq"] - t["gq"]).max()),
            "max_abs_dFdq": float(np.abs(e["gq"]).max()),
            "max_abs_d_dFdsigma": float(np.abs(e["gs"] - t["gs"]).max()),
            "max_abs_d_mu_ex": float(np.abs(e["mu"] - t["mu"]).max()),
            "ms_eval_taylor": t["ms"], "ms_eval_exact": e["ms"]}
    line = {"metric": "embedding-average difference, exact rule minus Taylor form (FP64)",
            "value": out["binary_alloy_fcc40_256k"]["dE_V_per_site"], "unit": "eV/site",
            "n_gpus": world, "steps": 1, "warmup": args.warmup, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic (seeded FCC lattices)", "vs_baseline": None,
            "config": {"workload": "embedding_average_taylor_vs_exact"}, "workloads": out}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    sys0 = W.config_binary_alloy()
    dt = sys0.dt_default()
    rl = O.r_list_for(sys0)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        st, off, idx = O.neighbors(sys0.q, sys0.L, rl, binned=True)
        fe = O.free_energy(sys0, (off, idx))
        boff, bidx = O.bonds(sys0, 0.5 * (sys0.a / np.sqrt(2.0) + sys0.a), off, idx)
        st, x1 = O.diffuse_step(sys0, fe["mu_ex"], (boff, bidx), dt)
        t1 = time.perf_counter()
        if i >= args.warmup:
            times.append(t1 - t0)
    per = float(np.mean(times))
    value = sys0.n / per
    cores = O.num_threads()
    line = {"metric": METRIC, "value": value, "unit": "site-evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded FCC binary alloy)", "impl": "reference",
            "config": {"workload": WORKLOAD, "sites": sys0.n, "species": 2, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": "site-evals/s", "cores": cores, "kind": "oracle",
                             "sample": "per step: one binned neighbour build, one free-energy/gradient "
                                       "evaluation and one Euler step of the full 256,000-site state"},
            "e2e": {"value": value, "unit": "site-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="ff", choices=["fp64", "mixed", "ff"])
    ap.add_argument("--fire-iters", type=int, default=FIRE_ITERS)
    ap.add_argument("--quick", action="store_true", help="main precision only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="binary",
                    choices=["binary", "ensemble", "unrolled_grad", "slab4m", "embedding"])
    ap.add_argument("--ensemble-steps", type=int, default=ENSEMBLE_STEPS)
    ap.add_argument("--pass-shape", default="",
                    help="lanes,threads[,pair_threads] of the passes (default: autotuned)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "unrolled_grad":
        run_unrolled_grad(args)
    elif args.workload == "slab4m":
        run_slab(args)
    elif args.workload == "embedding":
        run_embedding(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
