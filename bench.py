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


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


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
def k3_fp32_ops_per_pair(n_phi, n_f):
    """FP32-pipe operations the gradient pass spends on one (i, j) pair, counted
    from the algorithm: 12 nodes x (distance 2, switch 11, 5 per radial term,
    force/sigma accumulation 4.25) + the static point (distance 2, switch 11,
    5 per density term) + per-pair set-up and combination (separation 9,
    weights 3 n_phi + 4 n_f, sums 10 + 2 (n_phi + n_f))."""
    node = 2 + 11 + 5 * (n_phi + n_f) + 4.25
    static = 2 + 11 + 5 * n_f
    pair = 9 + 3 * n_phi + 4 * n_f + 10 + 2 * (n_phi + n_f)
    return 12 * node + static + pair


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
    sys0 = W.config_binary_alloy()
    n = sys0.n
    K = args.fire_iters
    fire = M.make_fire(check_every=K + 1)
    dt = sys0.dt_default()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def timed_arm(prec, steps, warmup, launches_out=None, kernel_events=False):
        stream = torch.cuda.Stream(dev)
        with torch.cuda.stream(stream):
            g = M.MxeSystem(sys0, prec, device=dev, stream=stream)
        q0, s0, x0 = g.q.clone(), g.sigma.clone(), g.x.clone()
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
            # average duration of the gradient pass (the dominant kernel), timed alone
            g.build_neighbors()
            g.free_energy_grad(with_mu=False)
            reps = 20
            A = M.lib()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ms = []
            for r in range(reps):
                with torch.cuda.stream(stream):
                    flush.fill_(float(r))
                ev[0].record(stream)
                M.mxe_free_energy_grad(g.ctx, g.state, M._ptr(g.F4), M._ptr(g.gq), M._ptr(g.gs),
                                       M._ptr(g.mu_ex), 0, True)
                ev[1].record(stream)
                stream.synchronize()
                ms.append(ev[0].elapsed_time(ev[1]))
            kern = float(np.median(ms))
            del A
        npairs = g.n_pairs
        g.close()
        return total_ms, kern, npairs

    main_prec = args.precision
    precs = [main_prec] + [p for p in ("fp64", "mixed", "ff") if p != main_prec and not args.quick]
    results = {}
    clocks = None
    for p in precs:
        steps = args.steps if p != "fp64" else max(1, min(args.steps, 3))
        warm = args.warmup if p != "fp64" else max(3, min(args.warmup, 3))
        sampler = ClockSampler(local) if p == main_prec else None
        if sampler:
            sampler.start()
        ms, _, npairs = timed_arm(p, steps, warm)
        if sampler:
            clocks = sampler.stop()
        t = torch.tensor([ms / steps], dtype=torch.float64)
        if world > 1:
            t = t.to(dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        results[p] = (float(t.item()), steps, warm, npairs)

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

    e2e_ms, h2d, d2h = e2e(main_prec, max(1, min(args.steps, 5)))
    t = torch.tensor([e2e_ms], dtype=torch.float64)
    if world > 1:
        t = t.to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_ms = float(t.item())

    # dominant kernel alone (roofline)
    _, kern_ms, npairs = timed_arm(main_prec, 1, 1, kernel_events=True)

    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    evals_per_step = n * (K + 2)
    ms, steps, warm, npairs = results[main_prec]
    value = world * evals_per_step / (ms / 1e3)
    dfn = M  # noqa: F841
    dp = sys0.pot
    n_phi = 3 if dp.cross_geomean else 2
    n_f = 2
    ops_launch = npairs * k3_fp32_ops_per_pair(n_phi, n_f)
    peak_ops = 152 * 128 * 2.07e9
    # the evaluation timed alone contains density + gradient + energy passes; the
    # gradient pass share of it comes from the ncu launch list (profiles/)
    k3_share = float(os.environ.get("MXE_K3_SHARE", "0.62"))
    k3_ms = kern_ms * k3_share if kern_ms else None
    achieved = ops_launch / (k3_ms / 1e3) / 1e12 if k3_ms else None
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
        "dtype": {"fp64": "f64", "mixed": "f32+f64acc", "ff": "f32+ff-acc"}[main_prec],
        "data": "synthetic (seeded FCC binary alloy, random-init composition)",
        "config": {"workload": WORKLOAD, "sites": n, "species": 2, "fire_iters_per_step": K,
                   "evals_per_step": K + 2, "neighbor_pairs": npairs, "parallelism": f"replicas{world}",
                   "l2": "flushed between steps (256 MB write)", "precision": main_prec},
        "diffusion_steps_per_s": world * 1e3 / ms,
        "precisions": {p: {"ms_per_step": r[0], "site_evals_per_s": world * evals_per_step / (r[0] / 1e3),
                           "steps": r[1]} for p, r in results.items()},
        "e2e": {"value": world * evals_per_step / (e2e_ms / 1e3), "unit": "site-evals/s",
                "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu", "kernel": "k_gradient", "achieved": achieved, "peak": peak_ops / 1e12,
                     "unit": "Tops/s (FP32 pipe)", "frac": (achieved / (peak_ops / 1e12)) if achieved else None,
                     "traffic": None, "kernel_ms": k3_ms, "ops_per_launch": ops_launch,
                     "peak_note": "152 SMs x 128 FP32 lanes x 2070 MHz (unit counts x max clock)"},
        "clocks": clocks,
        "gpu_launches": None,
    }
    # kernels per step: build 14, free energy 4 (+1 pack), diffuse 2, relax 1 + 5 (K + 1)
    pack = 0 if main_prec == "fp64" else 1
    line["gpu_launches"] = steps * (14 + 4 + pack + 2 + pack + 5 * (K + 1))
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
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "ff"])
    ap.add_argument("--fire-iters", type=int, default=FIRE_ITERS)
    ap.add_argument("--quick", action="store_true", help="main precision only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
