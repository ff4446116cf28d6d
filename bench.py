#!/usr/bin/env python
"""Benchmark of the FC2T2 transform: forward + backward query-evaluations per second.

Workload (default, ``uniform3d``): 3D, N = M = 2^20 sources and queries uniform in [0,1)^3,
w ~ N(0,1), Gaussian sigma = 0.02, 64^3 finest grid (5 levels), order 6 (84 coefficients per
cell); one step = forward y = f(q; p, w) plus backward (wbar, pbar) for the cotangent
ybar = y (L = sum y^2 / 2), all through the C ABI.  Metric: M / (t_fwd + t_bwd).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--m2l fp32]

Prints one JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload (the queries -- and, for the backward, the
sources -- with z < 1/8, about an eighth of each; the oracle evaluates only the cells these
need), reported in the same unit.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd query-evals/s"
UNIT = "query-evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--m2l", default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# --------------------------------------------------------------------------- arithmetic

def m2l_pairs_per_level(D: int, n: int):
    """Exact number of (target, source) cell pairs M2L visits per level: the parity window
    clipped to the grid, minus the 3^D hole above the finest level (per-dimension sums
    factorise because window and hole are products over dimensions)."""
    out, nl, lev = [], n, 0
    while nl >= 4:
        W = H = 0
        for t in range(nl):
            lo = -3 if t & 1 else -2
            W += sum(1 for o in range(lo, lo + 6) if 0 <= t + o < nl)
            H += sum(1 for o in (-1, 0, 1) if 0 <= t + o < nl)
        out.append(W ** D - (H ** D if lev > 0 else 0))
        nl //= 2
        lev += 1
    return out


def m2l_useful_flops(D: int, n: int, rho: int) -> int:
    """2 * C(rho + 2D, 2D) multiply-adds per interacting cell pair (|k| + |b| <= rho)."""
    return 2 * math.comb(rho + 2 * D, 2 * D) * sum(m2l_pairs_per_level(D, n))


def fp32_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 FLOP per FMA x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ helpers

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def slab_sample(x, frac=0.125):
    import numpy as np
    return np.nonzero(x[:, 2] < frac)[0]


def cpu_oracle_step(wl, sel_q, sel_p):
    """One oracle forward (at sel_q) + backward (at sel_p); returns seconds."""
    import numpy as np
    import oracle
    d = oracle.OracleDesc(dim=3, grid=wl.grid, order=wl.order, sigma=wl.sigma)
    p, w, q = (np.asarray(a, dtype=np.float64) for a in (wl.p, wl.w, wl.q))
    t0 = time.perf_counter()
    y = oracle.forward(d, p, w, q, sel=sel_q)
    ybar = np.zeros(q.shape[0])
    ybar[sel_q] = y                                   # cotangent on the sampled queries
    oracle.backward(d, p, w, q, ybar, sel=sel_p)
    return time.perf_counter() - t0


def run_reference(args, rank, world):
    """The oracle on the host cores, bounded sample per step (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    from paper_2111_00110_gb300 import workloads
    oracle.build()
    wl = workloads.uniform3d()
    sel_q = slab_sample(wl.q)
    sel_p = slab_sample(wl.p)
    for _ in range(args.warmup):
        cpu_oracle_step(wl, sel_q, sel_p)
    times = [cpu_oracle_step(wl, sel_q, sel_p) for _ in range(args.steps)]
    per_step = statistics.mean(times)
    value = len(sel_q) / per_step
    cores = os.cpu_count()
    sample = (f"{len(sel_q)} queries (forward) and {len(sel_p)} sources (backward) with z < 1/8 "
              f"of the uniform3d workload per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "uniform3d", "N": wl.N, "M": wl.M, "grid": wl.grid,
                   "order": wl.order, "sigma": wl.sigma, "dim": 3},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2111_00110_gb300 import build as _build
    from paper_2111_00110_gb300 import workloads
    from paper_2111_00110_gb300.transform import Plan

    _build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # weak scaling: every rank transforms its own independent point set
    wl = workloads.uniform3d(seed=2 + rank)
    D, n, rho = 3, wl.grid, wl.order
    plan = Plan(D, n, rho, wl.sigma, m2l=args.m2l, max_sources=wl.N, max_queries=wl.M, device=dev)
    p = torch.from_numpy(wl.p).to(dev)
    w = torch.from_numpy(wl.w).to(dev)
    q = torch.from_numpy(wl.q).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def step():
        y = plan.forward(p, w, q)
        plan.backward(p, w, q, y)

    for _ in range(max(args.warmup, 3 if args.warmup >= 3 else args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    plan.profile(True)
    plan.profile_read(reset=True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        flush.zero_()                       # evict L2 between timed steps (not timed)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    stage_ms, launches = plan.profile_read(reset=True)
    plan.profile(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    value = wl.M * args.steps * world / (total_ms / 1e3)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timing
    e2e = None
    if not args.no_e2e:
        hp, hw, hq = (torch.from_numpy(a).pin_memory() for a in (wl.p, wl.w, wl.q))
        dp, dw, dq = torch.empty_like(p), torch.empty_like(w), torch.empty_like(q)
        hwb = torch.empty(wl.N, dtype=torch.float32).pin_memory()
        hpb = torch.empty(wl.N, D, dtype=torch.float32).pin_memory()

        def e2e_step():
            dp.copy_(hp, non_blocking=True)
            dw.copy_(hw, non_blocking=True)
            dq.copy_(hq, non_blocking=True)
            y = plan.forward(dp, dw, dq)
            wbar, pbar = plan.backward(dp, dw, dq, y)
            hwb.copy_(wbar, non_blocking=True)
            hpb.copy_(pbar, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize(dev)
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(stream)
        for _ in range(args.steps):
            e2e_step()
        ee.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = es.elapsed_time(ee)
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        h2d = 4 * (wl.N * D + wl.N + wl.M * D)
        d2h = 4 * (wl.N + wl.N * D)
        e2e = {"value": wl.M * args.steps * world / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        return
    # ---- roofline of the dominant kernel (M2L; CUDA cores in FP32)
    peaks = load_peaks()
    m2l_flops = 2 * m2l_useful_flops(D, n, rho)            # forward + backward transforms
    m2l_ms = stage_ms["m2l"] / args.steps
    m2l_launches = launches["m2l"] / args.steps
    achieved = m2l_flops / (m2l_ms / 1e3) / 1e12
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    peak = fp32_peak_tflops(sm_max)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "m2l", "flops_per_step": m2l_flops, "launches_per_step": m2l_launches,
                "peak_basis": f"FP32 FMA: 152 SMs x 128 lanes x 2 x {sm_max:.0f} MHz"}
    step_stage_ms = {k: v / args.steps for k, v in stage_ms.items()}

    cpu = None
    if not args.no_cpu_baseline:
        try:
            import oracle
            oracle.build()
            sel_q, sel_p = slab_sample(wl.q), slab_sample(wl.p)
            secs = cpu_oracle_step(wl, sel_q, sel_p)
            cpu = {"value": len(sel_q) / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"one forward at the {len(sel_q)} queries and one backward at the "
                             f"{len(sel_p)} sources with z < 1/8 (oracle evaluates only the cells "
                             f"these need), {secs:.1f} s"}
        except Exception as exc:  # pragma: no cover
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {exc}"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "uniform3d", "dim": D, "N": wl.N, "M": wl.M, "grid": n,
                   "levels": plan_levels(n), "order": rho, "sigma": wl.sigma, "m2l": args.m2l,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": int(sum(launches.values())),
        "roofline": roofline,
        "stage_ms_per_step": step_stage_ms,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def plan_levels(n: int) -> int:
    return int(math.log2(n)) - 1


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            import torch
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
