#!/usr/bin/env python
"""Benchmark of the FC2T2 transform: forward + backward query-evaluations per second.

Workload (``uniform3d``): 3D, N = M = 2^20 sources and queries uniform in [0,1)^3, w ~ N(0,1),
Gaussian sigma = 0.02, 64^3 finest grid (5 levels), order 6 (84 coefficients per cell).  One step =
forward y = f(q; p, w) plus backward (wbar, pbar) for the cotangent ybar = y (L = sum y^2 / 2), all
through the C ABI.  Metric: M / (t_fwd + t_bwd) at a stated relative-L2 error against the FP64
oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--m2l MODE]

MODE "auto" (default) reports the fastest FP32-accurate path (the separable M2L: the Gaussian's
factored derivatives in three 1D passes on the CUDA cores, FP32) as `value`, and as `variants` the
tensor-core forms (BF16 x 3 and TF32 x 3 split operands, FP32-accurate; single-pass TF32 and BF16,
mixed precision) and the plain CUDA-core FP32 form, each with its measured error against the
oracle on a seeded sample (4096 queries for y, 4096 sources for wbar and pbar with a fixed seeded
cotangent).

Prints one JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload (the queries -- and, for the backward, the sources --
with z < 1/8, about an eighth of each; the oracle evaluates only the cells these need).
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
# nominal dense tensor-core ratios (TF32 : BF16 = 1.1 : 2.25 PFLOP/s per GPU)
TF32_PER_BF16 = 1.1 / 2.25
# DRAM bytes (read + write) of one transform's M2L launches of the current kernel builds, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum over the transform's M2L launches, on
# the same grid and order at 2^18 points: the M2L launches do not depend on the point count), by
# (M2L form, finest grid, coefficients per cell); None where no capture of the current build
# exists for that form, grid and order
M2L_TRAFFIC_BYTES = {("separable", 64, 84): 1078485760.0,
                     ("bf16x3", 64, 84): (464.0 + 82.8) * 1e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--m2l", default="auto",
                    choices=["auto", "separable", "tf32x3", "bf16x3", "tf32", "bf16", "fp32", "occupied"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-check", action="store_true", help="skip the oracle error check")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the ray-query (33.5M queries) and large fitting (2^24 points) workloads")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def fp32_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 FLOP per FMA x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def aggregate_max(value: float, world: int, device=None) -> float:
    """Max over ranks (timing); identity on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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
                 "--format=csv,noheader,nounits", "-lms", "20"],
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


def oracle_reference_sample(wl, n=4096, seed=12345, fit=False, exact=None):
    """Oracle y at n seeded queries, and (wbar, pbar) at n seeded sources for the seeded
    cotangent wl.ybar() -- the accuracy reference for every M2L form (``fit``: with the
    least-squares fitted operators); ``exact``: the direct sum at the same queries, computed once
    (the truncation error of each form is measured against it)."""
    import numpy as np
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    sq = np.sort(rng.choice(wl.M, size=n, replace=False))
    sp = np.sort(rng.choice(wl.N, size=n, replace=False))
    d = oracle.OracleDesc(dim=3, grid=wl.grid, order=wl.order, sigma=wl.sigma, fit=fit)
    p, w, q = (np.asarray(a, dtype=np.float64) for a in (wl.p, wl.w, wl.q))
    y = oracle.forward(d, p, w, q, sel=sq)
    wb, pb = oracle.backward(d, p, w, q, np.asarray(wl.ybar(), dtype=np.float64), sel=sp)
    if exact is None:
        exact = oracle.direct(d, p, w, q, sel=sq)
    return {"sq": sq, "sp": sp, "y": y, "wbar": wb, "pbar": pb, "exact": exact}


def rel_l2(a, b):
    import numpy as np
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


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


# ---------------------------------------------------------------------------- our path

class Measured:
    pass


def measure_mode(mode, wl, args, world, dev, flush, ref=None, do_e2e=False, clocks=False, steps=None, fit=False):
    """Time `steps` (default `args.steps`) fwd+bwd steps of one M2L form; per-stage device times
    from the library's events on the launching stream; optional end-to-end loop from pinned host
    buffers."""
    nsteps = args.steps if steps is None else steps
    import torch
    from paper_2111_00110_gb300.transform import Plan

    plan = Plan(3, wl.grid, wl.order, wl.sigma, m2l=mode, max_sources=wl.N, max_queries=wl.M, fit=fit, device=dev)
    p = torch.from_numpy(wl.p).to(dev)
    w = torch.from_numpy(wl.w).to(dev)
    q = torch.from_numpy(wl.q).to(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        # a training step's pair of calls: the backward reuses the forward's sorts of the same
        # (unchanged) arrays, as the autograd layer does
        y = plan.forward(p, w, q)
        plan.backward(p, w, q, y, reuse_forward=True)

    out = Measured()
    out.mode = mode
    out.grid = wl.grid
    out.info = plan.info()
    # accuracy against the oracle sample (a seeded cotangent for the backward)
    if ref is not None:
        y = plan.forward(p, w, q)
        wb, pb = plan.backward(p, w, q, torch.from_numpy(wl.ybar()).to(dev))
        torch.cuda.synchronize(dev)
        ys = y.cpu().numpy()[ref["sq"]]
        out.err = {"y": rel_l2(ys, ref["y"]),
                   "wbar": rel_l2(wb.cpu().numpy()[ref["sp"]], ref["wbar"]),
                   "pbar": rel_l2(pb.cpu().numpy()[ref["sp"]], ref["pbar"]),
                   "y_vs_exact_sum": rel_l2(ys, ref["exact"])}
    else:
        out.err = None
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    plan.profile_read(reset=True)           # (kernel launches are counted with profiling off too)
    sampler = ClockSampler(dev.index) if clocks else None
    if sampler:
        sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    torch.cuda.synchronize(dev)
    for i in range(nsteps):
        flush.zero_()                       # evict L2 between timed steps (not timed)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    out.clocks = sampler.stop() if sampler else None
    _, launches = plan.profile_read(reset=True)
    total_ms = aggregate_max(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world, dev)
    out.ms_per_step = total_ms / nsteps
    out.value = job_value(wl.M, nsteps, world, total_ms)
    out.launches = int(sum(launches.values()))
    out.launches_per_step = {k: v / nsteps for k, v in launches.items()}
    # per-stage device time from CUDA events around each stage, in separate untimed steps: with
    # the events on, a call runs its stages in order on the call's stream (no second stream), so
    # the stage times add up to a little more than the timed step
    nprof = min(nsteps, 10)
    plan.profile(True)
    plan.profile_read(reset=True)
    for _ in range(nprof):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    stage_ms, _ = plan.profile_read(reset=True)
    plan.profile(False)
    out.stage_ms = {k: v / nprof for k, v in stage_ms.items()}
    out.e2e = None
    if do_e2e:
        out.e2e = measure_e2e(plan, wl, p, w, q, nsteps, world, dev, stream)
    plan.close()
    return out


def measure_e2e(plan, wl, p, w, q, nsteps, world, dev, stream):
    """The bench step end to end through the public calls, from pinned host buffers: every step
    uploads its inputs (p, w, q) and reads its results (wbar, pbar) back to the host.

    serial: one stream, upload -> forward -> backward -> read back, step after step.
    overlapped (the reported value): the inputs are double-buffered on the device and the results
    on the host; step k+1's inputs are uploaded on one copy stream and step k's results read back
    on another while the compute stream runs step k.  The timed region runs from the first
    upload to the last read-back, so it still holds every step's copies."""
    import torch
    hp, hw, hq = (torch.from_numpy(a).pin_memory() for a in (wl.p, wl.w, wl.q))
    h2d = 4 * (wl.N * 3 + wl.N + wl.M * 3)
    d2h = 4 * (wl.N + wl.N * 3)

    def timed(run):
        run(2)
        torch.cuda.synchronize(dev)
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(stream)
        run(nsteps)
        ee.record(stream)
        torch.cuda.synchronize(dev)
        return aggregate_max(es.elapsed_time(ee), world, dev)

    dp, dw, dq = torch.empty_like(p), torch.empty_like(w), torch.empty_like(q)
    hwb = torch.empty(wl.N, dtype=torch.float32).pin_memory()
    hpb = torch.empty(wl.N, 3, dtype=torch.float32).pin_memory()

    def serial(n):
        for _ in range(n):
            dp.copy_(hp, non_blocking=True)
            dw.copy_(hw, non_blocking=True)
            dq.copy_(hq, non_blocking=True)
            y = plan.forward(dp, dw, dq)
            wbar, pbar = plan.backward(dp, dw, dq, y, reuse_forward=True)
            hwb.copy_(wbar, non_blocking=True)
            hpb.copy_(pbar, non_blocking=True)

    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    dev_in = [tuple(torch.empty_like(t) for t in (p, w, q)) for _ in range(2)]
    host_out = [(torch.empty(wl.N, dtype=torch.float32).pin_memory(),
                 torch.empty(wl.N, 3, dtype=torch.float32).pin_memory()) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]

    def upload(b):
        with torch.cuda.stream(up):
            for d, h in zip(dev_in[b], (hp, hw, hq)):
                d.copy_(h, non_blocking=True)
            ev_in[b].record(up)

    def overlapped(n):
        up.wait_stream(stream)
        down.wait_stream(stream)
        upload(0)
        used = [False, False]
        for k in range(n):
            b = k & 1
            if k + 1 < n:
                if used[1 - b]:
                    up.wait_event(ev_done[1 - b])     # step k-1 is done with those inputs
                upload(1 - b)
            stream.wait_event(ev_in[b])
            xp, xw, xq = dev_in[b]
            y = plan.forward(xp, xw, xq)
            wbar, pbar = plan.backward(xp, xw, xq, y, reuse_forward=True)
            ev_done[b].record(stream)
            used[b] = True
            with torch.cuda.stream(down):
                down.wait_event(ev_done[b])
                host_out[b][0].copy_(wbar, non_blocking=True)
                host_out[b][1].copy_(pbar, non_blocking=True)
            wbar.record_stream(down)
            pbar.record_stream(down)
        stream.wait_stream(down)

    serial_ms = timed(serial)
    overlap_ms = timed(overlapped)
    # the overlapped loop's last results against the serial loop's (same inputs and calls; the
    # sort's ranks within a cell come from atomics, so the two agree to rounding, not bitwise)
    last = host_out[(nsteps - 1) & 1]
    diff = max(rel_l2(last[0].numpy(), hwb.numpy()), rel_l2(last[1].numpy(), hpb.numpy()))
    return {"value": wl.M * nsteps * world / (overlap_ms / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": overlap_ms / nsteps,
            "copies": "overlapped: inputs double-buffered, step k+1 uploaded and step k read back on two "
                      "copy streams while step k computes",
            "rel_l2_vs_serial": diff,
            "serial": {"value": wl.M * nsteps * world / (serial_ms / 1e3), "ms_per_step": serial_ms / nsteps}}


def m2l_algorithmic_bytes(P: int, levels: int, grid: int) -> int:
    """Bytes the M2L must move per transform, whatever its form: every level's moment rows read
    once and its local rows written once (P FP32 values per row)."""
    return sum(2 * (grid >> l) ** 3 * P * 4 for l in range(levels))


def separable_bytes(P: int, levels: int, grid: int) -> int:
    """Bytes the separable M2L must move per transform: every pass reads its input rows once and
    writes its output rows once (P values per Taylor row, C(order+4, 4) per 4-indexed row; one
    chain of intermediates at the finest level, two above it)."""
    order = 0
    while (order + 1) * (order + 2) * (order + 3) // 6 < P:
        order += 1
    Q4 = (order + 1) * (order + 2) * (order + 3) * (order + 4) // 24
    total = 0
    for l in range(levels):
        G = (grid >> l) ** 3
        ch = 1 if l == 0 else 2
        total += G * 4 * ((P + ch * Q4) + (ch * Q4 + ch * Q4) + (ch * Q4 + P))
    return total


def roofline_for(m: Measured, peaks):
    """Roofline of the dominant kernel (the M2L contraction) for one measured form.

    `achieved` counts ALGORITHMIC flops: 2 x (number of |b| + |k| <= order coefficient products)
    per interacting cell pair, summed over the interaction lists of every level, two transforms
    per step.  On the tensor cores the kernel executes more than that (dense MMA tiles over the
    degree triangle, and three products per split form); `executed` reports those flops and the
    tensor-pipe fraction they reach.  Time = the M2L stage's CUDA events on the launching stream
    (the operand pack pass is a separate stage)."""
    m2l_ms = m.stage_ms["m2l"]                       # per step = two transforms
    useful = 2 * m.info["m2l_useful_flops"]
    issued = 2 * m.info["m2l_issued_flops"]
    achieved = useful / (m2l_ms / 1e3) / 1e12
    if m.mode == "separable":
        hbm = peaks.get("hbm_gbs")
        basis = "of measured hbm copy (MEASURED_PEAKS.json)"
        if hbm is None:
            hbm, basis = 6800.0, "of fallback hbm"
        # algorithmic bytes of the M2L (every level's moments read once, its locals written once)
        algo = 2 * m2l_algorithmic_bytes(m.info["coefficients"], m.info["levels"], m.grid)   # per step
        gbs = algo / (m2l_ms / 1e3) / 1e9
        inter = 2 * separable_bytes(m.info["coefficients"], m.info["levels"], m.grid)        # per step
        gbs_inter = inter / (m2l_ms / 1e3) / 1e9
        traffic = M2L_TRAFFIC_BYTES.get(("separable", m.grid, m.info["coefficients"]))
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": traffic, "traffic_unit": "bytes per transform (its M2L launches)",
                "traffic_ratio": None if traffic is None else traffic / (algo / 2),
                "kernel": "k_m2l_sep (passes X, Y, Z; finest level and levels above it)",
                "bytes_per_step": algo,
                "frac_with_intermediates": gbs_inter / hbm,
                "with_intermediates": {"bytes_per_step": inter, "achieved": gbs_inter,
                                       "what": "every pass reads its input rows and writes its output rows "
                                               "once, the 4-indexed intermediates included"},
                "useful_flops_per_step": useful,
                "useful_flops_achieved_tflops": achieved, "peak_basis": basis}
    if m.mode in ("fp32", "occupied"):
        # (the occupied-cell form on this workload: every cell holds points, so its pairs are all
        # the interacting pairs and the useful flops are the dense form's)
        sm = peaks.get("sm_max_mhz", 2070.0)
        peak = fp32_peak_tflops(sm)
        kernel = "k_m2l_occ (CUDA cores, FP32, work queue)" if m.mode == "occupied" else "m2l (CUDA cores, FP32)"
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": kernel, "flops_per_step": useful,
                "peak_basis": f"derived: 152 SMs x 128 FP32 lanes x 2 x {sm:.0f} MHz"}
    bf16 = peaks.get("bf16_tflops_sustained")
    basis = "of measured bf16 sustained (MEASURED_PEAKS.json)"
    if bf16 is None:
        bf16, basis = 1700.0, "of fallback bf16 sustained"
    peak = bf16 if m.mode in ("bf16", "bf16x3") else bf16 * TF32_PER_BF16
    if m.mode not in ("bf16", "bf16x3"):
        basis += " x nominal TF32/BF16 ratio 1.1/2.25"
    executed = issued / (m2l_ms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": M2L_TRAFFIC_BYTES.get((m.mode, m.grid, m.info["coefficients"])),
            "traffic_unit": "bytes per launch (one transform)",
            "kernel": f"k_m2l_tc (tcgen05, {m.mode})", "flops_per_step": useful,
            "executed": {"flops_per_step": issued, "achieved": executed, "frac": executed / peak},
            "peak_basis": basis}


def stage_roofline(m: Measured, wl, peaks):
    """HBM roofline of the memory-bound stages, per step (forward + backward): the bytes each
    stage must move (inputs read once, outputs written once) over its measured time."""
    hbm = peaks.get("hbm_gbs") or 6800.0
    P = m.info["coefficients"]
    Pp = (P + 3) // 4 * 4
    row = 4 * Pp
    G = [(wl.grid >> l) ** 3 for l in range(m.info["levels"])]
    N, M = wl.N, wl.M
    # per step: the forward sorts (p, w) (16 B read, a 16-byte record and a 4-byte index written
    # per point) and q (12 B read, 20 B written); the backward reuses both sorts and gathers ybar
    # into the record of each sorted query (index and ybar read, 4 B written)
    sort = (16 + 20) * N + (12 + 20) * M + (4 + 4 + 4) * M
    p2m = (16 * N + row * G[0]) + (16 * M + row * G[0])
    m2m = 2 * sum(row * (G[l] + G[l + 1]) for l in range(len(G) - 1))
    # L2L (parent row read, child row read and written) stops at level 1 when a transform has at
    # most 8 targets per finest cell (32 at orders >= 7); L2P then also reads the level-1 rows
    per_cell = 32 if wl.order >= 7 else 8

    def l2l_of(targets):
        stop = 1 if (len(G) > 1 and targets <= per_cell * G[0]) else 0
        return sum(row * (G[l + 1] + 2 * G[l]) for l in range(stop, len(G) - 1)), stop == 1

    l2l_f, two_f = l2l_of(M)
    l2l_b, two_b = l2l_of(N)
    l2l = l2l_f + l2l_b
    l2p = (16 * M + row * (G[0] + (G[1] if two_f else 0)) + 4 * M)
    l2p += (16 * N + row * (G[0] + (G[1] if two_b else 0)) + 16 * N)
    out = {}
    for name, b in (("sort", sort), ("p2m", p2m), ("m2m", m2m), ("l2l", l2l), ("l2p", l2p)):
        ms = m.stage_ms.get(name)
        if not ms:
            continue
        gbs = b / (ms / 1e3) / 1e9
        out[name] = {"bytes_per_step": b, "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm}
    return out


def measure_rays(dev, flush, steps, warmup):
    """Ray integrals (Sec. 6, integral-implicit layer) on the ray workload's sizes: 2^18 sphere-surface
    sources, the 512 x 512 pixel rays of its pinhole camera through the cube, 64^3, order 8, sigma
    0.01, separable M2L; a step is the forward ray integrals and their adjoint (wbar, pbar for
    L = sum y^2 / 2), timed with CUDA events on the launching stream."""
    import torch
    from paper_2111_00110_gb300 import workloads
    from paper_2111_00110_gb300.transform import Plan
    src = workloads.sphere_rays(width=4, height=4, samples=1)
    rays = torch.from_numpy(workloads.pinhole_rays(512, 512)).to(dev)
    p = torch.from_numpy(src.p).to(dev)
    w = torch.from_numpy(src.w).to(dev)
    plan = Plan(3, src.grid, src.order, src.sigma, m2l="separable", max_sources=src.N, max_queries=1, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        y = plan.ray_forward(p, w, rays)
        plan.ray_backward(p, w, rays, y)

    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize(dev)
    plan.profile_read(reset=True)
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        total += a.elapsed_time(b)
    _, launches = plan.profile_read(reset=True)
    plan.profile(True)
    step()
    torch.cuda.synchronize(dev)
    stage_ms, _ = plan.profile_read(reset=True)
    plan.profile(False)
    R = rays.shape[0]
    ms = total / steps
    out = {"workload": "sphere_rays sources, 512x512 pinhole rays", "N": src.N, "rays": R, "grid": src.grid,
           "order": src.order, "sigma": src.sigma, "m2l": "separable", "value": R / (ms / 1e3),
           "unit": "rays/s (ray integrals + adjoint)", "ms_per_step": ms, "steps": steps,
           "gpu_launches": int(sum(launches.values())),
           "stage_ms_per_step": {k: v for k, v in stage_ms.items() if v}}
    plan.close()
    return out


def measure_ray_queries(args, world, dev, flush, modes=("separable", "bf16x3", "tf32", "bf16"), n_ref=8192):
    """The ray-query workload as point queries: 2^18 sphere-surface sources, 512 x 512 pinhole rays x
    128 stratified samples (33,554,432 queries), 64^3, order 8, sigma 0.01; a forward + backward
    step per M2L form (the separable FP32 passes, BF16 x 3, and the mixed TF32 and BF16 forms), each
    with its error against the FP64 oracle at `n_ref` seeded queries (y) and sources (wbar, pbar)."""
    from paper_2111_00110_gb300 import workloads
    wl = workloads.sphere_rays()
    ref = None if args.no_check else oracle_reference_sample(wl, n=n_ref)
    out = {"workload": "sphere_rays: 2^18 sphere-surface sources, 512 x 512 rays x 128 samples",
           "N": wl.N, "M": wl.M, "grid": wl.grid, "order": wl.order, "sigma": wl.sigma,
           "unit": UNIT, "error_sample": f"{n_ref} seeded queries (y) and {n_ref} seeded sources (wbar, pbar)",
           "forms": {}}
    peaks = load_peaks()
    for mode in modes:
        m = measure_mode(mode, wl, args, world, dev, flush, ref=ref, steps=min(args.steps, 5))
        out["forms"][mode] = {"value": m.value, "ms_per_step": m.ms_per_step, "rel_l2_vs_oracle": m.err,
                              "stage_ms_per_step": m.stage_ms, "roofline": roofline_for(m, peaks)}
    return out


def measure_fit(dev, flush, steps, n=1 << 24, adam_steps=100, n_ref=2048, check=True):
    """The large fitting loop: 2^24 sources from 64 anisotropic Gaussians, 2^24 uniform queries,
    128^3, order 8, sigma 0.005; targets from the ground-truth set, w initialised to 0.1 N(0,1)
    (seed 5002), Adam (lr 1e-3) on (w, p) through the autograd layer.  The configured form is the
    mixed-precision (TF32) M2L: one timed forward + backward step, the device memory it holds (the
    library's plan workspace and the step's tensors; the backward rebuilds its own expansion from
    (q, ybar), so no expansion of the forward is kept), step 0 against the oracle at `n_ref`
    samples, and the loss over `adam_steps` steps.  The FP32 separable form is timed and checked on
    the same step 0 beside it."""
    import numpy as np
    import torch
    from paper_2111_00110_gb300 import workloads
    from paper_2111_00110_gb300.transform import Plan, fc2t2
    gt = workloads.fit_large(N=n, M=n)
    q = torch.from_numpy(gt.q).to(dev)
    w0 = (0.1 * np.random.default_rng(5002).standard_normal(n)).astype(np.float32)
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(7)
    sq = np.sort(rng.choice(n, size=n_ref, replace=False))
    sp = np.sort(rng.choice(n, size=n_ref, replace=False))
    target = None
    ref_y = None
    hi = float(np.nextafter(np.float32(1.0), np.float32(0.0)))
    out = {"workload": "fit_large: 2^24 sources (64 anisotropic Gaussians), 2^24 uniform queries",
           "N": n, "M": n, "grid": gt.grid, "order": gt.order, "sigma": gt.sigma,
           "unit": "query-evals/s (fwd+bwd through the autograd layer)"}
    for form in ("tf32", "separable"):
        torch.cuda.synchronize(dev)
        free0, _ = torch.cuda.mem_get_info(dev)
        plan = Plan(3, gt.grid, gt.order, gt.sigma, m2l=form, max_sources=n, max_queries=n, device=dev)
        torch.cuda.synchronize(dev)
        free1, _ = torch.cuda.mem_get_info(dev)
        if target is None:
            # targets: the configured (TF32) transform of the ground-truth set
            with torch.no_grad():
                target = plan.forward(torch.from_numpy(gt.p).to(dev), torch.from_numpy(gt.w).to(dev), q)
        p = torch.from_numpy(gt.p).to(dev).requires_grad_(True)
        w = torch.from_numpy(w0).to(dev).requires_grad_(True)

        def loss_and_grad():
            y = fc2t2(p, w, q, plan)
            loss = torch.mean((y - target) ** 2)
            loss.backward()
            return y, loss

        y, _ = loss_and_grad()
        torch.cuda.synchronize(dev)
        err = None
        if check:
            import oracle
            d = oracle.OracleDesc(dim=3, grid=gt.grid, order=gt.order, sigma=gt.sigma)
            f64 = lambda a: np.asarray(a, dtype=np.float64)
            if ref_y is None:
                ref_y = oracle.forward(d, f64(gt.p), f64(w0), f64(gt.q), sel=sq)
            ybar = (2.0 / n) * (y - target).detach().cpu().numpy()
            # (the cotangent depends on the form's own y: the backward reference is per form)
            wo, po = oracle.backward(d, f64(gt.p), f64(w0), f64(gt.q), f64(ybar), sel=sp)
            err = {"y": rel_l2(y.detach().cpu().numpy()[sq], ref_y), "wbar": rel_l2(w.grad.cpu().numpy()[sp], wo),
                   "pbar": rel_l2(p.grad.cpu().numpy()[sp], po)}
        torch.cuda.reset_peak_memory_stats(dev)
        for _ in range(2):
            w.grad = None
            p.grad = None
            loss_and_grad()
        torch.cuda.synchronize(dev)
        total_ms = 0.0
        for _ in range(steps):
            flush.zero_()
            w.grad = None
            p.grad = None
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            loss_and_grad()
            b.record(stream)
            torch.cuda.synchronize(dev)
            total_ms += a.elapsed_time(b)
        ms = total_ms / steps
        free2, _ = torch.cuda.mem_get_info(dev)
        res = {"m2l": form, "value": n / (ms / 1e3), "ms_per_step": ms, "steps": steps,
               "step0_rel_l2_vs_oracle": err,
               "memory": {"plan_workspace_bytes": int(free0 - free1),
                          "device_in_use_after_steps_bytes": int(free0 - free2),
                          "torch_peak_allocated_bytes": int(torch.cuda.max_memory_allocated(dev)),
                          "finest_expansion_bytes": int(gt.grid ** 3 * plan.info()["coefficients"] * 4)}}
        if form == "tf32":
            with torch.no_grad():
                w.copy_(torch.from_numpy(w0).to(dev))
                p.copy_(torch.from_numpy(gt.p).to(dev))
            opt = torch.optim.Adam([w, p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
            loss_t = []
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(adam_steps):
                opt.zero_grad()
                with torch.no_grad():
                    p.clamp_(0.0, hi)
                _, loss = loss_and_grad()
                opt.step()
                loss_t.append(loss.detach())
            b.record(stream)
            torch.cuda.synchronize(dev)
            losses = [float(x) for x in loss_t]
            res["adam"] = {"steps": adam_steps, "lr": 1e-3, "ms_total": a.elapsed_time(b),
                           "loss": {str(i): losses[i] for i in range(0, adam_steps, 10)} | {str(adam_steps - 1): losses[-1]}}
            out.update(res)
        else:
            out["fp32_separable"] = res
        plan.check()
        plan.close()
        del p, w
    return out


def measure_batched(dev, flush, steps, warmup, n_inst=64):
    """The batched workload: 64 independent clustered point sets (N_i = M_i log-uniform in
    [1024, 262144]), sigma 0.02, each with its grid (32^3 or 64^3), order (4, 6 or 8) and M2L form
    (separable line passes over the whole grid, at the automatic or 32 finest-level cells per CTA,
    or the occupied-cell work queue) chosen by the autotuner (fastest candidate within 1e-2 rel-L2
    of the exact sum), then refined for the batch (the choices timed as a whole batch against the
    same with the FP32 forms moved to the occupied-cell form).  A step is one batched
    forward and one batched backward call over all instances: each instance's sorts, P2M and M2M on
    its plan's stream, one persistent M2L launch for all occupied-cell instances of an order, then
    L2L and L2P per instance.  The step is captured in a CUDA graph and replayed; the same step
    launched eagerly, and the instances one call after another on one stream, for comparison."""
    import time
    import torch
    from paper_2111_00110_gb300 import autotune, workloads
    from paper_2111_00110_gb300.transform import Plan, backward_batched, forward_batched
    wls = [workloads.mixture(i) for i in range(n_inst)]
    ps = [torch.from_numpy(wl.p).to(dev) for wl in wls]
    ws = [torch.from_numpy(wl.w).to(dev) for wl in wls]
    qs = [torch.from_numpy(wl.q).to(dev) for wl in wls]
    t0 = time.time()
    choices = [autotune.autotune(p, w, q, wl.sigma, target=1e-2, grids=(32, 64), orders=(4, 6, 8),
                                 m2l=("occupied", "separable"), sample=512, reps=1, tiles=(0, 32))[0]
               for wl, p, w, q in zip(wls, ps, ws, qs)]
    stream = torch.cuda.current_stream(dev)

    def make_plans(cs):
        return [Plan(3, c.grid, c.order, wl.sigma, m2l=c.m2l, max_sources=wl.N, max_queries=wl.M, tile=c.tile,
                     device=dev) for c, wl in zip(cs, wls)]

    def time_batch(cs, reps=3):
        pls = make_plans(cs)
        try:
            for _ in range(2):
                backward_batched(pls, ps, ws, qs, forward_batched(pls, ps, ws, qs), reuse_forward=True)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                backward_batched(pls, ps, ws, qs, forward_batched(pls, ps, ws, qs), reuse_forward=True)
            b.record(stream)
            torch.cuda.synchronize(dev)
            return a.elapsed_time(b) / reps
        finally:
            for pl in pls:
                pl.close()

    # the per-instance choices against the same with the FP32 forms on the occupied-cell form
    # (one shared M2L launch), timed as whole batches
    choices, refinement = autotune.refine_batch(choices, time_batch)
    tune_s = time.time() - t0
    plans = make_plans(choices)

    def step_batched():
        ys = forward_batched(plans, ps, ws, qs)
        backward_batched(plans, ps, ws, qs, ys, reuse_forward=True)

    def step_sequential():
        for pl, p, w, q in zip(plans, ps, ws, qs):
            y = pl.forward(p, w, q)
            pl.backward(p, w, q, y, reuse_forward=True)

    def timed(fn):
        for _ in range(max(3, warmup)):
            fn()
        torch.cuda.synchronize(dev)
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            total += a.elapsed_time(b)
        return total / steps

    ms_eager = timed(step_batched)
    # the batched step captured once in a CUDA graph (every instance's launches, the plan streams'
    # fork / join and the shared M2L launches recorded once) and replayed
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step_batched()
    stream.wait_stream(side)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_batched()
    ms = timed(graph.replay)
    ms_seq = timed(step_sequential)
    queries = sum(wl.M for wl in wls)
    hist = {}
    for c in choices:
        key = f"{c.grid}^3 order {c.order} {c.m2l}" + (f" tile {c.tile}" if c.tile else "")
        hist[key] = hist.get(key, 0) + 1
    for pl in plans:
        pl.close()
    return {"workload": f"mixture, {n_inst} instances", "instances": n_inst, "queries": queries,
            "sigma": wls[0].sigma, "choices": hist, "autotune_s": tune_s, "batch_refinement": refinement,
            "value": queries / (ms / 1e3), "unit": "query-evals/s (fwd+bwd, all instances)",
            "ms_per_step": ms, "steps": steps, "timed": "the batched step replayed from a CUDA graph",
            "eager": {"ms_per_step": ms_eager, "value": queries / (ms_eager / 1e3)},
            "one_stream": {"ms_per_step": ms_seq, "value": queries / (ms_seq / 1e3)}}


def replica_workload(rank: int, **sizes):
    """The benchmark workload of one rank: weak scaling, every rank transforms its own
    independent point set (the uniform3d recipe drawn with seed 2 + rank)."""
    from paper_2111_00110_gb300 import workloads
    return workloads.uniform3d(seed=2 + rank, **sizes)


def job_value(units_per_rank: int, steps: int, world: int, job_ms: float) -> float:
    """Whole-job throughput: the units of every rank over the slowest rank's time."""
    return units_per_rank * steps * world / (job_ms / 1e3)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2111_00110_gb300 import build as _build
    from paper_2111_00110_gb300 import workloads

    _build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # weak scaling: every rank transforms its own independent point set
    wl = replica_workload(rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    ref = None
    if not args.no_check and rank == 0:
        ref = oracle_reference_sample(wl)
    primary = "separable" if args.m2l == "auto" else args.m2l
    main = measure_mode(primary, wl, args, world, dev, flush, ref=ref, do_e2e=not args.no_e2e, clocks=True)
    variants = {}
    if args.m2l == "auto":
        for mode in ("bf16x3", "tf32x3", "tf32", "bf16", "fp32", "occupied"):
            variants[mode] = measure_mode(mode, wl, args, world, dev, flush, ref=ref, steps=min(args.steps, 10))
        # the least-squares fitted operators (Sec. 3.1) on the tensor cores, checked against the
        # oracle's own fit
        ref_fit = None if ref is None else oracle_reference_sample(wl, fit=True, exact=ref["exact"])
        variants["bf16x3_fit"] = measure_mode("bf16x3", wl, args, world, dev, flush, ref=ref_fit,
                                              steps=min(args.steps, 10), fit=True)
    rays = measure_rays(dev, flush, min(args.steps, 10), args.warmup) if (args.m2l == "auto" and rank == 0) else None
    batched = measure_batched(dev, flush, min(args.steps, 5), args.warmup) if (args.m2l == "auto" and rank == 0) else None
    extra = args.m2l == "auto" and rank == 0 and not args.no_extra
    ray_queries = measure_ray_queries(args, world, dev, flush) if extra else None
    fit = measure_fit(dev, flush, min(args.steps, 5), check=not args.no_check) if extra else None
    if rank != 0:
        return
    peaks = load_peaks()
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

    def summary(m: Measured):
        return {"value": m.value, "ms_per_step": m.ms_per_step, "rel_l2_vs_oracle": m.err,
                "stage_ms_per_step": m.stage_ms, "roofline": roofline_for(m, peaks)}

    line = {
        "metric": METRIC, "value": main.value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main.ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "uniform3d", "dim": 3, "N": wl.N, "M": wl.M, "grid": wl.grid,
                   "levels": main.info["levels"], "order": wl.order, "sigma": wl.sigma, "m2l": primary,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
        "rel_l2_vs_oracle": main.err,
        "clocks": main.clocks,
        "e2e": main.e2e,
        "gpu_launches": main.launches,
        "roofline": roofline_for(main, peaks),
        "stage_roofline": {"peak_gbs": peaks.get("hbm_gbs"), "peak_basis": "of measured hbm copy (MEASURED_PEAKS.json)",
                           "stages": stage_roofline(main, wl, peaks)},
        "stage_ms_per_step": main.stage_ms,
        "variants": {k: summary(v) for k, v in variants.items()},
        "ray_integrals": rays,
        "ray_queries": ray_queries,
        "fit_large": fit,
        "batched": batched,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


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
