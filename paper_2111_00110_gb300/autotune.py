"""Per-instance choice of grid and expansion order (the batched workload's autotuner).

Each candidate (grid, order, M2L form) is built as a plan and run on the instance: its time is a
forward + backward step measured with CUDA events, its error the relative L2 distance to the exact
sum (``fc2t2_direct``, brute force on the device) on a seeded sample of queries.  The choice is the
fastest candidate whose error meets the target; when none does, the most accurate one.  The
selection rule is separate from the measurements so that it can be checked on the host.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import Callable, Iterable, List, Optional, Sequence, Tuple

import numpy as np


@dataclass
class Candidate:
    grid: int
    order: int
    m2l: str
    ms: float              # forward + backward, milliseconds
    err: float             # relative L2 error of y against the exact sum on the query sample
    tile: int = 0          # separable M2L: finest-level cells per CTA (0: the plan's automatic choice)


def select(cands: Sequence[Candidate], target: float) -> Candidate:
    """Fastest candidate with err <= target; if there is none, the most accurate (then fastest)."""
    if not cands:
        raise ValueError("no candidates")
    ok = [c for c in cands if c.err <= target]
    if ok:
        return min(ok, key=lambda c: (c.ms, c.err))
    return min(cands, key=lambda c: (c.err, c.ms))


def _rel_l2(a, b) -> float:
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.clamp(torch.linalg.vector_norm(b), min=1e-300))


def measure(p, w, q, sigma: float, grid: int, order: int, m2l: str, sample, ref, reps: int = 3,
            tile: int = 0) -> Candidate:
    """Time a forward + backward step of one candidate and its error on the query sample."""
    import torch
    from .transform import Plan
    dim = p.shape[1]
    plan = Plan(dim, grid, order, sigma, m2l=m2l, max_sources=max(p.shape[0], 1),
                max_queries=max(q.shape[0], 1), tile=tile, device=p.device)
    try:
        y = plan.forward(p, w, q)
        plan.backward(p, w, q, y)
        stream = torch.cuda.current_stream(p.device)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            y = plan.forward(p, w, q)
            plan.backward(p, w, q, y)
        b.record(stream)
        torch.cuda.synchronize(p.device)
        plan.check()
        err = _rel_l2(y[sample], ref)
        return Candidate(grid, order, m2l, a.elapsed_time(b) / reps, err, tile)
    finally:
        plan.close()


# M2L forms that compute the same operator in FP32 arithmetic: their truncation error against the
# exact sum is one (grid, order)'s, so once one of them misses the target the others need no run
FP32_FORMS = ("fp32", "separable", "occupied", "tf32x3", "bf16x3")


def autotune(p, w, q, sigma: float, target: float = 1e-2, grids: Iterable[int] = (32, 64),
             orders: Iterable[int] = (4, 6, 8), m2l: Iterable[str] = ("separable", "occupied"), sample: int = 1024,
             seed: int = 0, reps: int = 3, tiles: Iterable[int] = (0,)) -> Tuple[Candidate, List[Candidate]]:
    """Measure the (grid, order, M2L form, tile) candidates on the instance (p, w, q) and choose one.

    The forms differ in how the M2L's work is laid out on the GPU: the separable line passes
    sweep every cell of the grid in segments of ``tile`` cells per CTA at the finest level (each
    value of ``tiles``; 0 is the plan's automatic choice), the occupied-cell form takes work items
    of 32 occupied target cells from a queue (work in proportion to the occupied cell pairs).
    ``sample`` queries (seeded) are compared with the exact sum.  An FP32-accurate candidate of a
    (grid, order) whose first FP32-accurate candidate missed the target is skipped (same operator,
    same error).  Returns (choice, every measured candidate)."""
    from .transform import direct
    M = q.shape[0]
    rng = np.random.default_rng(seed)
    k = min(sample, M)
    idx = np.sort(rng.choice(M, size=k, replace=False)) if k < M else np.arange(M)
    import torch
    sample_idx = torch.as_tensor(idx, device=q.device, dtype=torch.long)
    ref = direct(p, w, q[sample_idx].contiguous(), sigma)
    cands = []
    for g in grids:
        for o in orders:
            missed = False
            for f in m2l:
                for t in (tuple(tiles) if f == "separable" else (0,)):
                    if missed and f in FP32_FORMS:
                        continue
                    c = measure(p, w, q, sigma, g, o, f, sample_idx, ref, reps, tile=t)
                    cands.append(c)
                    missed = missed or (f in FP32_FORMS and c.err > target)
    return select(cands, target), cands


def refine_batch(choices: Sequence[Candidate], time_batch: Callable[[Sequence[Candidate]], float]):
    """Batch-level refinement of per-instance choices.

    An instance timed alone does not see the batch: in a batched call the occupied-cell instances
    share one M2L launch, which an instance on another form does not join.  So the per-instance
    choices are timed as a whole batch (``time_batch(choices)``: ms per batched step) against the
    same choices with every FP32-accurate form moved to the occupied-cell form at the same grid and
    order (the same operator, hence the same error against the exact sum); the faster is kept.
    Returns (choices, {"per_instance_ms": ..., "occupied_ms": ...} or {} when nothing moves)."""
    alt = [replace(c, m2l="occupied", tile=0) if (c.m2l in FP32_FORMS and c.m2l != "occupied") else c
           for c in choices]
    if alt == list(choices):
        return list(choices), {}
    t_own, t_alt = time_batch(choices), time_batch(alt)
    return (alt if t_alt < t_own else list(choices)), {"per_instance_ms": t_own, "occupied_ms": t_alt}


def tune_batch(instances, sigma: float, target: float = 1e-2, **kw) -> List[Candidate]:
    """Choice per instance of a batch: ``instances`` yields (p, w, q) device tensors."""
    return [autotune(p, w, q, sigma, target, **kw)[0] for p, w, q in instances]
