"""PyTorch front end of the FC2T2 transform (arXiv 2111.00110).

``Plan`` wraps one ``fc2t2_plan`` of the C ABI; ``Plan.forward`` / ``Plan.backward`` pass
CUDA tensors' device pointers and the current stream to ``fc2t2_forward`` /
``fc2t2_backward``.  With C channels the weights are (C, N) and the values (C, M); with one
channel they may also be one-dimensional.  ``Plan.expand`` returns the accessor of Sec. 3
("How to use the implementation?", see ``accessor``).  ``FC2T2Function`` is the explicit layer of Sec. 4 as a
``torch.autograd.Function``: forward computes y = f(q; p, w), backward returns
(pbar, wbar, None) from the transposed transform (Sec. 4.1).  PyTorch only allocates memory
and supplies streams; every arithmetic step runs in the CUDA library.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import capi


def _ptr(t: Optional[torch.Tensor]) -> int:
    return 0 if t is None else t.data_ptr()


def _check_tensor(t: torch.Tensor, name: str, shape) -> None:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def resolve_m2l(m2l: str, dim: int, kernel: str, fit: bool) -> str:
    """The M2L form of a plan: "auto" takes the separable line passes where they apply (the
    Gaussian in 3D with Taylor operators: the fastest form, at FP32 accuracy), else plain FP32."""
    if m2l != "auto":
        return m2l
    return "separable" if (kernel == "gaussian" and dim == 3 and not fit) else "fp32"


class Plan:
    """A transform plan: dimension, finest grid, order, kernel, domain, workspace bounds, M2L form
    ("auto", "separable", "occupied", "fp32", "tf32", "bf16", "tf32x3", "bf16x3"); "occupied" runs the
    direct FP32 operator over the occupied cells only (clustered points)."""

    def __init__(self, dim: int, grid: int, order: int, sigma: float = 0.05, *,
                 kernel: str = "gaussian", poly_coef: Optional[Sequence[float]] = None,
                 lo: float = 0.0, hi: float = 1.0, m2l: str = "auto", check_domain: bool = False,
                 max_sources: int = 1 << 20, max_queries: int = 1 << 20, channels: int = 1, fit: bool = False,
                 tile: int = 0, device=None):
        self.dim, self.grid, self.order, self.channels = dim, grid, order, int(channels)
        m2l = resolve_m2l(m2l, dim, kernel, fit)
        self._serial = 0   # counts the calls that replace the plan's expansion
        self.sigma, self.kernel, self.lo, self.hi, self.m2l = sigma, kernel, lo, hi, m2l
        self.max_sources, self.max_queries = int(max_sources), int(max_queries)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        d = capi.PlanDesc()
        d.dim, d.grid, d.order = dim, grid, order
        d.kernel = capi.KERNELS[kernel]
        d.sigma = float(sigma)
        self._poly = None
        if poly_coef is not None:
            self._poly = np.ascontiguousarray(poly_coef, dtype=np.float64)
            d.poly_coef = self._poly.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            d.n_poly = int(self._poly.size)
        d.lo, d.hi = float(lo), float(hi)
        d.channels = self.channels
        d.m2l = capi.M2L_PREC[m2l]
        d.check_domain = 1 if check_domain else 0
        d.fit = 1 if fit else 0   # least-squares fitted M2L operators (Sec. 3.1)
        d.tile = int(tile)        # separable M2L: finest-level cells per CTA (0: automatic)
        self.tile = int(tile)
        d.max_sources, d.max_queries = self.max_sources, self.max_queries
        with torch.cuda.device(self.device):
            self._h = capi.plan_create(d)

    def close(self) -> None:
        if getattr(self, "_h", None):
            capi.plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, enable: bool = True) -> None:
        """Record per-stage CUDA events on every call (diagnostics)."""
        capi.profile_enable(self._h, enable)

    def profile_read(self, reset: bool = False):
        """(ms per stage, kernel launches per stage) accumulated since the last reset."""
        return capi.profile_read(self._h, reset)

    def info(self) -> dict:
        """Per-transform work of this plan (levels, P, M2L cell pairs and flops, device bytes)."""
        return capi.plan_query(self._h)

    def check(self) -> None:
        """Wait for the plan's work on the current stream and raise FC2T2Error if a bounded
        device-side wait gave up since the last check (or, with check_domain, a point was outside
        the domain in the last call)."""
        capi.plan_check(self._h, self._stream())

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _chan_shape(self, t: torch.Tensor, n: int):
        """(n,) for a one-dimensional tensor of a one-channel plan, else (C, n)."""
        if t.dim() == 1 and self.channels == 1:
            return (n,)
        return (self.channels, n)

    def expand(self, p: torch.Tensor, w: torch.Tensor):
        """Keep the expansion of (p, w) in the plan and return its accessor (``Expansion``)."""
        from .accessor import Expansion
        N = p.shape[0]
        _check_tensor(p, "p", (N, self.dim))
        _check_tensor(w, "w", self._chan_shape(w, N))
        self._serial += 1
        capi.expand(self._h, self._stream(), _ptr(p), _ptr(w), N)
        return Expansion(self, self._serial)

    def forward(self, p: torch.Tensor, w: torch.Tensor, q: torch.Tensor,
                out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """y[c, m] = sum_n psi(p[n] - q[m]) w[c, n] (Sec. 3, Eq. 1) through the series."""
        N, M = p.shape[0], q.shape[0]
        _check_tensor(p, "p", (N, self.dim))
        _check_tensor(w, "w", self._chan_shape(w, N))
        _check_tensor(q, "q", (M, self.dim))
        yshape = self._chan_shape(w, M)
        y = torch.empty(yshape, device=q.device, dtype=torch.float32) if out is None else out
        _check_tensor(y, "y", yshape)
        self._serial += 1
        capi.forward(self._h, self._stream(), _ptr(p), _ptr(w), N, _ptr(q), M, _ptr(y))
        return y

    def backward(self, p: torch.Tensor, w: torch.Tensor, q: torch.Tensor, ybar: torch.Tensor,
                 need_w: bool = True, need_p: bool = True, reuse_forward: bool = False):
        """(wbar, pbar) of Sec. 4.1 for the cotangent ybar; either may be skipped (None).

        ``reuse_forward``: the tensors are those of this plan's last forward call and unchanged
        since (as for an autograd layer's saved inputs), so that call's sorts are reused."""
        N, M = p.shape[0], q.shape[0]
        _check_tensor(p, "p", (N, self.dim))
        _check_tensor(w, "w", self._chan_shape(w, N))
        _check_tensor(q, "q", (M, self.dim))
        _check_tensor(ybar, "ybar", self._chan_shape(w, M))
        wbar = torch.empty(self._chan_shape(w, N), device=p.device, dtype=torch.float32) if need_w else None
        pbar = torch.empty(N, self.dim, device=p.device, dtype=torch.float32) if need_p else None
        self._serial += 1
        fn = capi.backward_reuse if reuse_forward else capi.backward
        fn(self._h, self._stream(), _ptr(p), _ptr(w), N, _ptr(q), M, _ptr(ybar), _ptr(wbar), _ptr(pbar))
        return wbar, pbar


    def backward_q(self, p: torch.Tensor, w: torch.Tensor, q: torch.Tensor, ybar: torch.Tensor) -> torch.Tensor:
        """qbar[m] = sum_c ybar[c, m] * grad y_c(q[m]) (the derivative of the local series at the
        queries)."""
        N, M = p.shape[0], q.shape[0]
        _check_tensor(p, "p", (N, self.dim))
        _check_tensor(w, "w", self._chan_shape(w, N))
        _check_tensor(q, "q", (M, self.dim))
        _check_tensor(ybar, "ybar", self._chan_shape(w, M))
        qbar = torch.empty(M, self.dim, device=q.device, dtype=torch.float32)
        self._serial += 1
        capi.backward_q(self._h, self._stream(), _ptr(p), _ptr(w), N, _ptr(q), M, _ptr(ybar), _ptr(qbar))
        return qbar

    def ray_forward(self, p: torch.Tensor, w: torch.Tensor, rays: torch.Tensor) -> torch.Tensor:
        """Integrals of the series of (p, w) along rays [R, 8] = (origin, direction, t0, t1):
        y[c, q] = int_{t0}^{t1} f_c(o_q + t r_q) dt (Sec. 6, the integral-implicit layer)."""
        N, R = p.shape[0], rays.shape[0]
        _check_tensor(p, "p", (N, self.dim))
        _check_tensor(w, "w", self._chan_shape(w, N))
        _check_tensor(rays, "rays", (R, 8))
        y = torch.empty(self._chan_shape(w, R), device=p.device, dtype=torch.float32)
        self._serial += 1
        capi.ray_forward(self._h, self._stream(), _ptr(p), _ptr(w), N, _ptr(rays), R, _ptr(y))
        return y

    def ray_backward(self, p: torch.Tensor, w: torch.Tensor, rays: torch.Tensor, ybar: torch.Tensor,
                     need_w: bool = True, need_p: bool = True):
        """(wbar, pbar) of ``ray_forward`` for the cotangent ybar (the rays inserted as sources)."""
        N, R = p.shape[0], rays.shape[0]
        _check_tensor(p, "p", (N, self.dim))
        _check_tensor(w, "w", self._chan_shape(w, N))
        _check_tensor(rays, "rays", (R, 8))
        _check_tensor(ybar, "ybar", self._chan_shape(w, R))
        wbar = torch.empty(self._chan_shape(w, N), device=p.device, dtype=torch.float32) if need_w else None
        pbar = torch.empty(N, self.dim, device=p.device, dtype=torch.float32) if need_p else None
        self._serial += 1
        capi.ray_backward(self._h, self._stream(), _ptr(p), _ptr(w), N, _ptr(rays), R, _ptr(ybar), _ptr(wbar),
                          _ptr(pbar))
        return wbar, pbar


class FC2T2RayFunction(torch.autograd.Function):
    """y = integrals of f(.; p, w) along fixed rays, with the adjoints of Sec. 6 (ray2M)."""

    @staticmethod
    def forward(ctx, p, w, rays, plan: "Plan"):
        p, w, rays = p.contiguous(), w.contiguous(), rays.contiguous()
        ctx.plan = plan
        ctx.save_for_backward(p, w, rays)
        return plan.ray_forward(p, w, rays)

    @staticmethod
    def backward(ctx, ybar):
        p, w, rays = ctx.saved_tensors
        need_p, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        wbar = pbar = None
        if need_p or need_w:
            wbar, pbar = ctx.plan.ray_backward(p, w, rays, ybar.contiguous(), need_w=need_w, need_p=need_p)
        return pbar, wbar, None, None


def fc2t2_rays(p: torch.Tensor, w: torch.Tensor, rays: torch.Tensor, plan: "Plan") -> torch.Tensor:
    """Differentiable ray integrals of the transform (Sec. 6)."""
    return FC2T2RayFunction.apply(p, w, rays, plan)


class FC2T2Function(torch.autograd.Function):
    """y = f(q; p, w) with hand-written adjoints (Sec. 4.1); the query gradient is computed when
    q requires it."""

    @staticmethod
    def forward(ctx, p, w, q, plan: Plan):
        p, w, q = p.contiguous(), w.contiguous(), q.contiguous()
        ctx.plan = plan
        ctx.save_for_backward(p, w, q)
        return plan.forward(p, w, q)

    @staticmethod
    def backward(ctx, ybar):
        p, w, q = ctx.saved_tensors
        need_p, need_w, need_q = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        ybar = ybar.contiguous()
        wbar = pbar = qbar = None
        if need_p or need_w:
            # the saved inputs are unchanged since the forward (autograd checks their versions);
            # the plan reuses that call's sorts if it still holds them
            wbar, pbar = ctx.plan.backward(p, w, q, ybar, need_w=need_w, need_p=need_p, reuse_forward=True)
        if need_q:
            qbar = ctx.plan.backward_q(p, w, q, ybar)
        return pbar, wbar, qbar, None


def fc2t2(p: torch.Tensor, w: torch.Tensor, q: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable explicit layer y = f(q; p, w) (Sec. 4)."""
    return FC2T2Function.apply(p, w, q, plan)


def direct(p: torch.Tensor, w: torch.Tensor, q: torch.Tensor, sigma: float) -> torch.Tensor:
    """Exact y[m] = sum_n exp(-|p[n] - q[m]|^2 / (2 sigma^2)) w[n] by brute force on the device
    (O(N M); for error measurements on query samples).  w is (N,) or (C, N); y is (M,) or (C, M)."""
    dim = p.shape[1]
    N, M = p.shape[0], q.shape[0]
    C = 1 if w.dim() == 1 else w.shape[0]
    _check_tensor(p, "p", (N, dim))
    _check_tensor(w, "w", (N,) if w.dim() == 1 else (C, N))
    _check_tensor(q, "q", (M, dim))
    d = capi.PlanDesc()
    d.dim, d.grid, d.order, d.kernel, d.sigma = dim, 4, 1, capi.KERNELS["gaussian"], float(sigma)
    d.lo, d.hi, d.channels = 0.0, 1.0, C
    y = torch.empty((M,) if w.dim() == 1 else (C, M), device=q.device, dtype=torch.float32)
    capi.direct(d, torch.cuda.current_stream(q.device).cuda_stream, _ptr(p), _ptr(w), N, _ptr(q), M, _ptr(y))
    return y


def forward_batched(plans: Sequence[Plan], ps, ws, qs):
    """Forward transforms of independent instances (one plan each, uneven N_i and M_i) through
    one ``fc2t2_forward_batched`` call on the current stream; returns the list of y_i."""
    n = len(plans)
    if not (len(ps) == len(ws) == len(qs) == n):
        raise ValueError("plans, ps, ws and qs must have the same length")
    ys = []
    for i, (pl, p, w, q) in enumerate(zip(plans, ps, ws, qs)):
        _check_tensor(p, f"p[{i}]", (p.shape[0], pl.dim))
        _check_tensor(w, f"w[{i}]", pl._chan_shape(w, p.shape[0]))
        _check_tensor(q, f"q[{i}]", (q.shape[0], pl.dim))
        ys.append(torch.empty(pl._chan_shape(w, q.shape[0]), device=q.device, dtype=torch.float32))
        pl._serial += 1
    stream = torch.cuda.current_stream(plans[0].device).cuda_stream if n else 0
    capi.forward_batched([pl._h for pl in plans], stream, [_ptr(p) for p in ps], [_ptr(w) for w in ws],
                         [p.shape[0] for p in ps], [_ptr(q) for q in qs], [q.shape[0] for q in qs],
                         [_ptr(y) for y in ys])
    return ys


def backward_batched(plans: Sequence[Plan], ps, ws, qs, ybars, reuse_forward: bool = False):
    """(wbar_i, pbar_i) of independent instances through one ``fc2t2_backward_batched`` call.

    ``reuse_forward``: the tensors are those of the plans' last ``forward_batched`` call and
    unchanged since, so that call's sorts are reused (``fc2t2_backward_batched_reuse``)."""
    n = len(plans)
    if not (len(ps) == len(ws) == len(qs) == len(ybars) == n):
        raise ValueError("plans, ps, ws, qs and ybars must have the same length")
    wbars, pbars = [], []
    for i, (pl, p, w, q, yb) in enumerate(zip(plans, ps, ws, qs, ybars)):
        _check_tensor(p, f"p[{i}]", (p.shape[0], pl.dim))
        _check_tensor(w, f"w[{i}]", pl._chan_shape(w, p.shape[0]))
        _check_tensor(q, f"q[{i}]", (q.shape[0], pl.dim))
        _check_tensor(yb, f"ybar[{i}]", pl._chan_shape(w, q.shape[0]))
        wbars.append(torch.empty(pl._chan_shape(w, p.shape[0]), device=p.device, dtype=torch.float32))
        pl._serial += 1
        pbars.append(torch.empty(p.shape[0], pl.dim, device=p.device, dtype=torch.float32))
    stream = torch.cuda.current_stream(plans[0].device).cuda_stream if n else 0
    capi.backward_batched([pl._h for pl in plans], stream, [_ptr(p) for p in ps], [_ptr(w) for w in ws],
                          [p.shape[0] for p in ps], [_ptr(q) for q in qs], [q.shape[0] for q in qs],
                          [_ptr(y) for y in ybars], [_ptr(t) for t in wbars], [_ptr(t) for t in pbars],
                          reuse=reuse_forward)
    return list(zip(wbars, pbars))
