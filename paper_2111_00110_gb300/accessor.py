"""The accessor of an expansion (Sec. 3, "How to use the implementation?").

``Plan.expand(p, w)`` keeps the expansion of the sources in the plan (``fc2t2_expand``) and
returns an :class:`Expansion`, which is indexed like an array of shape (C, n, n[, n]) whose
spatial axes take continuous positions:

* ``S[c, x, y, z]`` -- the field of channel(s) ``c`` at the points formed by broadcasting the
  spatial entries against each other;
* ``S.vol[c, x, y, z]`` -- on the meshgrid of the spatial entries (a scalar becomes an axis of
  length one);
* ``S.partials[...]`` / ``S.partials2[...]`` (and ``.partials.vol`` ...) -- the first partials
  (a trailing axis of ``dim`` values) and the second partials (``dim (dim + 1) / 2`` values,
  d^2/dx_i dx_k for i <= k in row-major order).

A spatial entry is a number, a one-dimensional sequence or tensor, or a slice ``a:b:c`` read as
``linspace(a, b, c)`` (``a`` and ``b`` default to the domain's ends ``lo`` and ``hi``; ``c`` is
required).  The channel entry is an int, a slice, a sequence of ints or ``...``; with only the
spatial entries given, every channel is returned.  The batch axis of the paper's accessor is a
list of expansions here (one plan per instance).

Points on the meshgrid are evaluated without forming a point list (``fc2t2_evaluate_grid``); point
queries are sorted by cell on the device (``fc2t2_evaluate``), in chunks of the plan's
``max_queries``.  An expansion is valid until the next transform call on its plan.
"""
from __future__ import annotations

from typing import List, Tuple

import torch

from . import capi

WIDTH = {"value": lambda d: 1, "partials": lambda d: d, "partials2": lambda d: d * (d + 1) // 2}


def parse_key(key, dim: int, lo: float, hi: float) -> Tuple[object, List[torch.Tensor], List[bool]]:
    """Split an accessor index into (channel selector, spatial entries, which entries were
    scalars).  Spatial entries are returned as CPU float32 tensors of dimension 0 (scalars) or 1."""
    if not isinstance(key, tuple):
        key = (key,)
    if any(k is Ellipsis for k in key):
        if key.count(Ellipsis) != 1 or key[0] is not Ellipsis or len(key) != dim + 1:
            raise IndexError(f"use [..., x0 .. x{dim - 1}] with {dim} spatial entries")
        chan, spatial = Ellipsis, key[1:]
    elif len(key) == dim:
        chan, spatial = Ellipsis, key
    elif len(key) == dim + 1:
        chan, spatial = key[0], key[1:]
    else:
        raise IndexError(f"expected {dim} spatial entries, optionally after a channel entry; got {len(key)}")
    coords, scalar = [], []
    for k in spatial:
        if isinstance(k, slice):
            if k.step is None or int(k.step) < 0:
                raise IndexError("a spatial slice a:b:c needs its count c (read as linspace(a, b, c))")
            a = lo if k.start is None else float(k.start)
            b = hi if k.stop is None else float(k.stop)
            coords.append(torch.linspace(a, b, int(k.step), dtype=torch.float64).to(torch.float32))
            scalar.append(False)
        elif isinstance(k, (int, float)):
            coords.append(torch.tensor(float(k), dtype=torch.float32))
            scalar.append(True)
        else:
            t = torch.as_tensor(k).detach().to("cpu", torch.float32)
            if t.dim() > 1:
                raise IndexError("spatial entries are numbers, one-dimensional sequences or slices")
            coords.append(t)
            scalar.append(t.dim() == 0)
    return chan, coords, scalar


def point_shape(coords: List[torch.Tensor]) -> Tuple[int, ...]:
    """Broadcast shape of the spatial entries of a point query."""
    return tuple(torch.broadcast_shapes(*[c.shape for c in coords]))


def grid_shape(coords: List[torch.Tensor]) -> Tuple[int, ...]:
    """Meshgrid shape of the spatial entries of a volume query (scalars become length 1)."""
    return tuple(int(c.numel()) for c in coords)


def select_channels(out: torch.Tensor, chan):
    if chan is Ellipsis:
        return out
    if isinstance(chan, (int, slice)):
        return out[chan]
    return out[torch.as_tensor(chan, dtype=torch.long, device=out.device)]


class _Query:
    def __init__(self, exp: "Expansion", what: str, vol: bool):
        self._exp, self._what, self._vol = exp, what, vol

    @property
    def vol(self) -> "_Query":
        return _Query(self._exp, self._what, True)

    def __getitem__(self, key):
        return self._exp._query(key, self._what, self._vol)


class Expansion:
    """The field of sources (p, w) held in a plan, indexed at continuous positions."""

    def __init__(self, plan, serial: int):
        self.plan, self._serial = plan, serial

    @property
    def shape(self) -> Tuple[int, ...]:
        return (self.plan.channels,)

    @property
    def vol(self) -> _Query:
        return _Query(self, "value", True)

    @property
    def partials(self) -> _Query:
        return _Query(self, "partials", False)

    @property
    def partials2(self) -> _Query:
        return _Query(self, "partials2", False)

    def __getitem__(self, key):
        return self._query(key, "value", False)

    def _check(self):
        if self.plan._serial != self._serial or self.plan._h is None:
            raise RuntimeError("this expansion has been replaced: its plan ran another transform since")

    def _query(self, key, what: str, vol: bool):
        self._check()
        pl = self.plan
        D, C, K = pl.dim, pl.channels, WIDTH[what](pl.dim)
        chan, coords, _ = parse_key(key, D, pl.lo, pl.hi)
        dev = pl.device
        stream = pl._stream()
        if vol:
            shape = grid_shape(coords)
            axes = [c.reshape(-1).to(dev).contiguous() for c in coords]
            out = torch.empty((C,) + shape + (K,), device=dev, dtype=torch.float32)
            capi.evaluate_grid(pl._h, stream, [a.data_ptr() if a.numel() else 0 for a in axes],
                               [int(a.numel()) for a in axes], what, out.data_ptr() if out.numel() else 0)
        else:
            shape = point_shape(coords)
            pts = torch.stack([c.expand(shape).reshape(-1) for c in coords], dim=1).to(dev).contiguous()
            M = pts.shape[0]
            out = torch.empty((C, M, K), device=dev, dtype=torch.float32)
            step = max(pl.max_queries, 1)
            for m0 in range(0, M, step):
                m1 = min(M, m0 + step)
                part = out if (m0 == 0 and m1 == M) else torch.empty((C, m1 - m0, K), device=dev, dtype=torch.float32)
                capi.evaluate(pl._h, stream, pts[m0:m1].data_ptr(), m1 - m0, what, part.data_ptr())
                if part is not out:
                    out[:, m0:m1] = part
            out = out.reshape((C,) + shape + (K,))
        if what == "value":
            out = out[..., 0]
        return select_channels(out, chan)
