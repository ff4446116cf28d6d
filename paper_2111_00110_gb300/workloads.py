"""Seeded synthetic workloads for the FC2T2 transform.

This module only draws random inputs; it holds none of the transform's arithmetic and is
shared by the tests, the benchmark and the smoke check.  Every generator draws in float64
with ``numpy.random.default_rng(seed)`` in the order (p, w, q) and returns float32 arrays
(the precision the transform consumes), plus the transform parameters.

The paper's own workloads (signed-distance fitting with 8m sources / 10m targets, and
radiance-field rays; Sec. 4.3 and Sec. 6.3) need meshes and image datasets that are not
available; these synthetic sets reproduce their shapes and sizes:

* ``uniform2d``   -- 2D, N = M = 4096 uniform in [0,1)^2, w ~ N(0,1), sigma 0.05,
                     32x32 grid, order 4, seed 0 (checkable against the direct sum).
* ``uniform3d``   -- 3D, N = M = 2^20 uniform in [0,1)^3, w ~ N(0,1), sigma 0.02,
                     64^3 grid, order 6, seed 2 (forward + backward).
* ``sphere_rays`` -- 3D, N = 2^18 sources near a sphere (radius 0.35 + N(0, 0.01) about
                     the cube centre), w ~ U(0,1); queries are 512x512 pinhole rays with
                     128 stratified samples each inside [0,1]^3 (33.5M queries), sigma 0.01,
                     64^3 grid, order 8, seed 3.
* ``mixture``     -- 3D instance i of a batch: N_i = M_i log-uniform in [1024, 262144],
                     8 isotropic Gaussian clusters (std 0.05), sigma 0.02, seed 1000 + i.
* ``fit_large``   -- 3D, N = M = 2^24, sources from 64 anisotropic Gaussians, queries
                     uniform, sigma 0.005, 128^3 grid, order 8, seeds 5001/5002.

``scaled(...)`` variants keep a workload's distributions but shrink N, M and the grid so
the oracle finishes in seconds.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class Workload:
    name: str
    dim: int
    grid: int
    order: int
    sigma: float
    p: np.ndarray            # [N, dim] float32
    w: np.ndarray            # [N] float32
    q: np.ndarray            # [M, dim] float32
    lo: float = 0.0
    hi: float = 1.0
    seed: int = 0
    ybar_seed: Optional[int] = None

    @property
    def N(self) -> int:
        return int(self.p.shape[0])

    @property
    def M(self) -> int:
        return int(self.q.shape[0])

    def ybar(self) -> np.ndarray:
        """A seeded cotangent for backward-only checks, N(0,1) float32 of length M."""
        rng = np.random.default_rng(self.seed + 7919 if self.ybar_seed is None else self.ybar_seed)
        return rng.standard_normal(self.M).astype(np.float32)

    def channel_weights(self, C: int) -> np.ndarray:
        """C channels of weights [C, N] (float32): channel 0 is ``w``, the others seeded N(0,1)."""
        rng = np.random.default_rng(self.seed + 104729)
        out = np.empty((C, self.N), dtype=np.float32)
        out[0] = self.w
        if C > 1:
            out[1:] = rng.standard_normal((C - 1, self.N)).astype(np.float32)
        return out

    def channel_ybar(self, C: int) -> np.ndarray:
        """C channels of seeded cotangents [C, M] (float32), channel 0 equal to ``ybar()``."""
        rng = np.random.default_rng(self.seed + 130363)
        out = np.empty((C, self.M), dtype=np.float32)
        out[0] = self.ybar()
        if C > 1:
            out[1:] = rng.standard_normal((C - 1, self.M)).astype(np.float32)
        return out


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def uniform(seed: int, dim: int, N: int, M: int, grid: int, order: int, sigma: float,
            name: str = "uniform") -> Workload:
    rng = np.random.default_rng(seed)
    p = rng.random((N, dim))
    w = rng.standard_normal(N)
    q = rng.random((M, dim))
    return Workload(name, dim, grid, order, sigma, _f32(p), _f32(w), _f32(q), seed=seed)


def uniform2d(N: int = 4096, M: int = 4096, grid: int = 32, order: int = 4,
              sigma: float = 0.05, seed: int = 0) -> Workload:
    """2D plain transform: 4096 uniform sources and queries, sigma 0.05, 32x32, order 4."""
    return uniform(seed, 2, N, M, grid, order, sigma, name="uniform2d")


def uniform3d(N: int = 1 << 20, M: int = 1 << 20, grid: int = 64, order: int = 6,
              sigma: float = 0.02, seed: int = 2) -> Workload:
    """3D forward+backward: 2^20 uniform sources and queries, sigma 0.02, 64^3, order 6."""
    return uniform(seed, 3, N, M, grid, order, sigma, name="uniform3d")


def _sphere_sources(rng, N: int):
    v = rng.standard_normal((N, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = 0.35 + 0.01 * rng.standard_normal((N, 1))
    p = 0.5 + r * v
    return np.clip(p, 0.0, np.nextafter(1.0, 0.0))


def pinhole_ray_samples(rng, width: int, height: int, samples: int) -> np.ndarray:
    """Stratified samples along pixel-centre rays of a pinhole camera at (0.5, 0.5, -1)
    looking along +z whose image exactly covers the z = 0 face of [0,1]^3 (vertical field
    of view 2 atan(0.5)); sample k of a ray is uniform in bin k of [t_in, t_out], the
    ray's slab intersection with the unit cube."""
    o = np.array([0.5, 0.5, -1.0])
    u = (np.arange(width) + 0.5) / width
    v = (np.arange(height) + 0.5) / height
    uu, vv = np.meshgrid(u, v, indexing="xy")
    # direction from the eye to the point (u, v, 0) on the z = 0 face
    d = np.stack([uu.ravel() - 0.5, vv.ravel() - 0.5, np.ones(uu.size)], axis=1)
    with np.errstate(divide="ignore"):
        inv = 1.0 / d
    t0 = (0.0 - o) * inv
    t1 = (1.0 - o) * inv
    tmin = np.minimum(t0, t1)
    tmax = np.maximum(t0, t1)
    t_in = np.max(tmin, axis=1)
    t_out = np.min(tmax, axis=1)
    R = d.shape[0]
    k = np.arange(samples)
    jitter = rng.random((R, samples))
    frac = (k[None, :] + jitter) / samples
    t = t_in[:, None] + frac * (t_out - t_in)[:, None]
    pts = o[None, None, :] + t[:, :, None] * d[:, None, :]
    return np.clip(pts.reshape(-1, 3), 0.0, np.nextafter(1.0, 0.0))


def pinhole_rays(width: int, height: int) -> np.ndarray:
    """Ray records [width * height, 8] (origin, direction, t_in, t_out) of the pixel-centre rays of
    the same pinhole camera as ``pinhole_ray_samples``: the ray through pixel (i, j) aims at the point
    ((i + 0.5) / width, (j + 0.5) / height, 0) of the cube's z = 0 face, and [t_in, t_out] is its
    slab intersection with the unit cube (float32)."""
    o = np.array([0.5, 0.5, -1.0])
    u = (np.arange(width) + 0.5) / width
    v = (np.arange(height) + 0.5) / height
    uu, vv = np.meshgrid(u, v, indexing="xy")
    d = np.stack([uu.ravel() - 0.5, vv.ravel() - 0.5, np.ones(uu.size)], axis=1)
    with np.errstate(divide="ignore"):
        inv = 1.0 / d
    t0 = (0.0 - o) * inv
    t1 = (1.0 - o) * inv
    t_in = np.max(np.minimum(t0, t1), axis=1)
    t_out = np.min(np.maximum(t0, t1), axis=1)
    out = np.concatenate([np.broadcast_to(o, d.shape), d, t_in[:, None], t_out[:, None]], axis=1)
    return _f32(out)


def sphere_rays(N: int = 1 << 18, width: int = 512, height: int = 512, samples: int = 128,
                grid: int = 64, order: int = 8, sigma: float = 0.01, seed: int = 3) -> Workload:
    """3D ray-query workload: sphere-surface sources, pinhole-ray stratified queries."""
    rng = np.random.default_rng(seed)
    p = _sphere_sources(rng, N)
    w = rng.random(N)
    q = pinhole_ray_samples(rng, width, height, samples)
    return Workload("sphere_rays", 3, grid, order, sigma, _f32(p), _f32(w), _f32(q), seed=seed)


def _mixture(rng, n: int, centres: np.ndarray, std: float) -> np.ndarray:
    out = np.empty((0, 3))
    while out.shape[0] < n:
        k = rng.integers(0, centres.shape[0], size=2 * n)
        x = centres[k] + std * rng.standard_normal((2 * n, 3))
        ok = np.all((x >= 0.0) & (x < 1.0), axis=1)
        out = np.concatenate([out, x[ok]], axis=0)
    return out[:n]


def mixture(i: int, grid: int = 64, order: int = 6, sigma: float = 0.02,
            n_override: Optional[int] = None) -> Workload:
    """Instance i of the batched workload: N_i = M_i log-uniform in [1024, 262144],
    8 isotropic clusters of std 0.05 with centres uniform in [0.15, 0.85]^3."""
    seed = 1000 + i
    rng = np.random.default_rng(seed)
    n = int(round(np.exp(rng.uniform(np.log(1024), np.log(262144)))))
    if n_override is not None:
        n = n_override
    centres = rng.uniform(0.15, 0.85, size=(8, 3))
    p = _mixture(rng, n, centres, 0.05)
    w = rng.standard_normal(n)
    q = _mixture(rng, n, centres, 0.05)
    return Workload(f"mixture{i}", 3, grid, order, sigma, _f32(p), _f32(w), _f32(q), seed=seed)


def fit_large(N: int = 1 << 24, M: int = 1 << 24, grid: int = 128, order: int = 8,
              sigma: float = 0.005, seed: int = 5001) -> Workload:
    """Large fitting workload: sources from 64 anisotropic Gaussians, uniform queries."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.1, 0.9, size=(64, 3))
    scales = rng.uniform(0.005, 0.05, size=(64, 3))
    rots = [np.linalg.qr(rng.standard_normal((3, 3)))[0] for _ in range(64)]
    out = np.empty((0, 3))
    while out.shape[0] < N:
        k = rng.integers(0, 64, size=N)
        z = rng.standard_normal((N, 3)) * scales[k]
        x = centres[k] + np.einsum("nij,nj->ni", np.stack(rots)[k], z)
        ok = np.all((x >= 0.0) & (x < 1.0), axis=1)
        out = np.concatenate([out, x[ok]], axis=0)
    p = out[:N]
    w = rng.standard_normal(N)
    q = rng.random((M, 3))
    return Workload("fit_large", 3, grid, order, sigma, _f32(p), _f32(w), _f32(q), seed=seed)


WORKLOADS = {
    "uniform2d": uniform2d,
    "uniform3d": uniform3d,
    "sphere_rays": sphere_rays,
    "mixture": mixture,
    "fit_large": fit_large,
}
