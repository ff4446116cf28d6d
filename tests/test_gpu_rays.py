"""GPU parity of the ray integrals (Sec. 6, the integral-implicit layer): integrals of the series
along rays (forward) and their adjoint (the rays inserted as sources, ray2M), against the FP64
oracle, which cuts the rays at the same faces but integrates each segment with the paper's
binomial line2poly / line2taylor formulas.

Tolerances: relative L2 <= 1e-5 and every element within 1e-4 of the largest magnitude (FP32
arithmetic; the adjoint's moments are summed with float atomics, in no fixed order)."""
import numpy as np
import pytest

import oracle
from paper_2111_00110_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL_L2 = 1e-5
ELEM = 1e-4


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_close(got, ref, rel=REL_L2, elem=ELEM, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    assert np.all(np.isfinite(got)), what
    scale = max(np.abs(ref).max(), 1e-30)
    err = rel_l2(got, ref)
    assert err <= rel, f"{what}: rel-L2 {err:.3e} > {rel:.1e}"
    worst = np.abs(got - ref).max() / scale
    assert worst <= elem, f"{what}: max element error {worst:.3e} of max |ref|"


@pytest.fixture(scope="module")
def lib():
    from paper_2111_00110_gb300 import build
    build.build()
    from paper_2111_00110_gb300 import capi
    return capi.load()


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in arrs]


def scene(seed, N, width, extra):
    """Sphere-surface sources and rays: a pinhole camera's pixel rays plus `extra` random rays
    (some starting outside the domain, some with zero length, some parallel to an axis)."""
    wl = workloads.sphere_rays(N=N, width=4, height=4, samples=1, seed=seed)
    cam = workloads.pinhole_rays(width, width)
    rng = np.random.default_rng(seed + 1)
    o = rng.random((extra, 3)) * 1.6 - 0.3
    d = rng.standard_normal((extra, 3))
    d[::7, 1] = 0.0                                   # parallel to the x-z plane
    t0 = -rng.random(extra)
    t1 = rng.random(extra) * 1.5
    t1[::11] = t0[::11]                               # zero length
    rand = np.concatenate([o, d, t0[:, None], t1[:, None]], axis=1).astype(np.float32)
    return wl.p, wl.w, np.concatenate([cam, rand], axis=0)


@pytest.mark.parametrize("grid,order,m2l", [(16, 4, "fp32"), (16, 6, "separable"), (8, 8, "fp32"),
                                            (32, 5, "separable"), (16, 6, "bf16x3"), (16, 6, "occupied")])
def test_ray_forward_and_adjoint(lib, grid, order, m2l):
    from paper_2111_00110_gb300.transform import Plan
    p, w, rays = scene(200 + order, 3000, 24, 300)
    R = rays.shape[0]
    ybar = np.random.default_rng(7).standard_normal(R).astype(np.float32)
    plan = Plan(3, grid, order, 0.08, m2l=m2l, max_sources=p.shape[0], max_queries=1)
    P_, W_, RAYS, YB = to_dev(p, w, rays, ybar)
    y = plan.ray_forward(P_, W_, RAYS)
    wbar, pbar = plan.ray_backward(P_, W_, RAYS, YB)
    torch.cuda.synchronize()
    plan.check()
    d = oracle.OracleDesc(dim=3, grid=grid, order=order, sigma=0.08)
    yo = oracle.ray_forward(d, p.astype(np.float64), w.astype(np.float64), rays.astype(np.float64))
    wo, po = oracle.ray_backward(d, p.astype(np.float64), w.astype(np.float64), rays.astype(np.float64),
                                 ybar.astype(np.float64))
    bar = (1e-5, 1e-4) if m2l != "bf16x3" else (2e-5, 2e-4)
    assert_close(y.cpu().numpy(), yo, *bar, what="ray integrals")
    assert_close(wbar.cpu().numpy(), wo, *bar, what="ray adjoint wbar")
    assert_close(pbar.cpu().numpy(), po, *bar, what="ray adjoint pbar")


def test_ray_channels_autograd(lib):
    """Channels and the autograd layer: L = sum y^2 over (C, R) ray integrals; the gradients equal
    the plan's adjoint and the oracle's, channel by channel (pbar summed)."""
    from paper_2111_00110_gb300.transform import Plan, fc2t2_rays
    C = 3
    p, w, rays = scene(230, 2000, 16, 100)
    wl = workloads.Workload("s", 3, 16, 6, 0.08, p, w, p[:1], seed=230)
    W = wl.channel_weights(C)
    plan = Plan(3, 16, 6, 0.08, m2l="separable", max_sources=p.shape[0], max_queries=1, channels=C)
    P_, W_, RAYS = to_dev(p, W, rays)
    P_.requires_grad_(True)
    W_.requires_grad_(True)
    y = fc2t2_rays(P_, W_, RAYS, plan)
    (y * y).sum().backward()
    torch.cuda.synchronize()
    assert y.shape == (C, rays.shape[0])
    d = oracle.OracleDesc(dim=3, grid=16, order=6, sigma=0.08)
    yb = 2.0 * y.detach().cpu().numpy().astype(np.float64)
    po = np.zeros(p.shape)
    for c in range(C):
        yo = oracle.ray_forward(d, p.astype(np.float64), W[c].astype(np.float64), rays.astype(np.float64))
        assert_close(y[c].detach().cpu().numpy(), yo, what=f"y[{c}]")
        wo, pc = oracle.ray_backward(d, p.astype(np.float64), W[c].astype(np.float64), rays.astype(np.float64), yb[c])
        assert_close(W_.grad[c].cpu().numpy(), wo, what=f"wbar[{c}]")
        po += pc
    assert_close(P_.grad.cpu().numpy(), po, what="pbar, 3 channels")


def test_ray_empty_and_unsupported(lib):
    from paper_2111_00110_gb300 import capi
    from paper_2111_00110_gb300.transform import Plan
    p, w, rays = scene(240, 500, 4, 10)
    plan = Plan(3, 8, 4, 0.1, m2l="fp32", max_sources=p.shape[0], max_queries=1)
    P_, W_, RAYS = to_dev(p, w, rays)
    assert plan.ray_forward(P_, W_, RAYS[:0].contiguous()).shape == (0,)
    y0 = plan.ray_forward(P_[:0].contiguous(), W_[:0].contiguous(), RAYS)
    wb, pb = plan.ray_backward(P_, W_, RAYS[:0].contiguous(), torch.zeros(0, device="cuda"))
    torch.cuda.synchronize()
    assert float(y0.abs().max()) == 0.0
    assert float(wb.abs().max()) == 0.0 and float(pb.abs().max()) == 0.0
    plan2 = Plan(2, 16, 4, 0.1, max_sources=10, max_queries=1)
    with pytest.raises(capi.FC2T2Error):
        plan2.ray_forward(torch.zeros(4, 2, device="cuda"), torch.zeros(4, device="cuda"), RAYS)
