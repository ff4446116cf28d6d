"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerance for the FP32 path: relative L2 error <= 1e-5 against the oracle, and every element
within 1e-4 of the largest output magnitude (FP32 arithmetic, unit roundoff 6e-8, summed over
at most a few thousand terms per output with cancellation factors below 5).
"""
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
    assert got.shape == ref.shape, what
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


def make_plan(dim, grid, order, sigma, N, M, **kw):
    from paper_2111_00110_gb300.transform import Plan
    kw.setdefault("m2l", "fp32")
    return Plan(dim, grid, order, sigma, max_sources=max(N, 1), max_queries=max(M, 1), **kw)


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in arrs]


def run_forward(plan, p, w, q):
    P_, W_, Q_ = to_dev(p, w, q)
    y = plan.forward(P_, W_, Q_)
    torch.cuda.synchronize()
    plan.check()
    return y.cpu().numpy()


def run_backward(plan, p, w, q, ybar):
    P_, W_, Q_, YB = to_dev(p, w, q, ybar)
    wbar, pbar = plan.backward(P_, W_, Q_, YB)
    torch.cuda.synchronize()
    plan.check()
    return wbar.cpu().numpy(), pbar.cpu().numpy()


def odesc(dim, grid, order, sigma, **kw):
    return oracle.OracleDesc(dim=dim, grid=grid, order=order, sigma=sigma, **kw)


def f64(*a):
    return [np.asarray(x, dtype=np.float64) for x in a]


# ------------------------------------------------------------------------------ forward

def test_uniform2d_forward(lib):
    """2D, N = M = 4096, sigma 0.05, 32x32, order 4 (the CPU-checkable workload)."""
    wl = workloads.uniform2d()
    plan = make_plan(2, wl.grid, wl.order, wl.sigma, wl.N, wl.M)
    y = run_forward(plan, wl.p, wl.w, wl.q)
    yo = oracle.forward(odesc(2, wl.grid, wl.order, wl.sigma), *f64(wl.p, wl.w, wl.q))
    assert_close(y, yo, what="uniform2d")
    # and the truncation error against the exact sum is the oracle's (about 1.1e-2)
    yd = oracle.direct(odesc(2, wl.grid, wl.order, wl.sigma), *f64(wl.p, wl.w, wl.q))
    assert rel_l2(y, yd) <= 2e-2


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6, 7, 8])
def test_every_order(lib, dim, order):
    grid = 16 if dim == 3 else 32
    wl = workloads.uniform(100 + 10 * dim + order, dim, 3001, 2503, grid, order, 0.06)
    plan = make_plan(dim, grid, order, wl.sigma, wl.N, wl.M)
    y = run_forward(plan, wl.p, wl.w, wl.q)
    yo = oracle.forward(odesc(dim, grid, order, wl.sigma), *f64(wl.p, wl.w, wl.q))
    assert_close(y, yo, what=f"D{dim} rho{order}")


@pytest.mark.parametrize("dim,grid", [(2, 4), (2, 8), (3, 4), (3, 8), (2, 128), (3, 32)])
def test_grid_sizes(lib, dim, grid):
    sigma = 2.0 / grid
    wl = workloads.uniform(7 + grid, dim, 2000, 1500, grid, 4, sigma)
    plan = make_plan(dim, grid, 4, sigma, wl.N, wl.M)
    y = run_forward(plan, wl.p, wl.w, wl.q)
    yo = oracle.forward(odesc(dim, grid, 4, sigma), *f64(wl.p, wl.w, wl.q))
    assert_close(y, yo, what=f"D{dim} n{grid}")


@pytest.mark.parametrize("dim,grid,order,m2l", [(3, 4, 4, "fp32"), (3, 8, 6, "separable"), (2, 8, 8, "fp32"),
                                                (3, 8, 8, "separable")])
def test_dense_cells(lib, dim, grid, order, m2l):
    """Many points per finest cell (hundreds to a few thousand, well past the 32 one P2M thread
    takes; the rest go through the overflow kernel's atomics), clustered so that a few cells hold
    most of them; forward and backward against the oracle.  (The FP32 bar holds for sums of a few
    thousand weights of random sign per coefficient: sqrt(n) times the unit roundoff is 4e-6 at
    n = 4000.)"""
    rng = np.random.default_rng(40 + dim + grid + order)
    N, M = 12000, 9000
    centre = rng.uniform(0.3, 0.7, size=dim)
    p = np.clip(centre + 0.05 * rng.standard_normal((N, dim)), 0.0, 0.999).astype(np.float32)
    p[: N // 3] = rng.random((N // 3, dim)).astype(np.float32)
    w = rng.standard_normal(N).astype(np.float32)
    q = np.clip(centre + 0.08 * rng.standard_normal((M, dim)), 0.0, 0.999).astype(np.float32)
    sigma = 1.5 / grid
    plan = make_plan(dim, grid, order, sigma, N, M, m2l=m2l)
    y = run_forward(plan, p, w, q)
    d = odesc(dim, grid, order, sigma)
    assert_close(y, oracle.forward(d, *f64(p, w, q)), what=f"dense forward D{dim} n{grid} rho{order}")
    ybar = rng.standard_normal(M).astype(np.float32)
    wbar, pbar = run_backward(plan, p, w, q, ybar)
    wo, po = oracle.backward(d, *f64(p, w, q, ybar))
    assert_close(wbar, wo, what="dense wbar")
    assert_close(pbar, po, what="dense pbar")


def test_dense_and_sparse_calls_alternate(lib):
    """One plan, calls whose P2M needs the overflow list (dense cells) alternating with calls that
    leave it empty: the list's counters are cleared between calls, so every result matches the
    oracle."""
    rng = np.random.default_rng(77)
    dim, grid, order, sigma, N, M = 3, 8, 5, 0.2, 8000, 3000
    dense = np.clip(0.5 + 0.04 * rng.standard_normal((N, dim)), 0.0, 0.999).astype(np.float32)
    sparse = rng.random((N, dim)).astype(np.float32)
    w = rng.standard_normal(N).astype(np.float32)
    q = rng.random((M, dim)).astype(np.float32)
    plan = make_plan(dim, grid, order, sigma, N, M, m2l="separable")
    d = odesc(dim, grid, order, sigma)
    for p in (dense, sparse, dense, sparse):
        y = run_forward(plan, p, w, q)
        assert_close(y, oracle.forward(d, *f64(p, w, q)), what="alternating forward")
    ybar = rng.standard_normal(M).astype(np.float32)
    wbar, _ = run_backward(plan, dense, w, q, ybar)
    assert_close(wbar, oracle.backward(d, *f64(dense, w, q, ybar))[0], what="alternating wbar")


@pytest.mark.parametrize("dim", [2, 3])
def test_polynomial_kernel_is_exact(lib, dim):
    """For a polynomial psi of degree <= rho the series equals the direct sum of Eq. 1."""
    mis = oracle.multi_indices(dim, 4)
    coef = np.zeros(len(mis))
    for i, m in enumerate(mis):
        if sum(m) in (0, 2, 4) and all(e % 2 == 0 for e in m):
            coef[i] = 1.0 / (1 + i)
    grid = 16
    wl = workloads.uniform(55 + dim, dim, 1500, 1200, grid, 4, 0.1)
    plan = make_plan(dim, grid, 4, 0.1, wl.N, wl.M, kernel="poly", poly_coef=coef)
    y = run_forward(plan, wl.p, wl.w, wl.q)
    d = odesc(dim, grid, 4, 0.1, kernel="poly", poly_coef=coef)
    yd = oracle.direct(d, *f64(wl.p, wl.w, wl.q))
    assert_close(y, yd, rel=2e-5, elem=2e-4, what="poly")


def test_clustered_sources_and_empty_cells(lib):
    """All sources in a few cells (long segments), most cells empty."""
    rng = np.random.default_rng(77)
    p = (0.3 + 0.01 * rng.standard_normal((4000, 3))).clip(0, 0.999)
    p[:1000] = 0.8 + 0.001 * rng.random((1000, 3))
    w = rng.standard_normal(4000)
    q = rng.random((3000, 3))
    plan = make_plan(3, 16, 5, 0.05, 4000, 3000)
    y = run_forward(plan, p, w, q)
    yo = oracle.forward(odesc(3, 16, 5, 0.05), *f64(p.astype(np.float32), w.astype(np.float32),
                                                  q.astype(np.float32)))
    assert_close(y, yo, what="clustered")


def test_points_on_faces_and_outside_are_clamped(lib):
    """Coordinates on cell faces, at hi and outside [lo, hi) bin by the FP32 rule on both sides."""
    rng = np.random.default_rng(5)
    grid = 16
    faces = rng.integers(0, grid + 1, size=(500, 3)) / grid
    outside = rng.uniform(-0.2, 1.2, size=(300, 3))
    p = np.concatenate([faces, outside, rng.random((700, 3))]).astype(np.float32)
    w = rng.standard_normal(p.shape[0]).astype(np.float32)
    q = np.concatenate([rng.random((600, 3)), faces[:200]]).astype(np.float32)
    plan = make_plan(3, grid, 3, 0.08, p.shape[0], q.shape[0])
    y = run_forward(plan, p, w, q)
    yo = oracle.forward(odesc(3, grid, 3, 0.08), *f64(p, w, q))
    assert_close(y, yo, what="faces")


def test_check_domain_reports_points_outside(lib):
    from paper_2111_00110_gb300 import capi
    p = np.array([[0.5, 0.5, 0.5], [1.5, 0.2, 0.2]], dtype=np.float32)
    w = np.ones(2, dtype=np.float32)
    q = np.array([[0.1, 0.2, 0.3]], dtype=np.float32)
    plan = make_plan(3, 8, 2, 0.1, 2, 1, check_domain=True)
    with pytest.raises(capi.FC2T2Error) as e:
        run_forward(plan, p, w, q)
    assert e.value.status == 4
    # inside points pass
    y = run_forward(plan, p[:1], w[:1], q)
    assert np.isfinite(y).all()


def test_empty_inputs(lib):
    plan = make_plan(3, 8, 3, 0.1, 10, 10)
    rng = np.random.default_rng(1)
    p, w, q = rng.random((10, 3)), rng.standard_normal(10), rng.random((10, 3))
    y = run_forward(plan, p[:0], w[:0], q)
    assert np.all(y == 0.0)
    assert run_forward(plan, p, w, q[:0]).shape == (0,)
    wbar, pbar = run_backward(plan, p, w, q[:0], np.zeros(0))
    assert np.all(wbar == 0.0) and np.all(pbar == 0.0)


def test_sizes_beyond_the_plan_are_rejected(lib):
    from paper_2111_00110_gb300 import capi
    plan = make_plan(2, 8, 2, 0.1, 10, 10)
    rng = np.random.default_rng(2)
    with pytest.raises(capi.FC2T2Error) as e:
        run_forward(plan, rng.random((11, 2)), rng.random(11), rng.random((5, 2)))
    assert e.value.status == 1


def test_repeated_calls_are_consistent(lib):
    wl = workloads.uniform(9, 3, 5000, 5000, 16, 4, 0.05)
    plan = make_plan(3, 16, 4, 0.05, wl.N, wl.M)
    y1 = run_forward(plan, wl.p, wl.w, wl.q)
    y2 = run_forward(plan, wl.p, wl.w, wl.q)
    assert rel_l2(y1, y2) <= 1e-6


# ----------------------------------------------------------------------------- backward

@pytest.mark.parametrize("dim,grid,order", [(2, 32, 4), (3, 16, 4), (3, 16, 6), (3, 8, 8)])
def test_backward_small(lib, dim, grid, order):
    wl = workloads.uniform(300 + grid + order, dim, 2100, 1900, grid, order, 0.06)
    ybar = wl.ybar()
    plan = make_plan(dim, grid, order, wl.sigma, wl.N, wl.M)
    wbar, pbar = run_backward(plan, wl.p, wl.w, wl.q, ybar)
    wo, po = oracle.backward(odesc(dim, grid, order, wl.sigma), *f64(wl.p, wl.w, wl.q, ybar))
    assert_close(wbar, wo, what="wbar")
    assert_close(pbar, po, what="pbar")


def test_autograd_function_matches_backward(lib):
    from paper_2111_00110_gb300.transform import fc2t2
    wl = workloads.uniform(31, 3, 3000, 2000, 16, 4, 0.05)
    plan = make_plan(3, 16, 4, 0.05, wl.N, wl.M)
    P_, W_, Q_ = to_dev(wl.p, wl.w, wl.q)
    P_.requires_grad_(True)
    W_.requires_grad_(True)
    y = fc2t2(P_, W_, Q_, plan)
    loss = (y * y).sum()
    loss.backward()
    torch.cuda.synchronize()
    yo = oracle.forward(odesc(3, 16, 4, 0.05), *f64(wl.p, wl.w, wl.q))
    wo, po = oracle.backward(odesc(3, 16, 4, 0.05), *f64(wl.p, wl.w, wl.q), 2.0 * yo)
    assert_close(W_.grad.cpu().numpy(), wo, what="autograd wbar")
    assert_close(P_.grad.cpu().numpy(), po, what="autograd pbar")


# ------------------------------------------------------------------------ full size

@pytest.mark.slow
def test_uniform3d_full_size_forward_backward(lib):
    """3D, N = M = 2^20, sigma 0.02, 64^3, order 6: forward and backward of L = sum y^2,
    against the oracle's full FP64 transform."""
    wl = workloads.uniform3d()
    plan = make_plan(3, wl.grid, wl.order, wl.sigma, wl.N, wl.M)
    y = run_forward(plan, wl.p, wl.w, wl.q)
    d = odesc(3, wl.grid, wl.order, wl.sigma)
    yo = oracle.forward(d, *f64(wl.p, wl.w, wl.q))
    assert_close(y, yo, what="uniform3d forward")
    ybar = 2.0 * y.astype(np.float32)
    wbar, pbar = run_backward(plan, wl.p, wl.w, wl.q, ybar)
    rng = np.random.default_rng(2024)
    sel = rng.choice(wl.N, size=4096, replace=False)
    wo, po = oracle.backward(d, *f64(wl.p, wl.w, wl.q, ybar), sel=sel)
    assert_close(wbar[sel], wo, what="uniform3d wbar")
    assert_close(pbar[sel], po, what="uniform3d pbar")


# ----------------------------------------------------------------- tensor-core M2L (3D)

# rel-L2 bars: TF32 x 3 is FP32-accurate; single-pass TF32 / BF16 are the mixed forms
TC_BARS = {"tf32x3": (1e-5, 1e-4), "bf16x3": (1e-5, 1e-4), "tf32": (1e-3, 1e-2), "bf16": (1e-2, 5e-2)}


# Target parity classes one tensor-core CTA accumulates, by (mode, order); 0 = the M2L stays on the
# CUDA cores (the operands do not fit shared memory).  Orders <= 5 share each moment view among
# four classes, 6 (and 7 for BF16) among two.
TC_CLASSES = {
    "bf16": {1: 4, 2: 4, 3: 4, 4: 4, 5: 4, 6: 2, 7: 2, 8: 1},
    "bf16x3": {1: 4, 2: 4, 3: 4, 4: 4, 5: 4, 6: 2, 7: 1, 8: 1},
    "tf32": {1: 4, 2: 4, 3: 4, 4: 4, 5: 4, 6: 2, 7: 1, 8: 1},
    "tf32x3": {1: 4, 2: 4, 3: 4, 4: 4, 5: 2, 6: 1, 7: 0, 8: 0},
}


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x3", "tf32", "bf16"])
@pytest.mark.parametrize("grid,order", [(16, 4), (16, 6), (32, 6), (8, 3), (8, 1), (16, 2), (16, 5), (16, 7),
                                        (16, 8)])
def test_tensor_core_m2l_forward(lib, mode, grid, order):
    wl = workloads.uniform(500 + grid + order, 3, 6000, 5000, grid, order, 1.3 / grid)
    plan = make_plan(3, grid, order, wl.sigma, wl.N, wl.M, m2l=mode)
    info = plan.info()
    assert info["m2l_classes_per_cta"] == TC_CLASSES[mode][order]
    assert info["m2l_tensor_cores"] == (1 if TC_CLASSES[mode][order] else 0)
    y = run_forward(plan, wl.p, wl.w, wl.q)
    yo = oracle.forward(odesc(3, grid, order, wl.sigma), *f64(wl.p, wl.w, wl.q))
    rel, elem = TC_BARS[mode]
    print(f"{mode} n{grid} rho{order}: rel-L2 {rel_l2(y, yo):.3e}")
    assert_close(y, yo, rel=rel, elem=elem, what=f"{mode} n{grid} rho{order}")


# ----------------------------------------------------------------- separable M2L (3D Gaussian)

@pytest.mark.parametrize("grid,order", [(16, 4), (16, 6), (32, 6), (8, 3), (8, 1), (16, 2), (16, 5), (16, 7),
                                        (16, 8), (4, 4), (64, 4)])
def test_separable_m2l_forward(lib, grid, order):
    wl = workloads.uniform(900 + grid + order, 3, 6000, 5000, grid, order, 1.3 / grid)
    plan = make_plan(3, grid, order, wl.sigma, wl.N, wl.M, m2l="separable")
    assert plan.info()["m2l_tensor_cores"] == 0
    y = run_forward(plan, wl.p, wl.w, wl.q)
    yo = oracle.forward(odesc(3, grid, order, wl.sigma), *f64(wl.p, wl.w, wl.q))
    print(f"separable n{grid} rho{order}: rel-L2 {rel_l2(y, yo):.3e}")
    assert_close(y, yo, what=f"separable n{grid} rho{order}")


def test_separable_m2l_backward(lib):
    wl = workloads.uniform(778, 3, 4000, 3500, 16, 6, 0.08)
    ybar = wl.ybar()
    plan = make_plan(3, 16, 6, wl.sigma, wl.N, wl.M, m2l="separable")
    wbar, pbar = run_backward(plan, wl.p, wl.w, wl.q, ybar)
    wo, po = oracle.backward(odesc(3, 16, 6, wl.sigma), *f64(wl.p, wl.w, wl.q, ybar))
    assert_close(wbar, wo, what="separable wbar")
    assert_close(pbar, po, what="separable pbar")


def test_default_plan_form(lib):
    """A plan made without an M2L form: the separable passes for the 3D Gaussian, plain FP32 for
    the 2D Gaussian; both against the oracle."""
    from paper_2111_00110_gb300.transform import Plan
    for dim, grid, order in ((3, 16, 6), (2, 32, 4)):
        wl = workloads.uniform(779 + dim, dim, 3000, 2500, grid, order, 1.3 / grid)
        plan = Plan(dim, grid, order, wl.sigma, max_sources=wl.N, max_queries=wl.M)
        assert plan.m2l == ("separable" if dim == 3 else "fp32")
        y = run_forward(plan, wl.p, wl.w, wl.q)
        yo = oracle.forward(odesc(dim, grid, order, wl.sigma), *f64(wl.p, wl.w, wl.q))
        assert_close(y, yo, what=f"default plan, {dim}D")


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x3", "tf32"])
def test_tensor_core_m2l_backward(lib, mode):
    wl = workloads.uniform(777, 3, 4000, 3500, 16, 6, 0.08)
    ybar = wl.ybar()
    plan = make_plan(3, 16, 6, wl.sigma, wl.N, wl.M, m2l=mode)
    wbar, pbar = run_backward(plan, wl.p, wl.w, wl.q, ybar)
    wo, po = oracle.backward(odesc(3, 16, 6, wl.sigma), *f64(wl.p, wl.w, wl.q, ybar))
    rel, elem = TC_BARS[mode]
    assert_close(wbar, wo, rel=rel, elem=elem, what=f"{mode} wbar")
    assert_close(pbar, po, rel=rel, elem=elem, what=f"{mode} pbar")


# ------------------------------------------------------------------------ query gradient

@pytest.mark.parametrize("m2l", ["fp32", "separable", "bf16x3"])
def test_query_gradient(lib, m2l):
    """qbar = ybar * grad y(q) through fc2t2_backward_q against the oracle (3D, 16^3, order 6)."""
    wl = workloads.uniform(779, 3, 5000, 4000, 16, 6, 0.08)
    ybar = wl.ybar()
    plan = make_plan(3, 16, 6, wl.sigma, wl.N, wl.M, m2l=m2l)
    P_, W_, Q_, YB = to_dev(wl.p, wl.w, wl.q, ybar)
    qbar = plan.backward_q(P_, W_, Q_, YB)
    torch.cuda.synchronize()
    plan.check()
    qo = oracle.backward_q(odesc(3, 16, 6, wl.sigma), *f64(wl.p, wl.w, wl.q, ybar))
    assert_close(qbar.cpu().numpy(), qo, what=f"qbar ({m2l})")


def test_autograd_query_gradient(lib):
    """The autograd layer returns qbar when q requires a gradient (and pbar, wbar as before)."""
    from paper_2111_00110_gb300.transform import fc2t2
    wl = workloads.uniform(780, 2, 3000, 2500, 32, 4, 0.05)
    plan = make_plan(2, 32, 4, wl.sigma, wl.N, wl.M)
    P_, W_, Q_ = [t.requires_grad_(True) for t in to_dev(wl.p, wl.w, wl.q)]
    y = fc2t2(P_, W_, Q_, plan)
    (y * y).sum().backward()
    torch.cuda.synchronize()
    d = odesc(2, 32, 4, wl.sigma)
    yo = oracle.forward(d, *f64(wl.p, wl.w, wl.q))
    qo = oracle.backward_q(d, *f64(wl.p, wl.w, wl.q, 2.0 * y.detach().cpu().numpy()))
    assert_close(Q_.grad.cpu().numpy(), qo, what="autograd qbar")
    assert rel_l2(y.detach().cpu().numpy(), yo) <= 1e-5


# ------------------------------------------------------------------------ sort reuse

def test_backward_reuse_matches_backward(lib):
    """fc2t2_backward_reuse after a forward on the same arrays equals fc2t2_backward (to the
    within-cell summation order of the sorts); after a forward on other arrays it falls back to
    sorting again, and still equals it."""
    wl = workloads.uniform(781, 3, 6000, 5000, 16, 6, 0.08)
    other = workloads.uniform(782, 3, 6000, 5000, 16, 6, 0.08)
    ybar = wl.ybar()
    for m2l in ("separable", "bf16x3"):
        plan = make_plan(3, 16, 6, wl.sigma, wl.N, wl.M, m2l=m2l)
        P_, W_, Q_, YB = to_dev(wl.p, wl.w, wl.q, ybar)
        P2, W2, Q2 = to_dev(other.p, other.w, other.q)
        wb0, pb0 = plan.backward(P_, W_, Q_, YB)
        plan.forward(P_, W_, Q_)
        wb1, pb1 = plan.backward(P_, W_, Q_, YB, reuse_forward=True)
        plan.forward(P2, W2, Q2)                       # the plan now holds other sorts
        wb2, pb2 = plan.backward(P_, W_, Q_, YB, reuse_forward=True)
        torch.cuda.synchronize()
        plan.check()
        for wb, pb in ((wb1, pb1), (wb2, pb2)):
            assert rel_l2(wb.cpu().numpy(), wb0.cpu().numpy()) <= 1e-6
            assert rel_l2(pb.cpu().numpy(), pb0.cpu().numpy()) <= 1e-6


# ----------------------------------------------- L2P with and without the finest L2L

@pytest.mark.parametrize("dim,order,m2l", [(3, 4, "fp32"), (3, 6, "separable"), (2, 5, "fp32"), (3, 8, "bf16x3")])
def test_l2p_without_finest_l2l_matches_l2l(lib, dim, order, m2l):
    """Up to a few targets per finest cell the transform skips the finest level's L2L (an exact
    re-centring) and evaluates the finest level's own M2L series plus level 1's local series at the
    targets; with more it runs L2L.  The same points evaluated both ways (the first targets of a
    larger call) agree, and both match the oracle."""
    grid = 8 if dim == 3 else 16
    G0 = grid ** dim
    per_cell = 32 if order >= 7 else 8
    few, many = G0 * per_cell // 2, G0 * per_cell + 1000       # below / above the switch
    wl = workloads.uniform(960 + dim + order, dim, 1500, many, grid, order, 0.15)
    plan = make_plan(dim, grid, order, wl.sigma, max(wl.N, many), many, m2l=m2l)
    P_, W_, Q_ = to_dev(wl.p, wl.w, wl.q)
    y_many = plan.forward(P_, W_, Q_)
    y_few = plan.forward(P_, W_, Q_[:few].contiguous())
    torch.cuda.synchronize()
    plan.check()
    assert rel_l2(y_few.cpu().numpy(), y_many[:few].cpu().numpy()) <= 1e-6
    d = odesc(dim, grid, order, wl.sigma)
    yo = oracle.forward(d, *f64(wl.p, wl.w, wl.q))
    bar = TC_BARS[m2l] if m2l in TC_BARS else (REL_L2, ELEM)
    assert_close(y_many.cpu().numpy(), yo, rel=bar[0], elem=bar[1], what="with L2L")
    assert_close(y_few.cpu().numpy(), yo[:few], rel=bar[0], elem=bar[1], what="from levels")
    # backward: the targets are the sources p (few of them here, so from levels), and the query
    # gradient at few / many queries
    ybar = np.random.default_rng(5).standard_normal(many).astype(np.float32)
    YB = to_dev(ybar)[0]
    wbar, pbar = plan.backward(P_, W_, Q_, YB)
    qb_many = plan.backward_q(P_, W_, Q_, YB)
    qb_few = plan.backward_q(P_, W_, Q_[:few].contiguous(), YB[:few].contiguous())
    torch.cuda.synchronize()
    wo, po = oracle.backward(d, *f64(wl.p, wl.w, wl.q, ybar))
    assert_close(wbar.cpu().numpy(), wo, rel=bar[0], elem=bar[1], what="wbar from levels")
    assert_close(pbar.cpu().numpy(), po, rel=bar[0], elem=bar[1], what="pbar from levels")
    assert rel_l2(qb_few.cpu().numpy(), qb_many[:few].cpu().numpy()) <= 1e-5


# ------------------------------------------------------- least-squares fitted operators

@pytest.mark.parametrize("dim,grid,order,m2l", [(3, 8, 4, "fp32"), (3, 16, 6, "bf16x3"), (3, 16, 5, "tf32x3"),
                                                (2, 16, 4, "fp32"), (3, 8, 6, "tf32"), (3, 16, 4, "occupied"),
                                                (2, 16, 6, "occupied")])
def test_fitted_operators(lib, dim, grid, order, m2l):
    """M2L with least-squares fitted coefficients (Sec. 3.1) against the oracle's own fit, forward
    and backward; with cells wider than the kernel the fitted transform is closer to the exact sum
    than the Taylor one."""
    sigma = 0.8 / grid                  # h / sigma = 1.25
    wl = workloads.uniform(990 + dim + order, dim, 2500, 2000, grid, order, sigma)
    ybar = wl.ybar()
    plan = make_plan(dim, grid, order, sigma, wl.N, wl.M, m2l=m2l, fit=True)
    y = run_forward(plan, wl.p, wl.w, wl.q)
    wbar, pbar = run_backward(plan, wl.p, wl.w, wl.q, ybar)
    d = odesc(dim, grid, order, sigma, fit=True)
    yo = oracle.forward(d, *f64(wl.p, wl.w, wl.q))
    wo, po = oracle.backward(d, *f64(wl.p, wl.w, wl.q, ybar))
    bar = TC_BARS[m2l] if m2l in TC_BARS else (REL_L2, ELEM)
    assert_close(y, yo, rel=bar[0], elem=bar[1], what=f"fitted forward ({m2l})")
    assert_close(wbar, wo, rel=bar[0], elem=bar[1], what=f"fitted wbar ({m2l})")
    assert_close(pbar, po, rel=bar[0], elem=bar[1], what=f"fitted pbar ({m2l})")
    if m2l == "fp32":
        exact = oracle.direct(d, *f64(wl.p, wl.w, wl.q))
        taylor = run_forward(make_plan(dim, grid, order, sigma, wl.N, wl.M), wl.p, wl.w, wl.q)
        assert rel_l2(y, exact) < 0.6 * rel_l2(taylor, exact)
