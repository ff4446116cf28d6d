"""GPU parity of the channel dimension and of the accessor (Sec. 3, "How to use the
implementation?"): transforms of C weight channels over shared points, and the expansion's value,
first and second partials at points and on meshgrids, against the FP64 oracle.

Channel c of a call is the transform of w[c]; the gradients with respect to positions sum the
channels' contributions.  Tolerances as for the single-channel parity: relative L2 <= 1e-5 and
every element within 1e-4 of the largest output magnitude (FP32 arithmetic)."""
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


def make_plan(dim, grid, order, sigma, N, M, **kw):
    from paper_2111_00110_gb300.transform import Plan
    kw.setdefault("m2l", "fp32")
    return Plan(dim, grid, order, sigma, max_sources=max(N, 1), max_queries=max(M, 1), **kw)


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in arrs]


def odesc(dim, grid, order, sigma, **kw):
    return oracle.OracleDesc(dim=dim, grid=grid, order=order, sigma=sigma, **kw)


def f64(*a):
    return [np.asarray(x, dtype=np.float64) for x in a]


# ------------------------------------------------------------------------------- channels

@pytest.mark.parametrize("dim,grid,order,m2l", [(3, 16, 4, "fp32"), (3, 16, 6, "separable"), (2, 32, 4, "fp32"),
                                                (3, 16, 5, "bf16x3"), (3, 16, 6, "occupied"), (2, 32, 5, "occupied")])
def test_channels_forward_backward(lib, dim, grid, order, m2l):
    """y[c], wbar[c] per channel and pbar, qbar summed over channels against the oracle run per
    channel; each channel agrees with a one-channel plan's transform of its weights."""
    C = 3
    wl = workloads.uniform(900 + dim + order, dim, 3000, 2500, grid, order, 0.08)
    W = wl.channel_weights(C)
    YB = wl.channel_ybar(C)
    plan = make_plan(dim, grid, order, wl.sigma, wl.N, wl.M, m2l=m2l, channels=C)
    single = make_plan(dim, grid, order, wl.sigma, wl.N, wl.M, m2l=m2l)
    P_, W_, Q_, YB_ = to_dev(wl.p, W, wl.q, YB)
    y = plan.forward(P_, W_, Q_)
    wbar, pbar = plan.backward(P_, W_, Q_, YB_)
    qbar = plan.backward_q(P_, W_, Q_, YB_)
    ys = [single.forward(P_, W_[c].contiguous(), Q_) for c in range(C)]
    torch.cuda.synchronize()
    plan.check()
    assert y.shape == (C, wl.M) and wbar.shape == (C, wl.N) and pbar.shape == (wl.N, dim)
    for c in range(C):   # (equal up to the within-cell summation order of the two sorts)
        assert rel_l2(y[c].cpu().numpy(), ys[c].cpu().numpy()) <= 1e-6, f"channel {c} vs a one-channel plan"
    d = odesc(dim, grid, order, wl.sigma)
    p64, q64 = f64(wl.p, wl.q)
    po_sum = np.zeros((wl.N, dim))
    qo_sum = np.zeros((wl.M, dim))
    for c in range(C):
        assert_close(y[c].cpu().numpy(), oracle.forward(d, p64, W[c].astype(np.float64), q64), what=f"y[{c}]")
        wo, po = oracle.backward(d, p64, W[c].astype(np.float64), q64, YB[c].astype(np.float64))
        assert_close(wbar[c].cpu().numpy(), wo, what=f"wbar[{c}]")
        po_sum += po
        qo_sum += oracle.backward_q(d, p64, W[c].astype(np.float64), q64, YB[c].astype(np.float64))
    assert_close(pbar.cpu().numpy(), po_sum, what="pbar (sum over channels)")
    assert_close(qbar.cpu().numpy(), qo_sum, what="qbar (sum over channels)")


def test_channels_autograd_and_reuse(lib):
    """The autograd layer with (C, N) weights: the backward reuses the forward's sorts and gives
    the same gradients as a fresh backward."""
    from paper_2111_00110_gb300.transform import fc2t2
    C = 4
    wl = workloads.uniform(911, 3, 4000, 3000, 16, 6, 0.08)
    W = wl.channel_weights(C)
    plan = make_plan(3, 16, 6, wl.sigma, wl.N, wl.M, m2l="separable", channels=C)
    P_, W_, Q_ = [t.requires_grad_(True) for t in to_dev(wl.p, W, wl.q)]
    y = fc2t2(P_, W_, Q_, plan)
    (y * y).sum().backward()
    torch.cuda.synchronize()
    ybar = 2.0 * y.detach()
    wb, pb = plan.backward(P_.detach(), W_.detach(), Q_.detach(), ybar)
    qb = plan.backward_q(P_.detach(), W_.detach(), Q_.detach(), ybar)
    torch.cuda.synchronize()
    plan.check()
    assert rel_l2(W_.grad.cpu().numpy(), wb.cpu().numpy()) <= 1e-6
    assert rel_l2(P_.grad.cpu().numpy(), pb.cpu().numpy()) <= 1e-6
    assert rel_l2(Q_.grad.cpu().numpy(), qb.cpu().numpy()) <= 1e-6
    d = odesc(3, 16, 6, wl.sigma)
    yb64 = ybar.cpu().numpy().astype(np.float64)
    po = sum(oracle.backward(d, *f64(wl.p, W[c], wl.q, yb64[c]))[1] for c in range(C))
    assert_close(P_.grad.cpu().numpy(), po, what="autograd pbar, 4 channels")


def test_channels_direct_and_empty(lib):
    """The exact device sum per channel, and empty inputs with channels."""
    from paper_2111_00110_gb300.transform import direct
    C = 2
    wl = workloads.uniform(912, 3, 700, 300, 16, 4, 0.08)
    W = wl.channel_weights(C)
    P_, W_, Q_ = to_dev(wl.p, W, wl.q)
    yd = direct(P_, W_, Q_, wl.sigma).cpu().numpy()
    d = odesc(3, 16, 4, wl.sigma)
    for c in range(C):
        assert rel_l2(yd[c], oracle.direct(d, *f64(wl.p, W[c], wl.q))) <= 1e-6
    plan = make_plan(3, 16, 4, wl.sigma, wl.N, wl.M, channels=C)
    y = plan.forward(P_[:0], W_[:, :0].contiguous(), Q_)
    torch.cuda.synchronize()
    assert y.shape == (C, wl.M) and float(y.abs().max()) == 0.0


# ------------------------------------------------------------------------------ accessor

ACC_CASES = [(3, 16, 4, "fp32", 1), (3, 16, 6, "separable", 2), (3, 8, 8, "fp32", 1), (3, 16, 1, "fp32", 1),
             (2, 32, 4, "fp32", 3), (2, 16, 8, "fp32", 1), (3, 16, 6, "bf16x3", 1), (3, 16, 6, "occupied", 2)]


@pytest.mark.parametrize("dim,grid,order,m2l,C", ACC_CASES)
def test_accessor_points(lib, dim, grid, order, m2l, C):
    """Value, first and second partials of the held expansion at points (sorted on the device)
    against the oracle's local series; the value equals the forward transform's y."""
    wl = workloads.uniform(920 + dim * 10 + order, dim, 2500, 1900, grid, order, 0.08)
    W = wl.channel_weights(C)
    plan = make_plan(dim, grid, order, wl.sigma, wl.N, wl.M, m2l=m2l, channels=C)
    P_, W_, Q_ = to_dev(wl.p, W, wl.q)
    y_fwd = plan.forward(P_, W_, Q_).reshape(C, -1).clone()
    S = plan.expand(P_, W_)
    cols = [Q_[:, i] for i in range(dim)]
    val = S[(Ellipsis,) + tuple(cols)]
    g = S.partials[(Ellipsis,) + tuple(cols)]
    h = S.partials2[(Ellipsis,) + tuple(cols)]
    torch.cuda.synchronize()
    plan.check()
    assert val.shape == (C, wl.M) and g.shape == (C, wl.M, dim) and h.shape == (C, wl.M, dim * (dim + 1) // 2)
    assert rel_l2(val.cpu().numpy(), y_fwd.cpu().numpy()) <= 1e-6
    d = odesc(dim, grid, order, wl.sigma)
    for c in range(C):
        vo, go, ho = oracle.partials(d, *f64(wl.p, W[c], wl.q))
        assert_close(val[c].cpu().numpy(), vo, what=f"value[{c}]")
        assert_close(g[c].cpu().numpy(), go, what=f"partials[{c}]")
        if order >= 2:
            assert_close(h[c].cpu().numpy(), ho, what=f"partials2[{c}]")
        else:
            assert float(h.abs().max()) == 0.0 and np.abs(ho).max() == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_accessor_polynomial_kernel_is_exact(lib, dim):
    """psi(x) = (1 - |x|^2)^2 at order 4: the series is the field, so the accessor's partials
    equal the oracle's (themselves pinned to sympy's closed forms)."""
    from itertools import product
    mis = [m for deg in range(5) for m in product(range(deg, -1, -1), repeat=dim) if sum(m) == deg]
    mis = sorted(set(mis), key=lambda m: (sum(m), [-e for e in m]))
    terms = {(0,) * dim: 1.0}
    for i in range(dim):
        e2 = tuple(2 if j == i else 0 for j in range(dim))
        e4 = tuple(4 if j == i else 0 for j in range(dim))
        terms[e2] = -2.0
        terms[e4] = 1.0
        for k in range(i + 1, dim):
            terms[tuple(2 if j in (i, k) else 0 for j in range(dim))] = 2.0
    coef = np.zeros(len(mis))
    for m, v in terms.items():
        coef[mis.index(m)] = v
    wl = workloads.uniform(930 + dim, dim, 800, 600, 8, 4, 0.1)
    from paper_2111_00110_gb300.transform import Plan
    plan = Plan(dim, 8, 4, kernel="poly", poly_coef=coef, max_sources=wl.N, max_queries=wl.M)
    P_, W_, Q_ = to_dev(wl.p, wl.w, wl.q)
    S = plan.expand(P_, W_)
    cols = tuple(Q_[:, i] for i in range(dim))
    g = S.partials[cols].cpu().numpy()
    h = S.partials2[cols].cpu().numpy()
    torch.cuda.synchronize()
    d = oracle.OracleDesc(dim=dim, grid=8, order=4, kernel="poly", poly_coef=coef)
    _, go, ho = oracle.partials(d, *f64(wl.p, wl.w, wl.q))
    assert_close(g[0], go, what="poly partials")
    assert_close(h[0], ho, what="poly partials2")


@pytest.mark.parametrize("dim", [2, 3])
def test_accessor_volume_equals_points(lib, dim):
    """A meshgrid query (the paper's `vol`) equals the point query at the meshgrid's points, and
    has the paper's shapes (a scalar entry becomes an axis of length one)."""
    C = 2
    wl = workloads.uniform(940 + dim, dim, 3000, 10, 16, 6, 0.08)
    W = wl.channel_weights(C)
    plan = make_plan(dim, 16, 6, wl.sigma, wl.N, 1 << 16, channels=C)
    P_, W_ = to_dev(wl.p, W)
    S = plan.expand(P_, W_)
    axes = [slice(0.0, 1.0, 33), slice(0.1, 0.8, 20)] + ([0.37] if dim == 3 else [])
    for what in ("value", "partials", "partials2"):
        q = S.vol if what == "value" else getattr(S, what).vol
        vol = q[(Ellipsis,) + tuple(axes)]
        K = {"value": (), "partials": (dim,), "partials2": (dim * (dim + 1) // 2,)}[what]
        assert vol.shape == (C, 33, 20) + ((1,) if dim == 3 else ()) + K
        grids = torch.meshgrid(torch.linspace(0.0, 1.0, 33), torch.linspace(0.1, 0.8, 20),
                               *([torch.tensor([0.37])] if dim == 3 else []), indexing="ij")
        pts = [t.reshape(-1).cuda() for t in grids]
        qp = S if what == "value" else getattr(S, what)
        ref = qp[(Ellipsis,) + tuple(pts)]
        torch.cuda.synchronize()
        assert torch.allclose(vol.reshape(ref.shape), ref, rtol=1e-6, atol=1e-6 * float(ref.abs().max())), what
    # the paper's example shapes
    assert S[(0,) + (0.5,) * dim].shape == ()
    assert S.partials[(Ellipsis,) + (0.0,) * dim].shape == (C, dim)
    assert S.partials2[(Ellipsis,) + (0.0,) * dim].shape == (C, dim * (dim + 1) // 2)
    if dim == 3:
        assert S.partials.vol[0, ::16, ::8, 0.0].shape == (16, 8, 1, 3)


def test_accessor_chunks_empty_and_staleness(lib):
    """Point queries beyond max_queries run in chunks; empty queries give empty outputs; an
    expansion whose plan ran another transform refuses to answer; evaluating with no expansion
    held is an error of the C ABI."""
    from paper_2111_00110_gb300 import capi
    wl = workloads.uniform(950, 3, 2000, 5000, 16, 4, 0.08)
    plan = make_plan(3, 16, 4, wl.sigma, wl.N, 1500)
    P_, W_, Q_ = to_dev(wl.p, wl.w, wl.q)
    with pytest.raises(capi.FC2T2Error):
        capi.evaluate(plan._h, 0, Q_.data_ptr(), 10, "value", Q_.data_ptr())
    S = plan.expand(P_, W_)
    v = S[Q_[:, 0], Q_[:, 1], Q_[:, 2]]
    torch.cuda.synchronize()
    vo = oracle.partials(odesc(3, 16, 4, wl.sigma), *f64(wl.p, wl.w, wl.q))[0]
    assert_close(v.cpu().numpy()[0], vo, what="chunked point query")
    assert S[Q_[:0, 0], Q_[:0, 1], Q_[:0, 2]].shape == (1, 0)
    assert S.vol[..., slice(0, 1, 0), 0.5, 0.5].shape == (1, 0, 1, 1)
    plan.forward(P_, W_, Q_[:1000].contiguous())
    with pytest.raises(RuntimeError):
        S[0.5, 0.5, 0.5]
