"""GPU parity of the M2L over occupied cells (``m2l="occupied"``) against the FP64 oracle.

The form sums, for every target cell with targets below it, the terms of the source cells of its
interaction list that hold sources (Sec. 3's M2L restricted to the pairs whose terms are nonzero
and read).  Every local series that L2P reads gets the terms of the full M2L, so the bars are the
FP32 path's: rel-L2 <= 1e-5 against the oracle, every element within 1e-4 of max |ref|; against the
plain FP32 form (the same operator and arithmetic) the outputs agree to rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2111_00110_gb300 import workloads
from test_gpu_parity import assert_close, f64, lib, make_plan, odesc, rel_l2, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def clustered(seed, dim, N, M, centres, std):
    """Sources and queries from a few isotropic clusters (independent draws, kept in [0, 1)^dim)."""
    rng = np.random.default_rng(seed)

    def draw(n):
        out = np.empty((0, dim))
        while out.shape[0] < n:
            k = rng.integers(0, len(centres), size=n)
            x = np.asarray(centres)[k] + std * rng.standard_normal((n, dim))
            out = np.concatenate([out, x[np.all((x >= 0) & (x < 1), axis=1)]])
        return out[:n].astype(np.float32)

    p = draw(N)
    w = rng.standard_normal(N).astype(np.float32)
    q = draw(M)
    return p, w, q


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("order", [1, 2, 4, 6, 7, 8])
def test_occupied_every_order(lib, dim, order):
    """Uniform points (every cell occupied: the full M2L through the work queue), forward and
    backward, against the oracle and element by element against the plain FP32 form."""
    grid = 16 if dim == 3 else 32
    wl = workloads.uniform(500 + 10 * dim + order, dim, 3001, 2503, grid, order, 0.06)
    occ = make_plan(dim, grid, order, wl.sigma, wl.N, wl.M, m2l="occupied")
    ref = make_plan(dim, grid, order, wl.sigma, wl.N, wl.M, m2l="fp32")
    P_, W_, Q_ = to_dev(wl.p, wl.w, wl.q)
    yb = dev(wl.ybar())
    y = occ.forward(P_, W_, Q_)
    wbar, pbar = occ.backward(P_, W_, Q_, yb)
    y32 = ref.forward(P_, W_, Q_)
    w32, p32 = ref.backward(P_, W_, Q_, yb)
    torch.cuda.synchronize()
    occ.check()
    d = odesc(dim, grid, order, wl.sigma)
    yo = oracle.forward(d, *f64(wl.p, wl.w, wl.q))
    wo, po = oracle.backward(d, *f64(wl.p, wl.w, wl.q, wl.ybar()))
    tag = f"D{dim} rho{order}"
    assert_close(y.cpu().numpy(), yo, what=f"{tag} y")
    assert_close(wbar.cpu().numpy(), wo, what=f"{tag} wbar")
    assert_close(pbar.cpu().numpy(), po, what=f"{tag} pbar")
    assert rel_l2(y.cpu().numpy(), y32.cpu().numpy()) <= 2e-6
    assert rel_l2(wbar.cpu().numpy(), w32.cpu().numpy()) <= 2e-6
    assert rel_l2(pbar.cpu().numpy(), p32.cpu().numpy()) <= 2e-6
    occ.close()
    ref.close()


CLUSTER_CASES = [(3, 32, 6, 4000, 3000), (3, 64, 4, 6000, 5000), (3, 32, 8, 2500, 2500), (2, 64, 6, 3000, 4000),
                 (2, 128, 8, 2000, 1500)]


@pytest.mark.parametrize("dim,grid,order,N,M", CLUSTER_CASES)
def test_occupied_clustered(lib, dim, grid, order, N, M):
    """Clustered sources and queries (most of the grid empty; target clusters that hold no source
    and source clusters with no target): forward, backward on the forward's sorts, and the query
    gradient against the oracle."""
    centres = [[0.2] * dim, [0.7] * dim, [0.25] + [0.8] * (dim - 1)]
    p, w, q = clustered(31 + grid + order, dim, N, M, centres[:2], 0.04)
    # a query cluster far from every source, and one source cluster with no queries
    rng = np.random.default_rng(7)
    q[: M // 5] = np.clip(np.asarray(centres[2]) + 0.02 * rng.standard_normal((M // 5, dim)), 0, 0.999).astype(np.float32)
    sigma = 1.5 / grid
    plan = make_plan(dim, grid, order, sigma, N, M, m2l="occupied")
    P_, W_, Q_ = to_dev(p, w, q)
    ybar = np.random.default_rng(8).standard_normal(M).astype(np.float32)
    YB = dev(ybar)
    y = plan.forward(P_, W_, Q_)
    wbar, pbar = plan.backward(P_, W_, Q_, YB, reuse_forward=True)
    qbar = plan.backward_q(P_, W_, Q_, YB)
    torch.cuda.synchronize()
    plan.check()
    d = odesc(dim, grid, order, sigma)
    yo = oracle.forward(d, *f64(p, w, q))
    wo, po = oracle.backward(d, *f64(p, w, q, ybar))
    qo = oracle.backward_q(d, *f64(p, w, q, ybar))
    tag = f"D{dim} n{grid} rho{order}"
    assert_close(y.cpu().numpy(), yo, what=f"{tag} y")
    assert_close(wbar.cpu().numpy(), wo, what=f"{tag} wbar")
    assert_close(pbar.cpu().numpy(), po, what=f"{tag} pbar")
    assert_close(qbar.cpu().numpy(), qo, what=f"{tag} qbar")
    plan.close()


@pytest.mark.parametrize("dim,grid", [(3, 4), (2, 4), (3, 8)])
def test_occupied_small_grids_and_single_cells(lib, dim, grid):
    """One level (grid 4) and two levels; all sources in one cell, queries in one other cell or
    next to it; an empty source set."""
    sigma = 2.0 / grid
    rng = np.random.default_rng(grid + dim)
    h = 1.0 / grid
    p = (np.full((300, dim), 0.5 * h) + 0.4 * h * rng.random((300, dim))).astype(np.float32)     # cell 0
    w = rng.standard_normal(300).astype(np.float32)
    for qc in (grid - 1, 1):
        q = (np.full((200, dim), (qc + 0.3) * h) + 0.4 * h * rng.random((200, dim))).astype(np.float32)
        plan = make_plan(dim, grid, 4, sigma, 300, 200, m2l="occupied")
        y = plan.forward(*to_dev(p, w, q))
        torch.cuda.synchronize()
        plan.check()
        yo = oracle.forward(odesc(dim, grid, 4, sigma), *f64(p, w, q))
        assert_close(y.cpu().numpy(), yo, what=f"D{dim} n{grid} query cell {qc}")
        # no sources: y = 0
        y0 = plan.forward(*to_dev(p[:0], w[:0], q))
        torch.cuda.synchronize()
        assert float(y0.abs().max()) == 0.0
        plan.close()


def test_occupied_polynomial_kernel_is_exact(lib):
    """psi(x) = (1 - |x|^2)^2 at order 4 on clustered points: the series is exact, so the occupied
    form equals the oracle (pinned to the direct sum for polynomial kernels)."""
    from itertools import product
    dim, grid, order = 3, 16, 4
    mis = [m for deg in range(5) for m in product(range(deg, -1, -1), repeat=dim) if sum(m) == deg]
    mis = sorted(set(mis), key=lambda m: (sum(m), [-e for e in m]))
    terms = {(0,) * dim: 1.0}
    for i in range(dim):
        terms[tuple(2 if j == i else 0 for j in range(dim))] = -2.0
        terms[tuple(4 if j == i else 0 for j in range(dim))] = 1.0
        for k in range(i + 1, dim):
            terms[tuple(2 if j in (i, k) else 0 for j in range(dim))] = 2.0
    coef = np.zeros(len(mis))
    for m, v in terms.items():
        coef[mis.index(m)] = v
    p, w, q = clustered(77, dim, 2000, 1500, [[0.3, 0.3, 0.3], [0.6, 0.7, 0.4]], 0.05)
    from paper_2111_00110_gb300.transform import Plan
    plan = Plan(dim, grid, order, kernel="poly", poly_coef=coef, m2l="occupied", max_sources=2000, max_queries=1500)
    y = plan.forward(*to_dev(p, w, q))
    torch.cuda.synchronize()
    plan.check()
    d = oracle.OracleDesc(dim=dim, grid=grid, order=order, kernel="poly", poly_coef=coef)
    yo = oracle.forward(d, *f64(p, w, q))
    assert_close(y.cpu().numpy(), yo, what="polynomial kernel")
    yd = oracle.direct(d, *f64(p, w, q))
    assert rel_l2(y.cpu().numpy(), yd) <= 1e-5
    plan.close()


def test_occupied_accessor_takes_every_cell(lib):
    """fc2t2_expand has no target set: the occupied form computes every cell's series, so the held
    expansion's value and partials at arbitrary points match the oracle."""
    dim, grid, order = 3, 16, 6
    p, w, _ = clustered(91, dim, 3000, 10, [[0.3, 0.4, 0.5]], 0.05)
    q = np.random.default_rng(92).random((2000, dim)).astype(np.float32)
    plan = make_plan(dim, grid, order, 0.1, 3000, 2000, m2l="occupied")
    P_, W_, Q_ = to_dev(p, w, q)
    S = plan.expand(P_, W_)
    cols = [Q_[:, i] for i in range(dim)]
    val = S[(Ellipsis,) + tuple(cols)]
    g = S.partials[(Ellipsis,) + tuple(cols)]
    torch.cuda.synchronize()
    plan.check()
    vo, go, _ = oracle.partials(odesc(dim, grid, order, 0.1), *f64(p, w, q))
    assert_close(val.reshape(-1).cpu().numpy(), vo, what="value")
    assert_close(g.reshape(-1, dim).cpu().numpy(), go, what="partials")
    plan.close()


def test_occupied_batched_one_launch(lib):
    """Instances of the clustered batched workload with occupied-cell plans of two orders (two M2L
    launches), one plan used twice in the batch (that instance runs on its own), a separable plan
    and an instance with no sources in the same call; every result against the oracle at sampled
    outputs, and the batched results equal to each plan's own calls."""
    from paper_2111_00110_gb300.transform import Plan, backward_batched, forward_batched
    spec = [(10, 64, 6, "occupied", None), (11, 32, 4, "occupied", 5000), (12, 64, 6, "occupied", 3000),
            (13, 32, 6, "separable", 4000), (14, 64, 4, "occupied", 20000)]
    wls = [workloads.mixture(i, grid=g, order=o, n_override=n) for i, g, o, m, n in spec]
    plans = [Plan(3, wl.grid, wl.order, wl.sigma, m2l=m, max_sources=wl.N, max_queries=wl.M)
             for wl, (_, _, _, m, _) in zip(wls, spec)]
    use = plans + [plans[1]]
    wl_use = wls + [workloads.mixture(15, grid=32, order=4, n_override=4000)]
    ps, ws, qs = [dev(wl.p) for wl in wl_use], [dev(wl.w) for wl in wl_use], [dev(wl.q) for wl in wl_use]
    ps[2], ws[2] = ps[2][:0], ws[2][:0]     # instance 2: no sources
    ybars = [dev(wl.ybar()) for wl in wl_use]
    ys = forward_batched(use, ps, ws, qs)
    grads = backward_batched(use, ps, ws, qs, ybars)
    torch.cuda.synchronize()
    for pl in plans:
        pl.check()
    assert float(ys[2].abs().max()) == 0.0
    for i, wl in enumerate(wl_use):
        if i == 2:
            continue
        rng = np.random.default_rng(wl.seed)
        sq = np.sort(rng.choice(wl.M, size=min(1024, wl.M), replace=False))
        sp = np.sort(rng.choice(wl.N, size=min(1024, wl.N), replace=False))
        d = odesc(3, wl.grid, wl.order, wl.sigma)
        yo = oracle.forward(d, *f64(wl.p, wl.w, wl.q), sel=sq)
        wo, po = oracle.backward(d, *f64(wl.p, wl.w, wl.q, wl.ybar()), sel=sp)
        tag = f"instance {i} n{wl.grid} rho{wl.order} N{wl.N}"
        assert_close(ys[i].cpu().numpy()[sq], yo, what=f"{tag} y")
        assert_close(grads[i][0].cpu().numpy()[sp], wo, what=f"{tag} wbar")
        assert_close(grads[i][1].cpu().numpy()[sp], po, what=f"{tag} pbar")
    # the backward on the forward's sorts (batched reuse) gives the same gradients
    ys = forward_batched(use, ps, ws, qs)
    grads_r = backward_batched(use, ps, ws, qs, ybars, reuse_forward=True)
    torch.cuda.synchronize()
    for i in range(len(use)):
        if i == 2:
            continue
        assert rel_l2(grads_r[i][0].cpu().numpy(), grads[i][0].cpu().numpy()) <= 1e-5
        assert rel_l2(grads_r[i][1].cpu().numpy(), grads[i][1].cpu().numpy()) <= 1e-5
    # the batched path and each plan's own calls agree to rounding
    for i in (0, 4):
        y1 = use[i].forward(ps[i], ws[i], qs[i])
        wb1, pb1 = use[i].backward(ps[i], ws[i], qs[i], ybars[i])
        torch.cuda.synchronize()
        assert rel_l2(ys[i].cpu().numpy(), y1.cpu().numpy()) <= 1e-5
        assert rel_l2(grads[i][0].cpu().numpy(), wb1.cpu().numpy()) <= 1e-5
        assert rel_l2(grads[i][1].cpu().numpy(), pb1.cpu().numpy()) <= 1e-5
    for pl in plans:
        pl.close()


def test_occupied_batched_many_instances_and_graph(lib):
    """More instances than one M2L launch takes (70 small instances: two launches), each equal to
    its own plan's call; and the batched forward + backward captured in a CUDA graph replays to the
    eager results.  (Two runs differ by rounding only: the cells hold up to hundreds of points, whose
    moments past the first 32 per cell are added with float atomics in no fixed order.)"""
    from paper_2111_00110_gb300.transform import Plan, backward_batched, forward_batched
    n_inst = 70
    rng = np.random.default_rng(2024)
    plans, ps, ws, qs, ybars = [], [], [], [], []
    for i in range(n_inst):
        N, M = int(rng.integers(50, 400)), int(rng.integers(50, 400))
        c = rng.uniform(0.2, 0.8, size=(2, 3))
        p, w, q = clustered(3000 + i, 3, N, M, c, 0.05)
        plans.append(Plan(3, 8, 4, 0.2, m2l="occupied", max_sources=N, max_queries=M))
        ps.append(dev(p)); ws.append(dev(w)); qs.append(dev(q))
        ybars.append(dev(rng.standard_normal(M)))
    ys = forward_batched(plans, ps, ws, qs)
    gs = backward_batched(plans, ps, ws, qs, ybars)
    torch.cuda.synchronize()
    for i in range(0, n_inst, 7):
        y1 = plans[i].forward(ps[i], ws[i], qs[i])
        wb1, pb1 = plans[i].backward(ps[i], ws[i], qs[i], ybars[i])
        torch.cuda.synchronize()
        assert rel_l2(ys[i].cpu().numpy(), y1.cpu().numpy()) <= 1e-5
        assert rel_l2(gs[i][0].cpu().numpy(), wb1.cpu().numpy()) <= 1e-5
        assert rel_l2(gs[i][1].cpu().numpy(), pb1.cpu().numpy()) <= 1e-5
    d = odesc(3, 8, 4, 0.2)
    for i in (0, 69):
        yo = oracle.forward(d, *f64(ps[i].cpu().numpy(), ws[i].cpu().numpy(), qs[i].cpu().numpy()))
        assert_close(ys[i].cpu().numpy(), yo, what=f"instance {i}")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        forward_batched(plans, ps, ws, qs)
        backward_batched(plans, ps, ws, qs, ybars)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        yg = forward_batched(plans, ps, ws, qs)
        gg = backward_batched(plans, ps, ws, qs, ybars)
    g.replay()
    torch.cuda.synchronize()
    for i in range(n_inst):
        assert rel_l2(yg[i].cpu().numpy(), ys[i].cpu().numpy()) <= 1e-5
        assert rel_l2(gg[i][1].cpu().numpy(), gs[i][1].cpu().numpy()) <= 1e-5
    del g
    for pl in plans:
        pl.close()
