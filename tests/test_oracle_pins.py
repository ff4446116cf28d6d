"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* kernel derivatives   -- symbolic differentiation with sympy;
* per-pair identity    -- the multi-level transform equals, for every (source, target)
                          pair, the order-rho Taylor polynomial of psi about the centre
                          offset of the unique level at which the pair interacts; computed
                          here by brute force in numpy from sympy derivatives (Sec. 3:
                          M2M/L2L are exact re-centrings, the per-level lists partition
                          all cell pairs);
* polynomial exactness -- for psi a polynomial of degree <= rho the series is exact, so
                          the transform equals the direct sum of Eq. 1;
* adjoint identity     -- Sec. 4.1: the backward transform is the transpose;
* finite differences   -- wbar and pbar (Sec. 4.1) against central differences of the
                          forward map with the binning held fixed;
* dense gradient       -- the exact gradient of the direct sum against its own central
                          differences, and the transform's gradients against it (agreement
                          to truncation error, falling with the order);
* truncation decay     -- error against the exact sum decreases with the order;
* special cases        -- one source / one target closed form, empty inputs, linearity,
                          permutation invariance;
* sensitivity          -- every deliberate mistake the oracle can be switched into makes
                          at least one of these pins fail.
"""
import itertools
import json
import os
from functools import lru_cache

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2111_00110_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers (independent)

def graded(dim, order):
    out = []
    for d in range(order + 1):
        if dim == 2:
            for a0 in range(d, -1, -1):
                out.append((a0, d - a0))
        else:
            for a0 in range(d, -1, -1):
                for a1 in range(d - a0, -1, -1):
                    out.append((a0, a1, d - a0 - a1))
    return out


@lru_cache(maxsize=None)
def sympy_derivs(kind, dim, order, sigma=None, poly=None):
    """Lambdified d^m psi for every graded m, |m| <= order."""
    xs = sp.symbols("x0:%d" % dim, real=True)
    if kind == "gaussian":
        psi = sp.exp(-sum(x ** 2 for x in xs) / (2 * sp.Float(sigma) ** 2))
    else:
        mons = graded(dim, 12)
        psi = sum(sp.Float(c) * sp.prod([x ** e for x, e in zip(xs, mons[i])])
                  for i, c in enumerate(poly) if c != 0)
        psi = sp.sympify(psi)
    fns = []
    for m in graded(dim, order):
        expr = psi
        for x, e in zip(xs, m):
            if e:
                expr = sp.diff(expr, x, e)
        fns.append(sp.lambdify(xs, expr, "numpy"))
    return fns


def eval_derivs(kind, dim, order, c, sigma=None, poly=None):
    fns = sympy_derivs(kind, dim, order, sigma, None if poly is None else tuple(poly))
    c = np.atleast_2d(c)
    out = np.empty((c.shape[0], len(fns)))
    for j, f in enumerate(fns):
        out[:, j] = np.broadcast_to(f(*[c[:, i] for i in range(dim)]), (c.shape[0],))
    return out


def bin_f32(x, n, lo=0.0, hi=1.0):
    """Finest-level cell per coordinate, every step rounded to float32."""
    xf = np.asarray(x, dtype=np.float32)
    t = (xf - np.float32(lo)) * np.float32(n / (hi - lo))
    c = np.floor(t).astype(np.int64)
    return np.clip(c, 0, n - 1)


def pairwise_reference(desc, p, w, q, kind="gaussian", poly=None):
    """Brute-force per-pair form: y_m = sum_n w_n T_rho[psi; c_nm](p_n - q_m)."""
    D, n, rho = desc.dim, desc.grid, desc.order
    h0 = (desc.hi - desc.lo) / n
    nlev = int(np.log2(n)) - 1
    sc = bin_f32(p, n, desc.lo, desc.hi)          # [N, D]
    tc = bin_f32(q, n, desc.lo, desc.hi)          # [M, D]
    S = sc[None, :, :]
    T = tc[:, None, :]
    lev = np.full((q.shape[0], p.shape[0]), -1, dtype=np.int64)
    for l in range(nlev):
        s_l, t_l = S >> l, T >> l
        if l == nlev - 1:
            parent_near = np.ones(lev.shape, dtype=bool)
        else:
            parent_near = np.all(np.abs((s_l >> 1) - (t_l >> 1)) <= 1, axis=2)
        near = np.all(np.abs(s_l - t_l) <= 1, axis=2)
        hit = parent_near if l == 0 else (parent_near & ~near)
        lev = np.where((lev < 0) & hit, l, lev)
    assert np.all(lev >= 0)
    hl = h0 * (2.0 ** lev)
    # z(s) - z(t) = (s - t) h at the interaction level
    off = ((S >> lev[..., None]) - (T >> lev[..., None])) * hl[..., None]
    x = p[None, :, :] - q[:, None, :]
    mis = graded(D, rho)
    offs = off.reshape(-1, D)
    uniq, inv = np.unique(offs, axis=0, return_inverse=True)
    dv = eval_derivs(kind, D, rho, uniq, sigma=desc.sigma, poly=poly)[inv.ravel()]
    u = x.reshape(-1, D) - offs
    from math import factorial
    acc = np.zeros(u.shape[0])
    for j, m in enumerate(mis):
        term = dv[:, j].copy()
        for i in range(D):
            term *= u[:, i] ** m[i] / factorial(m[i])
        acc += term
    A = acc.reshape(q.shape[0], p.shape[0])
    return A @ w


def small_inputs(seed, dim, N, M):
    rng = np.random.default_rng(seed)
    p = rng.random((N, dim)).astype(np.float32).astype(np.float64)
    w = rng.standard_normal(N)
    q = rng.random((M, dim)).astype(np.float32).astype(np.float64)
    return p, w, q


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------------ the pins

def test_multi_index_counts_match_paper():
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    for row in facts["coefficient_counts"]:
        mi = oracle.multi_indices(row["dim"], row["order"])
        assert mi.shape == (row["P"], row["dim"]), row
        assert [tuple(r) for r in mi] == graded(row["dim"], row["order"])
    for row in facts["memory_per_channel_MB"]:
        P = oracle.num_coeffs(3, row["order"])
        mb = row["cells_per_dim"] ** 3 * P * 4 / 1e6
        assert abs(mb - row["MB"]) <= 0.1, (row, mb)


@pytest.mark.parametrize("dim", [2, 3])
def test_gaussian_derivatives_vs_sympy(dim):
    rng = np.random.default_rng(1)
    for sigma in (0.02, 0.1):
        d = oracle.OracleDesc(dim=dim, grid=8, order=8, sigma=sigma)
        for _ in range(4):
            c = rng.uniform(-3 * sigma, 3 * sigma, size=dim)
            got = oracle.kernel_derivs(d, c)
            ref = eval_derivs("gaussian", dim, 8, c, sigma=sigma)[0]
            scale = np.abs(ref).max()
            assert np.max(np.abs(got - ref)) <= 1e-12 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_polynomial_derivatives_vs_sympy(dim):
    rng = np.random.default_rng(2)
    P4 = len(graded(dim, 4))
    coef = rng.standard_normal(P4)
    d = oracle.OracleDesc(dim=dim, grid=8, order=5, kernel="poly", poly_coef=coef)
    for _ in range(3):
        c = rng.uniform(-1, 1, size=dim)
        got = oracle.kernel_derivs(d, c)
        ref = eval_derivs("poly", dim, 5, c, poly=tuple(coef))[0]
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,grid,order", [(2, 8, 3), (2, 16, 4), (3, 8, 3), (3, 16, 2), (2, 32, 2),
                                            (3, 16, 6), (3, 8, 8)])
def test_per_pair_identity(dim, grid, order):
    p, w, q = small_inputs(10 + dim + grid + order, dim, 60, 50)
    sigma = 0.15 if grid == 8 else 0.08
    d = oracle.OracleDesc(dim=dim, grid=grid, order=order, sigma=sigma)
    y = oracle.forward(d, p, w, q)
    ref = pairwise_reference(d, p, w, q)
    assert rel(y, ref) <= 1e-12


POLYS_3D = {
    "one": {(0, 0, 0): 1.0},
    "r2": {(2, 0, 0): 1.0, (0, 2, 0): 1.0, (0, 0, 2): 1.0},
    "one_minus_r2_sq": {(0, 0, 0): 1.0, (2, 0, 0): -2.0, (0, 2, 0): -2.0, (0, 0, 2): -2.0,
                        (4, 0, 0): 1.0, (0, 4, 0): 1.0, (0, 0, 4): 1.0,
                        (2, 2, 0): 2.0, (2, 0, 2): 2.0, (0, 2, 2): 2.0},
    "odd_x": {(1, 0, 0): 1.0},
    "odd_mixed": {(1, 2, 0): 0.7, (0, 1, 1): -1.3, (0, 0, 3): 0.4},
}


def poly_coef(terms, dim, deg):
    mis = graded(dim, deg)
    c = np.zeros(len(mis))
    for m, v in terms.items():
        c[mis.index(m[:dim])] += v
    return c


@pytest.mark.parametrize("name", list(POLYS_3D))
@pytest.mark.parametrize("dim", [2, 3])
def test_polynomial_exactness(name, dim):
    terms = {m: v for m, v in POLYS_3D[name].items() if dim == 3 or m[2] == 0}
    deg = max(sum(m) for m in terms)
    coef = poly_coef(terms, dim, deg)
    for grid in (8, 16):
        d = oracle.OracleDesc(dim=dim, grid=grid, order=max(deg, 4), kernel="poly", poly_coef=coef)
        p, w, q = small_inputs(3 + grid, dim, 70, 40)
        y = oracle.forward(d, p, w, q)
        yd = oracle.direct(d, p, w, q)
        assert np.max(np.abs(y - yd)) <= 1e-11 * max(1.0, np.abs(yd).max()), (name, dim, grid)


@pytest.mark.parametrize("dim,grid,order", [(2, 16, 4), (3, 8, 4), (3, 16, 3)])
def test_adjoint_identity(dim, grid, order):
    p, w, q = small_inputs(40 + dim, dim, 80, 70)
    ybar = np.random.default_rng(5).standard_normal(q.shape[0])
    d = oracle.OracleDesc(dim=dim, grid=grid, order=order, sigma=0.1)
    y = oracle.forward(d, p, w, q)
    wbar, _ = oracle.backward(d, p, w, q, ybar)
    lhs, rhs = float(ybar @ y), float(wbar @ w)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(ybar) @ np.abs(y) + 1e-300)


def _loss(d, p, w, q, pc, qc):
    y = oracle.forward(d, p, w, q, src_cell=pc, tgt_cell=qc)
    return float(np.sum(y * y)), y


@pytest.mark.parametrize("dim", [2, 3])
def test_gradients_vs_central_differences(dim):
    grid, order = (16, 4) if dim == 2 else (8, 4)
    p, w, q = small_inputs(70 + dim, dim, 30, 40)
    d = oracle.OracleDesc(dim=dim, grid=grid, order=order, sigma=0.12)
    pc = oracle.bin_cells(d, p)
    qc = oracle.bin_cells(d, q)
    L0, y = _loss(d, p, w, q, pc, qc)
    wbar, pbar = oracle.backward(d, p, w, q, 2.0 * y, src_cell=pc, tgt_cell=qc)
    rng = np.random.default_rng(9)
    for n in rng.choice(p.shape[0], size=6, replace=False):
        # L is quadratic in w: the central difference is exact up to rounding
        eps = 1e-3
        wp, wm = w.copy(), w.copy()
        wp[n] += eps
        wm[n] -= eps
        fd = (_loss(d, p, wp, q, pc, qc)[0] - _loss(d, p, wm, q, pc, qc)[0]) / (2 * eps)
        assert abs(fd - wbar[n]) <= 1e-8 * (abs(wbar[n]) + np.sqrt(L0))
        for i in range(dim):
            vals = []
            for eps in (1e-3, 1e-4):
                pp, pm = p.copy(), p.copy()
                pp[n, i] += eps
                pm[n, i] -= eps
                fd = (_loss(d, pp, w, q, pc, qc)[0] - _loss(d, pm, w, q, pc, qc)[0]) / (2 * eps)
                vals.append(fd)
            scale = abs(pbar[n, i]) + 1e-3 * np.sqrt(L0) / d.sigma
            assert abs(vals[0] - pbar[n, i]) <= 2e-3 * scale
            assert abs(vals[1] - pbar[n, i]) <= 2e-5 * scale


@pytest.mark.parametrize("kind", ["gaussian", "poly"])
@pytest.mark.parametrize("dim", [2, 3])
def test_direct_gradient_vs_central_differences(kind, dim):
    """The dense gradient of <ybar, y> for the exact sum (Sec. 4.1 applied to Eq. 1) against
    central differences of the exact sum itself: exact to rounding in w (the sum is linear in w),
    second order in eps in p.  The polynomial is odd, so a sign slip in the gradient fails it."""
    p, w, q = small_inputs(200 + dim, dim, 25, 35)
    if kind == "gaussian":
        d = oracle.OracleDesc(dim=dim, grid=8, order=4, sigma=0.1)
    else:
        terms = {m: v for m, v in POLYS_3D["odd_mixed"].items() if dim == 3 or m[2] == 0}
        d = oracle.OracleDesc(dim=dim, grid=8, order=4, kernel="poly", poly_coef=poly_coef(terms, dim, 3))
    ybar = np.random.default_rng(201).standard_normal(q.shape[0])
    sel = np.array([0, 7, 13, 24])
    wbar, pbar = oracle.direct_grad(d, p, w, q, ybar, sel=sel)
    full_w, full_p = oracle.direct_grad(d, p, w, q, ybar)
    assert np.array_equal(full_w[sel], wbar) and np.array_equal(full_p[sel], pbar)
    L = lambda pp, ww: float(ybar @ oracle.direct(d, pp, ww, q))
    scale = np.abs(ybar) @ np.abs(oracle.direct(d, p, np.abs(w), q)) + 1e-300
    for j, n in enumerate(sel):
        wp, wm = w.copy(), w.copy()
        wp[n] += 1e-3
        wm[n] -= 1e-3
        assert abs((L(p, wp) - L(p, wm)) / 2e-3 - wbar[j]) <= 1e-10 * scale
        for i in range(dim):
            for eps, tol in ((1e-4, 1e-5), (1e-5, 1e-7)):
                pp, pm = p.copy(), p.copy()
                pp[n, i] += eps
                pm[n, i] -= eps
                fd = (L(pp, w) - L(pm, w)) / (2 * eps)
                assert abs(fd - pbar[j, i]) <= tol * (np.abs(full_p).max() + 1e-300), (n, i, eps)


def test_transform_gradients_approach_the_dense_gradient():
    """wbar and pbar of the transform (Sec. 4.1) against the exact gradient of the direct sum at
    the same cotangent: they agree to the truncation error of the series, which falls with the
    order (the 2D 32 x 32 workload, sigma 0.05)."""
    wl = workloads.uniform2d()
    p, w, q = (a.astype(np.float64) for a in (wl.p, wl.w, wl.q))
    ybar = np.random.default_rng(202).standard_normal(q.shape[0])
    d = oracle.OracleDesc(dim=2, grid=wl.grid, order=2, sigma=wl.sigma)
    wd, pd = oracle.direct_grad(d, p, w, q, ybar)
    ew, ep = [], []
    for order in (2, 4, 6, 8):
        d.order = order
        wb, pb = oracle.backward(d, p, w, q, ybar)
        ew.append(rel(wb, wd))
        ep.append(rel(pb, pd))
    assert all(a > b for a, b in zip(ew, ew[1:])), ew
    assert all(a > b for a, b in zip(ep, ep[1:])), ep
    assert ew[1] <= 2e-2 and ep[1] <= 8e-2, (ew, ep)


@pytest.mark.parametrize("dim", [2, 3])
def test_query_gradient_vs_central_differences(dim):
    """qbar = ybar * grad_x y(x)|_{x=q} (binning of q frozen) against central differences of
    L = sum(y^2) in the query positions; a mistake in the derivative of the local series (an
    index shift, a missing 1/h) fails it."""
    grid, order = (16, 4) if dim == 2 else (8, 4)
    p, w, q = small_inputs(90 + dim, dim, 30, 40)
    d = oracle.OracleDesc(dim=dim, grid=grid, order=order, sigma=0.12)
    pc = oracle.bin_cells(d, p)
    qc = oracle.bin_cells(d, q)
    L0, y = _loss(d, p, w, q, pc, qc)
    qbar = oracle.backward_q(d, p, w, q, 2.0 * y, src_cell=pc, tgt_cell=qc)
    rng = np.random.default_rng(11)
    for m in rng.choice(q.shape[0], size=6, replace=False):
        for i in range(dim):
            vals = []
            for eps in (1e-3, 1e-4):
                qp, qm = q.copy(), q.copy()
                qp[m, i] += eps
                qm[m, i] -= eps
                vals.append((_loss(d, p, w, qp, pc, qc)[0] - _loss(d, p, w, qm, pc, qc)[0]) / (2 * eps))
            scale = abs(qbar[m, i]) + 1e-3 * np.sqrt(L0) / d.sigma
            assert abs(vals[0] - qbar[m, i]) <= 2e-3 * scale
            assert abs(vals[1] - qbar[m, i]) <= 2e-5 * scale


def _accessor_reference(dim, coef, p, w, q):
    """Value, gradient and second partials in q of sum_n w_n psi(p_n - q) for a polynomial psi,
    from sympy's derivatives of psi: d/dq_i psi(p - q) = -psi_,i(p - q) and
    d^2/dq_i dq_k psi(p - q) = psi_,ik(p - q)."""
    mis = graded(dim, 2)
    diff = (p[:, None, :] - q[None, :, :]).reshape(-1, dim)
    der = eval_derivs("poly", dim, 2, diff, poly=tuple(coef)).reshape(p.shape[0], q.shape[0], -1)
    unit = [tuple(1 if j == i else 0 for j in range(dim)) for i in range(dim)]
    val = w @ der[:, :, 0]
    grad = np.stack([-(w @ der[:, :, mis.index(unit[i])]) for i in range(dim)], axis=1)
    hess = np.stack([w @ der[:, :, mis.index(tuple(a + b for a, b in zip(unit[i], unit[k])))]
                     for i in range(dim) for k in range(i, dim)], axis=1)
    return val, grad, hess


@pytest.mark.parametrize("name", ["r2", "one_minus_r2_sq", "odd_mixed"])
@pytest.mark.parametrize("dim", [2, 3])
def test_accessor_partials_polynomial_exact(name, dim):
    """For psi a polynomial of degree <= rho the local series is the field itself, so its value,
    first and second partials (the accessor's queries) equal the closed forms; a wrong lowering
    of an exponent, a missing 1/h, or a swapped (i, k) slot fails it."""
    terms = {m: v for m, v in POLYS_3D[name].items() if dim == 3 or m[2] == 0}
    deg = max(sum(m) for m in terms)
    coef = poly_coef(terms, dim, deg)
    d = oracle.OracleDesc(dim=dim, grid=8, order=max(deg, 4), kernel="poly", poly_coef=coef)
    p, w, q = small_inputs(120 + dim, dim, 50, 30)
    v, g, h = oracle.partials(d, p, w, q)
    rv, rg, rh = _accessor_reference(dim, coef, p, w, q)
    for a, b in ((v, rv), (g, rg), (h, rh)):
        assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.abs(b).max()), name


@pytest.mark.parametrize("dim", [2, 3])
def test_second_partials_vs_central_differences(dim):
    """Second partials of the Gaussian series at the queries against central differences of its
    first partials (binning of q frozen)."""
    grid, order = (16, 4) if dim == 2 else (8, 4)
    p, w, q = small_inputs(130 + dim, dim, 30, 40)
    d = oracle.OracleDesc(dim=dim, grid=grid, order=order, sigma=0.12)
    pc = oracle.bin_cells(d, p)
    qc = oracle.bin_cells(d, q)
    _, g, h = oracle.partials(d, p, w, q, src_cell=pc, tgt_cell=qc)
    slot, pos = {}, 0
    for i in range(dim):
        for k in range(i, dim):
            slot[(i, k)] = slot[(k, i)] = pos
            pos += 1
    rng = np.random.default_rng(13)
    scale = np.abs(h).max()
    for m in rng.choice(q.shape[0], size=6, replace=False):
        for k in range(dim):
            for eps, tol in ((1e-3, 2e-3), (1e-4, 2e-5)):
                qp, qm = q.copy(), q.copy()
                qp[m, k] += eps
                qm[m, k] -= eps
                gp = oracle.partials(d, p, w, qp, sel=[m], src_cell=pc, tgt_cell=qc)[1][0]
                gm = oracle.partials(d, p, w, qm, sel=[m], src_cell=pc, tgt_cell=qc)[1][0]
                fd = (gp - gm) / (2 * eps)
                for i in range(dim):
                    assert abs(fd[i] - h[m, slot[(i, k)]]) <= tol * scale, (m, i, k, eps)


def test_truncation_error_decays_with_order():
    wl = workloads.uniform2d()
    p = wl.p.astype(np.float64)
    w = wl.w.astype(np.float64)
    q = wl.q.astype(np.float64)
    d = oracle.OracleDesc(dim=2, grid=wl.grid, order=2, sigma=wl.sigma)
    yd = oracle.direct(d, p, w, q)
    errs = []
    for order in (2, 4, 6, 8):
        d.order = order
        errs.append(rel(oracle.forward(d, p, w, q), yd))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[1] <= 2e-2, errs


@pytest.mark.parametrize("dim", [2, 3])
def test_single_pair_closed_form(dim):
    rng = np.random.default_rng(11)
    d = oracle.OracleDesc(dim=dim, grid=16, order=4, sigma=0.1)
    from math import factorial
    for _ in range(5):
        p = rng.random((1, dim)).astype(np.float32).astype(np.float64)
        q = rng.random((1, dim)).astype(np.float32).astype(np.float64)
        w = np.array([rng.standard_normal()])
        y = oracle.forward(d, p, w, q)[0]
        ref = pairwise_reference(d, p, w, q)[0]
        assert abs(y - ref) <= 1e-12 * max(abs(ref), 1e-30)
        # same-cell pair: the expansion is about offset 0 at the finest level
        p2 = q + 1e-3
        y2 = oracle.forward(d, p2, w, q)[0]
        derivs = eval_derivs("gaussian", dim, 4, np.zeros(dim), sigma=0.1)[0]
        x = (p2 - q)[0]
        t = sum(derivs[j] * np.prod([x[i] ** m[i] / factorial(m[i]) for i in range(dim)])
                for j, m in enumerate(graded(dim, 4)))
        if np.all(bin_f32(p2, 16) == bin_f32(q, 16)):
            assert abs(y2 - w[0] * t) <= 1e-12 * abs(w[0] * t)


def test_empty_and_linearity_and_permutation():
    d = oracle.OracleDesc(dim=3, grid=8, order=3, sigma=0.1)
    p, w, q = small_inputs(21, 3, 50, 30)
    assert np.all(oracle.forward(d, p[:0], w[:0], q) == 0.0)
    assert oracle.forward(d, p, w, q[:0]).shape == (0,)
    y1 = oracle.forward(d, p, w, q)
    w2 = np.random.default_rng(3).standard_normal(w.shape)
    y2 = oracle.forward(d, p, w2, q)
    y12 = oracle.forward(d, p, 2.0 * w - 3.0 * w2, q)
    assert rel(y12, 2.0 * y1 - 3.0 * y2) <= 1e-13
    perm = np.random.default_rng(4).permutation(p.shape[0])
    assert rel(oracle.forward(d, p[perm], w[perm], q), y1) <= 1e-13


def test_selected_targets_match_full_evaluation():
    d = oracle.OracleDesc(dim=3, grid=16, order=3, sigma=0.05)
    p, w, q = small_inputs(31, 3, 200, 150)
    y = oracle.forward(d, p, w, q)
    sel = np.array([5, 0, 149, 77, 77])
    assert np.array_equal(oracle.forward(d, p, w, q, sel=sel), y[sel])


def test_binning_rule_edges():
    d = oracle.OracleDesc(dim=2, grid=32, order=2)
    x = np.array([[0.0, 1.0], [-0.25, 1.5], [0.5, 31.0 / 32.0], [np.nextafter(1.0, 0), 0.03125]])
    cells = oracle.bin_cells(d, x)
    c = bin_f32(x, 32)
    assert np.array_equal(cells, c[:, 0] + 32 * c[:, 1])
    assert cells[0] == 0 + 32 * 31 and cells[1] == 0 + 32 * 31


@pytest.mark.parametrize("fault", [f for f in oracle.FAULTS if f != "none"])
def test_each_planted_mistake_fails_a_pin(fault):
    """The pins above are sharp: every deliberate mistake breaks at least one of them."""
    caught = []
    # per-pair identity, Gaussian, 3D (three levels)
    p, w, q = small_inputs(55, 3, 60, 50)
    d = oracle.OracleDesc(dim=3, grid=16, order=3, sigma=0.08)
    y = oracle.forward(d, p, w, q, fault=fault)
    caught.append(rel(y, pairwise_reference(d, p, w, q)) > 1e-9)
    # polynomial exactness with an odd polynomial
    coef = poly_coef(POLYS_3D["odd_mixed"], 3, 3)
    dp = oracle.OracleDesc(dim=3, grid=16, order=3, kernel="poly", poly_coef=coef)
    yp = oracle.forward(dp, p, w, q, fault=fault)
    caught.append(np.max(np.abs(yp - oracle.direct(dp, p, w, q))) > 1e-9)
    assert any(caught), fault


# ---------------------------------------------------------------- rays (Sec. 6, integral layer)

def _clip(o, r, t0, t1, lo=0.0, hi=1.0):
    """Parameter range of o + t r inside [lo, hi)^3 within [t0, t1] (slab method), or None."""
    ta, tb = t0, t1
    for k in range(3):
        if r[k] == 0.0:
            if not (lo <= o[k] < hi):
                return None
            continue
        a, b = (lo - o[k]) / r[k], (hi - o[k]) / r[k]
        ta, tb = max(ta, min(a, b)), min(tb, max(a, b))
    return (ta, tb) if tb > ta else None


def _rays(seed, R, spread=1.0):
    rng = np.random.default_rng(seed)
    o = rng.random((R, 3)) * spread - 0.5 * (spread - 1.0)
    d = rng.standard_normal((R, 3))
    t0 = -rng.random(R) * 0.5
    t1 = rng.random(R) * 0.8
    return np.concatenate([o, d, t0[:, None], t1[:, None]], axis=1)


def _direct_ray(desc, p, w, rays, nodes=24):
    """Exact line integral of the direct sum for a polynomial kernel: Gauss-Legendre on the
    clipped range with enough nodes for its degree."""
    x, wq = np.polynomial.legendre.leggauss(nodes)
    out = np.zeros(rays.shape[0])
    for i, ray in enumerate(rays):
        rng_ = _clip(ray[:3], ray[3:6], ray[6], ray[7])
        if rng_ is None:
            continue
        ta, tb = rng_
        t = 0.5 * (tb - ta) * (x + 1.0) + ta
        q = ray[None, :3] + t[:, None] * ray[None, 3:6]
        out[i] = 0.5 * (tb - ta) * float(wq @ oracle.direct(desc, p, w, q))
    return out


@pytest.mark.parametrize("name", ["one", "r2", "one_minus_r2_sq", "odd_mixed"])
def test_ray_integral_polynomial_exact(name):
    """For psi a polynomial of degree <= rho the series is the field, so the integral of the series
    along a ray (cut at the cells it crosses, each cell's series restricted to the line) equals the
    integral of the direct sum; psi = 1 gives sum(w) times the length inside the domain."""
    terms = POLYS_3D[name]
    deg = max(sum(m) for m in terms)
    coef = poly_coef(terms, 3, deg)
    d = oracle.OracleDesc(dim=3, grid=8, order=max(deg, 4), kernel="poly", poly_coef=coef)
    p, w, _ = small_inputs(140, 3, 40, 1)
    rays = _rays(141, 25, spread=1.4)
    y = oracle.ray_forward(d, p, w, rays)
    ref = _direct_ray(d, p, w, rays)
    assert np.max(np.abs(y - ref)) <= 1e-10 * max(1.0, np.abs(ref).max()), name


def _gauss_ray_closed_form(p, w, rays, sigma):
    """int exp(-|p - o - t r|^2 / (2 sigma^2)) dt over the clipped range, by completing the square:
    exp(-c / (2 sigma^2)) sigma sqrt(pi/2) / |r| [erf(|r| (tb - t*) / (sigma sqrt 2)) - erf(..ta..)]."""
    from math import erf, sqrt, pi, exp
    out = np.zeros(rays.shape[0])
    for i, ray in enumerate(rays):
        rng_ = _clip(ray[:3], ray[3:6], ray[6], ray[7])
        if rng_ is None:
            continue
        ta, tb = rng_
        o, r = ray[:3], ray[3:6]
        rr = float(r @ r)
        acc = 0.0
        for pn, wn in zip(p, w):
            v = pn - o
            ts = float(r @ v) / rr
            c = float(v @ v) - float(r @ v) ** 2 / rr
            a = sqrt(rr) / (sigma * sqrt(2.0))
            acc += wn * exp(-c / (2 * sigma ** 2)) * sigma * sqrt(pi / 2) / sqrt(rr) * (erf(a * (tb - ts)) - erf(a * (ta - ts)))
        out[i] = acc
    return out


def test_ray_integral_gaussian_closed_form_and_decay():
    """Gaussian kernel: the series' ray integral approaches the closed-form line integral of the
    direct sum (erf), with the error falling as the order rises."""
    p, w, _ = small_inputs(150, 3, 60, 1)
    rays = _rays(151, 30)
    sigma = 0.15
    ref = _gauss_ray_closed_form(p, w, rays, sigma)
    errs = []
    for order in (2, 4, 6, 8):
        d = oracle.OracleDesc(dim=3, grid=8, order=order, sigma=sigma)
        errs.append(rel(oracle.ray_forward(d, p, w, rays), ref))
    assert errs[-1] <= 2e-3, errs
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_ray_adjoint_identity_and_linearity():
    """<ybar, F(w)> = <F^T(ybar), w> between the ray integral (line2poly) and its adjoint (ray2M
    with line2taylor), which are computed by different formulas; rays wholly outside or of zero
    length contribute nothing."""
    p, w, _ = small_inputs(160, 3, 50, 1)
    rays = _rays(161, 40, spread=1.5)
    rays[0, 6:8] = [0.3, 0.3]                       # zero length
    rays[1, :6] = [2.0, 2.0, 2.0, 1.0, 0.0, 0.0]   # outside the domain
    ybar = np.random.default_rng(162).standard_normal(40)
    d = oracle.OracleDesc(dim=3, grid=8, order=5, sigma=0.12)
    y = oracle.ray_forward(d, p, w, rays)
    wbar, _ = oracle.ray_backward(d, p, w, rays, ybar)
    assert y[0] == 0.0 and y[1] == 0.0
    assert abs(float(ybar @ y) - float(wbar @ w)) <= 1e-12 * (np.abs(ybar) @ np.abs(y))
    y2 = oracle.ray_forward(d, p, 2.0 * w + 1.0, rays)
    y1 = oracle.ray_forward(d, p, np.ones_like(w), rays)
    assert np.max(np.abs(y2 - (2.0 * y + y1))) <= 1e-12 * np.abs(y2).max()


def test_ray_source_gradient_vs_central_differences():
    """pbar of the ray adjoint against central differences of L = <ybar, F(p)> in the source
    positions (sources kept away from cell faces so the binning does not change)."""
    d = oracle.OracleDesc(dim=3, grid=8, order=4, sigma=0.12)
    rng = np.random.default_rng(170)
    p = (rng.integers(0, 8, (20, 3)) + 0.2 + 0.6 * rng.random((20, 3))) / 8.0
    w = rng.standard_normal(20)
    rays = _rays(171, 30)
    ybar = rng.standard_normal(30)
    _, pbar = oracle.ray_backward(d, p, w, rays, ybar)
    for n in range(0, 20, 4):
        for k in range(3):
            eps = 1e-5
            pp, pm = p.copy(), p.copy()
            pp[n, k] += eps
            pm[n, k] -= eps
            fd = (ybar @ oracle.ray_forward(d, pp, w, rays) - ybar @ oracle.ray_forward(d, pm, w, rays)) / (2 * eps)
            assert abs(fd - pbar[n, k]) <= 1e-6 * (np.abs(pbar).max() + 1e-30), (n, k, fd, pbar[n, k])


# ---------------------------------------------------------------- fitted operators (Sec. 3.1)

@pytest.mark.parametrize("name", ["r2", "one_minus_r2_sq", "odd_mixed"])
@pytest.mark.parametrize("dim", [2, 3])
def test_fitted_operators_exact_for_polynomial_kernels(name, dim):
    """A least-squares fit reproduces a polynomial of degree <= rho exactly, so the fitted
    coefficients equal the kernel's derivatives and the fitted transform equals the Taylor one."""
    terms = {m: v for m, v in POLYS_3D[name].items() if dim == 3 or m[2] == 0}
    deg = max(sum(m) for m in terms)
    coef = poly_coef(terms, dim, deg)
    order = max(deg, 4)
    d_fit = oracle.OracleDesc(dim=dim, grid=8, order=order, kernel="poly", poly_coef=coef, fit=True)
    d_tay = oracle.OracleDesc(dim=dim, grid=8, order=order, kernel="poly", poly_coef=coef)
    c = np.array([0.25, -0.125, 0.375][:dim])
    h = 0.125
    a, t = oracle.fit_coeffs(d_fit, c, h), oracle.kernel_derivs(d_tay, c)
    hm = np.array([h ** sum(m) for m in graded(dim, order)])   # compared in the scaled form h^|m| a_m
    assert np.max(np.abs((a - t) * hm)) <= 1e-11 * max(1.0, np.abs(t * hm).max())
    p, w, q = small_inputs(180 + dim, dim, 50, 40)
    y_fit, y_tay = oracle.forward(d_fit, p, w, q), oracle.forward(d_tay, p, w, q)
    assert np.max(np.abs(y_fit - y_tay)) <= 1e-9 * max(1.0, np.abs(y_tay).max())


@pytest.mark.parametrize("dim,order", [(2, 5), (3, 4), (3, 6)])
def test_fitted_operators_solve_the_least_squares_problem(dim, order):
    """The fitted coefficients are the weighted least-squares solution on the tensor
    Gauss-Legendre grid of order + 2 points per dimension over c + [-h, h]^dim: they agree with
    numpy's lstsq on that grid (nodes from numpy), and the residual is orthogonal to the basis."""
    import math
    sigma, h = 0.08, 0.125
    d = oracle.OracleDesc(dim=dim, grid=8, order=order, sigma=sigma, fit=True)
    c = np.array([0.25, 0.125, -0.375][:dim])
    a = oracle.fit_coeffs(d, c, h)
    K = order + 2
    x1, w1 = np.polynomial.legendre.leggauss(K)
    grids = np.meshgrid(*([x1] * dim), indexing="ij")
    xi = np.stack([g.ravel() for g in grids], axis=1)
    wts = np.prod(np.stack(np.meshgrid(*([w1] * dim), indexing="ij"), axis=-1).reshape(-1, dim), axis=1)
    mis = graded(dim, order)
    basis = np.stack([np.prod([xi[:, k] ** m[k] / math.factorial(m[k]) for k in range(dim)], axis=0)
                      for m in mis], axis=1)
    f = np.exp(-np.sum((c[None, :] + h * xi) ** 2, axis=1) / (2 * sigma ** 2))
    sw = np.sqrt(wts)
    b_ref = np.linalg.lstsq(basis * sw[:, None], f * sw, rcond=None)[0]
    b = a * np.array([h ** sum(m) for m in mis])
    assert np.max(np.abs(b - b_ref)) <= 1e-8 * np.abs(b_ref).max()
    resid = f - basis @ b
    assert np.max(np.abs(basis.T @ (wts * resid))) <= 1e-10 * np.abs(f).max()


def test_fitted_operators_reduce_the_error_of_coarse_grids():
    """With cells wider than the kernel (h / sigma 1.25-1.6) the fitted operators bring the
    transform closer to the exact sum than the Taylor coefficients at the same order (the paper's
    reason for the fit, Sec. 3.1)."""
    p, w, q = small_inputs(190, 3, 300, 250)
    for sigma, order in ((0.08, 4), (0.1, 4), (0.08, 6)):
        errs = []
        for fit in (False, True):
            d = oracle.OracleDesc(dim=3, grid=8, order=order, sigma=sigma, fit=fit)
            errs.append(rel(oracle.forward(d, p, w, q), oracle.direct(d, p, w, q)))
        assert errs[1] < 0.6 * errs[0], (sigma, order, errs)
