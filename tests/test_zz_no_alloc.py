"""The allocation-free forward transform (fc2t2_forward_noalloc) against the planned one and the
oracle.

fc2t2_forward_noalloc serves callers that cannot call cudaMalloc when they need a transform
(for example inside a framework that owns all device memory, or a real-time loop that must
not allocate); it keeps its intermediates in a static device array of the library.  This file
is collected last so that a run stopping at the first failure has already run every other test.

Tolerance: the FP32 bar of the parity tests (relative L2 <= 1e-5).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2111_00110_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL_L2 = 1e-5      # the FP32 tolerance of the parity tests


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_00110_gb300 import build
    build.build()
    from paper_2111_00110_gb300 import capi
    return capi.load()


def desc_for(wl):
    from paper_2111_00110_gb300 import capi
    d = capi.PlanDesc()
    d.dim, d.grid, d.order, d.kernel, d.sigma = wl.dim, wl.grid, wl.order, 0, wl.sigma
    d.lo, d.hi, d.channels, d.m2l, d.check_domain = 0.0, 1.0, 1, 0, 0
    d.max_sources, d.max_queries = wl.N, wl.M
    return d


def noalloc_forward(lib, wl, stream, n_src=None):
    """One call on `stream` (a torch.cuda.Stream or None for the current one)."""
    n = wl.N if n_src is None else n_src
    s = torch.cuda.current_stream() if stream is None else stream
    with torch.cuda.stream(s):
        p, w, q = (torch.from_numpy(a).cuda() for a in (wl.p, wl.w, wl.q))
        y = torch.full((wl.M,), float("nan"), device="cuda")
        d = desc_for(wl)
        st = lib.fc2t2_forward_noalloc(ctypes.byref(d), s.cuda_stream, p.data_ptr(), w.data_ptr(), n,
                                       q.data_ptr(), wl.M, y.data_ptr())
    assert st == 0, st
    torch.cuda.synchronize()
    return y.cpu().numpy()


def planned_forward(wl):
    from paper_2111_00110_gb300.transform import Plan
    plan = Plan(wl.dim, wl.grid, wl.order, wl.sigma, m2l="fp32", max_sources=wl.N, max_queries=wl.M)
    p, w, q = (torch.from_numpy(a).cuda() for a in (wl.p, wl.w, wl.q))
    y = plan.forward(p, w, q)
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    plan.close()
    return out


def oracle_forward(wl, sel=None):
    d = oracle.OracleDesc(dim=wl.dim, grid=wl.grid, order=wl.order, sigma=wl.sigma)
    f = lambda a: np.asarray(a, dtype=np.float64)
    return oracle.forward(d, f(wl.p), f(wl.w), f(wl.q), sel=sel)


def test_noalloc_matches_planned_forward_twice(lib):
    # two different problems back to back: the shared array must not carry state over
    first = workloads.uniform(901, 3, 20000, 15000, 16, 4, 0.06)
    second = workloads.uniform(902, 2, 30000, 25000, 64, 3, 0.03)
    for wl in (first, second):
        y_na = noalloc_forward(lib, wl, None)
        y_pl = planned_forward(wl)
        assert np.all(np.isfinite(y_na))
        assert rel_l2(y_na, y_pl) <= REL_L2
        assert rel_l2(y_na, oracle_forward(wl)) <= REL_L2


@pytest.mark.parametrize("dim,grid", [(3, 16), (2, 64)])
def test_noalloc_at_its_limits(lib, dim, grid):
    """N = M = 65536 (the largest sort), order 4 (the largest rows) and 4096 finest cells; 64^2
    has five levels, the most the array holds.  Run on a stream other than the current one, and
    checked against the oracle at 4096 seeded queries."""
    wl = workloads.uniform(904 + dim, dim, 65536, 65536, grid, 4, 1.3 / grid)
    side = torch.cuda.Stream()
    y_na = noalloc_forward(lib, wl, side)
    sel = np.sort(np.random.default_rng(905).choice(wl.M, size=4096, replace=False))
    assert np.all(np.isfinite(y_na))
    assert rel_l2(y_na[sel], oracle_forward(wl, sel=sel)) <= REL_L2
    assert rel_l2(y_na, planned_forward(wl)) <= REL_L2


def test_noalloc_dense_cells(lib):
    """65536 sources in 64 finest cells (about 1000 per cell: most go through P2M's overflow
    kernel), against the planned forward and the oracle."""
    wl = workloads.uniform(907, 3, 65536, 4000, 4, 4, 0.4)
    y_na = noalloc_forward(lib, wl, None)
    assert rel_l2(y_na, planned_forward(wl)) <= REL_L2
    assert rel_l2(y_na, oracle_forward(wl)) <= REL_L2


def test_noalloc_without_sources_gives_zero(lib):
    wl = workloads.uniform(906, 3, 1000, 3000, 16, 4, 0.06)
    noalloc_forward(lib, wl, None)                    # leaves nonzero coefficients in the array
    y = noalloc_forward(lib, wl, None, n_src=0)
    assert np.all(y == 0.0)


def test_noalloc_rejects_requests_beyond_its_limits(lib):
    wl = workloads.uniform(903, 3, 100, 100, 32, 4, 0.05)        # 32^3 cells > 4096
    d = desc_for(wl)
    st = lib.fc2t2_forward_noalloc(ctypes.byref(d), None, 1, 1, wl.N, 1, wl.M, 1)
    assert st == 1
    buf = ctypes.create_string_buffer(256)
    lib.fc2t2_last_error(buf, 256)
    assert b"4096" in buf.value
    d.grid, d.order = 16, 5
    assert lib.fc2t2_forward_noalloc(ctypes.byref(d), None, 1, 1, wl.N, 1, wl.M, 1) == 1
    d.order = 4
    assert lib.fc2t2_forward_noalloc(ctypes.byref(d), None, 1, 1, 70000, 1, wl.M, 1) == 1
    d.check_domain = 1                                             # never reported on this path
    assert lib.fc2t2_forward_noalloc(ctypes.byref(d), None, 1, 1, wl.N, 1, wl.M, 1) == 2
