"""The allocation-free forward transform (fc2t2_forward_noalloc) against the planned one.

fc2t2_forward_noalloc serves callers that cannot call cudaMalloc when they need a transform
(for example inside a framework that owns all device memory, or a real-time loop that must
not allocate); it keeps its intermediates in a static device array of the library.  This file
is collected last so that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

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


def noalloc_forward(lib, wl, stream):
    p, w, q = (torch.from_numpy(a).cuda() for a in (wl.p, wl.w, wl.q))
    y = torch.full((wl.M,), float("nan"), device="cuda")
    d = desc_for(wl)
    st = lib.fc2t2_forward_noalloc(ctypes.byref(d), stream, p.data_ptr(), w.data_ptr(), wl.N,
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


def test_noalloc_matches_planned_forward_twice(lib):
    stream = torch.cuda.current_stream().cuda_stream
    # two different problems back to back: the shared array must not carry state over
    first = workloads.uniform(901, 3, 20000, 15000, 16, 4, 0.06)
    second = workloads.uniform(902, 2, 30000, 25000, 64, 3, 0.03)
    for wl in (first, second):
        y_na = noalloc_forward(lib, wl, stream)
        y_pl = planned_forward(wl)
        assert np.all(np.isfinite(y_na))
        assert rel_l2(y_na, y_pl) <= REL_L2


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
