"""FP64 CPU oracle for the FC2T2 transform (arXiv 2111.00110, Sec. 3 and Sec. 4.1).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path: the transform lives in ``fc2t2_oracle.c`` (plain C, FP64), built
here with gcc and loaded through ctypes.

Public functions (all arrays are numpy, float64 unless stated):

* ``forward(desc, p, w, q, sel=None, src_cell=None, tgt_cell=None)`` -> y
    the multi-level approximation of Eq. 1, y_m = sum_n psi(p_n - q_m) w_n.
* ``backward(desc, p, w, q, ybar, sel=None, ...)`` -> (wbar, pbar)
    Sec. 4.1: wbar = f(p; q, ybar) (the transposed transform) and
    pbar = w * grad f(p; q, ybar).
* ``backward_q(desc, p, w, q, ybar, sel=None, ...)`` -> qbar (gradient at the queries).
* ``partials(desc, p, w, q, sel=None, ...)`` -> (value, first partials, second partials) of the
    forward series at the queries (the accessor of Sec. 3, "How to use the implementation?").
* ``ray_forward(desc, p, w, rays)`` / ``ray_backward(desc, p, w, rays, ybar)`` -> integrals of the
    series along rays (Sec. 6, integral-implicit layer) and their adjoint (w̄, p̄).
* ``direct(desc, p, w, q, sel=None)`` -> exact O(NM) sum of Eq. 1.
* ``direct_grad(desc, p, w, q, ybar, sel=None)`` -> (wbar, pbar) of <ybar, y> for that exact sum
    (the dense form of Sec. 4.1's Jacobian vector product).
* ``kernel_derivs(desc, c)`` -> d^m psi(c), |m| <= order, graded order.
* ``fit_coeffs(desc, c, h)`` -> the least-squares fitted replacements of d^m psi(c) (``fit=True``).
* ``multi_indices(dim, order)`` -> exponents [P, dim], graded order.
* ``bin_cells(desc, x)`` -> finest-level linear cell index per point (FP32 rule).

``desc`` is an :class:`OracleDesc`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fc2t2_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfc2t2_oracle.so")

_lock = threading.Lock()
_lib = None

FAULTS = {
    "none": 0,
    "drop_sign": 1,
    "drop_top_term": 2,
    "parity": 3,
    "no_l2l": 4,
    "m2m_sign": 5,
    "no_self": 6,
    "transpose": 7,
}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("grid", ctypes.c_int),
        ("order", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("poly_coef", ctypes.POINTER(ctypes.c_double)),
        ("n_poly", ctypes.c_int),
        ("lo", ctypes.c_double),
        ("hi", ctypes.c_double),
        ("fit", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_num_coeffs.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_num_coeffs.restype = ctypes.c_int
            lib.orc_multi_indices.argtypes = [ctypes.c_int, ctypes.c_int, P]
            lib.orc_multi_indices.restype = ctypes.c_int
            lib.orc_kernel_derivs.argtypes = [ctypes.POINTER(_Desc), P, P]
            lib.orc_kernel_derivs.restype = ctypes.c_int
            lib.orc_fit_coeffs.argtypes = [ctypes.POINTER(_Desc), P, ctypes.c_double, P]
            lib.orc_fit_coeffs.restype = ctypes.c_int
            lib.orc_bin.argtypes = [ctypes.POINTER(_Desc), P, ctypes.c_int64, P]
            lib.orc_bin.restype = ctypes.c_int
            lib.orc_transform.argtypes = [ctypes.POINTER(_Desc),
                                          P, P, ctypes.c_int64, P,
                                          P, ctypes.c_int64, P,
                                          P, ctypes.c_int64,
                                          P, P, ctypes.c_int]
            lib.orc_transform.restype = ctypes.c_int
            lib.orc_transform_h.argtypes = [ctypes.POINTER(_Desc),
                                            P, P, ctypes.c_int64, P,
                                            P, ctypes.c_int64, P,
                                            P, ctypes.c_int64,
                                            P, P, P, ctypes.c_int]
            lib.orc_transform_h.restype = ctypes.c_int
            lib.orc_ray_forward.argtypes = [ctypes.POINTER(_Desc), P, P, ctypes.c_int64, P, P, P, P,
                                            ctypes.c_int64, P]
            lib.orc_ray_forward.restype = ctypes.c_int
            lib.orc_ray_backward.argtypes = [ctypes.POINTER(_Desc), P, P, P, P, P, ctypes.c_int64, P,
                                             ctypes.c_int64, P, P, P]
            lib.orc_ray_backward.restype = ctypes.c_int
            lib.orc_direct.argtypes = [ctypes.POINTER(_Desc), P, P, ctypes.c_int64,
                                       P, ctypes.c_int64, P, ctypes.c_int64, P]
            lib.orc_direct.restype = ctypes.c_int
            lib.orc_direct_grad.argtypes = [ctypes.POINTER(_Desc), P, P, ctypes.c_int64,
                                            P, P, ctypes.c_int64, P, ctypes.c_int64, P, P]
            lib.orc_direct_grad.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class OracleDesc:
    """Transform description: dimension, finest grid, order, kernel, domain."""
    dim: int
    grid: int
    order: int
    kernel: str = "gaussian"          # "gaussian" or "poly"
    sigma: float = 0.05
    poly_coef: Optional[Sequence[float]] = None
    lo: float = 0.0
    hi: float = 1.0
    fit: bool = False                 # least-squares fitted M2L coefficients (Sec. 3.1)
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Desc:
        d = _Desc()
        d.dim, d.grid, d.order = self.dim, self.grid, self.order
        d.kernel = 0 if self.kernel == "gaussian" else 1
        d.sigma = float(self.sigma)
        if self.poly_coef is not None:
            arr = np.ascontiguousarray(self.poly_coef, dtype=np.float64)
            self._keep = [arr]
            d.poly_coef = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            d.n_poly = arr.size
        else:
            d.poly_coef = None
            d.n_poly = 0
        d.lo, d.hi = float(self.lo), float(self.hi)
        d.fit = 1 if self.fit else 0
        return d


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def num_coeffs(dim: int, order: int) -> int:
    return _load().orc_num_coeffs(dim, order)


def multi_indices(dim: int, order: int) -> np.ndarray:
    P = num_coeffs(dim, order)
    out = np.zeros((P, dim), dtype=np.int32)
    _load().orc_multi_indices(dim, order, out.ctypes.data)
    return out


def kernel_derivs(desc: OracleDesc, c) -> np.ndarray:
    c = _f64(c, (desc.dim,))
    out = np.zeros(num_coeffs(desc.dim, desc.order), dtype=np.float64)
    cd = desc.c()
    _load().orc_kernel_derivs(ctypes.byref(cd), c.ctypes.data, out.ctypes.data)
    return out


def fit_coeffs(desc: OracleDesc, c, h: float) -> np.ndarray:
    """The least-squares fitted coefficients a_m (|m| <= order, graded) that replace d^m psi(c) in
    M2L for cells of width h (Sec. 3.1; the fit is over the separations c + [-h, h]^dim)."""
    c = _f64(c, (desc.dim,))
    out = np.zeros(num_coeffs(desc.dim, desc.order), dtype=np.float64)
    cd = desc.c()
    _load().orc_fit_coeffs(ctypes.byref(cd), c.ctypes.data, float(h), out.ctypes.data)
    return out


def bin_cells(desc: OracleDesc, x) -> np.ndarray:
    x = _f64(x).reshape(-1, desc.dim)
    out = np.zeros(x.shape[0], dtype=np.int32)
    cd = desc.c()
    _load().orc_bin(ctypes.byref(cd), x.ctypes.data, x.shape[0], out.ctypes.data)
    return out


def transform(desc: OracleDesc, src, wt, tgt, sel=None, src_cell=None, tgt_cell=None,
              want_grad: bool = False, fault: str = "none", want_hess: bool = False):
    """Series value (and gradient) at targets of the transform of (src, wt); with ``want_hess``
    returns (value, gradient, second partials [n, dim(dim+1)/2])."""
    D = desc.dim
    src = _f64(src).reshape(-1, D)
    tgt = _f64(tgt).reshape(-1, D)
    wt = _f64(wt).reshape(-1)
    assert wt.shape[0] == src.shape[0]
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        n_sel = sel.shape[0]
    else:
        n_sel = tgt.shape[0]
    if src_cell is not None:
        src_cell = np.ascontiguousarray(src_cell, dtype=np.int32)
    if tgt_cell is not None:
        tgt_cell = np.ascontiguousarray(tgt_cell, dtype=np.int32)
    val = np.zeros(n_sel, dtype=np.float64)
    grad = np.zeros((n_sel, D), dtype=np.float64) if (want_grad or want_hess) else None
    hess = np.zeros((n_sel, D * (D + 1) // 2), dtype=np.float64) if want_hess else None
    cd = desc.c()
    rc = _load().orc_transform_h(ctypes.byref(cd), src.ctypes.data, wt.ctypes.data, src.shape[0],
                                 _ptr(src_cell), tgt.ctypes.data, tgt.shape[0], _ptr(tgt_cell),
                                 _ptr(sel), n_sel if sel is not None else -1,
                                 val.ctypes.data, _ptr(grad), _ptr(hess), FAULTS[fault])
    if rc != 0:
        raise ValueError(f"oracle transform rejected its arguments (rc={rc})")
    if want_hess:
        return val, grad, hess
    return (val, grad) if want_grad else val


def forward(desc: OracleDesc, p, w, q, sel=None, src_cell=None, tgt_cell=None, fault="none"):
    """y_m ~ sum_n psi(p_n - q_m) w_n (Eq. 1) through P2M, M2M, M2L, L2L, L2P."""
    return transform(desc, p, w, q, sel=sel, src_cell=src_cell, tgt_cell=tgt_cell, fault=fault)


def backward(desc: OracleDesc, p, w, q, ybar, sel=None, src_cell=None, tgt_cell=None,
             fault="none"):
    """Sec. 4.1: wbar = f(p; q, ybar), pbar = w * grad_x f(x; q, ybar)|_{x=p}.

    ``sel`` selects source indices n at which wbar/pbar are evaluated; ``src_cell`` and
    ``tgt_cell`` are the frozen cells of p and q (in the roles of the forward pass)."""
    w = _f64(w).reshape(-1)
    val, grad = transform(desc, q, ybar, p, sel=sel, src_cell=tgt_cell, tgt_cell=src_cell,
                          want_grad=True, fault=fault)
    ws = w if sel is None else w[np.asarray(sel, dtype=np.int64)]
    return val, grad * ws[:, None]


def backward_q(desc: OracleDesc, p, w, q, ybar, sel=None, src_cell=None, tgt_cell=None, fault="none"):
    """qbar_m = ybar_m * grad_x f(x; p, w)|_{x=q_m}: the derivative of the forward local series at
    the (selected) queries, the binning of q held fixed (as for pbar, Sec. 4.1)."""
    ybar = _f64(ybar).reshape(-1)
    _, grad = transform(desc, p, w, q, sel=sel, src_cell=src_cell, tgt_cell=tgt_cell, want_grad=True,
                        fault=fault)
    yb = ybar if sel is None else ybar[np.asarray(sel, dtype=np.int64)]
    return grad * yb[:, None]


def partials(desc: OracleDesc, p, w, q, sel=None, src_cell=None, tgt_cell=None, fault="none"):
    """The accessor's queries of the forward series of (p, w) at the (selected) queries (Sec. 3,
    "How to use the implementation?"): (value [n], first partials [n, dim], second partials
    [n, dim(dim+1)/2] for i <= k, row-major), the binning of q held fixed."""
    return transform(desc, p, w, q, sel=sel, src_cell=src_cell, tgt_cell=tgt_cell, want_hess=True,
                     fault=fault)


def _rays(rays):
    """Split rays [R, 8] = (origin (3), direction (3), t0, t1) into contiguous float64 arrays."""
    r = _f64(rays).reshape(-1, 8)
    return (np.ascontiguousarray(r[:, 0:3]), np.ascontiguousarray(r[:, 3:6]),
            np.ascontiguousarray(r[:, 6]), np.ascontiguousarray(r[:, 7]))


def ray_forward(desc: OracleDesc, p, w, rays):
    """Sec. 6, integral-implicit layer ("Line Integral"): y_q = int_{t0}^{t1} f(o_q + t r_q) dt of the series of (p, w),
    for rays [R, 8] (origin, direction, t0, t1; the part outside the domain box is dropped), through
    the cells each ray crosses (line2poly).  3D."""
    D = desc.dim
    p = _f64(p).reshape(-1, D)
    w = _f64(w).reshape(-1)
    o, r, t0, t1 = _rays(rays)
    y = np.zeros(o.shape[0], dtype=np.float64)
    cd = desc.c()
    rc = _load().orc_ray_forward(ctypes.byref(cd), p.ctypes.data, w.ctypes.data, p.shape[0], o.ctypes.data,
                                 r.ctypes.data, t0.ctypes.data, t1.ctypes.data, o.shape[0], y.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle ray transform rejected its arguments (rc={rc})")
    return y


def ray_backward(desc: OracleDesc, p, w, rays, ybar, src_cell=None):
    """Adjoint of ``ray_forward`` for the cotangent ybar [R]: the rays become the sources (ray2M,
    line2taylor) with weights ybar and p the targets; returns (wbar [N], pbar = w * gradient [N, 3]),
    the binning of p held fixed when ``src_cell`` is given."""
    D = desc.dim
    p = _f64(p).reshape(-1, D)
    w = _f64(w).reshape(-1)
    yb = _f64(ybar).reshape(-1)
    o, r, t0, t1 = _rays(rays)
    val = np.zeros(p.shape[0], dtype=np.float64)
    grad = np.zeros((p.shape[0], D), dtype=np.float64)
    if src_cell is not None:
        src_cell = np.ascontiguousarray(src_cell, dtype=np.int32)
    cd = desc.c()
    rc = _load().orc_ray_backward(ctypes.byref(cd), o.ctypes.data, r.ctypes.data, t0.ctypes.data, t1.ctypes.data,
                                  yb.ctypes.data, o.shape[0], p.ctypes.data, p.shape[0], _ptr(src_cell),
                                  val.ctypes.data, grad.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle ray transform rejected its arguments (rc={rc})")
    return val, grad * w[:, None]


def direct(desc: OracleDesc, p, w, q, sel=None):
    """Exact O(NM) sum of Eq. 1 at the selected targets."""
    D = desc.dim
    p = _f64(p).reshape(-1, D)
    q = _f64(q).reshape(-1, D)
    w = _f64(w).reshape(-1)
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        n_sel = sel.shape[0]
    else:
        n_sel = q.shape[0]
    val = np.zeros(n_sel, dtype=np.float64)
    cd = desc.c()
    _load().orc_direct(ctypes.byref(cd), p.ctypes.data, w.ctypes.data, p.shape[0],
                       q.ctypes.data, q.shape[0], _ptr(sel), n_sel if sel is not None else -1,
                       val.ctypes.data)
    return val


def direct_grad(desc: OracleDesc, p, w, q, ybar, sel=None):
    """Gradients of <ybar, y> for the exact sum y_m = sum_n psi(p_n - q_m) w_n (Eq. 1), at the
    selected sources: wbar_n = sum_m ybar_m psi(p_n - q_m) and
    pbar_n = w_n sum_m ybar_m grad psi(p_n - q_m) (Sec. 4.1 applied to the dense sum)."""
    D = desc.dim
    p = _f64(p).reshape(-1, D)
    q = _f64(q).reshape(-1, D)
    w = _f64(w).reshape(-1)
    yb = _f64(ybar).reshape(-1)
    assert yb.shape[0] == q.shape[0] and w.shape[0] == p.shape[0]
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        n_sel = sel.shape[0]
    else:
        n_sel = p.shape[0]
    wbar = np.zeros(n_sel, dtype=np.float64)
    pbar = np.zeros((n_sel, D), dtype=np.float64)
    cd = desc.c()
    _load().orc_direct_grad(ctypes.byref(cd), p.ctypes.data, w.ctypes.data, p.shape[0], q.ctypes.data,
                            yb.ctypes.data, q.shape[0], _ptr(sel), n_sel if sel is not None else -1,
                            wbar.ctypes.data, pbar.ctypes.data)
    return wbar, pbar
