"""ctypes binding of the C ABI declared in ``include/fc2t2.h``.

Argument marshalling only: every step of the transform runs in the CUDA library
``_build/libfc2t2.so``.  Importing this module never falls back to anything else: if the
library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfc2t2.so")

FC2T2_OK = 0
STATUS = {
    0: "FC2T2_OK",
    1: "FC2T2_ERR_INVALID_ARG",
    2: "FC2T2_ERR_UNSUPPORTED",
    3: "FC2T2_ERR_OOM",
    4: "FC2T2_ERR_DOMAIN",
    5: "FC2T2_ERR_CUDA",
    6: "FC2T2_ERR_TIMEOUT",
}
KERNELS = {"gaussian": 0, "poly": 1}
M2L_PREC = {"fp32": 0, "tf32": 1, "bf16": 2, "tf32x3": 3, "bf16x3": 4, "separable": 5, "occupied": 6}

# every entry point declared in include/fc2t2.h
EXPORTS = (
    "fc2t2_plan_create",
    "fc2t2_plan_destroy",
    "fc2t2_forward",
    "fc2t2_backward",
    "fc2t2_status_string",
    "fc2t2_last_error",
    "fc2t2_profile_enable",
    "fc2t2_profile_read",
    "fc2t2_forward_noalloc",
    "fc2t2_forward_batched",
    "fc2t2_backward_batched",
    "fc2t2_backward_batched_reuse",
    "fc2t2_plan_query",
    "fc2t2_plan_check",
    "fc2t2_direct",
    "fc2t2_backward_q",
    "fc2t2_backward_reuse",
    "fc2t2_expand",
    "fc2t2_evaluate",
    "fc2t2_evaluate_grid",
    "fc2t2_ray_forward",
    "fc2t2_ray_backward",
)
# what fc2t2_evaluate returns per point and channel
EVAL = {"value": 0, "partials": 1, "partials2": 2}
STAGES = ("sort", "p2m", "m2m", "m2l", "l2l", "l2p", "m2l_pack")


class PlanDesc(ctypes.Structure):
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
        ("channels", ctypes.c_int),
        ("m2l", ctypes.c_int),
        ("check_domain", ctypes.c_int),
        ("max_sources", ctypes.c_int64),
        ("max_queries", ctypes.c_int64),
        ("fit", ctypes.c_int),
        ("tile", ctypes.c_int),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("coefficients", ctypes.c_int),
        ("m2l_tensor_cores", ctypes.c_int),
        ("m2l_cell_pairs", ctypes.c_double),
        ("m2l_useful_flops", ctypes.c_double),
        ("m2l_issued_flops", ctypes.c_double),
        ("device_bytes", ctypes.c_int64),
        ("m2l_classes_per_cta", ctypes.c_int),
    ]


class FC2T2Error(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FileNotFoundError(
                f"{path} is missing: build it with `python -m paper_2111_00110_gb300.build`")
        lib = ctypes.CDLL(path)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.fc2t2_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(ctypes.c_void_p)]
        lib.fc2t2_plan_destroy.argtypes = [vp]
        lib.fc2t2_forward.argtypes = [vp, vp, vp, vp, i64, vp, i64, vp]
        lib.fc2t2_backward.argtypes = [vp, vp, vp, vp, i64, vp, i64, vp, vp, vp]
        lib.fc2t2_status_string.argtypes = [ctypes.c_int]
        lib.fc2t2_status_string.restype = ctypes.c_char_p
        lib.fc2t2_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
        lib.fc2t2_profile_enable.argtypes = [vp, ctypes.c_int]
        lib.fc2t2_profile_read.argtypes = [vp, vp, vp, ctypes.c_int]
        lib.fc2t2_forward_noalloc.argtypes = [ctypes.POINTER(PlanDesc), vp, vp, vp, i64, vp, i64, vp]
        lib.fc2t2_forward_batched.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.fc2t2_backward_batched.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.fc2t2_backward_batched_reuse.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.fc2t2_plan_query.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        lib.fc2t2_plan_check.argtypes = [vp, vp]
        lib.fc2t2_direct.argtypes = [ctypes.POINTER(PlanDesc), vp, vp, vp, i64, vp, i64, vp]
        lib.fc2t2_backward_q.argtypes = [vp, vp, vp, vp, i64, vp, i64, vp, vp]
        lib.fc2t2_backward_reuse.argtypes = [vp, vp, vp, vp, i64, vp, i64, vp, vp, vp]
        lib.fc2t2_expand.argtypes = [vp, vp, vp, vp, i64]
        lib.fc2t2_evaluate.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp]
        lib.fc2t2_evaluate_grid.argtypes = [vp, vp, vp, vp, ctypes.c_int, vp]
        lib.fc2t2_ray_forward.argtypes = [vp, vp, vp, vp, i64, vp, i64, vp]
        lib.fc2t2_ray_backward.argtypes = [vp, vp, vp, vp, i64, vp, i64, vp, vp, vp]
        for name in ("fc2t2_plan_create", "fc2t2_plan_destroy", "fc2t2_forward", "fc2t2_backward",
                     "fc2t2_last_error", "fc2t2_profile_enable", "fc2t2_profile_read",
                     "fc2t2_forward_noalloc", "fc2t2_forward_batched", "fc2t2_backward_batched",
                     "fc2t2_backward_batched_reuse", "fc2t2_plan_query"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def check(status: int):
    if status != FC2T2_OK:
        lib = load()
        buf = ctypes.create_string_buffer(512)
        lib.fc2t2_last_error(buf, 512)
        raise FC2T2Error(status, buf.value.decode(errors="replace"))


def plan_create(desc: PlanDesc) -> int:
    out = ctypes.c_void_p()
    check(load().fc2t2_plan_create(ctypes.byref(desc), ctypes.byref(out)))
    return out.value


def plan_destroy(plan: int) -> None:
    check(load().fc2t2_plan_destroy(plan))


def forward(plan: int, stream: int, p: int, w: int, N: int, q: int, M: int, y: int) -> None:
    check(load().fc2t2_forward(plan, stream, p, w, N, q, M, y))


def backward(plan: int, stream: int, p: int, w: int, N: int, q: int, M: int, ybar: int,
             wbar: int, pbar: int) -> None:
    check(load().fc2t2_backward(plan, stream, p, w, N, q, M, ybar, wbar, pbar))


def backward_reuse(plan: int, stream: int, p: int, w: int, N: int, q: int, M: int, ybar: int, wbar: int,
                   pbar: int) -> None:
    check(load().fc2t2_backward_reuse(plan, stream, p, w, N, q, M, ybar, wbar, pbar))


def backward_q(plan: int, stream: int, p: int, w: int, N: int, q: int, M: int, ybar: int, qbar: int) -> None:
    check(load().fc2t2_backward_q(plan, stream, p, w, N, q, M, ybar, qbar))


def expand(plan: int, stream: int, p: int, w: int, N: int) -> None:
    """Expand (p, w) into the plan for the accessor (device pointers)."""
    check(load().fc2t2_expand(plan, stream, p, w, N))


def evaluate(plan: int, stream: int, q: int, M: int, what: str, out: int) -> None:
    """Value / first / second partials of the held expansion at M points (device pointers)."""
    check(load().fc2t2_evaluate(plan, stream, q, M, EVAL[what], out))


def evaluate_grid(plan: int, stream: int, axes, counts, what: str, out: int) -> None:
    """The held expansion on the meshgrid of per-axis coordinates: axes are device pointers,
    counts their lengths (host lists, one entry per dimension)."""
    ax = (ctypes.c_void_p * len(axes))(*[a or None for a in axes])
    n = (ctypes.c_int64 * len(counts))(*counts)
    check(load().fc2t2_evaluate_grid(plan, stream, ctypes.addressof(ax), ctypes.addressof(n), EVAL[what], out))


def ray_forward(plan: int, stream: int, p: int, w: int, N: int, rays: int, R: int, y: int) -> None:
    """Integrals of the series along R rays [R][8] (device pointers)."""
    check(load().fc2t2_ray_forward(plan, stream, p, w, N, rays, R, y))


def ray_backward(plan: int, stream: int, p: int, w: int, N: int, rays: int, R: int, ybar: int, wbar: int,
                 pbar: int) -> None:
    """Adjoint of ray_forward: (wbar, pbar) at the sources for the cotangent ybar (device pointers)."""
    check(load().fc2t2_ray_backward(plan, stream, p, w, N, rays, R, ybar, wbar, pbar))


def direct(desc: PlanDesc, stream: int, p: int, w: int, N: int, q: int, M: int, y: int) -> None:
    """Brute-force sum of Eq. 1 on the device (device pointers)."""
    check(load().fc2t2_direct(ctypes.byref(desc), stream, p, w, N, q, M, y))


def plan_check(plan: int, stream: int) -> None:
    """Synchronise the stream; raise on a device-side timeout or (check_domain) domain error."""
    check(load().fc2t2_plan_check(plan, stream))


def profile_enable(plan: int, enable: bool) -> None:
    check(load().fc2t2_profile_enable(plan, 1 if enable else 0))


def profile_read(plan: int, reset: bool = False):
    """Per-stage accumulated device milliseconds and kernel launches (dicts by stage name)."""
    ms = (ctypes.c_double * len(STAGES))()
    n = (ctypes.c_int64 * len(STAGES))()
    check(load().fc2t2_profile_read(plan, ctypes.addressof(ms), ctypes.addressof(n), 1 if reset else 0))
    return dict(zip(STAGES, list(ms))), dict(zip(STAGES, list(n)))


def plan_query(plan: int) -> dict:
    info = PlanInfo()
    check(load().fc2t2_plan_query(plan, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in PlanInfo._fields_}


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[p or None for p in ptrs])
    return arr


def forward_batched(plans, stream, p, w, N, q, M, y) -> None:
    """Batched forward: lists of plan handles, device pointers and sizes, one entry per instance."""
    n = len(plans)
    i64 = ctypes.c_int64 * n
    check(load().fc2t2_forward_batched(n, ctypes.addressof(_keep(_ptr_array(plans))), stream,
                                       ctypes.addressof(_keep(_ptr_array(p))), ctypes.addressof(_keep(_ptr_array(w))),
                                       ctypes.addressof(_keep(i64(*N))), ctypes.addressof(_keep(_ptr_array(q))),
                                       ctypes.addressof(_keep(i64(*M))), ctypes.addressof(_keep(_ptr_array(y)))))
    _kept.clear()


def backward_batched(plans, stream, p, w, N, q, M, ybar, wbar, pbar, reuse: bool = False) -> None:
    n = len(plans)
    i64 = ctypes.c_int64 * n
    fn = load().fc2t2_backward_batched_reuse if reuse else load().fc2t2_backward_batched
    check(fn(n, ctypes.addressof(_keep(_ptr_array(plans))), stream,
                                        ctypes.addressof(_keep(_ptr_array(p))), ctypes.addressof(_keep(_ptr_array(w))),
                                        ctypes.addressof(_keep(i64(*N))), ctypes.addressof(_keep(_ptr_array(q))),
                                        ctypes.addressof(_keep(i64(*M))), ctypes.addressof(_keep(_ptr_array(ybar))),
                                        ctypes.addressof(_keep(_ptr_array(wbar))), ctypes.addressof(_keep(_ptr_array(pbar)))))
    _kept.clear()


_kept = []


def _keep(obj):
    _kept.append(obj)
    return obj
