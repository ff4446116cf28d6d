"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports every
entry point that include/fc2t2.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2111_00110_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fc2t2.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FC2T2_API\s+[\w\s\*]+?\b(fc2t2_\w+)\s*\(", text)))


def test_header_declares_the_binding_surface():
    assert declared_functions() == sorted(capi.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {capi.LIB_PATH}").read()
    exported = set(re.findall(r"\bT (fc2t2_\w+)", out))
    assert set(declared_functions()) <= exported


def test_status_strings(lib):
    for code in capi.STATUS:
        s = lib.fc2t2_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.fc2t2_status_string(0) == b"ok"


def _desc(**kw):
    d = capi.PlanDesc()
    d.dim, d.grid, d.order, d.kernel, d.sigma = 3, 16, 4, 0, 0.05
    d.lo, d.hi, d.channels, d.m2l, d.check_domain = 0.0, 1.0, 1, 0, 0
    d.max_sources, d.max_queries = 100, 100
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value,status", [
    ("dim", 4, 1), ("dim", 1, 1), ("grid", 12, 1), ("grid", 2, 1), ("grid", 2048, 1),
    ("order", 0, 1), ("order", 9, 1), ("sigma", 0.0, 1), ("sigma", -1.0, 1),
    ("hi", 0.0, 1), ("channels", 0, 1), ("channels", 4097, 1), ("m2l", 7, 2), ("fit", 2, 1), ("max_sources", -1, 1), ("kernel", 5, 1),
])
def test_bad_descriptors_are_rejected_on_the_host(lib, field, value, status):
    out = ctypes.c_void_p(123)
    st = lib.fc2t2_plan_create(ctypes.byref(_desc(**{field: value})), ctypes.byref(out))
    assert st == status
    assert out.value is None
    buf = ctypes.create_string_buffer(256)
    assert lib.fc2t2_last_error(buf, 256) == status
    assert len(buf.value) > 0


def test_polynomial_descriptor_needs_a_full_graded_block(lib):
    coef = (ctypes.c_double * 5)(*([1.0] * 5))   # 5 is not C(deg + 3, 3)
    d = _desc(kernel=1, n_poly=5)
    d.poly_coef = ctypes.cast(coef, ctypes.POINTER(ctypes.c_double))
    out = ctypes.c_void_p()
    assert lib.fc2t2_plan_create(ctypes.byref(d), ctypes.byref(out)) == 1


def test_separable_m2l_needs_the_gaussian_in_3d(lib):
    out = ctypes.c_void_p(123)
    assert lib.fc2t2_plan_create(ctypes.byref(_desc(m2l=5, dim=2)), ctypes.byref(out)) == 2
    coef = (ctypes.c_double * 4)(*([1.0] * 4))   # degree-1 polynomial in 3D: C(4, 3) = 4
    d = _desc(kernel=1, n_poly=4, m2l=5)
    d.poly_coef = ctypes.cast(coef, ctypes.POINTER(ctypes.c_double))
    assert lib.fc2t2_plan_create(ctypes.byref(d), ctypes.byref(out)) == 2
    assert out.value is None


def test_null_arguments(lib):
    assert lib.fc2t2_plan_create(None, None) == 1
    assert lib.fc2t2_forward(None, None, None, None, 0, None, 0, None) == 1
    assert lib.fc2t2_backward(None, None, None, None, 0, None, 0, None, None, None) == 1
    assert lib.fc2t2_plan_destroy(None) == 0
    assert lib.fc2t2_expand(None, None, None, None, 0) == 1
    assert lib.fc2t2_evaluate(None, None, None, 0, 0, None) == 1
    assert lib.fc2t2_evaluate_grid(None, None, None, None, 0, None) == 1


def test_fitted_operators_exclude_the_separable_m2l(lib):
    out = ctypes.c_void_p(123)
    assert lib.fc2t2_plan_create(ctypes.byref(_desc(m2l=5, fit=1)), ctypes.byref(out)) == 2
    assert out.value is None


def test_m2l_form_names_match_the_header():
    """The binding's M2L form names map to the header's enum values (OCCUPIED included)."""
    text = open(HEADER).read()
    vals = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"FC2T2_M2L_(\w+)\s*=\s*(\d+)", text)}
    assert vals == capi.M2L_PREC
    assert vals["occupied"] == 6


@pytest.mark.parametrize("tile", [1, 8, 48, 128, -16])
def test_tile_values_are_checked(lib, tile):
    out = ctypes.c_void_p(123)
    assert lib.fc2t2_plan_create(ctypes.byref(_desc(m2l=5, tile=tile)), ctypes.byref(out)) == 1
    assert out.value is None


@pytest.mark.parametrize("dim,kernel,fit", [(3, 0, 0), (2, 0, 1), (3, 1, 0)])
def test_occupied_m2l_descriptors_pass_validation(lib, dim, kernel, fit):
    """The occupied-cell M2L takes any kernel, 2D and 3D, and fitted operators: such a descriptor
    passes the host checks (without a GPU the plan then fails at its first device step, with a
    CUDA or memory error; with one it is built and released)."""
    coef = (ctypes.c_double * 4)(*([1.0] * 4))   # degree-1 polynomial in 3D: C(4, 3) = 4
    d = _desc(dim=dim, kernel=kernel, fit=fit, m2l=6)
    if kernel == 1:
        d.poly_coef = ctypes.cast(coef, ctypes.POINTER(ctypes.c_double))
        d.n_poly = 4
    out = ctypes.c_void_p(123)
    st = lib.fc2t2_plan_create(ctypes.byref(d), ctypes.byref(out))
    assert st in (0, 3, 5), st
    if st == 0:
        lib.fc2t2_plan_destroy(out)
    else:
        assert out.value is None
