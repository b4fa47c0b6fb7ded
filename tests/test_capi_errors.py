"""Argument errors of the C interface that are decided on the host, before
any device call: lq_create's checks of the lattice (section III.B) and of
the material (a nematic minimum S0 of Eq. (S0def) must exist; the one-
constant form has L2 = L3 = L4 = L6 = 0), the fault-injection switch and
the Frank-constant helper.  Each returns LQ_EINVAL, writes no handle and
leaves a message naming the problem.  These run without a GPU."""
import ctypes as C

import pytest

from paper_1911_07045_b300 import lqmin, synth


@pytest.fixture(scope="module")
def lib():
    from paper_1911_07045_b300 import build
    build.build()
    return lqmin.load()


def lattice(nx=8, ny=8, nz=8, spacing=1.0):
    return lqmin.Lattice(nx, ny, nz, spacing, (C.c_int * 3)(1, 1, 1))


def material(A=synth.A_5CB, B=synth.B_5CB, C_=synth.C_5CB, L=(2.32, 0.5, 0.3), n_constants=3,
             L4=0.0, L6=0.0):
    return lqmin.Material(A, B, C_, L[0], L[1], L[2], L4, L6, n_constants, 0.0,
                          (C.c_double * 3)(0, 0, 0), 0.0, (C.c_double * 3)(0, 0, 0), 0.0)


BAD_CREATE = {
    "zero size": (dict(nx=0), {}, lqmin.LQ_FP64, "positive"),
    "negative size": (dict(nz=-4), {}, lqmin.LQ_FP64, "positive"),
    "spacing other than 1": (dict(spacing=0.5), {}, lqmin.LQ_FP64, "spacing"),
    "two constants": ({}, dict(n_constants=2), lqmin.LQ_FP64, "n_constants"),
    "one constant with L2": ({}, dict(n_constants=1, L=(2.32, 0.5, 0.0)), lqmin.LQ_FP64,
                             "one-constant"),
    "one constant with L4": ({}, dict(n_constants=1, L=(2.32, 0.0, 0.0), L4=0.3), lqmin.LQ_FP64,
                             "one-constant"),
    "no nematic minimum (C < 0)": ({}, dict(C_=-1.0), lqmin.LQ_FP64, "nematic"),
    "no nematic minimum (B^2 < 24 A C)": ({}, dict(A=1.0, B=-0.1, C_=1.0), lqmin.LQ_FP64,
                                          "nematic"),
    "unknown precision": ({}, {}, 7, "precision"),
    "too many sites per x row index": (dict(nx=1, ny=1 << 16, nz=1 << 15), {}, lqmin.LQ_FP64,
                                       "too large"),
}


@pytest.mark.parametrize("case", sorted(BAD_CREATE))
def test_create_rejects_bad_arguments_on_the_host(lib, case):
    lat_kw, mat_kw, precision, why = BAD_CREATE[case]
    lat, mat = lattice(**lat_kw), material(**mat_kw)
    out = C.c_void_p(12345)
    st = lib.lq_create(C.byref(lat), C.byref(mat), precision, None, C.byref(out))
    assert st == lqmin.LQ_EINVAL
    assert out.value is None            # *out cleared, no handle
    assert why in lib.lq_create_error().decode()


def test_create_rejects_null_arguments(lib):
    lat, mat = lattice(), material()
    out = C.c_void_p()
    assert lib.lq_create(None, C.byref(mat), lqmin.LQ_FP64, None, C.byref(out)) == lqmin.LQ_EINVAL
    assert lib.lq_create(C.byref(lat), None, lqmin.LQ_FP64, None, C.byref(out)) == lqmin.LQ_EINVAL
    assert lib.lq_create(C.byref(lat), C.byref(mat), lqmin.LQ_FP64, None, None) == lqmin.LQ_EINVAL
    assert "null" in lib.lq_create_error().decode()


def test_inject_fault_checks_its_arguments(lib):
    assert lib.lq_inject_fault(99, 0) == lqmin.LQ_EINVAL
    assert lib.lq_inject_fault(-1, 0) == lqmin.LQ_EINVAL
    assert lib.lq_inject_fault(lqmin.LQ_FAULT_NONE, -1) == lqmin.LQ_EINVAL
    assert lib.lq_inject_fault(lqmin.LQ_FAULT_NONE, 0) == lqmin.LQ_OK


def test_frank_helper_rejects_nonpositive_or_nonfinite_input(lib):
    L = (C.c_double * 5)()
    assert lib.lq_frank_to_landau(1.0, 1.0, 1.0, 0.0, 0.0, 0.0, L) == lqmin.LQ_EINVAL
    assert lib.lq_frank_to_landau(1.0, 1.0, 1.0, 0.0, 0.0, -0.5, L) == lqmin.LQ_EINVAL
    assert lib.lq_frank_to_landau(float("nan"), 1.0, 1.0, 0.0, 0.0, 0.5, L) == lqmin.LQ_EINVAL
    assert lib.lq_frank_to_landau(1.0, 1.0, float("inf"), 0.0, 0.0, 0.5, L) == lqmin.LQ_EINVAL
    assert lib.lq_frank_to_landau(1.0, 1.0, 1.0, 0.0, 0.0, 0.5, None) == lqmin.LQ_EINVAL
    assert lib.lq_frank_to_landau(1.0, 1.0, 1.0, 0.0, 0.0, 0.5, L) == lqmin.LQ_OK


def test_bounds_counter_is_absent_from_the_release_library(lib):
    hits = C.c_uint32(7)
    assert lib.lq_bounds_check_hits(C.byref(hits)) == lqmin.LQ_EINVAL
    assert hits.value == 0
    assert lib.lq_bounds_check_hits(None) == lqmin.LQ_EINVAL
