"""Argument errors on a live solver, part-way through a FIRE run: every bad
call returns LQ_EINVAL with a message and changes nothing.  The objects, Q
and the minimiser state stay as they were, so the following FIRE steps
equal, bit for bit, those of a twin solver that never saw the bad calls."""
import ctypes as C

import numpy as np
import pytest

from _helpers import HOM, PLANAR, need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

SHAPE = (24, 20, 16)
OBJECTS = [dict(type="wall", axis=2, plane=0, anchor=PLANAR()),
           dict(type="sphere", c=(12.0, 10.0, 8.0), R=4.0, anchor=HOM())]
FP = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def d3(*v):
    return (C.c_double * 3)(*[float(x) for x in v])


def bad_calls(s, precision):
    """(name, thunk) pairs; each thunk makes one invalid call on ``s``."""
    lib, h = s.lib, s.h
    ok = lqmin.anchoring(lqmin.ND_HOMEOTROPIC, 1.0)
    bad_kind = lqmin.anchoring(7, 1.0)
    bad_w = lqmin.anchoring(lqmin.ND_HOMEOTROPIC, -1.0)

    def params(**kw):
        return C.byref(lqmin.fire_params(**dict(FP, **kw)))

    r = lqmin.Result()
    calls = [
        ("sphere R < 0", lambda: lib.lq_add_sphere(h, d3(5, 5, 5), -1.0, C.byref(ok))),
        ("sphere R NaN", lambda: lib.lq_add_sphere(h, d3(5, 5, 5), float("nan"), C.byref(ok))),
        ("droplet R = 0", lambda: lib.lq_add_droplet(h, d3(5, 5, 5), 0.0, C.byref(ok))),
        ("spherocylinder R < 0",
         lambda: lib.lq_add_spherocylinder(h, d3(3, 3, 3), d3(6, 6, 6), -0.5, C.byref(ok))),
        ("wall axis 3", lambda: lib.lq_add_wall(h, 3, 0, C.byref(ok))),
        ("unknown anchoring kind", lambda: lib.lq_add_sphere(h, d3(5, 5, 5), 2.0, C.byref(bad_kind))),
        ("negative anchoring strength",
         lambda: lib.lq_add_wall(h, 2, 15, C.byref(bad_w))),
        ("null anchoring", lambda: lib.lq_add_wall(h, 2, 15, None)),
        ("move a missing object", lambda: lib.lq_move_object(h, 5, d3(1, 0, 0))),
        ("move a wall by half a plane", lambda: lib.lq_move_object(h, 0, d3(0, 0, 0.5))),
        ("move by NaN", lambda: lib.lq_move_object(h, 1, d3(float("nan"), 0, 0))),
        ("index width 16", lambda: lib.lq_set_index_width(h, 16)),
        ("negative z chunk", lambda: lib.lq_set_zchunk(h, -1)),
        ("dt0 = 0", lambda: lib.lq_step(h, params(dt0=0.0), 3, C.byref(r))),
        ("dt_max < dt0", lambda: lib.lq_step(h, params(dt0=0.02, dt_max=0.01), 3, C.byref(r))),
        ("alpha0 > 1", lambda: lib.lq_minimize(h, params(alpha0=1.5), C.byref(r))),
        ("unknown method", lambda: lib.lq_step(h, params(method=9), 3, C.byref(r))),
        ("Nesterov momentum 1", lambda: lib.lq_step(h, params(method=lqmin.LQ_MIN_NESTEROV,
                                                               dt_max=FP["dt0"], momentum=1.0),
                                                   3, C.byref(r))),
        ("null parameters", lambda: lib.lq_step(h, None, 3, C.byref(r))),
        ("null q", lambda: lib.lq_set_q(h, None)),
        ("dipolar zero axis", lambda: lib.lq_init_dipolar(h, d3(12, 10, 8), d3(0, 0, 0), 2.0, 0.0)),
        ("dipolar rd = 0", lambda: lib.lq_init_dipolar(h, d3(12, 10, 8), d3(0, 0, 1), 0.0, 0.0)),
        ("boundary text with a short site line",
         lambda: lib.lq_add_boundary_text(h, b"object homeotropic 2.5\n 1 2\nend\n")),
    ]
    if precision == lqmin.LQ_FP32_BULK_FP64_RED:
        calls.append(("S outside the fixed-point range",
                      lambda: lib.lq_init_random_uniaxial(h, 3, 100.0)))
    return calls


@pytest.mark.parametrize("precision", [lqmin.LQ_FP64, lqmin.LQ_FP32_BULK_FP64_RED])
def test_bad_calls_change_nothing(precision):
    twins = []
    for _ in range(2):
        s = lqmin.Solver(SHAPE, synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, 0.5, 0.3,
                         precision=precision)
        s.add_objects(OBJECTS)
        s.set_q(synth.random_uniaxial_q(SHAPE, 21))
        s.step(lqmin.fire_params(**FP), 4)
        twins.append(s)
    a, b = twins
    q_before = a.get_q()
    for name, call in bad_calls(a, precision):
        st = call()
        assert st == lqmin.LQ_EINVAL, name
        assert a.lib.lq_last_error(a.h).decode(), name
    assert a.object_count() == b.object_count() == 2
    assert np.array_equal(a.get_q(), q_before)
    p = lqmin.fire_params(**FP)
    ra, rb = a.step(p, 6), b.step(p, 6)
    assert ra.iterations == rb.iterations == 10
    assert (ra.dt, ra.alpha, ra.npos, ra.max_force) == (rb.dt, rb.alpha, rb.npos, rb.max_force)
    assert np.array_equal(a.get_q(), b.get_q())
    assert np.array_equal(a.get_velocity(), b.get_velocity())
    assert np.array_equal(a.mask(), b.mask())
    a.close()
    b.close()


def test_batch_rejects_mixed_members_and_bad_tiling():
    """A batch needs one precision and one distortion form; tile heights are
    4 or 8 and z chunks >= 0.  Failed calls leave no batch, or the batch as
    it was."""
    def solver(precision=lqmin.LQ_FP64, L=(2.32, 0.5, 0.3)):
        s = lqmin.Solver((20, 16, 12), synth.A_5CB, synth.B_5CB, synth.C_5CB, *L,
                         precision=precision)
        s.set_q(synth.random_uniaxial_q((20, 16, 12), 5))
        return s
    a, b = solver(), solver()
    f32 = solver(precision=lqmin.LQ_FP32_BULK_FP64_RED)
    one = solver(L=(2.32, 0.0, 0.0))
    lib = a.lib
    out = C.c_void_p(99)
    for members in ([a, f32], [a, one]):
        arr = (C.c_void_p * len(members))(*[m.h.value for m in members])
        assert lib.lq_batch_create(arr, len(members), C.byref(out)) == lqmin.LQ_EINVAL
        assert out.value is None
    arr = (C.c_void_p * 2)(a.h.value, b.h.value)
    assert lib.lq_batch_create(arr, 0, C.byref(out)) == lqmin.LQ_EINVAL
    assert lib.lq_batch_create(None, 2, C.byref(out)) == lqmin.LQ_EINVAL
    batch = lqmin.Batch([a, b])
    before = batch.tiling()
    for ty, zc in ((5, 16), (4, -1), (8, -3)):
        assert lib.lq_batch_set_tiling(batch.h, ty, zc) == lqmin.LQ_EINVAL
        assert lib.lq_batch_last_error(batch.h).decode()
    assert batch.tiling() == before
    res = batch.step(lqmin.fire_params(**FP), 3)
    assert [r.iterations for r in res] == [3, 3]
    batch.close()
    for s in (a, b, f32, one):
        s.close()


def test_server_tickets_are_read_once_and_unknown_ones_refused():
    sv = lqmin.Server(1 << 30, max_active=4)
    cfg = dict(shape=(16, 16, 12), L1=2.32, objects=[])
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=200000, force_tol=1e-5))
    t = sv.submit(cfg, p, seed=3)
    r = lqmin.Result()
    lib = sv.lib
    assert lib.lq_server_wait(sv.h, C.c_uint64(t), 300.0, C.byref(r), None) == lqmin.LQ_OK
    assert r.fire_status == lqmin.FIRE_CONVERGED
    # handed back once: a second read, and a ticket never issued, are refused
    assert lib.lq_server_poll(sv.h, C.c_uint64(t), C.byref(r), None) == lqmin.LQ_EINVAL
    assert lib.lq_server_wait(sv.h, C.c_uint64(t), 1.0, C.byref(r), None) == lqmin.LQ_EINVAL
    assert lib.lq_server_poll(sv.h, C.c_uint64(t + 1000), C.byref(r), None) == lqmin.LQ_EINVAL
    assert lib.lq_server_poll(None, C.c_uint64(t), C.byref(r), None) == lqmin.LQ_EINVAL
    sv.close()
