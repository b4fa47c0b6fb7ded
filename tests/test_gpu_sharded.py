"""CUDA z slabs of one lattice (lq_slab_*), driven in one process by
``sharded.run_local`` (the same routing ``run_ranks`` uses between GPUs):
each slab's force equals the whole lattice's at its planes, and FIRE on two
or three slabs follows FIRE on the whole lattice -- in FP64 to 1e-11, in the
FP32 form to float rounding -- on periodic and open z axes with walls and
colloids.  Slabs refuse the whole-lattice calls."""
import ctypes as C

import numpy as np
import pytest

from _helpers import HOM, PLANAR, need_gpu
from paper_1911_07045_b300 import lqmin, sharded, synth

pytestmark = pytest.mark.gpu

FP = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)
CASES = {
    "periodic_z_3c": dict(shape=(34, 20, 24), periodic=(1, 1, 1), L=(2.32, 0.5, 0.3),
                          objects=[dict(type="sphere", c=(17.0, 10.0, 1.0), R=4.5, anchor=HOM())]),
    "open_z_walls_3c": dict(shape=(32, 18, 21), periodic=(1, 1, 0), L=(2.32, 0.5, 0.3),
                            objects=[dict(type="wall", axis=2, plane=0, anchor=PLANAR()),
                                     dict(type="wall", axis=2, plane=20, anchor=HOM()),
                                     dict(type="sphere", c=(16.0, 9.0, 10.0), R=4.0, anchor=HOM())]),
    "periodic_1c": dict(shape=(40, 16, 18), periodic=(1, 1, 1), L=(2.32, 0.0, 0.0),
                        objects=[dict(type="sphere", c=(20.0, 8.0, 17.0), R=3.5, anchor=HOM())]),
}


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def whole_solver(c, precision):
    s = lqmin.Solver(c["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, *c["L"], periodic=c["periodic"],
                     precision=precision)
    s.add_objects(c["objects"])
    return s


def own_planes(field, shape, z_lo, z_hi):
    nxy = shape[0] * shape[1]
    return field[:, z_lo * nxy:z_hi * nxy]


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_slab_force_is_the_whole_lattice_force(name, world):
    c = CASES[name]
    whole = whole_solver(c, 0)
    q0 = synth.random_uniaxial_q(c["shape"], 41)
    whole.set_q(q0)
    Fw = whole.force()
    lib = lqmin.load()
    pz = bool(c["periodic"][2])
    for r in range(world):
        z_lo, z_hi = sharded.slab_bounds(c["shape"][2], world, r)
        s = sharded.CudaSlab(whole, z_lo, z_hi)
        s.set_q(sharded.slab_field(q0, c["shape"], z_lo, z_hi, pz))
        out = np.empty((5, s.N))
        assert lib.lq_force(s.h, lqmin._ptr(out)) == lqmin.LQ_OK
        nxy = c["shape"][0] * c["shape"][1]
        got, want = out[:, nxy:s.N - nxy], own_planes(Fw, c["shape"], z_lo, z_hi)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
        s.close()
    whole.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fire_on_slabs_follows_the_whole_lattice(name, world, precision):
    c = CASES[name]
    steps = 12
    whole = whole_solver(c, precision)
    ref = whole_solver(c, precision)
    q0 = synth.random_uniaxial_q(c["shape"], 42)
    ref.set_q(q0)
    p = lqmin.fire_params(**FP)
    rr = ref.step(p, steps)
    pz = bool(c["periodic"][2])
    slabs = []
    for r in range(world):
        z_lo, z_hi = sharded.slab_bounds(c["shape"][2], world, r)
        s = sharded.CudaSlab(whole, z_lo, z_hi)
        s.set_q(sharded.slab_field(q0, c["shape"], z_lo, z_hi, pz))
        slabs.append(s)
    res = sharded.run_local(slabs, p, steps, pz)
    assert res.iterations == rr.iterations == steps
    assert res.npos == rr.npos
    assert abs(res.dt - rr.dt) <= 1e-14 * rr.dt
    qw = ref.get_q()
    tol = 1e-11 if precision == 0 else 2e-7
    for s in slabs:
        want = own_planes(qw, c["shape"], s.z_lo, s.z_hi)
        assert np.abs(s.own_q() - want).max() <= tol * np.abs(want).max()
        s.close()
    ref.close()
    whole.close()


def test_slabs_refuse_whole_lattice_calls():
    c = CASES["periodic_z_3c"]
    whole = whole_solver(c, 0)
    lib = lqmin.load()
    h = C.c_void_p()
    assert lib.lq_slab_create(whole.h, 5, 5, C.byref(h)) == lqmin.LQ_EINVAL
    assert lib.lq_slab_create(whole.h, -1, 4, C.byref(h)) == lqmin.LQ_EINVAL
    assert lib.lq_slab_create(whole.h, 0, c["shape"][2] + 1, C.byref(h)) == lqmin.LQ_EINVAL
    s = sharded.CudaSlab(whole, 0, 8)
    p = lqmin.fire_params(**FP)
    r = lqmin.Result()
    local = np.zeros(4)
    assert lib.lq_slab_step(s.h, lqmin._ptr(local)) == lqmin.LQ_EINVAL      # not started
    assert lib.lq_step(s.h, C.byref(p), 1, C.byref(r)) == lqmin.LQ_EINVAL
    assert lib.lq_minimize(s.h, C.byref(p), C.byref(r)) == lqmin.LQ_EINVAL
    assert lib.lq_fire_reset(s.h, C.byref(p)) == lqmin.LQ_EINVAL
    assert lib.lq_slab_create(s.h, 0, 2, C.byref(h)) == lqmin.LQ_EINVAL   # a slab of a slab
    a = lqmin.anchoring(*HOM())
    assert lib.lq_add_wall(s.h, 2, 1, C.byref(a)) == lqmin.LQ_EINVAL
    arr = (C.c_void_p * 1)(s.h.value)
    b = C.c_void_p()
    st = lib.lq_batch_create(C.cast(arr, C.c_void_p), 1, C.byref(b))
    assert st == lqmin.LQ_EINVAL
    assert lib.lq_slab_step(whole.h, lqmin._ptr(local)) == lqmin.LQ_EINVAL  # not a slab
    s.close()
    whole.close()
