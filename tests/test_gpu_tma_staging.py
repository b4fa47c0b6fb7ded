"""Tensor-copy staging of the FP32 form's three-constant step kernel.

The rows of each z plane that a tile and its ring need arrive in shared
memory as bulk tensor copies (lq_set_staging); the arithmetic of every site
is the one of the per-thread-load kernel, so the two stagings must give the
same q, v, F bit for bit, on every geometry kind, on open and periodic axes,
with ragged y and z extents, z chunks of one to five planes and both index
widths -- and both match the FP64 oracle within the FP32 form's tolerance."""
import numpy as np
import pytest

from _helpers import HOM, PLANAR, make_pair, need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

FP = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)
L3C = (2.32, 0.5, 0.3)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


CASES = {
    "periodic_bulk_ragged_y": dict(shape=(64, 22, 18), objects=[], periodic=(1, 1, 1)),
    "walls_colloid": dict(shape=(64, 28, 26), periodic=(1, 1, 1),
                          objects=[dict(type="wall", axis=2, plane=0, anchor=PLANAR()),
                                   dict(type="wall", axis=2, plane=25, anchor=HOM()),
                                   dict(type="sphere", c=(32.0, 14.0, 13.0), R=5.0, anchor=HOM())]),
    "open_axes": dict(shape=(32, 13, 11), periodic=(0, 0, 0),
                      objects=[dict(type="sphere", c=(16.0, 6.0, 5.0), R=3.2, anchor=HOM())]),
    "colloid_across_x_and_y_edges": dict(shape=(96, 14, 10), periodic=(1, 1, 1),
                                         objects=[dict(type="sphere", c=(0.5, 1.0, 5.0), R=4.0,
                                                       anchor=HOM())]),
    "droplet_rod": dict(shape=(64, 26, 24), periodic=(1, 1, 1),
                        objects=[dict(type="spherocylinder", c=(20.0, 10.0, 8.5), c2=(40.0, 15.0, 14.5),
                                      R=2.2, anchor=PLANAR()),
                                 dict(type="droplet", c=(31.5, 12.5, 11.5), R=11.2, anchor=HOM())]),
    "open_y_walls": dict(shape=(32, 18, 21), periodic=(1, 0, 1),
                         objects=[dict(type="wall", axis=1, plane=0, anchor=HOM()),
                                  dict(type="wall", axis=2, plane=20, anchor=PLANAR())]),
}


def make(c, staging, zchunk=0, idx64=False):
    s = lqmin.Solver(c["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, *L3C, periodic=c["periodic"],
                     precision=1)
    s.add_objects(c["objects"])
    s.set_staging(staging)
    if zchunk:
        s.set_zchunk(zchunk)
    if idx64:
        s.set_index_width(64)
    return s


@pytest.mark.parametrize("zchunk", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("name", sorted(CASES))
def test_tensor_copies_match_loads_bit_for_bit(name, zchunk):
    c = CASES[name]
    a, b = make(c, 1, zchunk), make(c, 2, zchunk)
    assert not a.uses_tensor_copies() and b.uses_tensor_copies()
    q0 = synth.random_uniaxial_q(c["shape"], 21)
    a.set_q(q0)
    b.set_q(q0)
    p = lqmin.fire_params(**FP)
    ra, rb = a.step(p, 7), b.step(p, 7)
    assert ra.iterations == rb.iterations == 7
    assert (ra.power, ra.norm_force, ra.norm_velocity, ra.max_force, ra.dt, ra.alpha) == \
           (rb.power, rb.norm_force, rb.norm_velocity, rb.max_force, rb.dt, rb.alpha)
    for x, y in ((a.get_q(), b.get_q()), (a.get_velocity(), b.get_velocity()),
                 (a.get_force(), b.get_force())):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_tensor_copies_with_64bit_indices():
    c = CASES["walls_colloid"]
    a, b = make(c, 1, 3), make(c, 2, 3, idx64=True)
    q0 = synth.random_uniaxial_q(c["shape"], 22)
    a.set_q(q0)
    b.set_q(q0)
    p = lqmin.fire_params(**FP)
    a.step(p, 4)
    b.step(p, 4)
    assert np.array_equal(a.get_q(), b.get_q())
    assert np.array_equal(a.get_force(), b.get_force())
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["walls_colloid", "open_axes", "colloid_across_x_and_y_edges"])
def test_tensor_copies_against_oracle(oracle_mod, name):
    """Five FIRE steps with tensor-copy staging against the FP64 oracle
    (the FP32 form's float rounding: q 2e-7, v and F 2e-6)."""
    c = CASES[name]
    s, o = make_pair(oracle_mod, c["shape"], L3C, c["objects"], periodic=c["periodic"], precision=1)
    s.set_staging(2)
    q0 = np.round(synth.random_uniaxial_q(c["shape"], 23) * 2.0 ** 28) / 2.0 ** 28
    s.set_q(q0)
    params = dict(FP, force_tol=1e-12)
    r = s.step(lqmin.fire_params(**params), 5)
    qo, vo, Fo, st = o.fire(q0, params, 5)
    sim = o.simulated()

    def rel(x, y):
        return float(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300))

    assert r.iterations == st["iter"] == 5
    assert rel(s.get_q()[:, sim], qo[:, sim]) < 2e-7
    assert rel(s.get_force()[:, sim], Fo[:, sim]) < 2e-6
    assert rel(s.get_velocity()[:, sim], vo[:, sim]) < 2e-6
    s.close()


def test_minimisation_is_the_same_with_either_staging():
    c = CASES["walls_colloid"]
    n = np.array([0.2, 0.1, 1.0])
    q0 = np.repeat(synth.uniaxial_q((n / np.linalg.norm(n))[:, None],
                                    synth.s0_closed_form(synth.A_5CB, synth.B_5CB, synth.C_5CB)),
                   int(np.prod(c["shape"])), axis=1)
    out = []
    for mode in (1, 2):
        s = make(c, mode)
        s.set_q(q0)
        code, r = s.minimize(lqmin.fire_params(**dict(FP, max_iter=100000, force_tol=1e-5)))
        assert code == lqmin.LQ_OK and r.fire_status == lqmin.FIRE_CONVERGED
        out.append((r.iterations, r.energy, s.get_q()))
        s.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])


def test_staging_modes_and_refusals():
    lib = lqmin.load()
    ok = make(CASES["open_axes"], 0)
    assert not ok.uses_tensor_copies()              # automatic: per-thread loads
    ok.set_staging(2)
    assert ok.uses_tensor_copies()
    ok.set_staging(1)
    assert not ok.uses_tensor_copies()
    assert lib.lq_set_staging(ok.h, 3) == lqmin.LQ_EINVAL
    assert lib.lq_set_staging(ok.h, -1) == lqmin.LQ_EINVAL
    ok.close()
    # x extent not a multiple of 32, one constant, FP64: per-thread loads only
    ragged = lqmin.Solver((33, 8, 8), synth.A_5CB, synth.B_5CB, synth.C_5CB, *L3C, precision=1)
    one_c = lqmin.Solver((32, 8, 8), synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, precision=1)
    fp64 = lqmin.Solver((32, 8, 8), synth.A_5CB, synth.B_5CB, synth.C_5CB, *L3C, precision=0)
    for s in (ragged, one_c, fp64):
        assert not s.uses_tensor_copies()
        assert lib.lq_set_staging(s.h, 2) == lqmin.LQ_EINVAL
        assert not s.uses_tensor_copies()
        s.close()


def test_copy_wait_that_runs_out_stops_fire_and_reports_it():
    """A plane whose copies never satisfy its barrier (injected on the host:
    the barrier expects more bytes than the copies deliver) must not hang
    the GPU: every wait gives up after about a second, the kernel stops with
    the stalled status, the entry point returns LQ_ECUDA, the context stays
    usable, and a FIRE restart runs exactly like a fresh solver."""
    import ctypes as C
    c = CASES["open_axes"]
    a, fresh = make(c, 2), make(c, 2)
    q0 = synth.random_uniaxial_q(c["shape"], 24)
    a.set_q(q0)
    p = lqmin.fire_params(**FP)
    a.step(p, 2)
    lib = lqmin.load()
    assert lib.lq_inject_fault(lqmin.LQ_FAULT_COPY_WAIT, 0) == lqmin.LQ_OK
    r = lqmin.Result()
    st = lib.lq_step(a.h, C.byref(p), 1, C.byref(r))        # one direct launch
    assert st == lqmin.LQ_ECUDA
    assert r.fire_status == lqmin.FIRE_STALLED
    assert b"tensor copy" in lib.lq_last_error(a.h)
    assert lib.lq_step(a.h, C.byref(p), 1, C.byref(r)) == lqmin.LQ_ECUDA   # stays stopped
    # restart from a fresh start state: the same trajectory as a fresh solver
    a.set_q(q0)
    fresh.set_q(q0)
    ra, rf = a.step(p, 5), fresh.step(p, 5)
    assert ra.fire_status == rf.fire_status == lqmin.FIRE_RUNNING
    assert np.array_equal(a.get_q(), fresh.get_q())
    a.close()
    fresh.close()
