"""Gradient descent and Nesterov's accelerated gradient (section III.C names
both; Fig. 2 compares gradient descent with FIRE) run by the same fused step
kernel as FIRE, against the oracle's textbook iterations: x <- x + eta F(x);
y_k = x_k + mu (x_k - x_{k-1}), x_{k+1} = y_k + eta F(y_k).  The solver's
state is y (where the force is evaluated) and the displacement of the
coming step, mu (x_k - x_{k-1}) + eta F(y_k)."""
import numpy as np
import pytest

from _helpers import HOM, PLANAR, make_pair, need_gpu, rand_q
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


GEOMS = {
    "bulk_1c": dict(shape=(24, 20, 18), L=(2.32, 0, 0), objects=[]),
    "colloid_walls_3c": dict(shape=(30, 28, 26), L=(2.32, 0.5, 0.3),
                             objects=[dict(type="wall", axis=2, plane=0, anchor=PLANAR()),
                                      dict(type="wall", axis=2, plane=25, anchor=PLANAR()),
                                      dict(type="sphere", c=(15.0, 14.0, 13.0), R=5.0,
                                           anchor=HOM())]),
}
METHODS = {"gd": (lqmin.LQ_MIN_GD, 0.01, 0.0), "nesterov": (lqmin.LQ_MIN_NESTEROV, 0.01, 0.9)}


@pytest.mark.parametrize("name", sorted(GEOMS))
@pytest.mark.parametrize("mname", sorted(METHODS))
def test_descent_steps_match_oracle(oracle_mod, name, mname):
    g = GEOMS[name]
    method, eta, mu = METHODS[mname]
    s, o = make_pair(oracle_mod, g["shape"], g["L"], g["objects"])
    q0 = synth.random_uniaxial_q(g["shape"], 21)
    s.set_q(q0)
    p = lqmin.descent_params(method, eta, momentum=mu, max_iter=10 ** 6, force_tol=1e-14)
    sim = o.simulated()
    r = s.step(p, 1)
    ro = o.descent(q0, method, eta, mu=mu, max_iter=10 ** 6, force_tol=1e-14, max_steps=1)
    assert r.iterations == ro["iter"] == 1 and r.fire_status == lqmin.FIRE_RUNNING
    assert rel(s.get_q()[:, sim], ro["y"][:, sim]) < 1e-13
    assert rel(s.get_force()[:, sim], ro["F"][:, sim]) < 1e-11
    step = ro["y"] + eta * ro["F"] - ro["x"]
    assert rel(s.get_velocity()[:, sim], step[:, sim]) < 1e-11
    assert r.dt == eta
    r = s.step(p, 59)
    ro = o.descent(None, method, eta, mu=mu, max_iter=10 ** 6, force_tol=1e-14, max_steps=59,
                   state=ro)
    assert r.iterations == ro["iter"] == 60
    assert rel(s.get_q()[:, sim], ro["y"][:, sim]) < 1e-11
    assert abs(r.max_force - ro["rmax"]) <= 1e-9 * ro["rmax"]


def test_fp32_form_nesterov_steps(oracle_mod):
    g = GEOMS["colloid_walls_3c"]
    s, o = make_pair(oracle_mod, g["shape"], g["L"], g["objects"],
                     precision=lqmin.LQ_FP32_BULK_FP64_RED)
    q0 = synth.random_uniaxial_q(g["shape"], 22)
    s.set_q(q0)
    p = lqmin.descent_params(lqmin.LQ_MIN_NESTEROV, 0.01, momentum=0.9, max_iter=10 ** 6,
                             force_tol=1e-14)
    r = s.step(p, 30)
    ro = o.descent(q0, oracle_mod.NESTEROV, 0.01, mu=0.9, max_iter=10 ** 6, force_tol=1e-14,
                   max_steps=30)
    sim = o.simulated()
    assert r.iterations == ro["iter"] == 30
    assert np.abs(s.get_q()[:, sim] - ro["y"][:, sim]).max() < 1e-5
    assert abs(r.max_force - ro["rmax"]) <= 1e-4 * ro["rmax"]


def test_nesterov_minimisation_reaches_the_oracle_minimum(oracle_mod):
    """From a near-uniform start between homeotropic walls (a unique
    minimum), Nesterov converges to the force tolerance and the energy of the
    oracle's own Nesterov minimum."""
    shape = (20, 18, 16)
    objs = [dict(type="wall", axis=2, plane=0, anchor=HOM()),
            dict(type="wall", axis=2, plane=15, anchor=HOM())]
    s, o = make_pair(oracle_mod, shape, (2.32, 0.5, 0.3), objs)
    n = np.array([0.3, 0.2, 1.0])
    q0 = np.repeat(synth.uniaxial_q((n / np.linalg.norm(n))[:, None], o.S0), o.N, axis=1)
    q0 = q0 + 0.01 * rand_q(o.N, 4, 1.0)
    s.set_q(q0)
    p = lqmin.descent_params(lqmin.LQ_MIN_NESTEROV, 0.01, momentum=0.9, max_iter=200000,
                             force_tol=1e-8)
    code, r = s.minimize(p)
    assert code == lqmin.LQ_OK and r.fire_status == lqmin.FIRE_CONVERGED
    ro = o.descent(q0, oracle_mod.NESTEROV, 0.01, mu=0.9, max_iter=200000, force_tol=1e-8,
                   max_steps=200000)
    assert ro["status"] == oracle_mod.CONVERGED
    Eo = o.energy(ro["y"])[0]
    assert abs(r.energy - Eo) <= 1e-10 * abs(Eo)
    assert abs(r.iterations - ro["iter"]) <= 2


def test_switching_minimiser_restarts_from_the_current_q(oracle_mod):
    g = GEOMS["bulk_1c"]
    s, o = make_pair(oracle_mod, g["shape"], g["L"], g["objects"])
    s.set_q(synth.random_uniaxial_q(g["shape"], 23))
    fire = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14))
    s.step(fire, 10)
    q = s.get_q()
    p = lqmin.descent_params(lqmin.LQ_MIN_GD, 0.01, max_iter=10 ** 6, force_tol=1e-14)
    r = s.step(p, 5)
    ro = o.descent(q, oracle_mod.GD, 0.01, max_iter=10 ** 6, force_tol=1e-14, max_steps=5)
    assert r.iterations == 5
    assert rel(s.get_q(), ro["y"]) < 1e-12


def test_batch_nesterov_matches_alone():
    """One-constant lattices under Nesterov in the persistent batch kernel
    advance bit for bit as alone."""
    cfgs = [dict(shape=(40, 24, 20), objects=[dict(type="sphere", c=(20.0, 12.0, 10.0), R=5.0,
                                                    anchor=HOM())]),
            dict(shape=(32, 32, 32), objects=[])]
    A, B, C = synth.A_5CB, synth.B_5CB, synth.C_5CB
    alone, mixed = [], []
    for k, c in enumerate(cfgs):
        for lst in (alone, mixed):
            s = lqmin.Solver(c["shape"], A, B, C, 2.32, precision=lqmin.LQ_FP32_BULK_FP64_RED)
            s.add_objects(c["objects"])
            s.set_q(synth.random_uniaxial_q(c["shape"], 40 + k))
            lst.append(s)
    batch = lqmin.Batch(mixed)
    ty, zc = batch.tiling()
    p = lqmin.descent_params(lqmin.LQ_MIN_NESTEROV, 0.01, momentum=0.8, max_iter=10 ** 6,
                             force_tol=1e-14)
    res = batch.step(p, 17)
    for a, m, rb in zip(alone, mixed, res):
        a.set_zchunk(zc)
        ra = a.step(p, 17)
        assert ra.iterations == rb.iterations == 17
        assert np.array_equal(a.get_q(), m.get_q())
        assert np.array_equal(a.get_force(), m.get_force())
    batch.close()


def test_invalid_minimiser_parameters():
    s = lqmin.Solver((8, 8, 8), synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32)
    s.init_random_uniaxial(1)
    for p in (lqmin.descent_params(lqmin.LQ_MIN_NESTEROV, 0.01, momentum=1.0),
              lqmin.descent_params(lqmin.LQ_MIN_GD, -0.01),
              lqmin.fire_params(method=7)):
        st = s.lib.lq_step(s.h, p, 1, None)
        assert st == lqmin.LQ_EINVAL
