"""FIRE through the C interface against the oracle's Algorithm 1: one fused
step, K steps, a full minimisation, checkpoint/resume, and the failure
statuses (divergence, max_iter, wall-clock limit) -- all raised on the host
from device flags, with nothing that faults the GPU."""
import numpy as np
import pytest

from _helpers import HOM, PLANAR, make_pair, need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

FP = dict(synth.FIRE_DEFAULTS)


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
    "droplet_rod_3c": dict(shape=(28, 26, 24), L=(2.32, 0.5, 0.3),
                           objects=[dict(type="spherocylinder", c=(9.0, 10.0, 8.5),
                                         c2=(18.0, 15.0, 14.5), R=2.2, anchor=PLANAR()),
                                    dict(type="droplet", c=(13.5, 12.5, 11.5), R=11.2,
                                         anchor=HOM())],
                           # the oracle's own trajectory turns ill-conditioned between
                           # steps 150 and 180 (a 1e-13 change in q0 grows to 1e-3)
                           steps=150),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_one_step_and_k_steps_match_oracle(oracle_mod, name):
    g = GEOMS[name]
    s, o = make_pair(oracle_mod, g["shape"], g["L"], g["objects"])
    q0 = synth.random_uniaxial_q(g["shape"], 11)
    s.set_q(q0)
    params = dict(FP, max_iter=10 ** 6, force_tol=1e-12)
    p = lqmin.fire_params(**params)
    r = s.step(p, 1)
    qo, vo, Fo, st = o.fire(q0, params, 1)
    sim = o.simulated()   # object sites: ignored by both, zero on the GPU
    assert r.iterations == st["iter"] == 1
    assert rel(s.get_q()[:, sim], qo[:, sim]) < 1e-12
    assert rel(s.get_velocity()[:, sim], vo[:, sim]) < 1e-12
    assert rel(s.get_force()[:, sim], Fo[:, sim]) < 1e-12
    assert (r.dt, r.alpha, r.npos) == (st["dt"], st["alpha"], st["npos"])
    # k - 1 more steps: k in total (200 by default)
    k = g.get("steps", 200)
    r = s.step(p, k - 1)
    qo, vo, Fo, st = o.fire(qo, params, k - 1, state=st, v=vo, F=Fo)
    assert r.iterations == st["iter"] == k
    assert np.abs(s.get_q()[:, sim] - qo[:, sim]).max() < 1e-9
    assert r.npos == st["npos"]
    assert abs(r.dt - st["dt"]) <= 1e-12 * st["dt"] and abs(r.alpha - st["alpha"]) <= 1e-12


def test_small_periodic_full_minimisation_matches_oracle(oracle_mod):
    """32^3 periodic one-constant bulk from random directors (seed 1) to
    max|F| < 1e-9: both reach the uniform texture at S0 (energy N f0)."""
    cfg = synth.config_small_periodic()
    s, o = make_pair(oracle_mod, cfg["shape"], (cfg["L1"], 0, 0), [])
    q0 = synth.random_uniaxial_q(cfg["shape"], cfg["seed"])
    s.set_q(q0)
    params = dict(FP, max_iter=100000, force_tol=cfg["tol"])
    st_code, r = s.minimize(lqmin.fire_params(**params))
    assert st_code == lqmin.LQ_OK and r.fire_status == lqmin.FIRE_CONVERGED
    qo, vo, Fo, st = o.fire(q0, params, 100000)
    assert st["status"] == oracle_mod.CONVERGED
    Eo = o.energy(qo)[0]
    assert abs(r.energy - Eo) <= 1e-10 * abs(Eo)
    assert r.max_force < cfg["tol"]
    # the unique minimum reached from here is the uniform texture, E = N f0;
    # the path there (defect annihilations, FIRE restarts) amplifies rounding
    # differences, so the iteration counts are reported, not compared
    f0 = 0.75 * synth.A_5CB * o.S0 ** 2 + 0.25 * synth.B_5CB * o.S0 ** 3 + \
        9.0 / 16.0 * synth.C_5CB * o.S0 ** 4
    assert abs(r.energy - o.N * f0) <= 1e-10 * abs(o.N * f0)
    print(f"iterations: gpu {r.iterations}, oracle {st['iter']}")


def test_checkpoint_resume_is_bitwise(oracle_mod):
    g = GEOMS["colloid_walls_3c"]
    for prec in (0, 1):
        s, _ = make_pair(oracle_mod, g["shape"], g["L"], g["objects"], precision=prec)
        s.init_random_uniaxial(5)
        p = lqmin.fire_params(**dict(FP, max_iter=10 ** 6, force_tol=1e-12))
        s.step(p, 37)
        ck = s.get_state()
        s.step(p, 41)
        qa, va, ra = s.get_q(), s.get_velocity(), s.fire_result()
        s.set_state(ck)
        s.step(p, 41)
        qb, vb, rb = s.get_q(), s.get_velocity(), s.fire_result()
        assert np.array_equal(qa, qb) and np.array_equal(va, vb)
        assert ra.iterations == rb.iterations == 78 and ra.dt == rb.dt


def test_statuses_without_faults(oracle_mod):
    g = GEOMS["bulk_1c"]
    s, _ = make_pair(oracle_mod, g["shape"], g["L"], g["objects"])
    s.init_random_uniaxial(2)
    # max_iter reached
    code, r = s.minimize(lqmin.fire_params(**dict(FP, max_iter=7, force_tol=1e-14)))
    assert code == lqmin.LQ_ENOTCONVERGED and r.iterations == 7
    # a time step far beyond stability: the reductions overflow and FIRE
    # reports divergence from the device flag
    s.init_random_uniaxial(2)
    code, r = s.minimize(lqmin.fire_params(**dict(FP, dt0=50.0, dt_max=50.0, max_iter=5000,
                                                   force_tol=1e-14)))
    assert code == lqmin.LQ_EDIVERGED and r.fire_status == lqmin.FIRE_DIVERGED
    # wall-clock limit
    s.init_random_uniaxial(2)
    code, r = s.minimize(lqmin.fire_params(**dict(FP, max_iter=10 ** 9, force_tol=0.0,
                                                   wall_timeout_s=0.05)))
    assert code == lqmin.LQ_ETIMEOUT
    # the solver stays usable afterwards
    s.init_random_uniaxial(2)
    r = s.step(lqmin.fire_params(**dict(FP, max_iter=10, force_tol=1e-14)), 3)
    assert r.iterations == 3 and np.isfinite(r.max_force)


def test_fp32_form_one_step(oracle_mod):
    """FP32 form: Q on the 2^-28 fixed-point grid, v and F in float, the
    stencil in float; one FIRE step agrees with the FP64 oracle to float
    accuracy."""
    g = GEOMS["colloid_walls_3c"]
    s, o = make_pair(oracle_mod, g["shape"], g["L"], g["objects"], precision=1)
    q0 = np.round(synth.random_uniaxial_q(g["shape"], 11) * 2.0 ** 28) / 2.0 ** 28
    s.set_q(q0)
    params = dict(FP, max_iter=10 ** 6, force_tol=1e-12)
    r = s.step(lqmin.fire_params(**params), 1)
    qo, vo, Fo, st = o.fire(q0, params, 1)
    sim = o.simulated()
    assert rel(s.get_q()[:, sim], qo[:, sim]) < 1e-7
    assert rel(s.get_force()[:, sim], Fo[:, sim]) < 5e-6
    assert rel(s.get_velocity()[:, sim], vo[:, sim]) < 5e-6


def test_fp32_form_reaches_fp64_minimum(oracle_mod):
    """FP32-bulk / FP64-reduction form: from a smooth start both precisions
    settle in the same basin; final energy within 1e-6 relative and the
    per-site order parameter within 1e-4 of the FP64 oracle."""
    shape = (28, 28, 24)
    objs = [dict(type="wall", axis=2, plane=0, anchor=HOM()),
            dict(type="wall", axis=2, plane=23, anchor=HOM()),
            dict(type="sphere", c=(14.0, 14.0, 12.0), R=5.0, anchor=HOM())]
    L = (2.32, 0.5, 0.3)
    s, o = make_pair(oracle_mod, shape, L, objs, precision=1)
    # smooth start: uniform director along z, slightly tilted
    n = np.array([0.1, 0.05, 1.0])
    n /= np.linalg.norm(n)
    q0 = np.repeat(synth.uniaxial_q(n[:, None], o.S0), o.N, axis=1)
    params = dict(FP, max_iter=200000, force_tol=1e-6)
    qo, vo, Fo, st = o.fire(q0, params, 200000)
    assert st["status"] == oracle_mod.CONVERGED
    s.set_q(q0)
    code, r = s.minimize(lqmin.fire_params(**params))
    assert code == lqmin.LQ_OK, (r.iterations, r.max_force)
    Eo = o.energy(qo)[0]
    assert abs(r.energy - Eo) <= 1e-6 * abs(Eo)
    sim = o.simulated()
    assert np.abs(s.order_field()[sim] - o.order_field(qo)[sim]).max() < 1e-4


FP32_KERNELS = {
    # one constant on a lattice narrower than 256 sites: 32-wide tiles
    "one_constant_32wide": dict(shape=(40, 20, 18), L=(2.32, 0.0, 0.0), extra={},
                                objects=[dict(type="sphere", c=(20.0, 10.0, 9.0), R=4.5,
                                              anchor=HOM())]),
    # one constant, 256 sites wide: 64-wide tiles
    "one_constant_64wide": dict(shape=(256, 10, 12), L=(2.32, 0.0, 0.0), extra={},
                                objects=[dict(type="wall", axis=2, plane=0, anchor=HOM()),
                                         dict(type="wall", axis=2, plane=11, anchor=PLANAR()),
                                         dict(type="sphere", c=(128.0, 5.0, 6.0), R=3.0,
                                              anchor=HOM())]),
    # three constants: the kernel that reads the own site's v, F again at the kick
    "three_constants": dict(GEOMS["colloid_walls_3c"], extra={}),
    # the chiral term and a field: the third kernel form
    "chiral_field": dict(GEOMS["colloid_walls_3c"],
                         extra=dict(L4=0.7, H=(0.3, -0.2, 0.5), mu0_dchi=1.3)),
}


@pytest.mark.parametrize("name", sorted(FP32_KERNELS))
def test_fp32_form_steps_in_every_kernel_form(oracle_mod, name):
    """Five FIRE steps of the FP32 form against the FP64 oracle in each of
    its kernel forms.  The one-constant and chiral kernels keep each own
    site's cv v + (cF + dt/2) F in shared memory from its drift to its kick;
    a wrong or stale coefficient there shows as an O(1e-2) error in v."""
    c = FP32_KERNELS[name]
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], precision=1, **c["extra"])
    q0 = np.round(synth.random_uniaxial_q(c["shape"], 12) * 2.0 ** 28) / 2.0 ** 28
    s.set_q(q0)
    params = dict(FP, max_iter=10 ** 6, force_tol=1e-12)
    r = s.step(lqmin.fire_params(**params), 5)
    qo, vo, Fo, st = o.fire(q0, params, 5)
    sim = o.simulated()
    assert r.iterations == st["iter"] == 5
    assert abs(r.dt - st["dt"]) <= 1e-12 * st["dt"]
    # measured: q 1.7e-8, F 1.2e-7 to 1.4e-7, v 1.4e-7 to 1.7e-7 (float rounding)
    assert rel(s.get_q()[:, sim], qo[:, sim]) < 2e-7
    assert rel(s.get_force()[:, sim], Fo[:, sim]) < 2e-6
    assert rel(s.get_velocity()[:, sim], vo[:, sim]) < 2e-6


@pytest.mark.parametrize("zchunk", [1, 2, 3, 5])
@pytest.mark.parametrize("name", ["one_constant_32wide", "one_constant_64wide", "chiral_field"])
def test_fp32_kept_kick_part_with_short_z_chunks(oracle_mod, name, zchunk):
    """Chunks of one to five planes exercise the first and last planes of
    the three-plane store of the kick's old-state part; five FIRE steps
    still match the oracle to float accuracy."""
    c = FP32_KERNELS[name]
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], precision=1, zchunk=zchunk,
                     **c["extra"])
    q0 = np.round(synth.random_uniaxial_q(c["shape"], 13) * 2.0 ** 28) / 2.0 ** 28
    s.set_q(q0)
    params = dict(FP, max_iter=10 ** 6, force_tol=1e-12)
    r = s.step(lqmin.fire_params(**params), 5)
    qo, vo, Fo, st = o.fire(q0, params, 5)
    sim = o.simulated()
    assert r.iterations == st["iter"] == 5
    assert rel(s.get_q()[:, sim], qo[:, sim]) < 2e-7
    assert rel(s.get_velocity()[:, sim], vo[:, sim]) < 2e-6
