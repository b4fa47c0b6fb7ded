"""Serving: requests of different sizes and geometries arrive while others
run, are admitted by the HBM budget, share the persistent-kernel launches,
and each result equals the same minimisation run alone -- bit for bit for
one-constant requests, within the FP32 form's tolerance otherwise."""
import time

import numpy as np
import pytest

from _helpers import HOM, PLANAR, need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

A, B, C = synth.A_5CB, synth.B_5CB, synth.C_5CB


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def requests():
    hom = HOM()
    return [
        dict(shape=(32, 32, 24), L1=2.32, objects=[dict(type="sphere", c=(16.0, 16.0, 12.0), R=5.0,
                                                        anchor=hom)], seed=11),
        dict(shape=(48, 24, 20), L1=2.32, objects=[dict(type="wall", axis=2, plane=0, anchor=hom),
                                                   dict(type="wall", axis=2, plane=19, anchor=hom)],
             seed=12),
        dict(shape=(24, 24, 24), L1=2.32, L2=0.5, L3=0.3,
             objects=[dict(type="sphere", c=(12.0, 12.0, 12.0), R=4.0, anchor=hom)], seed=13),
        dict(shape=(40, 40, 16), L1=2.32, objects=[
            dict(type="anchored", xyz=np.stack(np.meshgrid(np.arange(40), np.arange(40), [1],
                                                           indexing="ij"), -1).reshape(-1, 3),
                 kinds=1, W=5.3, dirs=[1.0, 0.0, 0.0]),
            dict(type="wall", axis=2, plane=0, anchor=hom),
            dict(type="wall", axis=2, plane=15, anchor=PLANAR())], seed=14),
        dict(shape=(28, 36, 20), L1=2.32, objects=[], seed=15),
        dict(shape=(26, 24, 24), L1=2.32,
             objects=[dict(type="spherocylinder", c=(9.0, 11.0, 10.0), c2=(15.0, 13.0, 13.0),
                           R=2.0, anchor=PLANAR()),
                      dict(type="droplet", c=(12.5, 11.5, 11.5), R=10.5, anchor=hom)], seed=16),
    ]


def params():
    # convergence to max|F| < 1e-6: two runs that differ by rounding then agree in S
    # to ~|F| / (slowest stiffness ~0.03) = 3e-5
    return lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=200000, force_tol=1e-6))


def alone(cfg):
    s = lqmin.Solver(cfg["shape"], A, B, C, cfg["L1"], cfg.get("L2", 0.0), cfg.get("L3", 0.0),
                     precision=lqmin.LQ_FP32_BULK_FP64_RED)
    s.add_objects(cfg["objects"])
    s.init_random_uniaxial(cfg["seed"])
    code, r = s.minimize(params())
    S = s.order_field()
    s.close()
    return code, r, S


def test_served_results_equal_alone_results():
    sv = lqmin.Server(hbm_budget_bytes=8 << 30, max_active=8)
    tickets = []
    for cfg in requests():           # staggered arrivals: later ones join running work
        tickets.append(sv.submit(cfg, params(), seed=cfg["seed"], want_S=True))
        time.sleep(0.02)
    served = [sv.wait(t, timeout=300, S=True) for t in tickets]
    stats = sv.stats()
    sv.close()
    assert stats["completed"] == len(tickets)
    for cfg, (code, r, S) in zip(requests(), served):
        ca, ra, Sa = alone(cfg)
        assert code == ca == lqmin.LQ_OK and r.fire_status == lqmin.FIRE_CONVERGED
        if cfg.get("L2", 0.0) == 0.0:
            assert r.iterations == ra.iterations
            assert r.energy == ra.energy and np.array_equal(S, Sa)
        else:
            assert abs(r.energy - ra.energy) <= 1e-6 * abs(ra.energy)
            assert np.abs(S - Sa).max() < 1e-4
        assert r.seconds > 0


def test_budget_admits_one_at_a_time_and_refuses_oversized():
    cfgs = requests()[:3]
    one = max(int(np.prod(c["shape"])) for c in cfgs) * 200 + (2 << 20)
    sv = lqmin.Server(hbm_budget_bytes=one, max_active=8)
    tickets = [sv.submit(c, params(), seed=c["seed"]) for c in cfgs]
    seen_active = 0
    deadline = time.time() + 300
    while sv.stats()["completed"] < len(tickets) and time.time() < deadline:
        seen_active = max(seen_active, sv.stats()["active"])
        time.sleep(0.002)
    assert sv.stats()["completed"] == len(tickets) and seen_active == 1
    for t in tickets:
        code, r, _ = sv.poll(t)
        assert code == lqmin.LQ_OK
    with pytest.raises(lqmin.LqError):
        sv.submit(dict(shape=(400, 400, 400), L1=2.32, objects=[]), params())
    sv.close()


def test_failed_request_does_not_stop_the_server():
    sv = lqmin.Server(hbm_budget_bytes=4 << 30)
    bad_q = np.full((5, 16 * 16 * 16), 3.0)          # outside the FP32 form's |q| < 2
    t_bad = sv.submit(dict(shape=(16, 16, 16), L1=2.32, objects=[]), params(), q0=bad_q)
    t_ok = sv.submit(requests()[4], params(), seed=15)
    code_bad, _, _ = sv.wait(t_bad, timeout=120)
    code_ok, r, _ = sv.wait(t_ok, timeout=300)
    assert code_bad == lqmin.LQ_EINVAL and code_ok == lqmin.LQ_OK
    sv.close()
