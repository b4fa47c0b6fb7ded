"""Host-side fault injection (no device fault is ever made): a device
allocation or a step-kernel launch that fails on request, the status the
library returns, and that the failing solver, other solvers and the server
keep working afterwards."""
import numpy as np
import pytest

from _helpers import HOM, need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

A, B, C = synth.A_5CB, synth.B_5CB, synth.C_5CB
FP = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    lqmin.inject_fault(lqmin.LQ_FAULT_NONE)


def mk(shape=(24, 20, 18), objects=(), prec=lqmin.LQ_FP64):
    s = lqmin.Solver(shape, A, B, C, 2.32, 0.5, 0.3, precision=prec)
    s.add_objects(list(objects))
    return s


SPHERE = dict(type="sphere", c=(12.0, 10.0, 9.0), R=4.0, anchor=HOM())


def test_allocation_failure_in_create_returns_enomem():
    other = mk()
    other.init_random_uniaxial(1)
    lqmin.inject_fault(lqmin.LQ_FAULT_DEVICE_ALLOC, 0)
    with pytest.raises(lqmin.LqError) as e:
        mk((16, 16, 16))
    assert e.value.status == lqmin.LQ_ENOMEM
    s = mk((16, 16, 16))                       # the injection was one-shot
    s.init_random_uniaxial(2)
    r = other.step(lqmin.fire_params(**FP), 5)
    assert r.iterations == 5 and r.fire_status == lqmin.FIRE_RUNNING


@pytest.mark.parametrize("after", [0, 1, 2, 4])
def test_allocation_failure_in_geometry_build_is_recoverable(after):
    s = mk(objects=[SPHERE])
    lqmin.inject_fault(lqmin.LQ_FAULT_DEVICE_ALLOC, after)
    with pytest.raises(lqmin.LqError) as e:
        s.geometry_info()
    assert e.value.status == lqmin.LQ_ENOMEM
    fresh = mk(objects=[SPHERE])
    assert s.geometry_info() == fresh.geometry_info()
    assert np.array_equal(s.mask(), fresh.mask())
    q = synth.random_uniaxial_q(s.shape, 3)
    s.set_q(q)
    fresh.set_q(q)
    assert np.array_equal(s.force(), fresh.force())


@pytest.mark.parametrize("prec", [lqmin.LQ_FP64, lqmin.LQ_FP32_BULK_FP64_RED])
@pytest.mark.parametrize("after", [0, 1, 3])
def test_step_launch_failure_returns_ecuda_and_the_solver_recovers(prec, after):
    a, b = mk(objects=[SPHERE], prec=prec), mk(prec=prec)
    for s in (a, b):
        s.init_random_uniaxial(4)
    p = lqmin.fire_params(**FP)
    a.step(p, 1)
    lqmin.inject_fault(lqmin.LQ_FAULT_STEP_LAUNCH, after)
    a.set_q(a.get_q())                         # the next step starts FIRE afresh
    with pytest.raises(lqmin.LqError) as e:
        a.step(p, 200)
    assert e.value.status == lqmin.LQ_ECUDA
    rb = b.step(p, 20)                         # another solver is untouched
    assert rb.iterations == 20
    # the failed solver restarts from a state it reads back and then runs
    # exactly like a fresh solver from that state
    q = a.get_q()
    fresh = mk(objects=[SPHERE], prec=prec)
    for s in (a, fresh):
        s.set_q(q)
    ra, rf = a.step(p, 30), fresh.step(p, 30)
    assert ra.iterations == rf.iterations == 30
    assert np.array_equal(a.get_q(), fresh.get_q())


def test_batch_launch_failure_returns_ecuda_and_the_batch_recovers():
    solvers = [mk(objects=[SPHERE], prec=lqmin.LQ_FP32_BULK_FP64_RED),
               mk(prec=lqmin.LQ_FP32_BULK_FP64_RED)]
    for k, s in enumerate(solvers):
        s.init_random_uniaxial(10 + k)
    batch = lqmin.Batch(solvers)
    p = lqmin.fire_params(**FP)
    batch.step(p, 3)
    lqmin.inject_fault(lqmin.LQ_FAULT_STEP_LAUNCH, 0)
    with pytest.raises(lqmin.LqError) as e:
        batch.step(p, 5)
    assert e.value.status == lqmin.LQ_ECUDA
    res = batch.step(p, 5)
    assert all(r.fire_status == lqmin.FIRE_RUNNING for r in res)
    batch.close()


def test_served_request_whose_allocation_fails():
    sv = lqmin.Server(hbm_budget_bytes=4 << 30)
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=200000, force_tol=1e-6))
    cfg = dict(shape=(24, 24, 20), L1=2.32, objects=[])
    lqmin.inject_fault(lqmin.LQ_FAULT_DEVICE_ALLOC, 0)
    t_bad = sv.submit(cfg, p, seed=1)
    code_bad, _, _ = sv.wait(t_bad, timeout=120)
    t_ok = sv.submit(cfg, p, seed=2)
    code_ok, r, _ = sv.wait(t_ok, timeout=300)
    assert code_bad == lqmin.LQ_ENOMEM and code_ok == lqmin.LQ_OK
    assert r.fire_status == lqmin.FIRE_CONVERGED
    sv.close()


def test_injection_arguments_are_checked():
    with pytest.raises(lqmin.LqError):
        lqmin.inject_fault(lqmin.LQ_FAULT_COPY_WAIT + 1)     # no such kind
    with pytest.raises(lqmin.LqError):
        lqmin.inject_fault(-1)
    with pytest.raises(lqmin.LqError):
        lqmin.inject_fault(lqmin.LQ_FAULT_DEVICE_ALLOC, -1)
    lqmin.inject_fault(lqmin.LQ_FAULT_NONE)                   # nothing stays armed


def test_served_round_with_a_failed_launch_is_retried():
    """A persistent-kernel round of the server whose launch fails is rebuilt
    and retried; the request still converges."""
    import time
    sv = lqmin.Server(hbm_budget_bytes=4 << 30)
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=400000, force_tol=1e-6))
    t = sv.submit(dict(shape=(48, 48, 40), L1=2.32, objects=[]), p, seed=3)
    t0 = time.time()
    # inject once the solve runs its rounds (its admission, which also
    # launches a step kernel, is over): the failed launch is a round's
    while sv.stats()["site_updates_issued"] == 0 and time.time() - t0 < 60:
        time.sleep(0.005)
    lqmin.inject_fault(lqmin.LQ_FAULT_STEP_LAUNCH, 0)
    code, r, _ = sv.wait(t, timeout=300)
    assert code == lqmin.LQ_OK and r.fire_status == lqmin.FIRE_CONVERGED
    sv.close()
