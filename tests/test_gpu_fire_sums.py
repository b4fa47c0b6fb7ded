"""FIRE reductions of the FP32-bulk form, checked against FP64 (Algorithm 1's
power P = F.v, the norms |F|^2 and |v|^2, and the convergence residual, the
largest site |F|^2).  After a few fused steps the device's sums must equal
the same sums recomputed exactly (math.fsum of FP64 products, which are exact
for FP32 operands) from the FP32 velocity and force the step stored, to
1e-12 relative, in every kernel form that forms them: three constants,
one constant (32- and 64-wide tiles), the chiral form, and a batch."""
import math

import numpy as np
import pytest

from _helpers import HOM, PLANAR, need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

FP = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def stored_v_f(s):
    """The FP32 form's stored velocity and force (Q is fixed point; v, F are
    float32), read from a checkpoint: header, then q, v, F arrays."""
    buf = s.get_state()
    arr = 5 * s.N * 4
    hdr = len(buf) - 3 * arr
    v = np.frombuffer(buf[hdr + arr:hdr + 2 * arr].tobytes(), dtype=np.float32).reshape(5, s.N)
    F = np.frombuffer(buf[hdr + 2 * arr:hdr + 3 * arr].tobytes(), dtype=np.float32).reshape(5, s.N)
    return v.astype(np.float64), F.astype(np.float64)


def exact_sums(s):
    v, F = stored_v_f(s)
    sim = (s.mask() & 1) != 0
    v, F = v[:, sim], F[:, sim]
    P = math.fsum((F * v).ravel())
    F2 = math.fsum((F * F).ravel())
    V2 = math.fsum((v * v).ravel())
    site = np.array([math.fsum(col) for col in (F * F).T])
    return P, F2, V2, float(site.max()), math.fsum(np.abs(F * v).ravel())


def check(s, r):
    P, F2, V2, R2, Pabs = exact_sums(s)
    assert P > 0.0 and Pabs < 100.0 * P      # not a cancellation-dominated state
    assert abs(r.power - P) <= 1e-12 * abs(P), (r.power, P)
    assert abs(r.norm_force ** 2 - F2) <= 1e-12 * F2, (r.norm_force ** 2, F2)
    assert abs(r.norm_velocity ** 2 - V2) <= 1e-12 * V2, (r.norm_velocity ** 2, V2)
    assert abs(r.max_force ** 2 - R2) <= 1e-12 * R2, (r.max_force ** 2, R2)


OBJS = [dict(type="wall", axis=2, plane=0, anchor=PLANAR()),
        dict(type="sphere", c=(15.0, 13.0, 11.0), R=5.0, anchor=HOM())]
FORMS = {
    "three_constants": dict(shape=(36, 26, 22), L=(2.32, 0.5, 0.3), objects=OBJS),
    "one_constant": dict(shape=(36, 26, 22), L=(2.32, 0.0, 0.0), objects=OBJS),
    "one_constant_wide_tiles": dict(shape=(256, 10, 8), L=(2.32, 0.0, 0.0), objects=[]),
    "chiral_field": dict(shape=(36, 26, 22), L=(2.32, 0.5, 0.3), objects=OBJS,
                         extra=dict(L4=0.6, H=(0.3, -0.2, 0.5), mu0_dchi=1.3)),
}


@pytest.mark.parametrize("name", sorted(FORMS))
def test_fp32_form_fire_sums_are_fp64_exact(name):
    g = FORMS[name]
    s = lqmin.Solver(g["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, *g["L"], precision=1,
                     **g.get("extra", {}))
    s.add_objects(g["objects"])
    s.set_q(synth.random_uniaxial_q(g["shape"], 5))
    p = lqmin.fire_params(**FP)
    for n in (3, 4):          # two readings in a row
        r = s.step(p, n)
        check(s, r)
    s.close()


def test_fp32_form_fire_sums_in_a_batch():
    shapes = [(40, 24, 20), (32, 32, 16)]
    solvers = []
    for k, shape in enumerate(shapes):
        s = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, 0.0, 0.0, precision=1)
        s.add_objects([dict(type="sphere", c=tuple(x / 2.0 for x in shape), R=4.0, anchor=HOM())])
        s.set_q(synth.random_uniaxial_q(shape, 20 + k))
        solvers.append(s)
    batch = lqmin.Batch(solvers)
    res = batch.step(lqmin.fire_params(**FP), 5)
    for s, r in zip(solvers, res):
        check(s, r)
    batch.close()
    for s in solvers:
        s.close()
