"""The CUDA path against closed forms of the mathematics, with no oracle in
between: the bulk force of a uniform uniaxial state is the derivative of the
Landau polynomial of Eq. (fphase) along the uniaxial family (and vanishes at
S0 of Eq. (S0def)), and a small Q_xy plane wave is an eigenvector of the
one-constant distortion force with the eigenvalue of the periodic second
difference (the averaged one-sided differences of section III.B)."""
import math

import numpy as np
import pytest

from _helpers import need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

A, B, C = synth.A_5CB, synth.B_5CB, synth.C_5CB


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def df_dS(S):
    """d/dS of the bulk density of Q = 3/2 S (nn - I/3): tr Q^2 = 3 S^2 / 2,
    tr Q^3 = 3 S^3 / 4, so f = 3A S^2/4 + B S^3/4 + 9C S^4/16."""
    return 1.5 * A * S + 0.75 * B * S * S + 2.25 * C * S ** 3


@pytest.mark.parametrize("precision", [lqmin.LQ_FP64, lqmin.LQ_FP32_BULK_FP64_RED])
def test_uniform_uniaxial_force_is_the_polynomial_derivative(precision):
    shape = (12, 10, 8)
    N = shape[0] * shape[1] * shape[2]
    s = lqmin.Solver(shape, A, B, C, 2.32, 0.5, 0.3, precision=precision)
    S0 = synth.s0_closed_form(A, B, C)
    n = synth.random_directors(1, 7)
    tol = 1e-12 if precision == lqmin.LQ_FP64 else 2e-6
    for S in (0.2, 0.45, 0.8, S0):
        q = np.repeat(synth.uniaxial_q(n, S), N, axis=1)
        if precision == lqmin.LQ_FP32_BULK_FP64_RED:
            q = np.round(q * 2.0 ** 28) / 2.0 ** 28
        s.set_q(q)
        F = s.force()
        # every site alike; no distortion force on a uniform state
        assert np.abs(F - F[:, :1]).max() <= tol * max(np.abs(F).max(), 1e-12)
        proj = -(F[:, 0] * q[:, 0]).sum() / S
        if S == S0:
            assert abs(proj) < (1e-13 if precision == lqmin.LQ_FP64 else 1e-6)
        else:
            assert abs(proj - df_dS(S)) <= tol * abs(df_dS(S))
    s.close()


@pytest.mark.parametrize("precision,nx,eps,tol", [
    (lqmin.LQ_FP64, 16, 1e-6, 1e-9),
    # 256 wide: the FP32 form's 64-wide one-constant tiles
    (lqmin.LQ_FP32_BULK_FP64_RED, 256, 5e-4, 5e-5),
])
def test_plane_wave_is_an_eigenvector_of_the_one_constant_force(precision, nx, eps, tol):
    """Q_xy = eps cos(2 pi m x / nx) about Q = 0: the force on Q_xy is
    -(2A + 2 L1 lambda_m) q with lambda_m = 2 (1 - cos(2 pi m / nx)); the
    factor 2 is the symmetric pair Q_xy = Q_yx.  Q_xz and Q_yz stay
    force-free; Q_xx and Q_yy see only the B term, of order eps^2.  The FP32
    form stores Q on the 2^-28 grid: rounding moves each value by at most
    d = 2^-29, which the operator maps to at most (2|A| + 8 L1) d, so its
    force is compared with the exact wave's within that bound."""
    shape = (nx, 4, 6)
    L1 = 2.32
    N = shape[0] * shape[1] * shape[2]
    s = lqmin.Solver(shape, A, B, C, L1, precision=precision)
    x = np.tile(np.arange(nx), shape[1] * shape[2]).astype(float)
    for m in (1, 3, nx // 4):
        q = np.zeros((5, N))
        q[1] = eps * np.cos(2 * math.pi * m * x / nx)
        s.set_q(q)
        F = s.force()
        lam = 2 * (1 - math.cos(2 * math.pi * m / nx))
        want = -(2 * A + 2 * L1 * lam) * q[1]
        bound = tol * eps * abs(2 * A + 2 * L1 * lam)
        if precision == lqmin.LQ_FP32_BULK_FP64_RED:
            bound += (2 * abs(A) + 8 * L1) * 2.0 ** -29
        assert np.abs(F[1] - want).max() <= bound
        assert np.abs(F[[2, 4]]).max() <= (1e-30 if precision == lqmin.LQ_FP64 else 1e-12)
        assert np.abs(F[[0, 3]]).max() <= 2 * abs(B) * eps ** 2
    s.close()


@pytest.mark.parametrize("precision", [lqmin.LQ_FP64, lqmin.LQ_FP32_BULK_FP64_RED])
@pytest.mark.parametrize("kind", [lqmin.ND_HOMEOTROPIC, lqmin.FG_PLANAR])
def test_wall_anchoring_energy_of_a_uniform_director(precision, kind):
    """A wall at z = 0 (normal nu = e_z) and a uniform uniaxial state at S0
    with director n, c = n . nu.  Per boundary site (area weight 1):
    Nobili-Durand homeotropic W |Q - Q0|^2 = W (9 S0^2 / 2)(1 - c^2);
    Fournier-Galatola planar W |Qt - P Qt P|^2 = W (9 S0^2 / 4)(2 c^2 - c^4)
    (Qt = Q + S0/2 I = 3 S0/2 nn, P = I - nu nu).  The aligned state (c = 1
    homeotropic, c = 0 planar) feels no force anywhere."""
    shape = (8, 6, 10)
    W = 1.7
    s = lqmin.Solver(shape, A, B, C, 2.32, 0.5, 0.3, precision=precision)
    s.add_wall(2, 0, kind, W)
    S0 = synth.s0_closed_form(A, B, C)
    N = shape[0] * shape[1] * shape[2]
    _, nanch = s.geometry_info()
    assert nanch == 2 * shape[0] * shape[1]      # planes z = 1 and z = 9 (periodic)
    tol = 1e-12 if precision == lqmin.LQ_FP64 else 1e-6
    for c in (1.0, 0.6, 0.0):
        n = np.array([[math.sqrt(1 - c * c)], [0.0], [c]])
        q = np.repeat(synth.uniaxial_q(n, S0), N, axis=1)
        if precision == lqmin.LQ_FP32_BULK_FP64_RED:
            q = np.round(q * 2.0 ** 28) / 2.0 ** 28
        s.set_q(q)
        _, parts = s.energy()
        if kind == lqmin.ND_HOMEOTROPIC:
            per = W * 4.5 * S0 ** 2 * (1 - c * c)
        else:
            per = W * 2.25 * S0 ** 2 * (2 * c * c - c ** 4)
        assert abs(parts[2] - nanch * per) <= tol * max(nanch * per, 1.0)
        assert abs(parts[1]) <= tol        # uniform: no distortion energy
        aligned = (c == 1.0) if kind == lqmin.ND_HOMEOTROPIC else (c == 0.0)
        if aligned:
            sim = s.mask() & 1
            assert np.abs(s.force()[:, sim.astype(bool)]).max() < (1e-12 if tol == 1e-12 else 1e-6)
    s.close()


@pytest.mark.parametrize("precision,tol", [(lqmin.LQ_FP64, 1e-12),
                                           (lqmin.LQ_FP32_BULK_FP64_RED, 2e-6)])
def test_fire_from_rest_on_a_harmonic_bulk_is_velocity_verlet(precision, tol):
    """With B = C = 0 the bulk density A/2 tr Q^2 is harmonic in q:
    -dF/dq_xx = -A (2 q_xx + q_yy), -dF/dq_xz = -2A q_xz, so q_xx = q_yy is a
    mode with w^2 = 3A and q_xz one with w^2 = 2A.  FIRE with alpha0 = 0 and
    f_inc = 1 is plain velocity Verlet while P > 0, and velocity Verlet from
    rest follows q_n = q_0 cos(n theta), cos theta = 1 - w^2 dt^2 / 2
    (the Stormer recurrence), for every mode and every site."""
    shape = (6, 4, 4)
    N = shape[0] * shape[1] * shape[2]
    Ah, dt = 1.0, 0.05
    s = lqmin.Solver(shape, Ah, 0.0, 0.0, 2.32, 0.5, 0.3, precision=precision, S0=0.5)
    q0 = np.zeros((5, N))
    q0[0] = q0[3] = 0.125
    q0[2] = 0.25
    s.set_q(q0)
    p = lqmin.fire_params(dt0=dt, dt_max=dt, alpha0=0.0, f_alpha=0.99, f_inc=1.0, f_dec=0.5,
                          n_min=5, max_iter=10 ** 6, force_tol=1e-14)
    n = 10
    r = s.step(p, n)
    assert r.iterations == n and r.dt == dt and r.npos == n
    q = s.get_q()
    for c, w2 in ((0, 3 * Ah), (3, 3 * Ah), (2, 2 * Ah)):
        theta = math.acos(1 - w2 * dt * dt / 2)
        want = q0[c] * math.cos(n * theta)
        assert np.abs(q[c] - want).max() <= tol * abs(want[0])
    assert np.abs(q[[1, 4]]).max() == 0.0
    s.close()


@pytest.mark.parametrize("method", [lqmin.LQ_MIN_GD, lqmin.LQ_MIN_NESTEROV])
def test_descent_on_a_harmonic_bulk_follows_its_recurrence(method):
    """The same harmonic bulk, modes w^2 = 3A (q_xx = q_yy) and 2A (q_xz):
    gradient descent with step eta gives a_n = (1 - eta w^2)^n a_0; Nesterov
    with momentum mu gives a_{k+1} = (1 - eta w^2) b_k, b_k = a_k + mu (a_k -
    a_{k-1}), a_{-1} = a_0, and the state it holds is the evaluation point
    b_n."""
    shape = (6, 4, 4)
    N = shape[0] * shape[1] * shape[2]
    Ah, eta, mu, n = 1.0, 0.05, 0.7, 25
    s = lqmin.Solver(shape, Ah, 0.0, 0.0, 2.32, 0.5, 0.3, S0=0.5)
    q0 = np.zeros((5, N))
    q0[0] = q0[3] = 0.125
    q0[2] = 0.25
    s.set_q(q0)
    m = mu if method == lqmin.LQ_MIN_NESTEROV else 0.0
    r = s.step(lqmin.descent_params(method, eta, momentum=m, max_iter=10 ** 6, force_tol=1e-14), n)
    assert r.iterations == n
    q = s.get_q()
    for c, w2 in ((0, 3 * Ah), (3, 3 * Ah), (2, 2 * Ah)):
        a_prev = a = 1.0
        for _ in range(n):
            b = a + m * (a - a_prev)
            a_prev, a = a, (1 - eta * w2) * b
        held = a + m * (a - a_prev)
        want = q0[c] * held
        assert np.abs(q[c] - want).max() <= 1e-12 * abs(q0[c, 0])
    assert np.abs(q[[1, 4]]).max() == 0.0
    s.close()


def test_batched_fire_from_rest_on_harmonic_bulks_is_velocity_verlet():
    """Three lattices of different sizes and stiffness in one batch (one
    persistent launch per iteration): each follows its own velocity Verlet
    closed form, as above."""
    dt, n = 0.05, 12
    cases = [((6, 4, 4), 1.0), ((40, 9, 7), 0.6), ((33, 20, 5), 1.4)]
    solvers, q0s = [], []
    for shape, Ah in cases:
        N = shape[0] * shape[1] * shape[2]
        s = lqmin.Solver(shape, Ah, 0.0, 0.0, 2.32, 0.5, 0.3, S0=0.5)
        q0 = np.zeros((5, N))
        q0[0] = q0[3] = 0.125
        q0[2] = 0.25
        s.set_q(q0)
        solvers.append(s)
        q0s.append(q0)
    batch = lqmin.Batch(solvers)
    p = lqmin.fire_params(dt0=dt, dt_max=dt, alpha0=0.0, f_alpha=0.99, f_inc=1.0, f_dec=0.5,
                          n_min=5, max_iter=10 ** 6, force_tol=1e-14)
    res = batch.step(p, n)
    for (shape, Ah), s, q0, r in zip(cases, solvers, q0s, res):
        assert r.iterations == n
        q = s.get_q()
        for c, w2 in ((0, 3 * Ah), (3, 3 * Ah), (2, 2 * Ah)):
            theta = math.acos(1 - w2 * dt * dt / 2)
            want = q0[c] * math.cos(n * theta)
            assert np.abs(q[c] - want).max() <= 1e-12 * abs(want[0])
    batch.close()
    for s in solvers:
        s.close()


def test_l2_and_l3_agree_on_a_periodic_lattice_without_objects():
    """On a fully periodic lattice without objects the averaged L2 and L3
    terms are equal for every Q (centred differences commute and sum by
    parts), so the GPU's energies and forces with (L2, L3) = (1, 0) and
    (0, 1) agree, at a size the oracle is never run on."""
    shape = (96, 80, 64)
    q = synth.random_uniaxial_q(shape, 17)
    out = []
    for L2, L3 in ((1.0, 0.0), (0.0, 1.0)):
        s = lqmin.Solver(shape, A, B, C, 0.0, L2, L3, n_constants=3)
        s.set_q(q)
        out.append((s.energy()[1][1], s.force()))
        s.close()
    (e2, F2), (e3, F3) = out
    assert abs(e2 - e3) <= 1e-11 * abs(e2)
    assert np.abs(F2 - F3).max() <= 1e-10 * np.abs(F2).max()


def test_swapping_x_and_y_maps_energy_and_force():
    """The mirror x <-> y of lattice, objects and Q (Q'_xx = Q_yy, Q'_xy =
    Q_xy, Q'_xz = Q_yz, ...) leaves the bulk, L1, L2, L3 and anchoring
    energy unchanged and maps the force the same way."""
    n = 40
    shape = (n, n, 24)
    c = (17.0, 17.0, 12.0)     # on the diagonal: the sphere is its own mirror image
    objs = [dict(type="wall", axis=2, plane=0, anchor=(lqmin.FG_PLANAR, 1.0, (0, 0, 1))),
            dict(type="sphere", c=c, R=6.0, anchor=(lqmin.ND_HOMEOTROPIC, 5.3, (0, 0, 1)))]
    q = synth.random_uniaxial_q(shape, 18)
    qs = q.reshape(5, shape[2], n, n)            # [c][z][y][x]
    perm = [3, 1, 4, 0, 2]                       # (xx, xy, xz, yy, yz) <- (yy, xy, yz, xx, xz)
    qm = qs[perm].transpose(0, 1, 3, 2).reshape(5, -1)
    res = []
    for state in (q, qm):
        s = lqmin.Solver(shape, A, B, C, 2.32, 0.5, 0.3)
        s.add_objects(objs)
        s.set_q(state)
        res.append((s.energy(), s.force()))
        s.close()
    (E, parts), F = res[0]
    (Em, partsm), Fm = res[1]
    assert abs(E - Em) <= 1e-12 * abs(E)
    assert np.allclose(parts, partsm, rtol=1e-12, atol=1e-12 * abs(E))
    Fmap = F.reshape(5, shape[2], n, n)[perm].transpose(0, 1, 3, 2).reshape(5, -1)
    assert np.abs(Fm - Fmap).max() <= 1e-10 * np.abs(F).max()


@pytest.mark.parametrize("precision,tol", [(lqmin.LQ_FP64, 1e-10),
                                           (lqmin.LQ_FP32_BULK_FP64_RED, 1e-5)])
def test_chiral_term_is_odd_under_the_mirror(precision, tol):
    """The chiral density eps_lik Q_lj dQ_ij/dx_k changes sign under a
    reflection: with only L4 (no bulk, no other elastic term) the mirror
    x <-> y of Q negates the energy and the mapped force."""
    n = 32
    shape = (n, n, 20)
    q = synth.random_uniaxial_q(shape, 19)
    if precision == lqmin.LQ_FP32_BULK_FP64_RED:
        q = np.round(q * 2.0 ** 28) / 2.0 ** 28
    perm = [3, 1, 4, 0, 2]
    qm = q.reshape(5, shape[2], n, n)[perm].transpose(0, 1, 3, 2).reshape(5, -1)
    res = []
    for state in (q, qm):
        s = lqmin.Solver(shape, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, precision=precision, L4=0.7,
                         n_constants=3, S0=0.5)
        s.set_q(state)
        res.append((s.energy()[1][1], s.force()))
        s.close()
    (e, F), (em, Fm) = res
    assert abs(e) > 1.0
    assert abs(e + em) <= tol * abs(e)
    Fmap = F.reshape(5, shape[2], n, n)[perm].transpose(0, 1, 3, 2).reshape(5, -1)
    assert np.abs(Fm + Fmap).max() <= tol * np.abs(F).max()
