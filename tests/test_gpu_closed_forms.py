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
