"""Pins of the CPU oracle to things other than itself: closed forms the paper
states, hand-derived values, invariants of the continuum and of the
discretisation, finite differences of its own energy, and library routines
for special cases.  No GPU.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1911_07045_b300 import synth

A, B, C = synth.A_5CB, synth.B_5CB, synth.C_5CB
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def s0_poly(A_, B_, C_):
    # Eq. (S0def), written independently of the oracle
    return (-B_ + math.sqrt(B_ * B_ - 24 * A_ * C_)) / (6 * C_)


def f_of_S(S, A_=A, B_=B, C_=C):
    # Eq. (fphaseS): the uniaxial reduction of the bulk energy
    return 0.75 * A_ * S ** 2 + 0.25 * B_ * S ** 3 + 9.0 / 16.0 * C_ * S ** 4


def df_dS(S, A_=A, B_=B, C_=C):
    return 1.5 * A_ * S + 0.75 * B_ * S ** 2 + 2.25 * C_ * S ** 3


def rand_q(N, seed, scale=0.3):
    return np.random.default_rng(seed).normal(scale=scale, size=(5, N))


def full_Q(q):
    """(N,3,3) tensors from (5,N) components."""
    N = q.shape[1]
    Q = np.zeros((N, 3, 3))
    Q[:, 0, 0], Q[:, 0, 1], Q[:, 0, 2] = q[0], q[1], q[2]
    Q[:, 1, 0], Q[:, 1, 1], Q[:, 1, 2] = q[1], q[3], q[4]
    Q[:, 2, 0], Q[:, 2, 1], Q[:, 2, 2] = q[2], q[4], -q[0] - q[3]
    return Q


def comps(Q):
    return np.stack([Q[:, 0, 0], Q[:, 0, 1], Q[:, 0, 2], Q[:, 1, 1], Q[:, 1, 2]])


# ---- paper's printed numbers ------------------------------------------------

def test_paper_5cb_numbers(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "paper_5cb.json")))
    S0 = oracle_mod.uniaxial_s0(g["A"], g["B"], g["C"])
    assert abs(S0 - g["S0_printed"]) < g["S0_printed_digits"]
    # K = L1 9 S0^2 / 2  and  dx^2 = L1 / (L1~ |A|)
    L1 = 2 * g["K_newton"] / (9 * S0 ** 2)
    dx_nm = math.sqrt(L1 / (g["L1_tilde"] * abs(g["A"]))) * 1e9
    assert abs(dx_nm - g["dx_nm_printed"]) < g["dx_nm_printed_digits"]
    # lattice-unit constants have the same S0 (S0 depends on ratios only)
    assert abs(oracle_mod.uniaxial_s0(A, B, C) - S0) < 1e-14


def test_rapini_papoular_identity(oracle_mod):
    """Uniaxial Q at S0 at angle theta to the preferred axis: Nobili-Durand
    energy = 9/2 S0^2 W sin^2(theta), i.e. the Rapini-Papoular form with
    W_RP = 9 S0^2 W_ND up to a constant."""
    g = json.load(open(os.path.join(GOLD, "paper_5cb.json")))
    W = 1.7
    for theta in (0.0, 0.3, 1.0, math.pi / 2):
        nu = np.array([0.0, 0.0, 1.0])
        o = oracle_mod.Oracle((3, 3, 3), A, B, C, 1.0, objects=[dict(
            type="anchored", xyz=[[1, 1, 1]], kinds=[oracle_mod.ND_ORIENTED], W=[W],
            dirs=[nu])])
        S0 = o.S0
        n = np.array([math.sin(theta), 0.0, math.cos(theta)])
        q = np.repeat(synth.uniaxial_q(n[:, None], S0), 27, axis=1)
        _, parts = o.energy(q)
        rp = -0.5 * g["W_RP_over_W_ND_over_S0sq"] * S0 ** 2 * W * math.cos(theta) ** 2
        assert abs(parts[2] - (4.5 * S0 ** 2 * W + rp)) < 1e-13
        assert abs(parts[2] - 4.5 * S0 ** 2 * W * math.sin(theta) ** 2) < 1e-13


def test_fournier_galatola_values(oracle_mod):
    """Planar-degenerate form: 0 for any in-plane director at S0, and
    9/4 S0^2 W cos^2 t (1 + sin^2 t) for a director tilted by t from nu."""
    W = 0.8
    nu = np.array([1.0, 2.0, 2.0]) / 3.0
    t1 = np.cross(nu, [0, 0, 1.0]); t1 /= np.linalg.norm(t1)
    t2 = np.cross(nu, t1)
    o = oracle_mod.Oracle((3, 3, 3), A, B, C, 1.0, objects=[dict(
        type="anchored", xyz=[[0, 2, 1]], kinds=[oracle_mod.FG_PLANAR], W=[W], dirs=[nu])])
    S0 = o.S0
    for phi in (0.0, 0.7, 2.0):
        n = math.cos(phi) * t1 + math.sin(phi) * t2
        q = np.repeat(synth.uniaxial_q(n[:, None], S0), 27, axis=1)
        assert abs(o.energy(q)[1][2]) < 1e-14
    for t in (0.2, 0.9, 1.3):
        n = math.cos(t) * nu + math.sin(t) * t1
        q = np.repeat(synth.uniaxial_q(n[:, None], S0), 27, axis=1)
        want = 2.25 * S0 ** 2 * W * math.cos(t) ** 2 * (1 + math.sin(t) ** 2)
        assert abs(o.energy(q)[1][2] - want) < 1e-13


# ---- bulk --------------------------------------------------------------------

@pytest.mark.parametrize("mat", [(A, B, C), (-1.0, -12.3256, 10.0581)])
def test_uniform_s0_is_stationary(oracle_mod, mat):
    A_, B_, C_ = mat
    S0 = s0_poly(A_, B_, C_)
    assert abs(df_dS(S0, A_, B_, C_)) < 1e-13
    shape = (3, 4, 2)
    N = 24
    n = synth.random_directors(1, 11)
    q = np.repeat(synth.uniaxial_q(n, S0), N, axis=1)
    o = oracle_mod.Oracle(shape, A_, B_, C_, 2.32, 0.5, 0.3)
    E, parts = o.energy(q)
    assert abs(E - N * f_of_S(S0, A_, B_, C_)) < 1e-13 * N
    assert parts[1] == 0.0
    assert np.abs(o.force(q)).max() < 1e-14


@pytest.mark.parametrize("S", [0.1, 0.3, 0.75, -0.2])
def test_uniform_uniaxial_force_is_polynomial_derivative(oracle_mod, S):
    n = synth.random_directors(1, 7)
    q = np.repeat(synth.uniaxial_q(n, S), 8, axis=1)
    o = oracle_mod.Oracle((2, 2, 2), A, B, C, 2.32)
    E, _ = o.energy(q)
    assert abs(E - 8 * f_of_S(S)) < 1e-14
    F = o.force(q)
    # -F . dq/dS = df/dS along the uniaxial family q(S) = S q(1)
    proj = -(F[:, 0] * q[:, 0] / S).sum()
    assert abs(proj - df_dS(S)) < 1e-13


def test_bulk_gradient_biaxial_fd(oracle_mod):
    """Uniform biaxial Q: the force on one site of a 1^3 lattice equals a
    central difference of Eq. (fphase) written out with numpy traces."""
    def f_bulk(q5):
        Q = full_Q(q5[:, None])[0]
        t2 = np.trace(Q @ Q)
        return A / 2 * t2 + B / 3 * np.trace(Q @ Q @ Q) + C / 4 * t2 * t2
    q = np.array([0.21, -0.13, 0.07, -0.05, 0.19])
    o = oracle_mod.Oracle((1, 1, 1), A, B, C, 2.32)
    F = o.force(q[:, None])[:, 0]
    h = 1e-5
    for c in range(5):
        e = np.zeros(5); e[c] = h
        fd = -(f_bulk(q + e) - f_bulk(q - e)) / (2 * h)
        assert abs(fd - F[c]) < 1e-9


# ---- hand-derived chain ---------------------------------------------------------

@pytest.mark.parametrize("Ls", [(2.32, 0.0, 0.0), (1.3, 0.5, 0.3)])
@pytest.mark.parametrize("periodic_yz", [0, 1])
def test_chain3_hand_values(oracle_mod, Ls, periodic_yz):
    g = json.load(open(os.path.join(GOLD, "chain3_hand.json")))
    L1, L2, L3 = Ls
    o = oracle_mod.Oracle((3, 1, 1), A, B, C, L1, L2, L3,
                          periodic=(0, periodic_yz, periodic_yz))
    q = np.zeros((5, 3))
    q[1] = g["a"]
    E, parts = o.energy(q)
    e = g["energy"]
    want = e["A"] * A + e["C"] * C + e["L1"] * L1 + e["L2"] * L2 + e["L3"] * L3
    assert abs(E - want) < 1e-12
    F = o.force(q)
    for s in range(3):
        f = g["force_q1"][s]
        want = f["L1"] * L1 + f["L23"] * (L2 + L3) + f["A"] * A + f["C"] * C
        assert abs(F[1, s] - want) < 1e-12
    for s in range(3):
        assert abs(F[0, s] - g["force_q0_q3_B"][s] * B) < 1e-12
        assert abs(F[3, s] - g["force_q0_q3_B"][s] * B) < 1e-12
    assert np.abs(F[[2, 4]]).max() < 1e-14


# ---- force = -gradient ------------------------------------------------------------

HOM = lambda W: (0, W, (0.0, 0.0, 1.0))
GEOMS = {
    "bulk_1c": dict(shape=(4, 3, 5), L=(2.32, 0, 0), periodic=(1, 1, 1), objects=[]),
    "wall_nd_3c": dict(shape=(5, 4, 5), L=(2.32, 0.5, 0.3), periodic=(1, 1, 1),
                       objects=[dict(type="wall", axis=2, plane=0, anchor=HOM(2.0))]),
    "sphere_nd_3c": dict(shape=(6, 6, 6), L=(1.1, 0.9, -0.4), periodic=(1, 1, 1),
                         objects=[dict(type="sphere", c=(3, 3, 3), R=1.5, anchor=HOM(5.3))]),
    "fg_walls_open_y": dict(shape=(4, 5, 6), L=(2.32, 0.5, 0.3), periodic=(1, 0, 1),
                            objects=[dict(type="wall", axis=2, plane=0, anchor=(2, 1.0, (0, 0, 1))),
                                     dict(type="wall", axis=2, plane=4, anchor=(2, 1.5, (0, 0, 1)))]),
    "custom_open_x": dict(shape=(5, 4, 4), L=(1.0, 0.7, 0.2), periodic=(0, 1, 1),
                          objects=[dict(type="sites", xyz=[[2, 1, 1], [2, 2, 1], [3, 2, 1]],
                                        anchor=(1, 3.0, (0.6, 0.0, 0.8))),
                                   dict(type="anchored", xyz=[[0, 0, 0], [4, 3, 3], [1, 1, 1]],
                                        kinds=[2, 1, 0], W=[1.0, 2.0, 0.5],
                                        dirs=[[0, 1, 0], [1, 1, 0], [0, 0, 1]])]),
    "tiny_2cube": dict(shape=(2, 2, 3), L=(1.5, 0.4, 0.6), periodic=(1, 1, 0), objects=[]),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_force_is_minus_gradient(oracle_mod, name):
    gdef = GEOMS[name]
    o = oracle_mod.Oracle(gdef["shape"], A, B, C, *gdef["L"], periodic=gdef["periodic"],
                          objects=gdef["objects"])
    q = rand_q(o.N, 5)
    F = o.force(q)
    sim = o.simulated()
    assert np.all(F[:, ~sim] == 0)
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(25):
        i = int(rng.choice(np.nonzero(sim)[0]))
        c = int(rng.integers(5))
        vals = []
        for s in (+1, -1, +2, -2):
            qq = q.copy()
            qq[c, i] += s * h
            vals.append(o.energy(qq)[0])
        # 4th-order central difference
        fd = -(8 * (vals[0] - vals[1]) - (vals[2] - vals[3])) / (12 * h)
        assert abs(fd - F[c, i]) < 1e-7 * max(1.0, abs(F[c, i])), (i, c, fd, F[c, i])


# ---- distortion pins ------------------------------------------------------------------

def test_uniform_field_zero_distortion_with_objects(oracle_mod):
    for gname in ("wall_nd_3c", "sphere_nd_3c", "custom_open_x", "fg_walls_open_y"):
        gdef = GEOMS[gname]
        o = oracle_mod.Oracle(gdef["shape"], A, B, C, *gdef["L"], periodic=gdef["periodic"],
                              objects=gdef["objects"])
        n = np.array([0.3, -0.5, 0.8]); n /= np.linalg.norm(n)
        q = np.repeat(synth.uniaxial_q(n[:, None], o.S0), o.N, axis=1)
        _, parts = o.energy(q)
        assert parts[1] == 0.0
        o0 = oracle_mod.Oracle(gdef["shape"], A, B, C, 0.0, periodic=gdef["periodic"],
                               objects=gdef["objects"])
        # the force is the bulk + anchoring force alone
        assert np.abs(o.force(q) - o0.force(q)).max() < 1e-14


@pytest.mark.parametrize("m", [1, 2, 3])
def test_twist_texture_energy(oracle_mod, m):
    shape = (3, 2, 12)
    L1 = 2.32
    o = oracle_mod.Oracle(shape, A, B, C, L1, 0.5, 0.3)
    q = synth.texture_q(shape, "twist", m)
    E, parts = o.energy(q)
    N = o.N
    k = math.pi * m / shape[2]
    S0 = o.S0
    assert abs(parts[1] / N - 2.25 * S0 ** 2 * L1 * math.sin(k) ** 2) < 1e-13
    assert abs(parts[0] / N - f_of_S(S0)) < 1e-13


@pytest.mark.parametrize("m", [1, 2])
def test_splay_bend_texture_energy(oracle_mod, m):
    shape = (2, 3, 10)
    L1, L2, L3 = 2.32, 0.5, 0.3
    o = oracle_mod.Oracle(shape, A, B, C, L1, L2, L3)
    q = synth.texture_q(shape, "splaybend", m)
    _, parts = o.energy(q)
    k = math.pi * m / shape[2]
    S0 = o.S0
    want = 2.25 * S0 ** 2 * math.sin(k) ** 2 * (L1 + (L2 + L3) / 2)
    assert abs(parts[1] / o.N - want) < 1e-13


def test_plane_wave_discrete_laplacian(oracle_mod):
    """A small Q_xy wave eps cos(2 pi m x / L) about Q = 0: the force on
    Q_xy is -(2A + 2 L1 lambda_m) q with lambda_m = 2 (1 - cos(2 pi m / L)),
    the eigenvalue of the periodic second difference; the factor 2 is the
    symmetric pair Q_xy = Q_yx."""
    L, L1, eps = 8, 2.32, 1e-6
    o = oracle_mod.Oracle((L, 3, 2), A, B, C, L1)
    x = np.tile(np.arange(L), 6).astype(float)
    for m in (1, 2, 3):
        q = np.zeros((5, o.N))
        q[1] = eps * np.cos(2 * math.pi * m * x / L)
        F = o.force(q)
        lam = 2 * (1 - math.cos(2 * math.pi * m / L))
        want = -(2 * A + 2 * L1 * lam) * q[1]
        assert np.abs(F[1] - want).max() < 1e-9 * eps
        # only the second-order B Q.Q term reaches the other components
        assert np.abs(F[[0, 3]]).max() <= abs(B) * eps ** 2 * (1 + 1e-9)
        assert np.abs(F[[2, 4]]).max() < 1e-30


def test_l2_l3_summation_by_parts_identity(oracle_mod):
    """On a fully periodic lattice without objects the averaged L2 and L3
    terms are equal for every Q (centred differences commute and sum by
    parts), so energies and forces with (L2, L3) = (1, 0) and (0, 1) agree."""
    shape = (4, 5, 3)
    o2 = oracle_mod.Oracle(shape, A, B, C, 0.0, 1.0, 0.0)
    o3 = oracle_mod.Oracle(shape, A, B, C, 0.0, 0.0, 1.0)
    o1 = oracle_mod.Oracle(shape, A, B, C, 1.0, 0.0, 0.0)
    q = rand_q(o2.N, 9)
    e2, e3, e1 = o2.energy(q)[1][1], o3.energy(q)[1][1], o1.energy(q)[1][1]
    assert abs(e2 - e3) < 1e-12 * abs(e2)
    assert abs(e2 - e1) > 1e-3 * abs(e1)  # and they are not the L1 term
    assert np.abs(o2.force(q) - o3.force(q)).max() < 1e-12


def test_l2_l3_differ_on_a_ramp_in_a_closed_box(oracle_mod):
    """Q_xx = a x, Q_zz = -a x, Q_xy = b y in a box closed along x and y:
    every difference is uniform, so each site's average is the continuum
    value: L1 (a^2+b^2) + (L2+L3)(a^2+b^2)/2 + L2 a b (the L3 cross term
    dQ_iy/dx dQ_ix/dy vanishes, the L2 cross term dQ_xx/dx dQ_xy/dy does not)."""
    shape = (4, 5, 3)
    a, b = 0.07, -0.11
    for L1, L2, L3 in ((0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (2.32, 0.5, 0.3)):
        o = oracle_mod.Oracle(shape, A, B, C, L1, L2, L3, periodic=(0, 0, 1))
        N = o.N
        x = np.tile(np.arange(4), 15).astype(float)
        y = np.tile(np.repeat(np.arange(5), 4), 3).astype(float)
        q = np.zeros((5, N))
        q[0] = a * x
        q[1] = b * y
        want = L1 * (a * a + b * b) + (L2 + L3) * (a * a + b * b) / 2 + L2 * a * b
        assert abs(o.energy(q)[1][1] / N - want) < 1e-14


def _rot_q(q, R):
    Q = full_Q(q)
    return comps(np.einsum("ab,nbc,dc->nad", R, Q, R))


def test_global_rotation_invariance_bulk_l1(oracle_mod):
    gdef = GEOMS["sphere_nd_3c"]
    o = oracle_mod.Oracle(gdef["shape"], A, B, C, 2.32, objects=[
        dict(type="sphere", c=(3, 3, 3), R=1.5, anchor=HOM(0.0))])
    q = rand_q(o.N, 21)
    rng = np.random.default_rng(4)
    R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    E, parts = o.energy(q)
    E2, parts2 = o.energy(_rot_q(q, R))
    assert abs(E - E2) < 1e-12 * abs(E)


def _lattice_rotation(shape_L, R, q, objects):
    """Rotate field and geometry by a cubic lattice rotation R (integer
    matrix) about the origin, wrapping coordinates into [0, L)."""
    L = shape_L
    N = L ** 3
    idx = np.arange(N)
    xyz = np.stack([idx % L, (idx // L) % L, idx // (L * L)])
    new = (R @ xyz) % L
    j = new[0] + L * (new[1] + L * new[2])
    qr = np.zeros_like(q)
    qr[:, j] = _rot_q(q, R)
    objs = []
    for ob in objects:
        ob = dict(ob)
        if ob["type"] == "sphere":
            ob["c"] = tuple(float(v) for v in (R @ np.array(ob["c"])) % L)
        elif ob["type"] == "wall":
            ax = int(np.nonzero(R[:, ob["axis"]])[0][0])
            ob["plane"] = int((R[ax, ob["axis"]] * ob["plane"]) % L)
            ob["axis"] = ax
        elif ob["type"] in ("sites", "anchored"):
            ob["xyz"] = ((R @ np.array(ob["xyz"]).T) % L).T
            if "dirs" in ob:
                ob["dirs"] = (R @ np.array(ob["dirs"], float).T).T
        if "anchor" in ob:
            k, W, d = ob["anchor"]
            ob["anchor"] = (k, W, tuple(R @ np.array(d, float)))
        objs.append(ob)
    return qr, objs


@pytest.mark.parametrize("rot", ["z90", "x90", "y180"])
def test_cubic_lattice_rotation_invariance(oracle_mod, rot):
    R = {"z90": np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]),
         "x90": np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]]),
         "y180": np.array([[-1, 0, 0], [0, 1, 0], [0, 0, -1]])}[rot]
    L = 6
    objects = [dict(type="wall", axis=2, plane=0, anchor=(2, 1.0, (0, 0, 1))),
               dict(type="sphere", c=(3.0, 2.0, 3.0), R=1.2, anchor=HOM(5.3)),
               dict(type="anchored", xyz=[[1, 4, 4], [5, 5, 2]], kinds=[1, 2], W=[2.0, 1.0],
                    dirs=[[1.0, 2.0, 0.5], [0.0, 0.6, 0.8]])]
    o = oracle_mod.Oracle((L, L, L), A, B, C, 2.32, 0.5, 0.3, objects=objects)
    q = rand_q(o.N, 8)
    qr, objr = _lattice_rotation(L, R, q, objects)
    orr = oracle_mod.Oracle((L, L, L), A, B, C, 2.32, 0.5, 0.3, objects=objr)
    E, parts = o.energy(q)
    Er, partsr = orr.energy(qr)
    assert np.allclose(parts, partsr, rtol=1e-12, atol=1e-12)
    # forces: the 3x3 derivative rotates as a tensor
    F, Fr = o.force(q), orr.force(qr)
    idx = np.arange(o.N)
    xyz = np.stack([idx % L, (idx // L) % L, idx // (L * L)])
    new = (R @ xyz) % L
    j = new[0] + L * (new[1] + L * new[2])
    # the force pairs with a perturbation: F.dq invariant for dq rotated alike
    dq = rand_q(o.N, 77, 1.0)
    dqr = np.zeros_like(dq)
    dqr[:, j] = _rot_q(dq, R)
    assert abs((F * dq).sum() - (Fr * dqr).sum()) < 1e-10 * np.abs(F * dq).sum()


def test_symmetric_traceless_structure(oracle_mod):
    q = rand_q(10, 3)
    Q = full_Q(q)
    assert np.abs(Q - Q.transpose(0, 2, 1)).max() == 0
    assert np.abs(np.trace(Q, axis1=1, axis2=2)).max() < 1e-15


# ---- eigen readback ---------------------------------------------------------------------

def test_eigen_uniaxial_and_biaxial(oracle_mod):
    rng = np.random.default_rng(12)
    for _ in range(20):
        Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        n, m_, l = Rm[:, 0], Rm[:, 1], Rm[:, 2]
        S, SB = rng.uniform(0.1, 0.8), rng.uniform(0.0, 0.1)
        Q = 1.5 * S * (np.outer(n, n) - np.eye(3) / 3) + 0.5 * SB * (np.outer(m_, m_) - np.outer(l, l))
        ev, vec = oracle_mod.eig_sym3(comps(Q[None])[:, 0])
        want = sorted([S, (-S + SB) / 2, (-S - SB) / 2], reverse=True)
        assert np.allclose(ev, want, atol=1e-14)
        assert abs(abs(vec[0] @ n) - 1) < 1e-10
    for _ in range(20):
        q = rng.normal(size=5)
        ev, _ = oracle_mod.eig_sym3(q)
        assert np.allclose(ev, np.linalg.eigvalsh(full_Q(q[:, None])[0])[::-1], atol=1e-14)


# ---- geometry ---------------------------------------------------------------------------

def test_geometry_sphere_and_walls(oracle_mod):
    L = 12
    c, R = (5.0, 6.0, 6.0), 3.4
    o = oracle_mod.Oracle((L, L, L), A, B, C, 1.0, objects=[
        dict(type="wall", axis=2, plane=0, anchor=HOM(1.0)),
        dict(type="sphere", c=c, R=R, anchor=HOM(2.0))])
    sim = o.simulated().reshape(L, L, L)   # [z, y, x]
    zz, yy, xx = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    inside = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= R * R
    assert np.array_equal(~sim, inside | (zz == 0))
    sites, kind, W, q0, nu = o.records()
    S0 = o.S0
    for s, k, w, qq in zip(sites, kind, W, q0):
        x, y, z = s % L, (s // L) % L, s // (L * L)
        assert k == 1
        if z in (1, L - 1):
            assert w == 1.0
            assert np.allclose(qq, synth.uniaxial_q(np.array([[0.0], [0], [1]]), S0)[:, 0])
        else:
            assert w == 2.0
            d = np.array([x - c[0], y - c[1], z - c[2]])
            assert np.allclose(qq, synth.uniaxial_q((d / np.linalg.norm(d))[:, None], S0)[:, 0])
    # every simulated face neighbour of an object site has a record
    touched = np.zeros_like(sim)
    obj = ~sim
    for ax in range(3):
        for sh in (1, -1):
            touched |= np.roll(obj, sh, axis=ax)
    assert np.array_equal(np.sort(sites), np.nonzero((touched & sim).ravel())[0])


def _face_touched(obj):
    """Sites with a face neighbour in ``obj`` (periodic rolls; [z, y, x] arrays)."""
    t = np.zeros_like(obj)
    for ax in range(3):
        for sh in (1, -1):
            t |= np.roll(obj, sh, axis=ax)
    return t


def _segment_distance_sampled(P, p0, p1, shape, periodic, n=801):
    """Distance of the points P (m, 3) to the segment p0..p1 over all periodic
    images, by sampling the segment at n points (an independent route to the
    nearest point) -- returns the distance and the offset to the sampled
    nearest point."""
    ts = np.linspace(0.0, 1.0, n)
    seg = np.asarray(p0)[None, :] + ts[:, None] * (np.asarray(p1) - np.asarray(p0))[None, :]
    L = np.asarray(shape, dtype=float)
    best = np.full(len(P), np.inf)
    off = np.zeros((len(P), 3))
    shifts = [[-1, 0, 1] if p else [0] for p in periodic]
    for img in np.array(np.meshgrid(*shifts)).reshape(3, -1).T:
        d = P[:, None, :] + img * L - seg[None, :, :]
        r = np.sqrt((d * d).sum(2))
        k = r.argmin(1)
        rk = r[np.arange(len(P)), k]
        better = rk < best
        best[better] = rk[better]
        off[better] = d[np.arange(len(P)), k][better]
    return best, off


def test_geometry_droplet_is_the_complement_of_a_sphere(oracle_mod):
    """A droplet (Fig. 3) of radius R about c fills exactly the sites a sphere
    of the same c and R removes, wrapping across periodic faces; its boundary
    sites are the ball's sites with a face neighbour outside, anchored along
    the radius."""
    L = 14
    for c, R in (((6.5, 7.0, 6.2), 5.3), ((1.0, 7.0, 12.5), 4.5)):
        drop = oracle_mod.Oracle((L, L, L), A, B, C, 1.0, objects=[
            dict(type="droplet", c=c, R=R, anchor=HOM(2.0))])
        sph = oracle_mod.Oracle((L, L, L), A, B, C, 1.0, objects=[
            dict(type="sphere", c=c, R=R, anchor=HOM(2.0))])
        assert np.array_equal(drop.simulated(), ~sph.simulated())
        sim = drop.simulated().reshape(L, L, L)
        assert abs(sim.sum() - 4 / 3 * np.pi * R ** 3) < 0.15 * 4 / 3 * np.pi * R ** 3
        sites, kind, W, q0, nu = drop.records()
        assert np.array_equal(np.sort(sites), np.nonzero((_face_touched(~sim) & sim).ravel())[0])
        for s, qq in zip(sites, q0):
            x, y, z = s % L, (s // L) % L, s // (L * L)
            d = np.array([x - c[0], y - c[1], z - c[2]])
            d -= L * np.round(d / L)
            assert np.allclose(qq, synth.uniaxial_q((d / np.linalg.norm(d))[:, None], drop.S0)[:, 0],
                               atol=1e-14)
    # a droplet larger than the lattice's inscribed ball's diagonal is the bulk
    big = oracle_mod.Oracle((6, 5, 4), A, B, C, 1.0, objects=[
        dict(type="droplet", c=(3.0, 2.0, 2.0), R=5.0, anchor=HOM(2.0))])
    assert big.simulated().all() and len(big.records()[0]) == 0


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 0)])
def test_geometry_spherocylinder_against_sampled_segment(oracle_mod, periodic):
    """Object sites of a spherocylinder (Fig. 3) are the sites within R of its
    axis segment, found here by sampling the segment over all periodic
    images; boundary normals point from the nearest axis point to the site."""
    shape = (20, 13, 11)
    p0, p1, R = (4.3, 5.1, 4.0), (14.6, 8.2, 6.7), 2.6
    o = oracle_mod.Oracle(shape, A, B, C, 1.0, periodic=periodic, objects=[
        dict(type="spherocylinder", c=p0, c2=p1, R=R, anchor=HOM(2.0))])
    nx, ny, nz = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(float)
    dist, off = _segment_distance_sampled(P, p0, p1, shape, periodic)
    sim = o.simulated()
    clear = np.abs(dist - R) > 1e-3
    assert clear.sum() > 0.95 * len(P)
    assert np.array_equal(sim[clear], (dist > R)[clear])
    assert 0.7 * (np.pi * R * R * np.linalg.norm(np.subtract(p1, p0)) + 4 / 3 * np.pi * R ** 3) \
        < (~sim).sum() < 1.3 * (np.pi * R * R * np.linalg.norm(np.subtract(p1, p0)) +
                                4 / 3 * np.pi * R ** 3)
    sites, kind, W, q0, nu = o.records()
    assert len(sites) > 50
    for s, qq in zip(sites, q0):
        n = off[s] / np.linalg.norm(off[s])
        ref = synth.uniaxial_q(n[:, None], o.S0)[:, 0]
        assert np.abs(qq - ref).max() < 2e-3


def test_geometry_spherocylinder_of_zero_length_is_a_sphere(oracle_mod):
    shape = (13, 12, 11)
    for c, R in (((6.0, 5.5, 5.2), 3.3), ((0.5, 11.0, 5.0), 2.8)):
        a = oracle_mod.Oracle(shape, A, B, C, 1.0, objects=[
            dict(type="spherocylinder", c=c, c2=c, R=R, anchor=(2, 1.5, (0.0, 0.0, 1.0)))])
        b = oracle_mod.Oracle(shape, A, B, C, 1.0, objects=[
            dict(type="sphere", c=c, R=R, anchor=(2, 1.5, (0.0, 0.0, 1.0)))])
        assert np.array_equal(a.simulated(), b.simulated())
        ra, rb = a.records(), b.records()
        for u, v in zip(ra, rb):
            assert np.array_equal(u, v)


def _degree(field, centre, radius, n_theta=120, n_phi=240):
    """Topological degree of a unit-vector field on a sphere: the signed
    solid angle its image sweeps over a triangulated (theta, phi) mesh,
    divided by 4 pi (outward orientation)."""
    th = np.linspace(0.0, np.pi, n_theta + 1)
    ph = np.linspace(0.0, 2 * np.pi, n_phi + 1)
    T, P = np.meshgrid(th, ph, indexing="ij")
    pts = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    n = field(np.asarray(centre)[None, :] + radius * pts.reshape(-1, 3)).reshape(pts.shape)

    def omega(a, b, c):
        num = np.einsum("...i,...i", a, np.cross(b, c))
        den = 1 + np.einsum("...i,...i", a, b) + np.einsum("...i,...i", b, c) + \
            np.einsum("...i,...i", c, a)
        return 2 * np.arctan2(num, den)

    a, b = n[:-1, :-1], n[1:, :-1]
    c, d = n[1:, 1:], n[:-1, 1:]
    # (theta, phi) increasing is the outward orientation of (e_theta, e_phi)
    tot = omega(a, b, c).sum() + omega(a, c, d).sum()
    return tot / (4 * np.pi)


def test_degree_routine_on_textbook_fields():
    radial = lambda x: x / np.linalg.norm(x, axis=1, keepdims=True)
    assert _degree(radial, (0, 0, 0), 1.0) == pytest.approx(1.0, abs=1e-9)
    mirror = lambda x: radial(x) * np.array([1.0, 1.0, -1.0])   # reflected in z = 0
    assert _degree(mirror, (0, 0, 0), 1.0) == pytest.approx(-1.0, abs=1e-9)
    half_turn = lambda x: radial(x) * np.array([-1.0, -1.0, 1.0])   # rotated by pi about z
    assert _degree(half_turn, (0, 0, 0), 1.0) == pytest.approx(1.0, abs=1e-9)
    assert _degree(lambda x: -radial(x), (0, 0, 0), 1.0) == pytest.approx(-1.0, abs=1e-9)
    uniform = lambda x: np.tile([0.3, 0.4, 0.866], (len(x), 1))
    assert _degree(uniform, (0, 0, 0), 1.0) == pytest.approx(0.0, abs=1e-9)


@pytest.mark.parametrize("axis", [(0, 0, 1), (0.3, -0.5, 0.8)])
def test_dipolar_director_hedgehog_charges_and_far_field(oracle_mod, axis):
    """The dipolar start pairs a radial hedgehog at the colloid centre with
    a hyperbolic hedgehog at rd along the axis, of opposite charges and total
    charge zero, and is uniform along the axis far away (section IV.A).  As a
    vector field continuous away from the two points, n ~ -u/|u| near the
    centre (theta_h ~ pi there: degree -1) and n ~ w/|w| turned by pi about
    the axis near the defect (degree +1)."""
    R = 8.0
    rd = 1.25 * R
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    f = lambda x: oracle_mod.dipolar_director(x, axis, rd)
    assert _degree(f, (0, 0, 0), 0.3 * rd) == pytest.approx(-1.0, abs=1e-6)
    assert _degree(f, rd * a, 0.3 * rd) == pytest.approx(1.0, abs=1e-6)
    assert _degree(f, 0.5 * rd * a, 4 * rd) == pytest.approx(0.0, abs=1e-6)
    # unit vectors; radial on the colloid surface opposite the defect
    rng = np.random.default_rng(3)
    x = rng.normal(size=(500, 3)) * 3 * R
    n = f(x)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-14)
    assert np.allclose(np.abs(f(-R * a[None, :]) @ a), 1.0, atol=1e-14)
    # far field: n -> a, the deviation falling like rd / r
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    for r in (1e3 * rd, 1e5 * rd):
        dev = 1 - f(r * d) @ a
        assert dev.max() < (2 * rd / r) ** 2
    # rotating the point about the axis rotates the director with it
    from scipy.spatial.transform import Rotation
    rot = Rotation.from_rotvec(0.7 * a).as_matrix()
    assert np.allclose(f(x @ rot.T), f(x) @ rot.T, atol=1e-12)


def test_dipolar_q_is_uniaxial_on_the_lattice(oracle_mod):
    shape = (24, 22, 20)
    c, R = (11.5, 10.7, 9.3), 4.0
    o = oracle_mod.Oracle(shape, A, B, C, 1.0, objects=[
        dict(type="sphere", c=c, R=R, anchor=HOM(5.0))])
    q = oracle_mod.dipolar_q(o, c, (0, 0, 1), 1.25 * R, o.S0)
    sim = o.simulated()
    assert np.all(q[:, ~sim] == 0)
    for i in np.nonzero(sim)[0][::97]:
        ev, _ = oracle_mod.eig_sym3(q[:, i])
        assert np.allclose(sorted(ev), [-o.S0 / 2, -o.S0 / 2, o.S0], atol=1e-13)


# ---- FIRE ---------------------------------------------------------------------------------

FP = dict(dt0=0.1, dt_max=0.25, alpha0=0.2, f_alpha=0.5, f_inc=2.0, f_dec=0.5, n_min=2,
          max_iter=100, force_tol=0.0)


def test_fire_scalar_machine_scripted(oracle_mod):
    st = dict(dt=0.1, alpha=0.2, npos=0, iter=0, initialized=1, status=0)
    expect = [  # (P, a, b/(nv/nF), dt, alpha, npos) by hand from Algorithm 1
        (+1.0, 0.8, 0.2, 0.1, 0.2, 1),
        (+1.0, 0.8, 0.2, 0.1, 0.2, 2),
        (+1.0, 0.8, 0.2, 0.2, 0.1, 3),
        (+1.0, 0.9, 0.1, 0.25, 0.05, 4),
        (-1.0, 0.0, 0.0, 0.125, 0.2, 0),
        (0.0, 0.0, 0.0, 0.0625, 0.2, 0),
        (+2.0, 0.8, 0.2, 0.0625, 0.2, 1),
    ]
    nF, nv = 2.0, 3.0
    for P, a_w, b_w, dt_w, al_w, np_w in expect:
        a, b, st = oracle_mod.fire_scalars(FP, st, P, nF, nv)
        assert abs(a - a_w) < 1e-15 and abs(b - b_w * nv / nF) < 1e-15
        assert abs(st["dt"] - dt_w) < 1e-15 and abs(st["alpha"] - al_w) < 1e-15
        assert st["npos"] == np_w
    a, b, st = oracle_mod.fire_scalars(FP, st, 1.0, 0.0, 3.0)
    assert (a, b) == (1.0, 0.0)


def test_fire_single_site_reaches_uniaxial_s0(oracle_mod):
    o = oracle_mod.Oracle((1, 1, 1), A, B, C, 2.32, 0.5, 0.3)
    q0 = np.array([[0.30], [0.05], [-0.02], [-0.12], [0.04]])
    params = dict(synth.FIRE_DEFAULTS, max_iter=200000, force_tol=1e-12)
    q, v, F, st = o.fire(q0, params, 200000)
    assert st["status"] == oracle_mod.CONVERGED
    ev, _ = oracle_mod.eig_sym3(q[:, 0])
    S0 = o.S0
    assert np.allclose(ev, [S0, -S0 / 2, -S0 / 2], atol=1e-10)
    assert abs(o.energy(q)[0] - f_of_S(S0)) < 1e-14


def test_fire_fixed_point_and_descent(oracle_mod):
    o = oracle_mod.Oracle((4, 4, 4), A, B, C, 2.32)
    n = synth.random_directors(1, 5)
    q = np.repeat(synth.uniaxial_q(n, o.S0), o.N, axis=1)
    params = dict(synth.FIRE_DEFAULTS, max_iter=100, force_tol=1e-12)
    q2, v, F, st = o.fire(q, params, 10)
    assert st["status"] == oracle_mod.CONVERGED and st["iter"] == 0
    assert np.array_equal(q2, q)
    # from random directors the energy stays above N f0 and goes down
    q = synth.random_uniaxial_q((4, 4, 4), 3)
    E0 = o.energy(q)[0]
    params = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-9)
    q2, v, F, st = o.fire(q, params, 400)
    E1 = o.energy(q2)[0]
    assert E1 < E0
    assert E1 >= o.N * f_of_S(o.S0) - 1e-12


def test_fire_reduces_to_velocity_verlet_on_a_harmonic_well(oracle_mod):
    """With alpha0 = 0 (no mixing) and an unreachable N_min, and while P > 0,
    FIRE is plain velocity Verlet.  For f = A/2 tr Q^2 with only Q_xy set,
    f = A q1^2 and F = -omega^2 q1 with omega^2 = 2A; one Verlet step of size
    h is the linear map [q, v] -> [q (1 - h^2 w2/2) + h v,
    v (1 - h^2 w2/2) - h w2 q (1 - h^2 w2/4)] (textbook form)."""
    Ah, h = 0.5, 0.1
    w2 = 2 * Ah
    o = oracle_mod.Oracle((1, 1, 1), Ah, 0.0, 0.0, 1.0)
    q = np.zeros((5, 1)); q[1, 0] = 1.0
    params = dict(dt0=h, dt_max=1.0, alpha0=0.0, f_alpha=1.0, f_inc=1.0, f_dec=0.5,
                  n_min=10 ** 6, max_iter=10 ** 6, force_tol=0.0)
    M = np.array([[1 - h * h * w2 / 2, h], [-h * w2 * (1 - h * h * w2 / 4), 1 - h * h * w2 / 2]])
    for k in (1, 5, 12):
        qk, vk, Fk, st = o.fire(q, params, k)
        want = np.linalg.matrix_power(M, k) @ np.array([1.0, 0.0])
        assert st["iter"] == k
        assert abs(qk[1, 0] - want[0]) < 1e-14 and abs(vk[1, 0] - want[1]) < 1e-14
        assert abs(Fk[1, 0] + w2 * qk[1, 0]) < 1e-15


# ---- gradient descent and Nesterov's accelerated gradient (section III.C) ----

def test_descent_single_site_reaches_uniaxial_s0(oracle_mod):
    """Gradient descent and Nesterov from a biaxial single site (no
    distortion) stop at the uniaxial bulk minimum: eigenvalues (S0, -S0/2,
    -S0/2) with S0 from the closed form of Eq. (S0def)."""
    q0 = np.array([[0.30], [0.05], [-0.02], [-0.12], [0.04]])
    S0 = synth.s0_closed_form(A, B, C)
    for method, eta, mu in ((oracle_mod.GD, 0.5, 0.0), (oracle_mod.NESTEROV, 0.2, 0.8)):
        o = oracle_mod.Oracle((1, 1, 1), A, B, C, 2.32, 0.5, 0.3)
        r = o.descent(q0, method, eta, mu=mu, max_iter=100000, force_tol=1e-12, max_steps=100000)
        assert r["status"] == oracle_mod.CONVERGED
        ev, _ = oracle_mod.eig_sym3(r["y"][:, 0])
        assert np.allclose(ev, [S0, -S0 / 2, -S0 / 2], atol=1e-10)


def test_gradient_descent_lowers_the_energy_every_step(oracle_mod):
    """A small step is a descent direction: the energy of a three-constant
    lattice with a colloid and a wall falls at every step (a sign error in
    the update or the force raises it)."""
    objs = [dict(type="sphere", c=(3.0, 3.0, 2.5), R=1.5, anchor=(0, 5.3, (0, 0, 1))),
            dict(type="wall", axis=2, plane=0, anchor=(2, 1.0, (0, 0, 1)))]
    o = oracle_mod.Oracle((7, 6, 6), A, B, C, 2.32, 0.5, 0.3, objects=objs)
    q = synth.random_uniaxial_q((7, 6, 6), 11)
    E = o.energy(q)[0]
    r = None
    for _ in range(30):
        r = o.descent(q, oracle_mod.GD, 0.01, max_steps=1, state=r)
        En = o.energy(r["x"])[0]
        assert En < E
        E = En
    assert r["iter"] == 30 and np.array_equal(r["x"], r["y"])


def test_nesterov_on_a_plane_wave_follows_its_recurrence(oracle_mod):
    """With A = B = C = 0 the energy is quadratic and a Q_xy wave
    eps cos(2 pi m x / L) is an eigenvector of the force, F = -lam q with
    lam = 2 L1 (2 - 2 cos(2 pi m / L)) (the symmetric pair Q_xy = Q_yx
    times the periodic second difference).  Nesterov's amplitudes then obey
    a_{k+1} = (1 - eta lam) b_k, b_k = a_k + mu (a_k - a_{k-1}), a_{-1} = a_0;
    the oracle's iterates (x) and evaluation points (y) must follow it."""
    L, L1, eps, eta, mu = 12, 1.3, 1e-3, 0.05, 0.7
    o = oracle_mod.Oracle((L, 2, 2), 0.0, 0.0, 0.0, L1)
    x = np.tile(np.arange(L), 4).astype(float)
    for m in (1, 3):
        wave = np.cos(2 * math.pi * m * x / L)
        q = np.zeros((5, o.N))
        q[1] = eps * wave
        lam = 2 * L1 * (2 - 2 * math.cos(2 * math.pi * m / L))
        a_prev, a = eps, eps
        r = None
        for k in range(40):
            r = o.descent(q, oracle_mod.NESTEROV, eta, mu=mu, max_steps=1, force_tol=0.0,
                          state=r)
            b = a + mu * (a - a_prev)
            a_prev, a = a, (1 - eta * lam) * b
            b_next = a + mu * (a - a_prev)
            assert np.abs(r["x"][1] - a * wave).max() <= 1e-12 * eps
            assert np.abs(r["y"][1] - b_next * wave).max() <= 1e-12 * eps
            assert np.abs(r["F"][1] + lam * b_next * wave).max() <= 1e-11 * eps
        assert np.abs(r["x"][[0, 2, 3, 4]]).max() == 0.0


def test_nesterov_without_momentum_is_gradient_descent(oracle_mod):
    o = oracle_mod.Oracle((6, 5, 4), A, B, C, 2.32, 0.5, 0.3)
    q = synth.random_uniaxial_q((6, 5, 4), 5)
    g = o.descent(q, oracle_mod.GD, 0.02, max_steps=25, force_tol=0.0)
    n = o.descent(q, oracle_mod.NESTEROV, 0.02, mu=0.0, max_steps=25, force_tol=0.0)
    assert np.array_equal(g["x"], n["x"]) and np.array_equal(g["F"], n["F"])


# ---- chiral L4, cubic L6 and external fields (Eq. fdistortionFull, section II) ----

EXTRA = dict(L4=0.7, L6=0.9, H=(0.3, -0.2, 0.5), mu0_dchi=1.3, E=(0.1, 0.4, 0.2), eps0_deps=-0.6)


def _twist_helix(L, k, S):
    """Uniaxial Q at order S with n = (cos kz, sin kz, 0), all sites."""
    z = np.repeat(np.arange(L[2]), L[0] * L[1]).astype(float)
    n = np.stack([np.cos(k * z), np.sin(k * z), np.zeros_like(z)])
    return synth.uniaxial_q(n, S)


@pytest.mark.parametrize("m", [1, 2, 5])
def test_twist_helix_energy_with_chiral_and_cubic_terms(oracle_mod, m):
    """A twist helix along z on a periodic lattice: every site sees the same
    averaged differences (Q(z+1) - Q(z-1)) / 2 and squares, so per site
      L1:  (9 S^2 / 8) L1 (1 - cos 2k)
      L4:  (9 S^2 / 16) L4 sin 2k     (eps_lik Q_lj dQ_ij/dz, only k = z)
      L6:  L6/2 Q_zz <|dQ/dz|^2> = -(9 L6 S^3 / 16) (1 - cos 2k)
    and the L2, L3 terms vanish (Q_iz = 0 for i != z, Q_zz constant)."""
    shape = (2, 3, 24)
    k = 2 * math.pi * m / shape[2]
    S = 0.53
    o = oracle_mod.Oracle(shape, A, B, C, 2.32, 0.5, 0.3, L4=0.7, L6=0.9)
    _, parts = o.energy(_twist_helix(shape, k, S))
    per = (9 * S ** 2 / 8 * 2.32 * (1 - math.cos(2 * k)) + 9 * S ** 2 / 16 * 0.7 * math.sin(2 * k)
           - 9 * 0.9 * S ** 3 / 16 * (1 - math.cos(2 * k)))
    assert abs(parts[1] - o.N * per) < 1e-12 * o.N


def test_chiral_term_picks_a_handedness(oracle_mod):
    """L4 < 0 favours the helix with k > 0, L4 > 0 the other; the lattice
    energy of the twist helix is lowest at tan 2k = -L4 / (2 L1) (from the
    closed form above with L6 = 0)."""
    shape = (1, 1, 120)
    for L4 in (-0.5, 0.5):
        o = oracle_mod.Oracle(shape, 0.0, 0.0, 0.0, 2.32, L4=L4)
        ks = 2 * math.pi * np.arange(-6, 7) / shape[2]
        E = [o.energy(_twist_helix(shape, k, 0.5))[1][1] for k in ks]
        kbest = ks[int(np.argmin(E))]
        kstar = -0.5 * math.atan(L4 / (2 * 2.32))
        assert np.sign(kbest) == np.sign(kstar)
        assert abs(kbest - kstar) <= math.pi / shape[2]


def test_field_energy_and_alignment(oracle_mod):
    """Uniaxial limit of the field term: -(1/2) S mu0_dchi (H.n)^2 + const;
    minimising a single site aligns the director with H for mu0_dchi > 0 and
    turns it perpendicular for mu0_dchi < 0."""
    H = np.array([0.6, 0.0, 0.8])
    for chi in (2.0, -2.0):
        o = oracle_mod.Oracle((1, 1, 1), A, B, C, 2.32, H=tuple(H), mu0_dchi=chi)
        qpar = synth.uniaxial_q(H[:, None], o.S0)
        nperp = np.array([0.8, 0.0, -0.6])
        qper = synth.uniaxial_q(nperp[:, None], o.S0)
        dE = o.energy(qpar)[0] - o.energy(qper)[0]
        assert abs(dE - (-0.5 * o.S0 * chi * 1.0)) < 1e-13
        q0 = synth.uniaxial_q(np.array([[0.3], [0.9], [0.3]]) / math.sqrt(0.99), o.S0)
        r = o.descent(q0, oracle_mod.NESTEROV, 0.05, mu=0.5, force_tol=1e-12, max_steps=200000,
                      max_iter=200000)
        assert r["status"] == oracle_mod.CONVERGED
        Qf = full_Q(r["y"])[0]
        # the largest-eigenvalue axis: along H for chi > 0, perpendicular for chi < 0
        w, V = np.linalg.eigh(Qf)
        nmax = V[:, int(np.argmax(w))]
        assert (abs(np.dot(nmax, H)) > 1 - 1e-6) if chi > 0 else (abs(np.dot(nmax, H)) < 1e-6)


EXTRA_GEOMS = ["sphere_nd_3c", "fg_walls_open_y", "custom_open_x", "tiny_2cube"]


@pytest.mark.parametrize("name", EXTRA_GEOMS)
def test_force_is_minus_gradient_with_chiral_cubic_and_fields(oracle_mod, name):
    gdef = GEOMS[name]
    o = oracle_mod.Oracle(gdef["shape"], A, B, C, *gdef["L"], periodic=gdef["periodic"],
                          objects=gdef["objects"], **EXTRA)
    q = rand_q(o.N, 6)
    F = o.force(q)
    sim = o.simulated()
    assert np.all(F[:, ~sim] == 0)
    rng = np.random.default_rng(5)
    h = 1e-5
    for _ in range(25):
        i = int(rng.choice(np.nonzero(sim)[0]))
        c = int(rng.integers(5))
        vals = []
        for s in (+1, -1, +2, -2):
            qq = q.copy()
            qq[c, i] += s * h
            vals.append(o.energy(qq)[0])
        fd = -(8 * (vals[0] - vals[1]) - (vals[2] - vals[3])) / (12 * h)
        assert abs(fd - F[c, i]) < 1e-7 * max(1.0, abs(F[c, i])), (i, c, fd, F[c, i])


def test_chiral_energy_is_odd_under_reflection(oracle_mod):
    """Mirroring x -> -x (lattice and Q -> M Q M) flips the sign of the L4
    energy and keeps every other term: eps_lik is a pseudotensor."""
    L = 6
    M = np.diag([-1.0, 1.0, 1.0])
    q = rand_q(L ** 3, 9)
    idx = np.arange(L ** 3)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    j = ((-x) % L) + L * (y + L * z)
    qm = np.zeros_like(q)
    qm[:, j] = comps(np.einsum("ab,nbc,dc->nad", M, full_Q(q), M))
    base = oracle_mod.Oracle((L, L, L), A, B, C, 2.32, 0.5, 0.3, L6=0.9)
    chi = oracle_mod.Oracle((L, L, L), A, B, C, 2.32, 0.5, 0.3, L4=0.7, L6=0.9)
    e4 = chi.energy(q)[1][1] - base.energy(q)[1][1]
    e4m = chi.energy(qm)[1][1] - base.energy(qm)[1][1]
    assert abs(e4) > 1e-3
    assert abs(e4 + e4m) < 1e-11 * abs(e4)
    assert abs(base.energy(q)[0] - base.energy(qm)[0]) < 1e-11 * abs(base.energy(q)[0])


@pytest.mark.parametrize("rot", ["z90", "x90"])
def test_cubic_rotation_invariance_with_chiral_and_cubic_terms(oracle_mod, rot):
    R = {"z90": np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]),
         "x90": np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]])}[rot]
    L = 6
    objects = [dict(type="sphere", c=(3.0, 2.0, 3.0), R=1.2, anchor=HOM(5.3))]
    o = oracle_mod.Oracle((L, L, L), A, B, C, 2.32, 0.5, 0.3, objects=objects, L4=0.7, L6=0.9)
    q = rand_q(o.N, 10)
    qr, objr = _lattice_rotation(L, R, q, objects)
    orr = oracle_mod.Oracle((L, L, L), A, B, C, 2.32, 0.5, 0.3, objects=objr, L4=0.7, L6=0.9)
    assert np.allclose(o.energy(q)[1], orr.energy(qr)[1], rtol=1e-12, atol=1e-12)


# ---- Frank constants -> distortion constants ---------------------------------------------

def _frank_oseen_and_q_gradient(n_expr, X, K1, K2, K3, K24, q0, S):
    """Frank-Oseen density Eq. (FOfull) of a director field written in
    sympy, and Q = 3/2 S (n n - I/3) with its gradient, as numpy callables."""
    import sympy as sp
    x, y, z = X
    n = n_expr / sp.sqrt(n_expr.dot(n_expr))
    div = sum(sp.diff(n[i], X[i]) for i in range(3))
    curl = sp.Matrix([sp.diff(n[2], y) - sp.diff(n[1], z), sp.diff(n[0], z) - sp.diff(n[2], x),
                      sp.diff(n[1], x) - sp.diff(n[0], y)])
    bend = sp.Matrix([sum(n[j] * sp.diff(n[i], X[j]) for j in range(3)) for i in range(3)])
    saddle = sum(sp.diff((bend - n * div)[i], X[i]) for i in range(3))
    fo = (K1 * div ** 2 + K2 * (n.dot(curl) + q0) ** 2 + K3 * bend.dot(bend) + K24 * saddle) / 2
    Q = sp.Rational(3, 2) * S * (n * n.T - sp.eye(3) / 3)
    d = sp.Array([[[sp.diff(Q[i, j], X[k]) for k in range(3)] for j in range(3)] for i in range(3)])
    return (sp.lambdify(X, fo, "numpy"), sp.lambdify(X, Q, "numpy"), sp.lambdify(X, d, "numpy"))


@pytest.mark.parametrize("K", [(1.3, 0.7, 1.9, 0.45, 0.21), (0.6, 0.6, 0.6, 0.6, 0.0),
                               (1.0, 0.5, 2.0, 0.0, -0.4)])
def test_frank_mapping_reproduces_the_frank_oseen_density(oracle_mod, K):
    """With the identifications of section II, the oracle's Eq.
    (fdistortionFull) at a uniaxial Q equals Eq. (FOfull) pointwise, up to
    the constant K2 q0^2 / 2, for a smooth twisted, splayed and bent field."""
    import sympy as sp
    K1, K2, K3, K24, q0 = K
    S = 0.6
    X = sp.symbols("x y z", real=True)
    x, y, z = X
    field = sp.Matrix([sp.sin(0.7 * y) + 0.3 * z, 0.5 + 0.4 * x * z,
                       1 + 0.2 * x + 0.3 * sp.cos(0.9 * y)])
    fo, Qf, df = _frank_oseen_and_q_gradient(field, X, K1, K2, K3, K24, q0, S)
    Ls = oracle_mod.frank_to_landau(K1, K2, K3, K24, q0, S)
    o = oracle_mod.Oracle((2, 2, 2), -1.0, -1.0, 1.0, Ls["L1"], Ls["L2"], Ls["L3"],
                          L4=Ls["L4"], L6=Ls["L6"])
    for pt in [(0.3, -0.2, 0.5), (1.1, 0.7, -0.4), (-0.6, 0.2, 0.9), (2.0, -1.5, 0.1)]:
        want = float(fo(*pt)) - K2 * q0 * q0 / 2
        got = o.distortion_density(np.array(Qf(*pt), float), np.array(df(*pt), float))
        assert got == pytest.approx(want, rel=1e-12, abs=1e-14)
    if K[:4] == (K1,) * 4 and q0 == 0:   # one-constant case, Eq. (fd1)
        assert Ls["L1"] == pytest.approx(2 * K1 / (9 * S * S), rel=1e-15)
        assert Ls["L2"] == Ls["L3"] == Ls["L4"] == Ls["L6"] == 0.0
