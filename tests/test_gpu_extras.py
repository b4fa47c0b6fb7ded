"""The chiral L4 and cubic L6 terms of Eq. (fdistortionFull) and the
external-field term (section II) on the GPU against the oracle: force,
energy, a FIRE step, the FP32 form, batches and the allocation-free energy."""
import numpy as np
import pytest

from _helpers import CASES, force_rel_err, make_pair, need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

EXTRA = dict(L4=0.7, L6=0.9, H=(0.3, -0.2, 0.5), mu0_dchi=1.3, E=(0.1, 0.4, 0.2), eps0_deps=-0.6)
FIELDS = dict(H=(0.3, -0.2, 0.5), mu0_dchi=1.3, E=(0.1, 0.4, 0.2), eps0_deps=-0.6)
THREE_CASES = [n for n in sorted(CASES) if CASES[n]["L"][1] != 0.0 or CASES[n]["L"][2] != 0.0]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("name", THREE_CASES)
@pytest.mark.parametrize("zchunk", [0, 3])
def test_chiral_cubic_fields_force_and_energy_fp64(oracle_mod, name, zchunk):
    c = CASES[name]
    per = c.get("periodic", (1, 1, 1))
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per, zchunk=zchunk, **EXTRA)
    q = synth.random_uniaxial_q(c["shape"], 31)
    s.set_q(q)
    sim = o.simulated()
    assert force_rel_err(s.force(), o.force(q), sim) < 1e-10
    Eg, pg = s.energy()
    Eo, po = o.energy(q)
    assert abs(Eg - Eo) <= 1e-12 * abs(Eo)
    assert np.allclose(pg, po, rtol=1e-12, atol=1e-12 * abs(Eo))


@pytest.mark.parametrize("name", ["bulk1c_ragged", "sphere_nd_1c", "walls_nd_3c"])
def test_fields_alone_force(oracle_mod, name):
    """Fields without L4 / L6 keep the regular fast path (one- and
    three-constant): the field force is the same at every site."""
    c = CASES[name]
    per = c.get("periodic", (1, 1, 1))
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per, **FIELDS)
    q = synth.random_uniaxial_q(c["shape"], 32)
    s.set_q(q)
    assert force_rel_err(s.force(), o.force(q), o.simulated()) < 1e-10
    assert abs(s.energy()[0] - o.energy(q)[0]) <= 1e-12 * abs(o.energy(q)[0])


def test_chiral_cubic_fp32_form(oracle_mod):
    c = CASES["sphere_walls_fg_3c"]
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"],
                     precision=lqmin.LQ_FP32_BULK_FP64_RED, **EXTRA)
    q = synth.random_uniaxial_q(c["shape"], 33)
    s.set_q(q)
    assert force_rel_err(s.force(), o.force(q), o.simulated()) < 5e-5


def test_chiral_cubic_fire_steps(oracle_mod):
    c = CASES["walls_nd_3c"]
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], **EXTRA)
    q0 = synth.random_uniaxial_q(c["shape"], 34)
    s.set_q(q0)
    params = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-12)
    r = s.step(lqmin.fire_params(**params), 20)
    qo, vo, Fo, st = o.fire(q0, params, 20)
    sim = o.simulated()
    assert r.iterations == st["iter"] == 20
    assert np.abs(s.get_q()[:, sim] - qo[:, sim]).max() < 1e-11
    assert abs(r.dt - st["dt"]) <= 1e-12 * st["dt"]


def test_chiral_helix_relaxes_toward_its_pitch(oracle_mod):
    """A twist helix with L4 < 0 relaxes toward positive twist: starting
    from the uniform state plus a small twist, FIRE increases the twist
    energy gain (the L4 part of the energy falls below zero)."""
    shape = (4, 4, 40)
    s = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, 0.0, 0.0, L4=-0.5,
                     n_constants=3)
    z = np.repeat(np.arange(shape[2]), shape[0] * shape[1]).astype(float)
    k = 2 * np.pi / shape[2]
    n = np.stack([np.cos(k * z), np.sin(k * z), np.zeros_like(z)])
    S0 = synth.s0_closed_form(synth.A_5CB, synth.B_5CB, synth.C_5CB)
    s.set_q(synth.uniaxial_q(n, S0))
    E0 = s.energy()[0]
    code, r = s.minimize(lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=100000,
                                                  force_tol=1e-7)))
    assert code == lqmin.LQ_OK
    assert r.energy < E0


def test_batch_mixing_chiral_and_plain_lattices(oracle_mod):
    """A batch with one chiral/cubic lattice runs every member through the
    general path; each still matches its solve alone within rounding."""
    A, B, C = synth.A_5CB, synth.B_5CB, synth.C_5CB
    cfgs = [dict(shape=(24, 20, 18), extra=EXTRA),
            dict(shape=(20, 16, 12), extra={})]
    alone, mixed = [], []
    for k, c in enumerate(cfgs):
        for lst in (alone, mixed):
            s = lqmin.Solver(c["shape"], A, B, C, 2.32, 0.5, 0.3, **c["extra"])
            s.set_q(synth.random_uniaxial_q(c["shape"], 50 + k))
            lst.append(s)
    batch = lqmin.Batch(mixed)
    ty, zc = batch.tiling()
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14))
    res = batch.step(p, 12)
    for a, m, rb in zip(alone, mixed, res):
        a.set_zchunk(zc)
        ra = a.step(p, 12)
        assert ra.iterations == rb.iterations == 12
        qa = a.get_q()
        assert np.abs(qa - m.get_q()).max() <= 1e-12 * np.abs(qa).max()
    batch.close()


def test_noalloc_energy_with_chiral_cubic_fields(oracle_mod):
    import ctypes as C
    import torch
    c = CASES["sphere_walls_fg_3c"]
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], **EXTRA)
    q = synth.random_uniaxial_q(c["shape"], 35)
    nx, ny, nz = c["shape"]
    qd = torch.tensor(q, dtype=torch.float64, device="cuda").contiguous()
    md = torch.tensor(s.mask(), dtype=torch.uint8, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    lat = lqmin.Lattice(nx, ny, nz, 1.0, (C.c_int * 3)(1, 1, 1))
    mat = lqmin.Material(synth.A_5CB, synth.B_5CB, synth.C_5CB, *c["L"], EXTRA["L4"], EXTRA["L6"], 3,
                         0.0, (C.c_double * 3)(*EXTRA["H"]), EXTRA["mu0_dchi"],
                         (C.c_double * 3)(*EXTRA["E"]), EXTRA["eps0_deps"])
    st = s.lib.lq_energy_noalloc(C.byref(lat), C.byref(mat), C.c_void_p(qd.data_ptr()),
                                 C.c_void_p(md.data_ptr()), C.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert st == lqmin.LQ_OK
    _, po = o.energy(q)
    # bulk (with fields) and distortion (with L4, L6); anchoring is not part of it
    assert np.allclose(out.cpu().numpy()[:2], po[:2], rtol=1e-12, atol=1e-10)


CHIRAL = dict(L4=0.7, H=(0.3, -0.2, 0.5), mu0_dchi=1.3)


@pytest.mark.parametrize("name", THREE_CASES)
@pytest.mark.parametrize("zchunk", [0, 3])
def test_chiral_alone_regular_path_fp64(oracle_mod, name, zchunk):
    """The chiral term without the cubic one (L6 = 0) runs the regular-site
    path on regular planes (central differences) and the general path
    elsewhere: force and energy against the oracle on every three-constant
    geometry."""
    c = CASES[name]
    per = c.get("periodic", (1, 1, 1))
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per, zchunk=zchunk, **CHIRAL)
    q = synth.random_uniaxial_q(c["shape"], 34)
    s.set_q(q)
    sim = o.simulated()
    assert force_rel_err(s.force(), o.force(q), sim) < 1e-10
    Eg, pg = s.energy()
    Eo, po = o.energy(q)
    assert abs(Eg - Eo) <= 1e-12 * abs(Eo)


@pytest.mark.parametrize("name", ["bulk3c_ragged", "sphere_walls_fg_3c"])
def test_chiral_alone_fp32_form_and_steps(oracle_mod, name):
    c = CASES[name]
    per = c.get("periodic", (1, 1, 1))
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per,
                     precision=lqmin.LQ_FP32_BULK_FP64_RED, **CHIRAL)
    q = np.round(synth.random_uniaxial_q(c["shape"], 35) * 2.0 ** 28) / 2.0 ** 28
    s.set_q(q)
    assert force_rel_err(s.force(), o.force(q), o.simulated()) < 5e-5
    f64, _ = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per, **CHIRAL)
    fp = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)
    f64.set_q(q)
    r = f64.step(lqmin.fire_params(**fp), 60)
    qo, vo, Fo, st = o.fire(q, fp, 60)
    assert r.iterations == st["iter"] == 60
    sim = o.simulated()
    assert np.abs(f64.get_q()[:, sim] - qo[:, sim]).max() < 1e-9


@pytest.mark.parametrize("precision", [lqmin.LQ_FP64, lqmin.LQ_FP32_BULK_FP64_RED])
@pytest.mark.parametrize("L6", [0.0, 0.9])
def test_helix_energy_on_the_gpu_is_the_closed_form(precision, L6):
    """A twist helix n = (cos kz, sin kz, 0) on a periodic lattice: every
    site sees the same averaged differences, so the distortion energy per
    site is (9 S^2/8) L1 (1 - cos 2k) + (9 S^2/16) L4 sin 2k
    - (9 L6 S^3/16)(1 - cos 2k), with no L2, L3 part (Q_iz = 0 for i != z).
    The GPU's energy equals N times that, and the lowest-energy helix among
    the lattice's wave numbers is the one nearest tan 2k = -L4 / (2 L1)
    (with L6 = 0); no bulk terms (A = B = C = 0, S0 given)."""
    shape = (4, 4, 120)
    S, L1 = 0.5, 2.32
    z = np.repeat(np.arange(shape[2]), shape[0] * shape[1]).astype(float)
    N = shape[0] * shape[1] * shape[2]
    for L4 in (-0.5, 0.5):
        s = lqmin.Solver(shape, 0.0, 0.0, 0.0, L1, 0.5, 0.3, precision=precision, L4=L4, L6=L6,
                         n_constants=3, S0=S)
        ks = 2 * np.pi * np.arange(-6, 7) / shape[2]
        E = []
        for k in ks:
            n = np.stack([np.cos(k * z), np.sin(k * z), np.zeros_like(z)])
            q = synth.uniaxial_q(n, S)
            if precision == lqmin.LQ_FP32_BULK_FP64_RED:
                q = np.round(q * 2.0 ** 28) / 2.0 ** 28
            s.set_q(q)
            _, parts = s.energy()
            per = (9 * S ** 2 / 8 * L1 * (1 - np.cos(2 * k)) + 9 * S ** 2 / 16 * L4 * np.sin(2 * k)
                   - 9 * L6 * S ** 3 / 16 * (1 - np.cos(2 * k)))
            # FP32 form: the energy of the fixed-point-rounded state
            tol = 1e-12 if precision == lqmin.LQ_FP64 else 2e-6
            assert abs(parts[1] - N * per) <= tol * N * max(abs(per), 1e-3)
            E.append(parts[1])
        if L6 == 0.0:
            kbest = ks[int(np.argmin(E))]
            kstar = -0.5 * np.arctan(L4 / (2 * L1))
            assert np.sign(kbest) == np.sign(kstar)
            assert abs(kbest - kstar) <= np.pi / shape[2]
        s.close()
