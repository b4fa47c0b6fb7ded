"""CUDA path against the CPU oracle: geometry, force, energy, order field and
the random start, through the C interface (FP64 and the FP32 form)."""
import numpy as np
import pytest

from _helpers import CASES, HOM, PLANAR, force_rel_err, make_pair, need_gpu, rand_q
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

FORCE_TOL_FP64 = 1e-10     # per-site relative, normalised as in force_rel_err
ENERGY_TOL_FP64 = 1e-12    # relative total energy
# FP32 form: stencil and bulk in single precision; unit roundoff 6e-8 times
# the number of terms that cancel (O(10^2)) bounds the relative force error
FORCE_TOL_FP32 = 5e-5


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _mask_from_oracle(o, shape, periodic):
    nx, ny, nz = shape
    sim = o.simulated().reshape(nz, ny, nx)
    m = sim.astype(np.uint8)
    rec_sites = o.records()[0]
    anch = np.zeros(nx * ny * nz, bool)
    anch[rec_sites] = True
    m |= (anch.reshape(nz, ny, nx).astype(np.uint8) << 1)
    for k, ax in enumerate((2, 1, 0)):  # x, y, z in [z, y, x] order
        n = shape[k]
        for sgn, bit in ((+1, 2 + 2 * k), (-1, 3 + 2 * k)):
            nb = np.roll(sim, -sgn, axis=ax)
            if not periodic[k]:
                idx = [slice(None)] * 3
                idx[ax] = n - 1 if sgn > 0 else 0
                nb = nb.copy()
                nb[tuple(idx)] = False
            m |= ((nb & sim).astype(np.uint8) << bit)
    return m.ravel()


@pytest.mark.parametrize("name", sorted(CASES))
def test_geometry_masks_match_oracle(oracle_mod, name):
    c = CASES[name]
    per = c.get("periodic", (1, 1, 1))
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per)
    want = _mask_from_oracle(o, c["shape"], per)
    got = s.mask()
    assert np.array_equal(got, want)
    nsim, nrec = s.geometry_info()
    assert nsim == int(o.simulated().sum()) and nrec == int(o.geom.nrec)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("zchunk", [0, 1, 3])
def test_force_and_energy_fp64(oracle_mod, name, zchunk):
    c = CASES[name]
    per = c.get("periodic", (1, 1, 1))
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per, zchunk=zchunk)
    q = rand_q(o.N, 17)
    s.set_q(q)
    Fo = o.force(q)
    Fg = s.force()
    sim = o.simulated()
    assert force_rel_err(Fg, Fo, sim) < FORCE_TOL_FP64
    assert np.all(Fg[:, ~sim] == 0)
    Eo, po = o.energy(q)
    Eg, pg = s.energy()
    assert abs(Eg - Eo) <= ENERGY_TOL_FP64 * abs(Eo)
    assert np.allclose(pg, po, rtol=1e-12, atol=1e-12 * abs(Eo))
    # object sites read back as zero
    qg = s.get_q()
    assert np.array_equal(qg[:, sim], q[:, sim]) and np.all(qg[:, ~sim] == 0)


@pytest.mark.parametrize("name", ["walls_nd_3c", "sphere_walls_fg_3c", "bulk1c_ragged",
                                  "custom_open_x_3c", "spherocylinder_fg_3c",
                                  "droplet_with_rod_open_3c"])
def test_force_fp32_form(oracle_mod, name):
    c = CASES[name]
    per = c.get("periodic", (1, 1, 1))
    s, o = make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per, precision=1)
    q = np.round(rand_q(o.N, 5) * 2.0 ** 28) / 2.0 ** 28   # on the form's fixed-point grid
    s.set_q(q)
    Fo = o.force(q)
    assert force_rel_err(s.force(), Fo, o.simulated()) < FORCE_TOL_FP32
    Eo, po = o.energy(q)
    Eg, pg = s.energy()               # FP64 arithmetic on the FP32 state
    # bulk and distortion see the same (FP32-representable) Q: FP64 agreement
    assert abs(pg[0] - po[0]) <= 1e-12 * abs(po[0]) + 1e-12
    assert abs(pg[1] - po[1]) <= 1e-12 * abs(po[1]) + 1e-12
    # the FP32 form keeps its anchoring targets on its Q grid (Q0) or in
    # float (nu)
    assert abs(pg[2] - po[2]) <= 1e-6 * abs(po[2]) + 1e-9
    assert abs(Eg - Eo) <= 1e-7 * abs(Eo)


def test_colloid_slab_128_full_force(oracle_mod):
    """The 128^3 homeotropic slab with a centred colloid (three constants)."""
    cfg = synth.config_colloid_slab()
    s, o = make_pair(oracle_mod, cfg["shape"], (cfg["L1"], cfg["L2"], cfg["L3"]), cfg["objects"])
    q = synth.random_uniaxial_q(cfg["shape"], cfg["seed"])
    s.set_q(q)
    assert force_rel_err(s.force(), o.force(q), o.simulated()) < FORCE_TOL_FP64
    Eo, _ = o.energy(q)
    Eg, _ = s.energy()
    assert abs(Eg - Eo) <= ENERGY_TOL_FP64 * abs(Eo)


def test_order_field_and_random_start(oracle_mod):
    shape = (20, 12, 9)
    objs = [dict(type="sphere", c=(10.0, 6.0, 4.0), R=3.0, anchor=HOM())]
    s, o = make_pair(oracle_mod, shape, (2.32, 0, 0), objs)
    s.init_random_uniaxial(77, 0.0)
    qg = s.get_q()
    want = synth.random_uniaxial_q(shape, 77)
    sim = o.simulated()
    assert np.abs(qg[:, sim] - want[:, sim]).max() < 1e-15
    assert np.all(qg[:, ~sim] == 0)
    q = rand_q(o.N, 3)
    s.set_q(q)
    assert np.abs(s.order_field() - o.order_field(q)).max() < 1e-12


def test_empty_lattice_all_object_sites(oracle_mod):
    shape = (4, 3, 1)
    objs = [dict(type="wall", axis=2, plane=0, anchor=HOM())]
    s, o = make_pair(oracle_mod, shape, (2.32, 0.5, 0.3), objs)
    assert s.geometry_info() == (0, 0)
    s.set_q(rand_q(12, 1))
    assert np.all(s.force() == 0)
    assert s.energy()[0] == 0.0


@pytest.mark.parametrize("name", ["bulk3c_ragged", "sphere_walls_fg_3c", "custom_open_x_3c",
                                  "droplet_with_rod_open_3c", "sphere_nd_1c"])
@pytest.mark.parametrize("prec", [0, 1])
def test_index64_kernels_equal_index32(oracle_mod, name, prec):
    """The 64-bit-index instantiation of the step kernels (the path of
    lattices above about 950^3 sites) computes exactly what the 32-bit one
    does: forced on small lattices, forces and FIRE trajectories agree bit
    for bit, and with the oracle."""
    c = CASES[name]
    per = c.get("periodic", (1, 1, 1))
    pair = [make_pair(oracle_mod, c["shape"], c["L"], c["objects"], per, precision=prec)
            for _ in range(2)]
    (a, o), (b, _) = pair
    b.set_index_width(64)
    q = rand_q(o.N, 23)
    if prec == 1:
        q = np.round(q * 2.0 ** 28) / 2.0 ** 28
    for s in (a, b):
        s.set_q(q)
    Fa, Fb = a.force(), b.force()
    assert np.array_equal(Fa, Fb)
    tol = FORCE_TOL_FP64 if prec == 0 else FORCE_TOL_FP32
    assert force_rel_err(Fb, o.force(q), o.simulated()) < tol
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14))
    ra, rb = a.step(p, 150), b.step(p, 150)
    assert ra.iterations == rb.iterations == 150 and ra.max_force == rb.max_force
    assert np.array_equal(a.get_q(), b.get_q())
    with pytest.raises(lqmin.LqError):
        b.set_index_width(32)


def test_index64_member_in_a_batch():
    """A batch with a member forced to 64-bit indices runs the 64-bit batch
    kernel for all; one-constant members still advance bit for bit as alone."""
    shape = (40, 26, 22)
    mk = lambda: lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32,
                              precision=lqmin.LQ_FP32_BULK_FP64_RED)
    alone, mixed = [mk(), mk()], [mk(), mk()]
    for lst in (alone, mixed):
        lst[0].add_objects([dict(type="sphere", c=(20.0, 13.0, 11.0), R=5.0, anchor=HOM())])
        for k, s in enumerate(lst):
            s.set_q(synth.random_uniaxial_q(shape, 70 + k))
    mixed[1].set_index_width(64)
    batch = lqmin.Batch(mixed)
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14))
    res = batch.step(p, 33)
    for a, m, rb in zip(alone, mixed, res):
        a.set_zchunk(batch.tiling()[1])
        ra = a.step(p, 33)
        assert ra.iterations == rb.iterations == 33
        assert np.array_equal(a.get_q(), m.get_q())
    batch.close()


def test_empty_and_zero_length_inputs():
    """Empty site lists and boundary text, zero steps, and a lattice with no
    simulated site at all: nothing changes, nothing divides by zero."""
    shape = (10, 9, 8)
    s = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32)
    s.add_object_sites(np.zeros((0, 3), np.int32))
    s.add_anchored_sites(np.zeros((0, 3), np.int32), [], [], np.zeros((0, 3)))
    s.add_boundary_text("# nothing here\n")
    assert s.object_count() == 2 and s.geometry_info() == (np.prod(shape), 0)
    s.init_random_uniaxial(2)
    q = s.get_q()
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=1000, force_tol=1e-9))
    r = s.step(p, 0)
    assert r.iterations == 0 and r.fire_status == lqmin.FIRE_RUNNING
    assert np.array_equal(s.get_q(), q)
    # every site an object site: converged at once, zero residual
    e = lqmin.Solver((4, 3, 1), synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32)
    e.add_objects([dict(type="wall", axis=2, plane=0, anchor=HOM())])
    e.init_random_uniaxial(1)
    st, r = e.minimize(p)
    assert st == lqmin.LQ_OK and r.fire_status == lqmin.FIRE_CONVERGED
    assert r.max_force == 0.0 and r.rms_force == 0.0 and np.isfinite(r.energy)


def test_wide_tiles_of_wide_one_constant_fp32_lattices(oracle_mod):
    """One-constant FP32 lattices at least 256 sites wide run 64-wide tiles
    (the ragged last tile here holds 4 columns); force and FIRE steps against
    the oracle."""
    shape = (260, 12, 10)
    objs = [dict(type="sphere", c=(130.0, 6.0, 5.0), R=3.5, anchor=HOM()),
            dict(type="wall", axis=1, plane=0, anchor=PLANAR()),
            dict(type="sites", xyz=[[0, 5, 5], [63, 5, 5], [64, 5, 5], [259, 7, 3]],
                 anchor=HOM(2.0))]
    s, o = make_pair(oracle_mod, shape, (2.32, 0.0, 0.0), objs, precision=1)
    q = np.round(rand_q(o.N, 41) * 2.0 ** 28) / 2.0 ** 28
    s.set_q(q)
    sim = o.simulated()
    assert force_rel_err(s.force(), o.force(q), sim) < FORCE_TOL_FP32
    fp = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)
    r = s.step(lqmin.fire_params(**fp), 40)
    qo, vo, Fo, st = o.fire(q, fp, 40)
    assert r.iterations == st["iter"] == 40
    assert np.abs(s.get_q()[:, sim] - qo[:, sim]).max() < 1e-5


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dtype", [0, 1])
def test_set_q_from_device_memory(prec, dtype):
    """lq_set_q_device takes Q from a device array of doubles or floats (a
    torch tensor here) and equals the same values given through host memory;
    the FP32 form refuses values outside its fixed-point range."""
    import torch
    shape = (20, 18, 16)
    objs = [dict(type="sphere", c=(10.0, 9.0, 8.0), R=3.5, anchor=HOM())]
    a = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, 0.5, 0.3, precision=prec)
    b = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, 0.5, 0.3, precision=prec)
    for s in (a, b):
        s.add_objects(objs)
    q = synth.random_uniaxial_q(shape, 9)
    t = torch.tensor(q, dtype=torch.float64 if dtype == 0 else torch.float32, device="cuda")
    torch.cuda.synchronize()
    a.set_q_device(t.data_ptr(), dtype)
    b.set_q(t.cpu().double().numpy())
    assert np.array_equal(a.get_q(), b.get_q())
    assert np.array_equal(a.force(), b.force())
    if prec == 1:
        bad = torch.full_like(t, 3.0)
        torch.cuda.synchronize()
        with pytest.raises(lqmin.LqError):
            a.set_q_device(bad.data_ptr(), dtype)
    with pytest.raises(lqmin.LqError):
        a.set_q_device(t.data_ptr(), 2)
