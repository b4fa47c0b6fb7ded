"""Objects after creation (section VI: objects moved and the liquid crystal
re-minimised, repeated for a potential of mean force; energy terms changed
between minimisations), solver clones, sweeps over object positions in one
batch, the custom boundary text format and the dipolar start of section
IV.A -- all through the C interface, against the oracle built with the
same (moved, changed) description."""
import numpy as np
import pytest

from _helpers import HOM, PLANAR, force_rel_err, make_pair, need_gpu, rand_q
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

A, B, C = synth.A_5CB, synth.B_5CB, synth.C_5CB
FP = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _oracle(oracle_mod, shape, L, objects, periodic=(1, 1, 1), **extra):
    return oracle_mod.Oracle(shape, A, B, C, *L, periodic=periodic, objects=list(objects), **extra)


def _moved(spec, shift):
    spec = dict(spec)
    if spec["type"] == "wall":
        spec["plane"] = spec["plane"] + int(shift[spec["axis"]])
    elif spec["type"] in ("sphere", "droplet"):
        spec["c"] = tuple(np.add(spec["c"], shift))
    elif spec["type"] == "spherocylinder":
        spec["c"] = tuple(np.add(spec["c"], shift))
        spec["c2"] = tuple(np.add(spec["c2"], shift))
    return spec


def test_moved_objects_match_the_oracle_built_at_the_new_positions(oracle_mod):
    shape, L = (32, 30, 26), (2.32, 0.5, 0.3)
    objs = [dict(type="wall", axis=2, plane=0, anchor=HOM(1.0)),
            dict(type="sphere", c=(12.0, 14.0, 12.0), R=5.0, anchor=HOM()),
            dict(type="spherocylinder", c=(20.0, 6.0, 8.0), c2=(26.0, 9.0, 15.0), R=2.5,
                 anchor=PLANAR())]
    s, o0 = make_pair(oracle_mod, shape, L, objs)
    q = rand_q(o0.N, 31)
    s.set_q(q)
    shifts = {0: (0.0, 0.0, 3.0), 1: (2.5, -1.25, 0.5), 2: (-3.0, 2.0, 1.0)}
    for k, sh in shifts.items():
        s.move_object(k, sh)
    moved = [_moved(objs[k], shifts[k]) for k in range(3)]
    o1 = _oracle(oracle_mod, shape, L, moved)
    sim0, sim1 = o0.simulated(), o1.simulated()
    assert np.array_equal(s.mask() & 1, sim1.astype(np.uint8))
    # the state: Q kept where both lattices simulate, 0 on freed sites
    want = np.where(sim0 & sim1, q, 0.0)
    got = s.get_q()
    assert np.array_equal(got, want)
    assert force_rel_err(s.force(), o1.force(want), sim1) < 1e-12
    Eo = o1.energy(want)[0]
    assert abs(s.energy()[0] - Eo) <= 1e-12 * abs(Eo)
    assert s.object_count() == 3


def test_move_rules_and_site_lists_wrap(oracle_mod):
    shape = (12, 10, 8)
    s = lqmin.Solver(shape, A, B, C, 2.32)
    s.add_objects([dict(type="wall", axis=0, plane=2, anchor=HOM()),
                   dict(type="sites", xyz=[[11, 0, 0], [11, 1, 0]], anchor=HOM())])
    with pytest.raises(lqmin.LqError):
        s.move_object(0, (0.5, 0, 0))        # walls move by whole planes
    with pytest.raises(lqmin.LqError):
        s.move_object(1, (1.0, 0.5, 0))      # site lists by lattice vectors
    with pytest.raises(lqmin.LqError):
        s.move_object(2, (1, 0, 0))          # no such object
    s.move_object(0, (-3, 7, 7))             # plane 2 - 3 wraps to 11
    s.move_object(1, (1, -1, 0))             # (0, 9, 0), (0, 0, 0)
    o = oracle_mod.Oracle(shape, A, B, C, 2.32, objects=[
        dict(type="wall", axis=0, plane=11, anchor=HOM()),
        dict(type="sites", xyz=[[0, 9, 0], [0, 0, 0]], anchor=HOM())])
    assert np.array_equal(s.mask() & 1, o.simulated().astype(np.uint8))
    s.clear_objects()
    assert s.object_count() == 0 and s.geometry_info() == (np.prod(shape), 0)


def test_step_after_a_geometry_change_uses_the_new_geometry(oracle_mod):
    """Steps captured before an object is added must not run on the old
    geometry tables: stepping after the change equals a fresh solver."""
    shape, L = (24, 22, 20), (2.32, 0.5, 0.3)
    s = lqmin.Solver(shape, A, B, C, *L)
    s.set_q(synth.random_uniaxial_q(shape, 5))
    p = lqmin.fire_params(**FP)
    s.step(p, 130)                     # long enough to capture and replay graphs
    sphere = dict(type="sphere", c=(11.0, 10.0, 9.0), R=4.0, anchor=HOM())
    s.add_objects([sphere])
    q = s.get_q()
    fresh = lqmin.Solver(shape, A, B, C, *L)
    fresh.add_objects([sphere])
    fresh.set_q(q)
    r1, r2 = s.step(p, 130), fresh.step(p, 130)
    assert r1.iterations == r2.iterations == 130
    assert np.array_equal(s.get_q(), fresh.get_q())


def test_set_material_matches_the_oracle_with_the_new_constants(oracle_mod):
    shape = (28, 24, 22)
    objs = [dict(type="wall", axis=2, plane=0, anchor=HOM(2.0)),
            dict(type="sphere", c=(13.0, 12.0, 11.0), R=4.5, anchor=PLANAR())]
    s = lqmin.Solver(shape, A, B, C, 2.32)
    s.add_objects(objs)
    q = rand_q(np.prod(shape), 12)
    s.set_q(q)
    s.step(lqmin.fire_params(**FP), 20)
    q = s.get_q()
    A2, B2, C2 = -0.3, -2.2, 1.9
    new = dict(L2=0.6, L3=-0.2, L4=0.4, L6=0.3, H=(0.2, 0.1, 0.5), mu0_dchi=0.7)
    s.set_material(A2, B2, C2, 1.9, **new)
    o = oracle_mod.Oracle(shape, A2, B2, C2, 1.9, new["L2"], new["L3"], objects=objs,
                          L4=new["L4"], L6=new["L6"], H=new["H"], mu0_dchi=new["mu0_dchi"])
    sim = o.simulated()
    assert np.array_equal(s.get_q(), q)
    assert force_rel_err(s.force(), o.force(q), sim) < 1e-11
    Eg, pg = s.energy()
    Eo, po = o.energy(q)
    assert abs(Eg - Eo) <= 1e-11 * abs(Eo)
    assert np.allclose(pg, po, rtol=1e-11, atol=1e-11 * abs(Eo))   # anchoring at the new S0
    # and back to one constant
    s.set_material(A, B, C, 2.32)
    o1 = oracle_mod.Oracle(shape, A, B, C, 2.32, objects=objs)
    assert force_rel_err(s.force(), o1.force(q), sim) < 1e-12
    with pytest.raises(lqmin.LqError):
        s.set_material(A, B, C, 2.32, L2=0.5, n_constants=1)


def test_clone_is_an_independent_copy(oracle_mod):
    shape = (26, 24, 20)
    objs = [dict(type="droplet", c=(12.5, 11.5, 9.5), R=9.0, anchor=HOM())]
    for prec in (lqmin.LQ_FP64, lqmin.LQ_FP32_BULK_FP64_RED):
        s = lqmin.Solver(shape, A, B, C, 2.32, 0.5, 0.3, precision=prec)
        s.add_objects(objs)
        s.init_random_uniaxial(3)
        p = lqmin.fire_params(**FP)
        s.step(p, 10)
        c = s.clone()
        assert np.array_equal(c.mask(), s.mask()) and c.object_count() == 1
        assert np.array_equal(c.get_q(), s.get_q())
        assert np.array_equal(c.force(), s.force())
        # both restart FIRE from the same Q: identical trajectories
        q = s.get_q()
        s.set_q(q)
        ra, rb = s.step(p, 25), c.step(p, 25)
        assert ra.iterations == rb.iterations and np.array_equal(s.get_q(), c.get_q())
        c.move_object(0, (1.0, 0.0, 0.0))
        assert not np.array_equal(c.mask(), s.mask())
        c.close()
        s.close()


def test_batch_follows_member_changes():
    """A batch built before its members' geometry or material changed
    rebuilds its tables: its steps equal the members stepped alone."""
    shape = (30, 26, 24)
    mk = lambda: lqmin.Solver(shape, A, B, C, 2.32)
    alone, mixed = [mk(), mk()], [mk(), mk()]
    sphere = dict(type="sphere", c=(14.0, 13.0, 12.0), R=5.0, anchor=HOM())
    for lst in (alone, mixed):
        lst[0].add_objects([sphere])
        for k, s in enumerate(lst):
            s.set_q(synth.random_uniaxial_q(shape, 60 + k))
    batch = lqmin.Batch(mixed)
    p = lqmin.fire_params(**FP)
    batch.step(p, 8)
    for a in alone:
        a.set_zchunk(batch.tiling()[1])
        a.step(p, 8)
    for lst in (alone, mixed):
        lst[0].move_object(0, (3.0, -2.0, 1.5))
        lst[1].add_objects([dict(type="wall", axis=1, plane=0, anchor=PLANAR())])
        lst[1].set_material(A, B, C, 1.7)
    res = batch.step(p, 9)
    for a, m, rb in zip(alone, mixed, res):
        ra = a.step(p, 9)
        assert ra.iterations == rb.iterations
        assert np.array_equal(a.get_q(), m.get_q())
    batch.close()


def test_pmf_sweep_equals_each_position_minimised_alone(oracle_mod):
    """A potential-of-mean-force sweep (section VI) minimises every
    position in one batch; each equals its clone moved and minimised alone,
    and the energy at each minimum is the oracle's energy of that state."""
    shape = (28, 24, 24)
    objs = [dict(type="wall", axis=2, plane=0, anchor=HOM(1.0)),
            dict(type="wall", axis=2, plane=23, anchor=HOM(1.0)),
            dict(type="sphere", c=(13.0, 12.0, 11.5), R=4.0, anchor=HOM(2.0))]
    base = lqmin.Solver(shape, A, B, C, 2.32)
    base.add_objects(objs)
    base.init_random_uniaxial(17)
    p = lqmin.fire_params(**dict(FP, max_iter=4000, force_tol=1e-6))
    base.minimize(p)
    shifts = np.array([[0.0, 0.0, 0.0], [1.5, 0.0, 0.0], [3.0, 0.0, 0.0], [0.0, 2.0, 1.0]])
    q_base = base.get_q()
    st, res = base.pmf_sweep(2, shifts, p)
    assert st in (lqmin.LQ_OK, lqmin.LQ_ENOTCONVERGED)
    assert np.array_equal(base.get_q(), q_base)      # base untouched
    for sh, rb in zip(shifts, res):
        c = base.clone()
        c.move_object(2, sh)
        c.set_zchunk(0)
        st1, ra = c.minimize(p)
        assert ra.iterations == rb.iterations and ra.energy == rb.energy
        o = oracle_mod.Oracle(shape, A, B, C, 2.32,
                              objects=objs[:2] + [_moved(objs[2], sh)])
        Eo = o.energy(c.get_q())[0]
        assert abs(rb.energy - Eo) <= 1e-11 * abs(Eo)
        c.close()
    assert len({r.energy for r in res}) == len(res)


def test_pmf_scan_moves_and_reminimises_in_place():
    shape = (24, 20, 20)
    s = lqmin.Solver(shape, A, B, C, 2.32)
    s.add_objects([dict(type="sphere", c=(10.0, 10.0, 10.0), R=3.5, anchor=HOM())])
    s.init_random_uniaxial(4)
    p = lqmin.fire_params(**dict(FP, max_iter=3000, force_tol=1e-6))
    out = s.pmf_scan(0, [[1.0, 0, 0]] * 3, p)
    assert len(out) == 3 and all(st in (lqmin.LQ_OK, lqmin.LQ_ENOTCONVERGED) for st, _ in out)
    ref = lqmin.Solver(shape, A, B, C, 2.32)
    ref.add_objects([dict(type="sphere", c=(13.0, 10.0, 10.0), R=3.5, anchor=HOM())])
    assert np.array_equal(ref.mask(), s.mask())


BOUNDARY = """# two custom objects and a patch of oriented anchoring
object homeotropic 2.5
  10 10 10
  11 10 10
  10 11 10
  10 10 11
end
object planar 1.0 0 0 1
  3 4 5
  3 4 6
end
boundary
  0 0 1  oriented 3.0  0.0 1.0 0.0
  1 0 1  planar 1.5  0 0 1
  2 0 1  homeotropic 0.5  0 0 1
  5 5 5  1 2e-1 1 1 0
end
"""


def test_boundary_text_equals_the_in_memory_objects(oracle_mod, tmp_path):
    shape, L = (20, 18, 16), (2.32, 0.5, 0.3)
    objs = [dict(type="sites", xyz=[[10, 10, 10], [11, 10, 10], [10, 11, 10], [10, 10, 11]],
                 anchor=(0, 2.5, (0, 0, 1))),
            dict(type="sites", xyz=[[3, 4, 5], [3, 4, 6]], anchor=(2, 1.0, (0, 0, 1))),
            dict(type="anchored", xyz=[[0, 0, 1], [1, 0, 1], [2, 0, 1], [5, 5, 5]],
                 kinds=[1, 2, 0, 1], W=[3.0, 1.5, 0.5, 0.2],
                 dirs=[[0, 1, 0], [0, 0, 1], [0, 0, 1], [1, 1, 0]])]
    a, o = make_pair(oracle_mod, shape, L, objs)
    b = lqmin.Solver(shape, A, B, C, *L)
    b.add_boundary_text(BOUNDARY)
    f = tmp_path / "boundary.txt"
    f.write_text(BOUNDARY)
    c = lqmin.Solver(shape, A, B, C, *L)
    c.load_boundary_file(str(f))
    q = rand_q(o.N, 8)
    Fo = o.force(q)
    for s in (a, b, c):
        s.set_q(q)
        assert s.object_count() == 3
        assert np.array_equal(s.mask(), a.mask())
        assert force_rel_err(s.force(), Fo, o.simulated()) < 1e-12
    # a bad text changes nothing
    with pytest.raises(lqmin.LqError, match="line 3"):
        b.add_boundary_text("object planar 1\n1 2 3\nobject planar 1\n")
    with pytest.raises(lqmin.LqError):
        b.load_boundary_file(str(tmp_path / "missing.txt"))
    assert b.object_count() == 3


@pytest.mark.parametrize("prec", [lqmin.LQ_FP64, lqmin.LQ_FP32_BULK_FP64_RED])
def test_dipolar_start_matches_the_oracle(oracle_mod, prec):
    shape = (36, 34, 40)
    c, R = (17.5, 16.25, 14.0), 6.0
    for axis in ((0.0, 0.0, 1.0), (0.4, -0.3, 0.866)):
        s = lqmin.Solver(shape, A, B, C, 2.32, precision=prec)
        s.add_objects([dict(type="sphere", c=c, R=R, anchor=HOM())])
        s.init_dipolar(c, axis, R=R)
        o = oracle_mod.Oracle(shape, A, B, C, 2.32,
                              objects=[dict(type="sphere", c=c, R=R, anchor=HOM())])
        want = oracle_mod.dipolar_q(o, c, axis, 1.25 * R, o.S0)
        tol = 1e-13 if prec == lqmin.LQ_FP64 else 2.0 ** -28
        assert np.abs(s.get_q() - want).max() <= tol
    with pytest.raises(lqmin.LqError):
        s.init_dipolar(c, (0, 0, 0), rd=5.0)
    with pytest.raises(lqmin.LqError):
        s.init_dipolar(c, (0, 0, 1), rd=-1.0)


def test_solvers_driven_from_several_threads_match_sequential_runs():
    """Distinct solvers may be used from different threads: two lattices
    minimised concurrently (the binding releases the interpreter lock in
    every call) end where they end when run one after the other."""
    import threading
    shapes = [(30, 26, 22), (28, 28, 20)]
    objs = [[dict(type="sphere", c=(15.0, 13.0, 11.0), R=4.0, anchor=HOM())], []]
    p = lqmin.fire_params(**dict(FP, max_iter=3000, force_tol=1e-8))

    def make(k):
        s = lqmin.Solver(shapes[k], A, B, C, 2.32, 0.5, 0.3)
        s.add_objects(objs[k])
        s.init_random_uniaxial(50 + k)
        return s

    seq = []
    for k in range(2):
        s = make(k)
        s.minimize(p)
        seq.append(s.get_q())
        s.close()
    par = [make(0), make(1)]
    errors = []

    def run(s):
        try:
            s.minimize(p)
        except Exception as e:   # reported below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(s,)) for s in par]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors
    for s, q in zip(par, seq):
        assert np.array_equal(s.get_q(), q)
