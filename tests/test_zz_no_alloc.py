"""lq_energy_noalloc: the energy entry point for callers that cannot let a
library allocate device memory (their memory is reserved up front by their
own allocator or budget, or their loop cannot take the device-wide
synchronisation of cudaMalloc/cudaFree).  It uses only a static device
scratch array; the caller owns every input and output buffer.

The test calls it twice in a row through the C interface, on two different
Q fields, and compares each result with lq_energy's bulk and distortion
parts for the same field.  This file is collected last so that a failure
here leaves every other test already run."""
import ctypes as C

import pytest

from _helpers import HOM, PLANAR, need_gpu, rand_q
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_lq_energy():
    need_gpu()
    import torch
    shape = (37, 22, 19)
    objs = [dict(type="wall", axis=2, plane=0, anchor=PLANAR()),
            dict(type="sphere", c=(18.0, 11.0, 9.0), R=4.5, anchor=HOM())]
    L1, L2, L3 = 2.32, 0.5, 0.3
    per = (1, 0, 1)
    s = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, periodic=per)
    s.add_objects(objs)
    lib = lqmin.load()
    lat = lqmin.Lattice(*shape, 1.0, (C.c_int * 3)(*per))
    mat = lqmin.Material(synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, 0.0, 0.0, 3, 0.0)
    mask = torch.from_numpy(s.mask()).cuda()          # caller-owned device buffers
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for seed in (3, 4):                                # two calls in a row
        q = rand_q(s.N, seed)
        s.set_q(q)
        _, want = s.energy()
        qd = torch.from_numpy(q).cuda()
        torch.cuda.synchronize()
        st = lib.lq_energy_noalloc(C.byref(lat), C.byref(mat), C.c_void_p(qd.data_ptr()),
                                   C.c_void_p(mask.data_ptr()), C.c_void_p(out.data_ptr()), None)
        assert st == lqmin.LQ_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - want[0]) <= 1e-12 * abs(want[0])
        assert abs(got[1] - want[1]) <= 1e-12 * abs(want[1])
        assert got[2] == 0.0
    # sizes beyond the static scratch are refused
    big = lqmin.Lattice(2, 2, 4097, 1.0, (C.c_int * 3)(1, 1, 1))
    st = lib.lq_energy_noalloc(C.byref(big), C.byref(mat), C.c_void_p(qd.data_ptr()),
                               C.c_void_p(mask.data_ptr()), C.c_void_p(out.data_ptr()), None)
    assert st == lqmin.LQ_EINVAL
    # lattice and material are checked as lq_create checks them
    bad_spacing = lqmin.Lattice(*shape, 0.5, (C.c_int * 3)(*per))
    one_c_with_l2 = lqmin.Material(synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, 0.0, 0.0, 0.0, 1, 0.0)
    two_consts = lqmin.Material(synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, 0.0, 0.0, 2, 0.0)
    for la, ma in ((bad_spacing, mat), (lat, one_c_with_l2), (lat, two_consts)):
        st = lib.lq_energy_noalloc(C.byref(la), C.byref(ma), C.c_void_p(qd.data_ptr()),
                                   C.c_void_p(mask.data_ptr()), C.c_void_p(out.data_ptr()), None)
        assert st == lqmin.LQ_EINVAL
    s.close()


def test_energy_noalloc_mask_for_other_periodic_flags():
    """A mask built on a fully periodic lattice, passed with a lattice that
    is open on every axis: its bits that name neighbours across the open
    edges count as absent neighbours, so the result is finite and equals
    lq_energy's bulk and distortion parts of the open lattice itself."""
    need_gpu()
    import torch
    shape = (24, 17, 13)
    objs = [dict(type="sphere", c=(12.0, 8.0, 6.0), R=3.5, anchor=HOM())]
    L1, L2, L3 = 2.32, 0.5, 0.3
    lib = lqmin.load()
    periodic = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, periodic=(1, 1, 1))
    periodic.add_objects(objs)
    open_ = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, periodic=(0, 0, 0))
    open_.add_objects(objs)
    q = rand_q(open_.N, 11)
    open_.set_q(q)
    _, want = open_.energy()
    lat = lqmin.Lattice(*shape, 1.0, (C.c_int * 3)(0, 0, 0))
    mat = lqmin.Material(synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, 0.0, 0.0, 3, 0.0)
    mask = torch.from_numpy(periodic.mask()).cuda()
    qd = torch.from_numpy(q).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = lib.lq_energy_noalloc(C.byref(lat), C.byref(mat), C.c_void_p(qd.data_ptr()),
                               C.c_void_p(mask.data_ptr()), C.c_void_p(out.data_ptr()), None)
    assert st == lqmin.LQ_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert abs(got[0] - want[0]) <= 1e-12 * abs(want[0])
    assert abs(got[1] - want[1]) <= 1e-12 * abs(want[1])
    periodic.close()
    open_.close()


def test_energy_noalloc_chiral_cubic_and_fields():
    """The chiral (L4) and cubic (L6) distortion terms and the magnetic and
    electric field terms: the two energy calls evaluate each of them in
    their own kernels, and the two results agree to 1e-12 in both parts on
    a lattice with an open axis, a wall and a colloid."""
    need_gpu()
    import torch
    shape = (21, 18, 16)
    objs = [dict(type="wall", axis=2, plane=0, anchor=HOM()),
            dict(type="sphere", c=(10.0, 9.0, 8.0), R=3.5, anchor=PLANAR())]
    per = (1, 1, 0)
    L1, L2, L3 = 2.32, 0.5, 0.3
    extra = dict(L4=0.7, L6=0.9, H=(0.3, -0.2, 0.5), mu0_dchi=1.3, E=(0.1, 0.4, 0.2), eps0_deps=-0.6)
    s = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, periodic=per, **extra)
    s.add_objects(objs)
    lib = lqmin.load()
    lat = lqmin.Lattice(*shape, 1.0, (C.c_int * 3)(*per))
    mat = lqmin.material(synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, **extra)
    mask = torch.from_numpy(s.mask()).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    q = rand_q(s.N, 17)
    s.set_q(q)
    _, want = s.energy()
    qd = torch.from_numpy(q).cuda()
    torch.cuda.synchronize()
    st = lib.lq_energy_noalloc(C.byref(lat), C.byref(mat), C.c_void_p(qd.data_ptr()),
                               C.c_void_p(mask.data_ptr()), C.c_void_p(out.data_ptr()), None)
    assert st == lqmin.LQ_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert abs(got[0] - want[0]) <= 1e-12 * abs(want[0])
    assert abs(got[1] - want[1]) <= 1e-12 * abs(want[1])
    # the terms are really there: without them both parts change
    plain = lqmin.Solver(shape, synth.A_5CB, synth.B_5CB, synth.C_5CB, L1, L2, L3, periodic=per)
    plain.add_objects(objs)
    plain.set_q(q)
    _, base = plain.energy()
    assert abs(base[0] - want[0]) > 1e-6 * abs(want[0])
    assert abs(base[1] - want[1]) > 1e-6 * abs(want[1])
    plain.close()
    s.close()
