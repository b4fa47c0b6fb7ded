"""Shared helpers of the GPU tests: build the CUDA solver and the oracle from
the same workload description and compare their outputs."""
import numpy as np
import pytest

from paper_1911_07045_b300 import synth


def need_gpu():
    try:
        import torch
        ok = torch.cuda.is_available()
    except Exception:
        ok = False
    if not ok:
        pytest.skip("no CUDA device")


def make_pair(oracle_mod, shape, L=(2.32, 0.0, 0.0), objects=(), periodic=(1, 1, 1),
              precision=0, A=synth.A_5CB, B=synth.B_5CB, C=synth.C_5CB, zchunk=0, **extra):
    """CUDA solver and oracle on the same lattice, material and objects;
    ``extra``: L4, L6, H, mu0_dchi, E, eps0_deps."""
    from paper_1911_07045_b300 import lqmin
    L1, L2, L3 = L
    s = lqmin.Solver(shape, A, B, C, L1, L2, L3, periodic=periodic, precision=precision, **extra)
    s.add_objects(list(objects))
    if zchunk:
        s.set_zchunk(zchunk)
    o = oracle_mod.Oracle(shape, A, B, C, L1, L2, L3, periodic=periodic, objects=list(objects),
                          **extra)
    return s, o


def force_rel_err(Fg, Fo, sim=None):
    """Per-site error of the 5-component force normalised by
    max(|F_site|, 1e-12 max_site |F|); returns the largest."""
    if sim is not None:
        Fg, Fo = Fg[:, sim], Fo[:, sim]
    if Fo.size == 0:
        return 0.0
    site = np.sqrt((Fo * Fo).sum(0))
    scale = np.maximum(site, 1e-12 * max(site.max(), 1e-300))
    err = np.sqrt(((Fg - Fo) ** 2).sum(0))
    return float((err / scale).max())


def rand_q(N, seed, scale=0.3):
    return np.random.default_rng(seed).normal(scale=scale, size=(5, N))


HOM = lambda W=5.3: (0, W, (0.0, 0.0, 1.0))
PLANAR = lambda W=1.0: (2, W, (0.0, 0.0, 1.0))

# geometries of the parity cases: ragged tiles, every object kind, open and
# periodic axes, tiny and degenerate lattices
CASES = {
    "bulk1c_ragged": dict(shape=(33, 17, 9), L=(2.32, 0.0, 0.0), objects=[]),
    "bulk3c_ragged": dict(shape=(35, 9, 11), L=(2.32, 0.5, 0.3), objects=[]),
    "walls_nd_3c": dict(shape=(40, 24, 20), L=(2.32, 0.5, 0.3),
                        objects=[dict(type="wall", axis=2, plane=0, anchor=HOM()),
                                 dict(type="wall", axis=2, plane=19, anchor=HOM())]),
    "sphere_nd_1c": dict(shape=(48, 40, 36), L=(2.32, 0.0, 0.0),
                         objects=[dict(type="sphere", c=(20.0, 18.0, 17.0), R=7.0, anchor=HOM())]),
    "sphere_walls_fg_3c": dict(shape=(36, 36, 30), L=(1.7, 0.9, -0.4),
                               objects=[dict(type="wall", axis=2, plane=0, anchor=PLANAR()),
                                        dict(type="wall", axis=2, plane=29, anchor=PLANAR(1.5)),
                                        dict(type="sphere", c=(17.5, 16.0, 14.0), R=5.5,
                                             anchor=HOM())]),
    "open_y_fg_3c": dict(shape=(24, 13, 16), L=(2.32, 0.5, 0.3), periodic=(1, 0, 1),
                         objects=[dict(type="wall", axis=0, plane=3, anchor=PLANAR()),
                                  dict(type="sphere", c=(14.0, 6.0, 8.0), R=3.2,
                                       anchor=(1, 2.0, (0.3, 0.4, 0.866)))]),
    "custom_open_x_3c": dict(shape=(21, 12, 10), L=(1.0, 0.7, 0.2), periodic=(0, 1, 1),
                             objects=[dict(type="anchored",
                                           xyz=[[0, 0, 0], [20, 11, 9], [5, 5, 5], [6, 5, 5]],
                                           kinds=[2, 1, 0, 1], W=[1.0, 2.0, 0.5, 3.0],
                                           dirs=[[0, 1, 0], [1, 1, 0], [0, 0, 1], [1, 0, 0]]),
                                      dict(type="sites",
                                           xyz=[[10, 4, 4], [10, 5, 4], [11, 5, 4], [11, 5, 5]],
                                           anchor=(1, 3.0, (0.6, 0.0, 0.8))),
                                      dict(type="wall", axis=1, plane=0, anchor=HOM(1.0))]),
    "droplet_nd_1c": dict(shape=(30, 28, 26), L=(2.32, 0.0, 0.0),
                          objects=[dict(type="droplet", c=(14.5, 13.8, 12.6), R=11.0,
                                        anchor=HOM())]),
    "spherocylinder_fg_3c": dict(shape=(40, 26, 24), L=(2.32, 0.5, 0.3),
                                 objects=[dict(type="wall", axis=2, plane=0, anchor=HOM(1.0)),
                                          dict(type="spherocylinder", c=(10.0, 12.5, 11.0),
                                               c2=(29.0, 14.0, 12.5), R=4.5, anchor=PLANAR())]),
    "droplet_with_rod_open_3c": dict(shape=(28, 26, 24), L=(1.7, 0.9, -0.4), periodic=(0, 0, 0),
                                     objects=[dict(type="spherocylinder", c=(9.0, 10.0, 8.5),
                                                   c2=(18.0, 15.0, 14.5), R=2.2,
                                                   anchor=(1, 2.0, (0.3, 0.4, 0.866))),
                                              dict(type="droplet", c=(13.5, 12.5, 11.5), R=11.2,
                                                   anchor=HOM(3.0))]),
    "tiny_1x1x1": dict(shape=(1, 1, 1), L=(2.32, 0.5, 0.3), objects=[]),
    "tiny_2x3x1_open": dict(shape=(2, 3, 1), L=(2.32, 0.5, 0.3), periodic=(0, 1, 0), objects=[]),
    "chain_open": dict(shape=(5, 1, 1), L=(1.3, 0.5, 0.3), periodic=(0, 1, 1), objects=[]),
}
