"""The benchmark workload at full size (512^3, four colloids, planar walls,
three constants, and the same geometry with one constant), in the launch
configurations the benchmark times (the one-constant FP32 form on 64-wide
tiles): one FIRE step of each precision form from a seeded random start,
compared with the oracle at sampled sites -- tile and chunk seams, the
walls, the colloid surfaces and random interior sites -- plus properties
that hold at any size.

Expected values at the samples come from the oracle alone: the force at q0
(Eq. 10 with the averaged differences of Eqs. 7-9), the velocity-Verlet drift
of Algorithm 1 from rest, q1 = q0 + dt0^2/2 F(q0), applied on the samples'
neighbourhood, and the force at q1.  On a small lattice the same composition
is checked against the oracle's own FIRE step first."""
import numpy as np
import pytest

from _helpers import force_rel_err, need_gpu
from paper_1911_07045_b300 import lqmin, synth

pytestmark = pytest.mark.gpu

L = 512
FP = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 12, force_tol=0.0)
TOL = {"fp64": dict(force=1e-10, q=1e-13, rmax=1e-12),
       "fp32": dict(force=5e-5, q=1e-8, rmax=1e-6)}


def neighbourhood(sites, shape):
    """Every site within L1 distance 2 of a sample (the support of the force
    at a site), wrapped periodically."""
    nx, ny, nz = shape
    x, y, z = sites % nx, (sites // nx) % ny, sites // (nx * ny)
    offs = [(a, b, c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)
            if abs(a) + abs(b) + abs(c) <= 2]
    out = [(((z + c) % nz) * ny + (y + b) % ny) * nx + (x + a) % nx for a, b, c in offs]
    return np.unique(np.concatenate(out))


def samples(cfg, seed=0):
    nx, ny, nz = cfg["shape"]
    r = np.random.default_rng(seed)
    pts = [r.integers(0, nx * ny * nz, 1500)]
    # tile seams (32 x 4, 32 x 8 and 64 x 4 tiles) and chunk seams along z
    xs = np.array([0, 1, 31, 32, 33, 63, 64, 65, 127, 128, 255, 256, 510, 511])
    ys = np.array([0, 3, 4, 7, 8, 11, 12, 255, 256, 511])
    zs = np.array([0, 1, 2, 3, 7, 8, 15, 16, 31, 32, 63, 64, 127, 128, 129, 255, 256,
                   383, 384, 508, 509, 510, 511])
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    grid = ((Z * ny + Y) * nx + X).ravel()
    pts.append(r.choice(grid, 600, replace=False))
    # shells around each colloid surface
    for o in cfg["objects"]:
        if o["type"] != "sphere":
            continue
        d = r.normal(size=(200, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        rad = o["R"] + r.uniform(-1.0, 2.0, 200)
        p = np.floor(np.asarray(o["c"]) + d * rad[:, None]).astype(np.int64)
        p %= np.array([nx, ny, nz])
        pts.append((p[:, 2] * ny + p[:, 1]) * nx + p[:, 0])
    return np.unique(np.concatenate(pts))


@pytest.fixture(scope="module", params=["three_constants", "one_constant"])
def workload(request, oracle_mod):
    need_gpu()
    cfg = synth.config_large(L)
    if request.param == "one_constant":
        cfg = dict(cfg, L2=0.0, L3=0.0)
    q0 = synth.random_uniaxial_q(cfg["shape"], cfg["seed"])
    o = oracle_mod.Oracle(cfg["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, cfg["L1"],
                          cfg["L2"], cfg["L3"], objects=cfg["objects"])
    sim = o.simulated()
    smp = samples(cfg)
    smp = smp[sim[smp]]
    nb = neighbourhood(smp, cfg["shape"])
    dt0 = FP["dt0"]
    F0_nb = o.force_sites(q0, nb)
    # q1 on the neighbourhood (object sites stay put), in place on a copy of
    # q0's neighbourhood values that is restored afterwards
    saved = q0[:, nb].copy()
    move = sim[nb]
    q0[:, nb[move]] += 0.5 * dt0 * dt0 * F0_nb[:, move]
    q1 = q0[:, smp].copy()
    F1 = o.force_sites(q0, smp)
    q0[:, nb] = saved
    return dict(cfg=cfg, q0=q0, smp=smp, q1=q1, F1=F1)


def test_composition_is_the_oracle_step(oracle_mod):
    """q1 = q0 + dt0^2/2 F(q0) and F1 = F(q1) from rest is the oracle's own
    first FIRE step (on a small copy of the workload's structure)."""
    cfg = synth.config_large(48)
    o = oracle_mod.Oracle(cfg["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, cfg["L1"],
                          cfg["L2"], cfg["L3"], objects=cfg["objects"])
    q0 = synth.random_uniaxial_q(cfg["shape"], cfg["seed"])
    sim = o.simulated()
    qo, vo, Fo, st = o.fire(q0, FP, 1)
    q1 = q0.copy()
    q1[:, sim] += 0.5 * FP["dt0"] ** 2 * o.force(q0)[:, sim]
    assert np.array_equal(q1, qo)
    assert np.array_equal(o.force(q1)[:, sim], Fo[:, sim])


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_fullsize_step_at_samples(workload, form):
    w = workload
    prec = lqmin.LQ_FP32_BULK_FP64_RED if form == "fp32" else lqmin.LQ_FP64
    import torch
    stream = torch.cuda.Stream()
    s = lqmin.solver_for(w["cfg"], precision=prec, stream=stream.cuda_stream)
    try:
        s.set_q(w["q0"])
        r = s.step(lqmin.fire_params(**FP), 1)
        assert r.iterations == 1 and r.fire_status == lqmin.FIRE_RUNNING
        smp = w["smp"]
        Fg = s.get_force()
        # the residual is the largest site force norm over the whole lattice
        norms = np.sqrt(np.einsum("ij,ij->j", Fg, Fg))
        assert r.max_force == pytest.approx(float(norms.max()), rel=TOL[form]["rmax"])
        Fs = Fg[:, smp]
        del Fg, norms
        assert force_rel_err(Fs, w["F1"]) < TOL[form]["force"]
        assert r.max_force >= np.sqrt((w["F1"] ** 2).sum(0)).max() * (1 - TOL[form]["force"])
        qs = s.get_q()[:, smp]
        assert np.abs(qs - w["q1"]).max() < TOL[form]["q"]
    finally:
        s.close()
