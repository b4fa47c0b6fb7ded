"""One lattice decomposed into z slabs (paper_1911_07045_b300/sharded.py) on
CPU ranks: the partition, the halo routing and the FP64 combination of FIRE's
sums, driven through ``run_ranks`` over gloo exactly as the GPU slabs are
driven over NCCL.  Each rank's slab is a plain CPU restatement of the step
(Algorithm 1 on the own planes, the force from the oracle of the whole
lattice, halo planes filled only by the exchange); two and three ranks must
reproduce the oracle's own FIRE on the whole lattice."""
import math
import os
import socket
import sys
import types

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1911_07045_b300 import sharded, synth  # noqa: E402

HOM = (0, 5.3, (0.0, 0.0, 1.0))
PLANAR = (2, 1.0, (0.0, 0.0, 1.0))
FP = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-12)
STEPS = 9
CASES = {
    "periodic_z": dict(shape=(9, 8, 12), periodic=(1, 1, 1),
                       objects=[dict(type="sphere", c=(4.0, 3.5, 2.0), R=2.2, anchor=HOM)]),
    "open_z_walls": dict(shape=(8, 7, 11), periodic=(1, 1, 0),
                         objects=[dict(type="wall", axis=2, plane=0, anchor=PLANAR),
                                  dict(type="sphere", c=(3.5, 3.0, 6.0), R=2.0, anchor=HOM)]),
}


def test_slab_bounds_partition_the_planes():
    for nz in (1, 2, 7, 12, 64):
        for world in range(1, min(nz, 9) + 1):
            b = [sharded.slab_bounds(nz, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == nz
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [h - l for l, h in b]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharded.slab_bounds(3, 4, 0)
    with pytest.raises(ValueError):
        sharded.slab_bounds(8, 2, 2)


def test_slab_field_takes_halos_with_the_periodicity():
    shape = (2, 3, 5)
    f = np.arange(2 * 30, dtype=float).reshape(2, 30)
    plane = lambda z: f[:, 6 * z:6 * z + 6]
    got = sharded.slab_field(f, shape, 0, 2, periodic_z=True).reshape(2, 4, 6)
    for k, z in enumerate((4, 0, 1, 2)):
        assert np.array_equal(got[:, k], plane(z))
    got = sharded.slab_field(f, shape, 3, 5, periodic_z=False).reshape(2, 4, 6)
    for k, z in enumerate((2, 3, 4)):
        assert np.array_equal(got[:, k], plane(z))
    assert not got[:, 3].any()


def test_halo_routing_and_combination():
    planes = [(f"lo{r}", f"hi{r}") for r in range(3)]
    assert sharded.neighbour_planes(planes, True) == [("hi2", "lo1"), ("hi0", "lo2"), ("hi1", "lo0")]
    assert sharded.neighbour_planes(planes, False) == [(None, "lo1"), ("hi0", "lo2"), ("hi1", None)]
    assert sharded.neighbour_planes([("lo", "hi")], True) == [("hi", "lo")]
    t = sharded.combine([[1.0, 2.0, 3.0, 4.0], [0.5, 0.25, 1.0, 9.0]])
    assert list(t) == [1.5, 2.25, 4.0, 9.0]


class OracleSlab:
    """Algorithm 1 on the own planes [z_lo, z_hi) of the whole lattice: the
    force from the oracle (which reads only the own planes, the halo planes
    and the neighbour bits of the masks), the drift on the own and halo
    planes, the sums over the own simulated sites, the FIRE scalar rules
    from the combined sums; halo planes are changed by the exchange only."""

    def __init__(self, o, shape, z_lo, z_hi, q0, periodic_z):
        import oracle
        self.oracle = oracle
        nx, ny, nz = shape
        nxy = nx * ny
        self.o = o
        self.q = np.array(q0, dtype=float).reshape(5, -1).copy()
        self.v = np.zeros_like(self.q)
        self.F = np.zeros_like(self.q)
        plane = lambda z: np.arange(z * nxy, (z + 1) * nxy)
        self.own = np.concatenate([plane(z) for z in range(z_lo, z_hi)])
        sim = o.simulated()
        self.own_sim = self.own[sim[self.own]]
        self.lo, self.hi = plane(z_lo), plane(z_hi - 1)
        self.below = plane((z_lo - 1) % nz) if (z_lo > 0 or periodic_z) else None
        self.above = plane(z_hi % nz) if (z_hi < nz or periodic_z) else None
        halo = [h for h in (self.below, self.above) if h is not None]
        d = np.concatenate([self.own] + halo)
        self.drift_sites = np.unique(d[sim[d]])

    def sums(self):
        F, v = self.F[:, self.own_sim], self.v[:, self.own_sim]
        site = (F * F).sum(0)
        return np.array([(F * v).sum(), site.sum(), (v * v).sum(), site.max() if site.size else 0.0])

    def start(self, params):
        self.params = params
        self.state = None
        self.v[:] = 0.0
        self.F[:, self.own] = self.o.force_sites(self.q, self.own)
        return self.sums()

    def step(self):
        dt = self.state["dt"]
        d = self.drift_sites
        self.q[:, d] += dt * self.v[:, d] + 0.5 * dt * dt * self.F[:, d]
        Fn = self.o.force_sites(self.q, self.own)
        self.v[:, self.own] += 0.5 * dt * (self.F[:, self.own] + Fn)
        self.F[:, self.own] = Fn
        self.state["iter"] += 1
        return self.sums()

    def finish(self, total):
        P, F2, V2, R2 = total
        p = self.params
        if self.state is None:
            self.state = dict(dt=p["dt0"], alpha=p["alpha0"], npos=0, iter=0, initialized=1, status=0,
                              P=P, normF=math.sqrt(F2), normv=math.sqrt(V2), rmax=math.sqrt(R2))
            if math.sqrt(R2) < p["force_tol"]:
                self.state["status"] = 1
        elif math.sqrt(R2) < p["force_tol"]:
            self.state["status"] = 1
        elif self.state["iter"] >= p["max_iter"]:
            self.state["status"] = 2
        else:
            a, b, st = self.oracle.fire_scalars(p, self.state, P, math.sqrt(F2), math.sqrt(V2))
            self.state.update(dt=st["dt"], alpha=st["alpha"], npos=st["npos"])
            own = self.own
            self.v[:, own] = a * self.v[:, own] + b * self.F[:, own]
        return types.SimpleNamespace(fire_status=self.state["status"], iterations=self.state["iter"])

    def planes(self):
        pack = lambda idx: np.concatenate([self.q[:, idx], self.v[:, idx], self.F[:, idx]])
        return pack(self.lo), pack(self.hi)

    def set_halos(self, below, above):
        for idx, pl in ((self.below, below), (self.above, above)):
            if idx is not None and pl is not None:
                self.q[:, idx], self.v[:, idx], self.F[:, idx] = pl[0:5], pl[5:10], pl[10:15]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, name, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_1911_07045_b300 import sharded as sh
    dist.init_process_group("gloo")
    c = CASES[name]
    o = oracle.Oracle(c["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, 0.5, 0.3,
                      periodic=c["periodic"], objects=c["objects"])
    q0 = synth.random_uniaxial_q(c["shape"], 31)
    z_lo, z_hi = sh.slab_bounds(c["shape"][2], world, rank)
    slab = OracleSlab(o, c["shape"], z_lo, z_hi, q0, bool(c["periodic"][2]))
    comm = sh.TorchComm(periodic_z=bool(c["periodic"][2]))
    res = sh.run_ranks(slab, comm, FP, STEPS)
    out.put((rank, slab.own, slab.q[:, slab.own], slab.v[:, slab.own], slab.F[:, slab.own],
             dict(slab.state), res.iterations))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_gloo_ranks_match_the_whole_lattice(oracle_mod, name, world):
    c = CASES[name]
    o = oracle_mod.Oracle(c["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, 0.5, 0.3,
                          periodic=c["periodic"], objects=c["objects"])
    q0 = synth.random_uniaxial_q(c["shape"], 31)
    qo, vo, Fo, st = o.fire(q0, FP, STEPS)
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sim = o.simulated()
    seen = np.zeros(o.N, dtype=bool)
    for rank, own, qs, vs, Fs, state, iters in got:
        assert iters == st["iter"] == STEPS
        assert state["npos"] == st["npos"]
        assert abs(state["dt"] - st["dt"]) <= 1e-14 * st["dt"]
        assert abs(state["alpha"] - st["alpha"]) <= 1e-14 * st["alpha"]
        m = sim[own]
        for x, y in ((qs, qo[:, own]), (vs, vo[:, own]), (Fs, Fo[:, own])):
            scale = max(np.abs(y[:, m]).max(), 1e-300)
            assert np.abs(x[:, m] - y[:, m]).max() <= 1e-11 * scale
        seen[own] = True
    assert seen.all()
