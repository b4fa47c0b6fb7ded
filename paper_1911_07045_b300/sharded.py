"""One lattice decomposed into z slabs over several processes, one GPU each.

Section III.B splits the lattice into sub-domains with halos; FIRE's power
and norms (Algorithm 1) are then sums over every sub-domain.  Here the
sub-domains are slabs of z planes (``lq_slab_*`` in the C interface): per
FIRE iteration every slab runs the fused step over its own planes and leaves
its sums (P, |F|^2, |v|^2, largest site |F|^2); the sums are combined in FP64
(three sums and a maximum), every slab applies the same FIRE scalar update,
and each slab's first and last own planes of q, v, F go to its neighbours'
halo planes, staged through host buffers.

The orchestration here only routes data: ``run_ranks`` drives one slab per
process over a ``torch.distributed`` group (NCCL between GPUs, gloo between
CPU processes), ``run_local`` several slabs in one process.  A slab is any
object with the methods of ``CudaSlab`` (start, step, finish, planes,
set_halos), so the same routing drives the CUDA slabs and, in the tests, a
plain CPU restatement of the step.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import lqmin


def slab_bounds(nz: int, world: int, rank: int):
    """Planes [z_lo, z_hi) of slab ``rank`` of ``world`` near-equal
    contiguous slabs of nz planes."""
    if not 0 < world <= nz or not 0 <= rank < world:
        raise ValueError(f"cannot cut {nz} planes into {world} slabs (rank {rank})")
    base, extra = divmod(nz, world)
    z_lo = rank * base + min(rank, extra)
    return z_lo, z_lo + base + (1 if rank < extra else 0)


def slab_field(field: np.ndarray, shape, z_lo: int, z_hi: int, periodic_z: bool) -> np.ndarray:
    """The planes of slab [z_lo, z_hi) of a whole-lattice field of shape
    (components, N): one halo plane below, the own planes, one halo plane
    above -- taken with the lattice's periodicity, zero beyond an open z
    edge; returned as (components, nx*ny*(z_hi - z_lo + 2))."""
    nx, ny, nz = shape
    f = np.asarray(field).reshape(field.shape[0], nz, ny * nx)
    planes = []
    for Z in range(z_lo - 1, z_hi + 1):
        if 0 <= Z < nz:
            planes.append(f[:, Z])
        elif periodic_z:
            planes.append(f[:, Z % nz])
        else:
            planes.append(np.zeros_like(f[:, 0]))
    return np.stack(planes, axis=1).reshape(field.shape[0], -1)


def combine(locals_) -> np.ndarray:
    """FP64 totals of the slabs' (P, |F|^2, |v|^2, largest site |F|^2):
    sums of the first three, maximum of the fourth."""
    a = np.asarray(locals_, dtype=np.float64).reshape(-1, 4)
    return np.array([a[:, 0].sum(), a[:, 1].sum(), a[:, 2].sum(), a[:, 3].max()])


def neighbour_planes(planes, periodic_z: bool):
    """Halo routing: ``planes[r] = (lower_own, upper_own)`` of slab r, slabs
    ordered along z; returns for every slab (below, above) -- the upper own
    plane of the slab beneath and the lower own plane of the slab above,
    wrapping around in a periodic lattice, None beyond an open edge."""
    n = len(planes)
    out = []
    for r in range(n):
        below = planes[r - 1][1] if (r > 0 or periodic_z) else None
        above = planes[(r + 1) % n][0] if (r < n - 1 or periodic_z) else None
        out.append((below, above))
    return out


class CudaSlab:
    """Planes [z_lo, z_hi) of a whole-lattice ``lqmin.Solver`` as a slab on
    the current device (lq_slab_create); ``whole`` supplies the geometry."""

    def __init__(self, whole: "lqmin.Solver", z_lo: int, z_hi: int):
        self.lib = lqmin.load()
        self.whole_shape = whole.shape
        self.z_lo, self.z_hi = z_lo, z_hi
        h = C.c_void_p()
        st = self.lib.lq_slab_create(whole.h, int(z_lo), int(z_hi), C.byref(h))
        if st != lqmin.LQ_OK:
            raise lqmin.LqError(st, self.lib.lq_last_error(whole.h).decode())
        self.h = h
        nx, ny, _ = whole.shape
        self.shape = (nx, ny, z_hi - z_lo + 2)
        self.N = nx * ny * (z_hi - z_lo + 2)
        n = C.c_size_t()
        self._ck(self.lib.lq_slab_plane_bytes(self.h, C.byref(n)))
        self.plane_bytes = n.value

    def _ck(self, st):
        if st != lqmin.LQ_OK:
            raise lqmin.LqError(st, self.lib.lq_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.lib.lq_destroy(self.h)
            self.h = None

    def set_q(self, q_slab: np.ndarray):
        """Q of every plane of the slab, halos included (see ``slab_field``)."""
        q = np.ascontiguousarray(q_slab, dtype=np.float64).reshape(5, self.N)
        self._ck(self.lib.lq_set_q(self.h, lqmin._ptr(q)))

    def own_q(self) -> np.ndarray:
        """Q of the own planes, (5, nx*ny*(z_hi - z_lo))."""
        out = np.empty((5, self.N))
        self._ck(self.lib.lq_get_q(self.h, lqmin._ptr(out)))
        nxy = self.shape[0] * self.shape[1]
        return out[:, nxy:self.N - nxy]

    def start(self, params: "lqmin.FireParams") -> np.ndarray:
        local = np.zeros(4)
        self._ck(self.lib.lq_slab_start(self.h, C.byref(params), lqmin._ptr(local)))
        return local

    def step(self) -> np.ndarray:
        local = np.zeros(4)
        self._ck(self.lib.lq_slab_step(self.h, lqmin._ptr(local)))
        return local

    def finish(self, total: np.ndarray) -> "lqmin.Result":
        t = np.ascontiguousarray(total, dtype=np.float64)
        r = lqmin.Result()
        self._ck(self.lib.lq_slab_finish(self.h, lqmin._ptr(t), C.byref(r)))
        return r

    def planes(self):
        """(lower own plane, upper own plane) of q, v, F as host bytes."""
        lo = np.empty(self.plane_bytes, dtype=np.uint8)
        hi = np.empty(self.plane_bytes, dtype=np.uint8)
        self._ck(self.lib.lq_slab_get_planes(self.h, lqmin._ptr(lo), lqmin._ptr(hi)))
        return lo, hi

    def set_halos(self, below, above):
        b = None if below is None else np.ascontiguousarray(below, dtype=np.uint8)
        a = None if above is None else np.ascontiguousarray(above, dtype=np.uint8)
        self._ck(self.lib.lq_slab_set_halos(self.h, None if b is None else lqmin._ptr(b),
                                            None if a is None else lqmin._ptr(a)))


def _one_iteration_local(slabs, periodic_z, local):
    total = combine(local)
    res = [s.finish(total) for s in slabs]
    routes = neighbour_planes([s.planes() for s in slabs], periodic_z)
    for s, (below, above) in zip(slabs, routes):
        s.set_halos(below, above)
    return res[0]


def run_local(slabs, params, steps: int, periodic_z: bool):
    """Start FIRE and run up to ``steps`` iterations on several slabs in one
    process (ordered along z); returns the FIRE state after the last one
    (the same on every slab)."""
    res = _one_iteration_local(slabs, periodic_z, [s.start(params) for s in slabs])
    for _ in range(steps):
        if res.fire_status != lqmin.FIRE_RUNNING:
            break
        res = _one_iteration_local(slabs, periodic_z, [s.step() for s in slabs])
    return res


class TorchComm:
    """The two collectives of a decomposed FIRE iteration over a
    ``torch.distributed`` group, one slab per rank in z order: the FP64
    totals of the slabs' sums, and the halo exchange between neighbouring
    ranks (point-to-point, staged through host buffers -- or through
    ``device`` tensors for NCCL)."""

    def __init__(self, periodic_z: bool, device: str = "cpu"):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.periodic_z = periodic_z
        self.device = device

    def total(self, local) -> np.ndarray:
        import torch
        d = self.dist
        s = torch.tensor(np.asarray(local[:3], dtype=np.float64), device=self.device)
        m = torch.tensor(np.asarray(local[3:4], dtype=np.float64), device=self.device)
        d.all_reduce(s, op=d.ReduceOp.SUM)
        d.all_reduce(m, op=d.ReduceOp.MAX)
        return np.concatenate([s.cpu().numpy(), m.cpu().numpy()])

    def exchange(self, lower, upper):
        """Send the own planes to the neighbours; returns (below, above)."""
        import torch
        d, r, w = self.dist, self.rank, self.world
        if w == 1:
            return (upper, lower) if self.periodic_z else (None, None)
        dn = r - 1 if (r > 0 or self.periodic_z) else None
        up = r + 1 if (r < w - 1 or self.periodic_z) else None
        dn = None if dn is None else dn % w
        up = None if up is None else up % w
        t_lo = torch.from_numpy(np.ascontiguousarray(lower)).to(self.device)
        t_hi = torch.from_numpy(np.ascontiguousarray(upper)).to(self.device)
        # every slab's planes have the same size and type
        below = torch.empty_like(t_lo) if dn is not None else None
        above = torch.empty_like(t_hi) if up is not None else None
        # my upper plane is the halo below the rank above me, my lower plane
        # the halo above the rank below.  Sends first (upper, then lower),
        # receives in the matching order (below, then above): with two
        # periodic ranks both planes travel between the same pair, and a
        # backend that matches messages in order (NCCL ignores tags) pairs
        # them right; tags name the direction where the backend uses them
        ops = []
        if up is not None:
            ops.append(d.P2POp(d.isend, t_hi, up, tag=1))
        if dn is not None:
            ops.append(d.P2POp(d.isend, t_lo, dn, tag=2))
        if dn is not None:
            ops.append(d.P2POp(d.irecv, below, dn, tag=1))
        if up is not None:
            ops.append(d.P2POp(d.irecv, above, up, tag=2))
        if ops:
            for q in d.batch_isend_irecv(ops):
                q.wait()
        return (None if below is None else below.cpu().numpy(),
                None if above is None else above.cpu().numpy())


def run_ranks(slab, comm: TorchComm, params, steps: int):
    """Start FIRE and run up to ``steps`` iterations of this rank's slab of
    the decomposed lattice (every rank calls it); returns the FIRE state
    after the last iteration (the same on every rank)."""
    def finish_and_exchange(local):
        res = slab.finish(comm.total(local))
        lo, hi = slab.planes()
        slab.set_halos(*comm.exchange(lo, hi))
        return res

    res = finish_and_exchange(slab.start(params))
    for _ in range(steps):
        if res.fire_status != lqmin.FIRE_RUNNING:
            break
        res = finish_and_exchange(slab.step())
    return res
