"""Thin ctypes binding of the C interface in ``include/lqmin.h``.

Only argument marshalling lives here: every step of the force + FIRE path
runs in the CUDA kernels of ``liblqmin.so``.  There is no CPU fallback: if
the library has not been built, or no CUDA device is present, the first call
raises.

The ``lq_*`` functions mirror the C calls one to one (same names, numpy
arrays for host buffers, ints for device pointers and streams).  ``Solver``
is a small convenience wrapper that owns one ``lq_solver`` handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblqmin.so")

LQ_OK, LQ_EINVAL, LQ_ENOMEM, LQ_ECUDA, LQ_ENOTCONVERGED, LQ_ETIMEOUT, LQ_EDIVERGED, LQ_EBUSY = range(8)
STATUS_NAMES = ["LQ_OK", "LQ_EINVAL", "LQ_ENOMEM", "LQ_ECUDA", "LQ_ENOTCONVERGED", "LQ_ETIMEOUT",
                "LQ_EDIVERGED", "LQ_EBUSY"]
LQ_FP64, LQ_FP32_BULK_FP64_RED = 0, 1
ND_HOMEOTROPIC, ND_ORIENTED, FG_PLANAR = 0, 1, 2
FIRE_RUNNING, FIRE_CONVERGED, FIRE_MAXITER, FIRE_DIVERGED, FIRE_STALLED = 0, 1, 2, 3, 4
LQ_MIN_FIRE, LQ_MIN_GD, LQ_MIN_NESTEROV = 0, 1, 2

# every symbol include/lqmin.h declares
EXPORTS = [
    "lq_create", "lq_destroy", "lq_last_error", "lq_create_error", "lq_add_wall", "lq_add_sphere",
    "lq_add_droplet", "lq_add_spherocylinder",
    "lq_add_object_sites", "lq_add_anchored_sites", "lq_geometry_info", "lq_get_mask", "lq_set_q",
    "lq_set_q_device", "lq_init_random_uniaxial", "lq_get_q", "lq_get_velocity", "lq_get_force",
    "lq_force", "lq_energy", "lq_order_field", "lq_fire_reset", "lq_step", "lq_minimize",
    "lq_fire_result", "lq_get_state", "lq_set_state", "lq_set_zchunk", "lq_device_bytes",
    "lq_energy_noalloc", "lq_batch_create", "lq_batch_destroy", "lq_batch_last_error",
    "lq_batch_set_tiling", "lq_batch_get_tiling", "lq_batch_set_tile", "lq_batch_get_tile",
    "lq_batch_autotune", "lq_batch_step",
    "lq_batch_minimize", "lq_server_create", "lq_server_destroy", "lq_server_submit",
    "lq_server_poll", "lq_server_wait", "lq_server_stats_get", "lq_boundary_check",
    "lq_add_boundary_text", "lq_load_boundary_file", "lq_object_count", "lq_move_object",
    "lq_clear_objects", "lq_set_material", "lq_clone", "lq_pmf_sweep", "lq_init_dipolar",
    "lq_frank_to_landau", "lq_set_index_width", "lq_inject_fault", "lq_bounds_check_hits",
    "lq_fp64_fma_rate", "lq_set_staging", "lq_get_staging",
    "lq_slab_create", "lq_slab_start", "lq_slab_step", "lq_slab_finish", "lq_slab_plane_bytes",
    "lq_slab_get_planes", "lq_slab_set_halos",
]


class LqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Lattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("spacing", C.c_double),
                ("periodic", C.c_int * 3)]


class Material(C.Structure):
    _fields_ = [("A", C.c_double), ("B", C.c_double), ("C", C.c_double), ("L1", C.c_double),
                ("L2", C.c_double), ("L3", C.c_double), ("L4", C.c_double), ("L6", C.c_double),
                ("n_constants", C.c_int), ("S0", C.c_double),
                ("H", C.c_double * 3), ("mu0_dchi", C.c_double),
                ("E", C.c_double * 3), ("eps0_deps", C.c_double)]


class Anchoring(C.Structure):
    _fields_ = [("kind", C.c_int), ("W", C.c_double), ("dir", C.c_double * 3)]


class FireParams(C.Structure):
    _fields_ = [("dt0", C.c_double), ("dt_max", C.c_double), ("alpha0", C.c_double),
                ("f_alpha", C.c_double), ("f_inc", C.c_double), ("f_dec", C.c_double),
                ("n_min", C.c_int), ("max_iter", C.c_int64), ("force_tol", C.c_double),
                ("wall_timeout_s", C.c_double), ("method", C.c_int), ("momentum", C.c_double)]


class Result(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("max_force", C.c_double), ("rms_force", C.c_double),
                ("norm_force", C.c_double), ("norm_velocity", C.c_double), ("power", C.c_double),
                ("dt", C.c_double), ("alpha", C.c_double), ("npos", C.c_int64),
                ("energy", C.c_double), ("fire_status", C.c_int), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Object(C.Structure):
    _fields_ = [("type", C.c_int), ("axis", C.c_int), ("plane", C.c_int), ("c", C.c_double * 3),
                ("R", C.c_double), ("anch", Anchoring), ("n", C.c_int64),
                ("xyz", C.c_void_p), ("per_site", C.c_void_p), ("c2", C.c_double * 3)]


class Request(C.Structure):
    _fields_ = [("lattice", Lattice), ("material", Material), ("n_objects", C.c_int),
                ("objects", C.c_void_p), ("q0", C.c_void_p), ("seed", C.c_uint64), ("S", C.c_double),
                ("params", FireParams), ("want_order_field", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int64), ("active", C.c_int64), ("completed", C.c_int64),
                ("bytes_in_use", C.c_size_t), ("budget", C.c_size_t), ("site_updates", C.c_double),
                ("site_updates_issued", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load ``liblqmin.so``; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1911_07045_b300.build` (nvcc, sm_103a)")
    lib = C.CDLL(path)
    p, i64, d = C.c_void_p, C.c_int64, C.c_double
    S = p  # lq_solver*
    sig = {
        "lq_create": (C.c_int, [C.POINTER(Lattice), C.POINTER(Material), C.c_int, p, C.POINTER(p)]),
        "lq_destroy": (None, [S]),
        "lq_last_error": (C.c_char_p, [S]),
        "lq_create_error": (C.c_char_p, []),
        "lq_add_wall": (C.c_int, [S, C.c_int, C.c_int, C.POINTER(Anchoring)]),
        "lq_add_sphere": (C.c_int, [S, C.POINTER(C.c_double), d, C.POINTER(Anchoring)]),
        "lq_add_droplet": (C.c_int, [S, C.POINTER(C.c_double), d, C.POINTER(Anchoring)]),
        "lq_add_spherocylinder": (C.c_int, [S, C.POINTER(C.c_double), C.POINTER(C.c_double), d,
                                            C.POINTER(Anchoring)]),
        "lq_add_object_sites": (C.c_int, [S, i64, p, C.POINTER(Anchoring)]),
        "lq_add_anchored_sites": (C.c_int, [S, i64, p, p]),
        "lq_geometry_info": (C.c_int, [S, C.POINTER(i64), C.POINTER(i64)]),
        "lq_get_mask": (C.c_int, [S, p]),
        "lq_set_q": (C.c_int, [S, p]),
        "lq_set_q_device": (C.c_int, [S, p, C.c_int]),
        "lq_init_random_uniaxial": (C.c_int, [S, C.c_uint64, d]),
        "lq_get_q": (C.c_int, [S, p]),
        "lq_get_velocity": (C.c_int, [S, p]),
        "lq_get_force": (C.c_int, [S, p]),
        "lq_force": (C.c_int, [S, p]),
        "lq_energy": (C.c_int, [S, C.POINTER(d), p]),
        "lq_order_field": (C.c_int, [S, p]),
        "lq_fire_reset": (C.c_int, [S, C.POINTER(FireParams)]),
        "lq_step": (C.c_int, [S, C.POINTER(FireParams), i64, C.POINTER(Result)]),
        "lq_minimize": (C.c_int, [S, C.POINTER(FireParams), C.POINTER(Result)]),
        "lq_fire_result": (C.c_int, [S, C.POINTER(Result)]),
        "lq_get_state": (C.c_int, [S, p, C.POINTER(C.c_size_t)]),
        "lq_set_state": (C.c_int, [S, p, C.c_size_t]),
        "lq_set_zchunk": (C.c_int, [S, C.c_int]),
        "lq_device_bytes": (C.c_size_t, [S]),
        "lq_energy_noalloc": (C.c_int, [C.POINTER(Lattice), C.POINTER(Material), p, p, p, p]),
        "lq_batch_create": (C.c_int, [p, C.c_int, C.POINTER(p)]),
        "lq_batch_destroy": (None, [p]),
        "lq_batch_last_error": (C.c_char_p, [p]),
        "lq_batch_set_tiling": (C.c_int, [p, C.c_int, C.c_int]),
        "lq_batch_get_tiling": (C.c_int, [p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "lq_batch_set_tile": (C.c_int, [p, C.c_int, C.c_int, C.c_int]),
        "lq_batch_get_tile": (C.c_int, [p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "lq_batch_autotune": (C.c_int, [p, C.POINTER(FireParams), C.c_int, C.POINTER(d)]),
        "lq_batch_step": (C.c_int, [p, C.POINTER(FireParams), i64, p]),
        "lq_batch_minimize": (C.c_int, [p, C.POINTER(FireParams), p]),
        "lq_server_create": (C.c_int, [C.c_size_t, C.c_int, C.c_int, C.POINTER(p)]),
        "lq_server_destroy": (None, [p]),
        "lq_server_submit": (C.c_int, [p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "lq_server_poll": (C.c_int, [p, C.c_uint64, C.POINTER(Result), p]),
        "lq_server_wait": (C.c_int, [p, C.c_uint64, d, C.POINTER(Result), p]),
        "lq_server_stats_get": (C.c_int, [p, C.POINTER(ServerStats)]),
        "lq_boundary_check": (C.c_int, [C.c_char_p, C.POINTER(i64), C.POINTER(i64), C.c_char_p,
                                        C.c_size_t]),
        "lq_add_boundary_text": (C.c_int, [S, C.c_char_p]),
        "lq_load_boundary_file": (C.c_int, [S, C.c_char_p]),
        "lq_object_count": (C.c_int, [S, C.POINTER(C.c_int)]),
        "lq_move_object": (C.c_int, [S, C.c_int, C.POINTER(C.c_double)]),
        "lq_clear_objects": (C.c_int, [S]),
        "lq_set_material": (C.c_int, [S, C.POINTER(Material)]),
        "lq_clone": (C.c_int, [S, p, C.POINTER(p)]),
        "lq_pmf_sweep": (C.c_int, [S, C.c_int, C.c_int, p, C.POINTER(FireParams), p]),
        "lq_init_dipolar": (C.c_int, [S, C.POINTER(C.c_double), C.POINTER(C.c_double), d, d]),
        "lq_frank_to_landau": (C.c_int, [d, d, d, d, d, d, C.POINTER(C.c_double)]),
        "lq_set_index_width": (C.c_int, [S, C.c_int]),
        "lq_inject_fault": (C.c_int, [C.c_int, i64]),
        "lq_bounds_check_hits": (C.c_int, [C.POINTER(C.c_uint32)]),
        "lq_fp64_fma_rate": (C.c_int, [i64, C.POINTER(d)]),
        "lq_set_staging": (C.c_int, [S, C.c_int]),
        "lq_get_staging": (C.c_int, [S, C.POINTER(C.c_int)]),
        "lq_slab_create": (C.c_int, [S, C.c_int, C.c_int, C.POINTER(p)]),
        "lq_slab_start": (C.c_int, [S, C.POINTER(FireParams), p]),
        "lq_slab_step": (C.c_int, [S, p]),
        "lq_slab_finish": (C.c_int, [S, p, C.POINTER(Result)]),
        "lq_slab_plane_bytes": (C.c_int, [S, C.POINTER(C.c_size_t)]),
        "lq_slab_get_planes": (C.c_int, [S, p, p]),
        "lq_slab_set_halos": (C.c_int, [S, p, p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def fire_params(dt0=1e-3, dt_max=1e-2, alpha0=0.99, f_alpha=0.99, f_inc=1.1, f_dec=0.5, n_min=5,
                max_iter=10 ** 9, force_tol=1e-9, wall_timeout_s=0.0, method=0,
                momentum=0.0) -> FireParams:
    """Minimiser parameters (lq_fire_params): FIRE by default; method
    LQ_MIN_GD / LQ_MIN_NESTEROV take dt0 as the step and momentum as mu."""
    return FireParams(dt0, dt_max, alpha0, f_alpha, f_inc, f_dec, n_min, max_iter, force_tol,
                      wall_timeout_s, int(method), float(momentum))


def descent_params(method, step, momentum=0.0, max_iter=10 ** 9, force_tol=1e-9,
                   wall_timeout_s=0.0) -> FireParams:
    """Gradient descent (LQ_MIN_GD) or Nesterov (LQ_MIN_NESTEROV) with step eta."""
    return fire_params(dt0=step, dt_max=step, max_iter=max_iter, force_tol=force_tol,
                       wall_timeout_s=wall_timeout_s, method=method, momentum=momentum)


def material(A, B, C_, L1, L2=0.0, L3=0.0, n_constants=None, S0=0.0, L4=0.0, L6=0.0,
             H=(0.0, 0.0, 0.0), mu0_dchi=0.0, E=(0.0, 0.0, 0.0), eps0_deps=0.0) -> Material:
    """lq_material; n_constants None picks 1 when L2..L6 are all zero."""
    if n_constants is None:
        n_constants = 1 if (L2 == 0.0 and L3 == 0.0 and L4 == 0.0 and L6 == 0.0) else 3
    return Material(A, B, C_, L1, L2, L3, L4, L6, n_constants, S0,
                    (C.c_double * 3)(*[float(v) for v in H]), float(mu0_dchi),
                    (C.c_double * 3)(*[float(v) for v in E]), float(eps0_deps))


def frank_to_landau(K1, K2, K3, K24, q0, S):
    """Distortion constants L1, L2, L3, L4, L6 from Frank constants (see
    ``lq_frank_to_landau``), as a dict of keyword arguments for Solver."""
    out = (C.c_double * 5)()
    st = load().lq_frank_to_landau(K1, K2, K3, K24, q0, S, out)
    if st != LQ_OK:
        raise LqError(st, "lq_frank_to_landau: S must be positive and inputs finite")
    return dict(zip(("L1", "L2", "L3", "L4", "L6"), list(out)))


LQ_FAULT_NONE, LQ_FAULT_DEVICE_ALLOC, LQ_FAULT_STEP_LAUNCH, LQ_FAULT_COPY_WAIT = 0, 1, 2, 3


def fp64_fma_rate(iters: int = 1 << 16) -> float:
    """Measured FP64 fused multiply-adds per second of the current device
    (lq_fp64_fma_rate): the ceiling of the FP64 form of the step."""
    lib = load()
    out = C.c_double()
    st = lib.lq_fp64_fma_rate(int(iters), C.byref(out))
    if st != LQ_OK:
        raise LqError(st, "lq_fp64_fma_rate")
    return out.value


def inject_fault(kind, after=0):
    """Host-side fault injection for tests (see ``lq_inject_fault``)."""
    st = load().lq_inject_fault(int(kind), int(after))
    if st != LQ_OK:
        raise LqError(st, "lq_inject_fault")


def boundary_check(text):
    """Parse boundary text (see ``lq_add_boundary_text``) without a solver:
    (number of blocks, number of site lines); raises LqError with the
    message naming the line."""
    lib = load()
    nb, ns = C.c_int64(), C.c_int64()
    err = C.create_string_buffer(256)
    st = lib.lq_boundary_check(text.encode(), C.byref(nb), C.byref(ns), err, len(err))
    if st != LQ_OK:
        raise LqError(st, err.value.decode())
    return nb.value, ns.value


def anchoring(kind, W, dir=(0.0, 0.0, 1.0)) -> Anchoring:
    return Anchoring(int(kind), float(W), (C.c_double * 3)(*[float(v) for v in dir]))


# lq_anchoring as a numpy record (int kind, 4 bytes of padding, double W,
# double dir[3]: 40 bytes), for per-site arrays marshalled without a Python loop
_ANCHOR_DTYPE = np.dtype([("kind", "<i4"), ("pad", "<i4"), ("W", "<f8"), ("dir", "<f8", (3,))])
assert _ANCHOR_DTYPE.itemsize == C.sizeof(Anchoring)


def anchoring_array(n, kinds, W, dirs) -> np.ndarray:
    """n lq_anchoring records in one contiguous array (kinds, W, dirs
    broadcast to n sites)."""
    arr = np.zeros(max(1, n), dtype=_ANCHOR_DTYPE)
    arr["kind"][:n] = np.broadcast_to(np.asarray(kinds), (n,))
    arr["W"][:n] = np.broadcast_to(np.asarray(W, dtype=float), (n,))
    arr["dir"][:n] = np.broadcast_to(np.asarray(dirs, dtype=float), (n, 3))
    return arr


class Solver:
    """One lattice on the current CUDA device (see ``lq_create``)."""

    def __init__(self, shape, A, B, C_, L1, L2=0.0, L3=0.0, periodic=(1, 1, 1), precision=LQ_FP64,
                 stream=None, n_constants=None, S0=0.0, L4=0.0, L6=0.0, H=(0.0, 0.0, 0.0),
                 mu0_dchi=0.0, E=(0.0, 0.0, 0.0), eps0_deps=0.0):
        lib = load()
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        lat = Lattice(nx, ny, nz, 1.0, (C.c_int * 3)(*[int(bool(p)) for p in periodic]))
        mat = material(A, B, C_, L1, L2, L3, n_constants, S0, L4, L6, H, mu0_dchi, E, eps0_deps)
        h = C.c_void_p()
        st = lib.lq_create(C.byref(lat), C.byref(mat), int(precision),
                           C.c_void_p(stream) if stream else None, C.byref(h))
        if st != LQ_OK:
            raise LqError(st, lib.lq_create_error().decode())
        self.h = h
        self.lib = lib
        self.precision = precision

    @classmethod
    def _wrap(cls, lib, h, shape, precision):
        self = cls.__new__(cls)
        self.lib, self.h, self.shape, self.precision = lib, h, tuple(shape), precision
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        return self

    def clone(self, stream=None):
        """A new solver with this one's lattice, material, objects and Q."""
        h = C.c_void_p()
        self._ck(self.lib.lq_clone(self.h, C.c_void_p(stream) if stream else None, C.byref(h)))
        return Solver._wrap(self.lib, h, self.shape, self.precision)

    def set_material(self, A, B, C_, L1, L2=0.0, L3=0.0, n_constants=None, S0=0.0, L4=0.0, L6=0.0,
                     H=(0.0, 0.0, 0.0), mu0_dchi=0.0, E=(0.0, 0.0, 0.0), eps0_deps=0.0):
        mat = material(A, B, C_, L1, L2, L3, n_constants, S0, L4, L6, H, mu0_dchi, E, eps0_deps)
        self._ck(self.lib.lq_set_material(self.h, C.byref(mat)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.lq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st, ok=(LQ_OK,)):
        if st not in ok:
            raise LqError(st, self.lib.lq_last_error(self.h).decode())
        return st

    # ---- geometry --------------------------------------------------------
    def add_wall(self, axis, plane, kind=ND_HOMEOTROPIC, W=0.0, dir=(0, 0, 1)):
        a = anchoring(kind, W, dir)
        self._ck(self.lib.lq_add_wall(self.h, int(axis), int(plane), C.byref(a)))

    def add_sphere(self, c, R, kind=ND_HOMEOTROPIC, W=0.0, dir=(0, 0, 1)):
        a = anchoring(kind, W, dir)
        cc = (C.c_double * 3)(*[float(v) for v in c])
        self._ck(self.lib.lq_add_sphere(self.h, cc, float(R), C.byref(a)))

    def add_droplet(self, c, R, kind=ND_HOMEOTROPIC, W=0.0, dir=(0, 0, 1)):
        a = anchoring(kind, W, dir)
        cc = (C.c_double * 3)(*[float(v) for v in c])
        self._ck(self.lib.lq_add_droplet(self.h, cc, float(R), C.byref(a)))

    def add_spherocylinder(self, p0, p1, R, kind=ND_HOMEOTROPIC, W=0.0, dir=(0, 0, 1)):
        a = anchoring(kind, W, dir)
        c0 = (C.c_double * 3)(*[float(v) for v in p0])
        c1 = (C.c_double * 3)(*[float(v) for v in p1])
        self._ck(self.lib.lq_add_spherocylinder(self.h, c0, c1, float(R), C.byref(a)))

    def add_object_sites(self, xyz, kind=ND_HOMEOTROPIC, W=0.0, dir=(0, 0, 1)):
        xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        a = anchoring(kind, W, dir)
        self._ck(self.lib.lq_add_object_sites(self.h, xyz.shape[0], _ptr(xyz), C.byref(a)))

    def add_anchored_sites(self, xyz, kinds, W, dirs):
        xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        n = xyz.shape[0]
        arr = anchoring_array(n, kinds, W, dirs)
        self._ck(self.lib.lq_add_anchored_sites(self.h, n, _ptr(xyz), _ptr(arr)))

    def add_objects(self, objects):
        """Objects in the dict format of ``synth`` (same as the oracle's)."""
        for o in objects:
            t = o["type"]
            if t == "wall":
                k, W, d = o.get("anchor", (ND_HOMEOTROPIC, 0.0, (0, 0, 1)))
                self.add_wall(o["axis"], o["plane"], k, W, d)
            elif t == "sphere":
                k, W, d = o.get("anchor", (ND_HOMEOTROPIC, 0.0, (0, 0, 1)))
                self.add_sphere(o["c"], o["R"], k, W, d)
            elif t == "droplet":
                k, W, d = o.get("anchor", (ND_HOMEOTROPIC, 0.0, (0, 0, 1)))
                self.add_droplet(o["c"], o["R"], k, W, d)
            elif t == "spherocylinder":
                k, W, d = o.get("anchor", (ND_HOMEOTROPIC, 0.0, (0, 0, 1)))
                self.add_spherocylinder(o["c"], o["c2"], o["R"], k, W, d)
            elif t == "sites":
                k, W, d = o.get("anchor", (ND_HOMEOTROPIC, 0.0, (0, 0, 1)))
                self.add_object_sites(o["xyz"], k, W, d)
            elif t == "anchored":
                self.add_anchored_sites(o["xyz"], o["kinds"], o["W"], o["dirs"])
            else:
                raise ValueError(t)

    def add_boundary_text(self, text):
        self._ck(self.lib.lq_add_boundary_text(self.h, text.encode()))

    def load_boundary_file(self, path):
        self._ck(self.lib.lq_load_boundary_file(self.h, os.fsencode(path)))

    def object_count(self):
        n = C.c_int()
        self._ck(self.lib.lq_object_count(self.h, C.byref(n)))
        return n.value

    def move_object(self, index, shift):
        sh = (C.c_double * 3)(*[float(v) for v in shift])
        self._ck(self.lib.lq_move_object(self.h, int(index), sh))

    def clear_objects(self):
        self._ck(self.lib.lq_clear_objects(self.h))

    def pmf_sweep(self, index, shifts, params: FireParams):
        """Minimise one clone per shift of object ``index`` in one batch;
        returns (status, results) with each result's energy at its minimum."""
        sh = np.ascontiguousarray(shifts, dtype=np.float64).reshape(-1, 3)
        out = (Result * len(sh))()
        st = self._ck(self.lib.lq_pmf_sweep(self.h, int(index), len(sh), _ptr(sh), C.byref(params),
                                            C.cast(out, C.c_void_p)),
                      ok=(LQ_OK, LQ_ENOTCONVERGED, LQ_ETIMEOUT, LQ_EDIVERGED))
        return st, list(out)

    def pmf_scan(self, index, shifts, params: FireParams):
        """Move object ``index`` by each shift in turn (cumulative) and
        re-minimise from the previous minimum; returns the results."""
        out = []
        for sh in np.asarray(shifts, dtype=np.float64).reshape(-1, 3):
            self.move_object(index, sh)
            out.append(self.minimize(params))
        return out

    def init_dipolar(self, c, axis=(0.0, 0.0, 1.0), rd=None, R=None, S=0.0):
        """Dipolar start (see ``lq_init_dipolar``); rd defaults to 1.25 R."""
        if rd is None:
            if R is None:
                raise ValueError("give rd or the colloid radius R")
            rd = 1.25 * float(R)
        cc = (C.c_double * 3)(*[float(v) for v in c])
        aa = (C.c_double * 3)(*[float(v) for v in axis])
        self._ck(self.lib.lq_init_dipolar(self.h, cc, aa, float(rd), float(S)))

    def geometry_info(self):
        a, b = C.c_int64(), C.c_int64()
        self._ck(self.lib.lq_geometry_info(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def mask(self):
        out = np.empty(self.N, dtype=np.uint8)
        self._ck(self.lib.lq_get_mask(self.h, _ptr(out)))
        return out

    # ---- state -----------------------------------------------------------
    def set_q(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(5, self.N)
        self._ck(self.lib.lq_set_q(self.h, _ptr(q)))

    def set_q_device(self, ptr: int, dtype: int):
        self._ck(self.lib.lq_set_q_device(self.h, C.c_void_p(ptr), int(dtype)))

    def init_random_uniaxial(self, seed, S=0.0):
        self._ck(self.lib.lq_init_random_uniaxial(self.h, C.c_uint64(seed), float(S)))

    def _get5(self, fn):
        out = np.empty((5, self.N))
        self._ck(fn(self.h, _ptr(out)))
        return out

    def get_q(self):
        return self._get5(self.lib.lq_get_q)

    def get_velocity(self):
        return self._get5(self.lib.lq_get_velocity)

    def get_force(self):
        return self._get5(self.lib.lq_get_force)

    def force(self):
        return self._get5(self.lib.lq_force)

    def energy(self):
        tot = C.c_double()
        parts = np.zeros(3)
        self._ck(self.lib.lq_energy(self.h, C.byref(tot), _ptr(parts)))
        return tot.value, parts

    def order_field(self):
        out = np.empty(self.N)
        self._ck(self.lib.lq_order_field(self.h, _ptr(out)))
        return out

    # ---- FIRE --------------------------------------------------------------
    def fire_reset(self, params: FireParams):
        self._ck(self.lib.lq_fire_reset(self.h, C.byref(params)))

    def step(self, params: FireParams, n: int) -> Result:
        r = Result()
        self._ck(self.lib.lq_step(self.h, C.byref(params), int(n), C.byref(r)))
        return r

    def minimize(self, params: FireParams):
        r = Result()
        st = self._ck(self.lib.lq_minimize(self.h, C.byref(params), C.byref(r)),
                      ok=(LQ_OK, LQ_ENOTCONVERGED, LQ_ETIMEOUT, LQ_EDIVERGED))
        return st, r

    def fire_result(self) -> Result:
        r = Result()
        self._ck(self.lib.lq_fire_result(self.h, C.byref(r)))
        return r

    def get_state(self) -> bytes:
        n = C.c_size_t()
        self._ck(self.lib.lq_get_state(self.h, None, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self._ck(self.lib.lq_get_state(self.h, _ptr(buf), C.byref(n)))
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._ck(self.lib.lq_set_state(self.h, _ptr(buf), buf.size))

    def set_zchunk(self, z):
        self._ck(self.lib.lq_set_zchunk(self.h, int(z)))

    def set_staging(self, mode):
        """0 automatic, 1 per-thread loads, 2 tensor copies (lq_set_staging)."""
        self._ck(self.lib.lq_set_staging(self.h, int(mode)))

    def uses_tensor_copies(self) -> bool:
        out = C.c_int()
        self._ck(self.lib.lq_get_staging(self.h, C.byref(out)))
        return bool(out.value)

    def set_index_width(self, bits):
        self._ck(self.lib.lq_set_index_width(self.h, int(bits)))

    def device_bytes(self):
        return self.lib.lq_device_bytes(self.h)


class Batch:
    """Several solvers advanced by one persistent kernel (see lq_batch_create).
    Keeps references to the solvers; destroy the batch before them."""

    def __init__(self, solvers):
        self.lib = load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        h = C.c_void_p()
        st = self.lib.lq_batch_create(arr, len(self.solvers), C.byref(h))
        if st != LQ_OK:
            raise LqError(st, "lq_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lq_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st, ok=(LQ_OK,)):
        if st not in ok:
            raise LqError(st, self.lib.lq_batch_last_error(self.h).decode())
        return st

    def tiling(self):
        a, b = C.c_int(), C.c_int()
        self._ck(self.lib.lq_batch_get_tiling(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_tiling(self, tile_y, zchunk):
        self._ck(self.lib.lq_batch_set_tiling(self.h, int(tile_y), int(zchunk)))

    def tile(self):
        """(tile width, tile height, z chunk) of the current tiling."""
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._ck(self.lib.lq_batch_get_tile(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def set_tile(self, tile_x, tile_y, zchunk):
        self._ck(self.lib.lq_batch_set_tile(self.h, int(tile_x), int(tile_y), int(zchunk)))

    def autotune(self, params: FireParams, launches=12):
        """Time every tiling (lq_batch_autotune); returns ((tile width,
        tile height, z chunk), milliseconds per launch of the fastest)."""
        ms = C.c_double()
        self._ck(self.lib.lq_batch_autotune(self.h, C.byref(params), int(launches), C.byref(ms)))
        return self.tile(), ms.value

    def step(self, params: FireParams, n: int):
        out = (Result * len(self.solvers))()
        self._ck(self.lib.lq_batch_step(self.h, C.byref(params), int(n), C.cast(out, C.c_void_p)))
        return list(out)

    def minimize(self, params: FireParams):
        out = (Result * len(self.solvers))()
        st = self._ck(self.lib.lq_batch_minimize(self.h, C.byref(params), C.cast(out, C.c_void_p)),
                      ok=(LQ_OK, LQ_ENOTCONVERGED, LQ_ETIMEOUT, LQ_EDIVERGED))
        return st, list(out)


OBJ_TYPES = {"wall": 0, "sphere": 1, "sites": 2, "anchored": 3, "droplet": 4,
             "spherocylinder": 5}


class Server:
    """Continuous-batching server (see lq_server_create) on the current device."""

    def __init__(self, hbm_budget_bytes, precision=LQ_FP32_BULK_FP64_RED, max_active=64):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.lq_server_create(int(hbm_budget_bytes), int(precision), int(max_active),
                                       C.byref(h))
        if st != LQ_OK:
            raise LqError(st, "lq_server_create")
        self.h = h
        self.sizes = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.lq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, cfg, params: FireParams, seed=0, q0=None, want_S=False, S=0.0,
               A=None, B=None, C_=None, periodic=(1, 1, 1)):
        """Queue the workload dict ``cfg`` (synth format); returns a ticket."""
        from . import synth
        nx, ny, nz = cfg["shape"]
        L2, L3 = cfg.get("L2", 0.0), cfg.get("L3", 0.0)
        mat = Material(synth.A_5CB if A is None else A, synth.B_5CB if B is None else B,
                       synth.C_5CB if C_ is None else C_, cfg["L1"], L2, L3, 0.0, 0.0,
                       1 if (L2 == 0.0 and L3 == 0.0) else 3, 0.0)
        lat = Lattice(nx, ny, nz, 1.0, (C.c_int * 3)(*cfg.get("periodic", periodic)))
        keep = []
        objs = (Object * max(1, len(cfg.get("objects", []))))()
        for o, spec in zip(objs, cfg.get("objects", [])):
            o.type = OBJ_TYPES[spec["type"]]
            if "anchor" in spec:
                o.anch = anchoring(*spec["anchor"])
            if spec["type"] == "wall":
                o.axis, o.plane = spec["axis"], spec["plane"]
            elif spec["type"] in ("sphere", "droplet", "spherocylinder"):
                o.c = (C.c_double * 3)(*spec["c"])
                o.R = spec["R"]
                if spec["type"] == "spherocylinder":
                    o.c2 = (C.c_double * 3)(*spec["c2"])
            else:
                xyz = np.ascontiguousarray(spec["xyz"], dtype=np.int32).reshape(-1, 3)
                keep.append(xyz)
                o.n = xyz.shape[0]
                o.xyz = xyz.ctypes.data
                if spec["type"] == "anchored":
                    per = anchoring_array(xyz.shape[0], spec["kinds"], spec["W"], spec["dirs"])
                    keep.append(per)
                    o.per_site = per.ctypes.data
        rq = Request(lat, mat, len(cfg.get("objects", [])), C.cast(objs, C.c_void_p).value, None,
                     int(seed), float(S), params, int(bool(want_S)))
        if q0 is not None:
            q0 = np.ascontiguousarray(q0, dtype=np.float64)
            keep.append(q0)
            rq.q0 = q0.ctypes.data
        t = C.c_uint64()
        st = self.lib.lq_server_submit(self.h, C.byref(rq), C.byref(t))
        if st != LQ_OK:
            raise LqError(st, "lq_server_submit")
        self.sizes[t.value] = nx * ny * nz
        return t.value

    def _out(self, ticket, S):
        return (np.empty(self.sizes[ticket]) if S else None)

    def poll(self, ticket, S=False):
        """None while busy, else (status, Result, S field or None)."""
        r = Result()
        Sbuf = self._out(ticket, S)
        st = self.lib.lq_server_poll(self.h, int(ticket), C.byref(r),
                                     None if Sbuf is None else Sbuf.ctypes.data)
        if st == LQ_EBUSY:
            return None
        return st, r, Sbuf

    def wait(self, ticket, timeout=0.0, S=False):
        r = Result()
        Sbuf = self._out(ticket, S)
        st = self.lib.lq_server_wait(self.h, int(ticket), float(timeout), C.byref(r),
                                     None if Sbuf is None else Sbuf.ctypes.data)
        if st == LQ_EBUSY:
            return None
        return st, r, Sbuf

    def stats(self):
        out = ServerStats()
        self.lib.lq_server_stats_get(self.h, C.byref(out))
        return out.as_dict()


def solver_for(cfg: dict, precision=LQ_FP64, stream=None, A=None, B=None, C_=None,
               periodic=(1, 1, 1)) -> Solver:
    """Solver for a ``synth`` workload dict (shape, L1/L2/L3, objects)."""
    from . import synth
    s = Solver(cfg["shape"], synth.A_5CB if A is None else A, synth.B_5CB if B is None else B,
               synth.C_5CB if C_ is None else C_, cfg["L1"], cfg.get("L2", 0.0), cfg.get("L3", 0.0),
               periodic=cfg.get("periodic", periodic), precision=precision, stream=stream)
    s.add_objects(cfg.get("objects", []))
    return s
