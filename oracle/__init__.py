"""Plain FP64 CPU oracle for the lattice Landau-de Gennes force and FIRE.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA path.  The arithmetic lives in ``lqoracle.c``
(see its header for the paper passages each routine follows); this module
marshals numpy arrays through ctypes, except for the dipolar initial
condition (``dipolar_director``), written here in numpy.

Every function is pinned by the ``-m "not gpu"`` tests in ``tests/`` against
closed forms, invariants, hand-derived values and finite differences.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lqoracle.c")
_HDR = os.path.join(_HERE, "lqoracle.h")
_LIB = os.path.join(_HERE, "liblqoracle.so")

ND_HOMEOTROPIC, ND_ORIENTED, FG_PLANAR = 0, 1, 2
WALL, SPHERE, SITES, ANCHORED, DROPLET, SPHEROCYLINDER = 0, 1, 2, 3, 4, 5
RUNNING, CONVERGED, MAXITER, DIVERGED = 0, 1, 2, 3


def _host_tag() -> str:
    """CPU model and flags: -march=native code is only reused on the same CPU."""
    model, flags = "", ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name") and not model:
                model = line.split(":", 1)[1].strip()
            if line.startswith("flags") and not flags:
                flags = line.split(":", 1)[1].strip()
    except OSError:
        pass
    import hashlib
    return hashlib.sha1((model + "|" + flags).encode()).hexdigest()


def build(force: bool = False) -> str:
    """Compile ``liblqoracle.so`` with gcc -O3 -march=native + OpenMP; rebuilt
    when the sources change or the host CPU differs from the build host."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    tagfile = _LIB + ".host"
    tag = _host_tag()
    stale = (not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest
             or not os.path.exists(tagfile) or open(tagfile).read().strip() != tag)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O3", "-march=native", "-fopenmp", "-fPIC", "-shared", "-std=c99",
             "-Wall", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
        with open(tagfile, "w") as f:
            f.write(tag + "\n")
    return _LIB


class _Model(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("periodic", C.c_int * 3),
                ("A", C.c_double), ("B", C.c_double), ("C", C.c_double),
                ("L1", C.c_double), ("L2", C.c_double), ("L3", C.c_double),
                ("S0", C.c_double), ("L4", C.c_double), ("L6", C.c_double),
                ("H", C.c_double * 3), ("mu0_dchi", C.c_double),
                ("E", C.c_double * 3), ("eps0_deps", C.c_double)]


class _AnchorSpec(C.Structure):
    _fields_ = [("kind", C.c_int), ("W", C.c_double), ("dir", C.c_double * 3)]


class _Object(C.Structure):
    _fields_ = [("type", C.c_int), ("axis", C.c_int), ("plane", C.c_int),
                ("c", C.c_double * 3), ("R", C.c_double),
                ("n", C.c_int64), ("xyz", C.POINTER(C.c_int32)),
                ("per_site", C.POINTER(_AnchorSpec)),
                ("anch", _AnchorSpec), ("c2", C.c_double * 3)]


class _Anchor(C.Structure):
    _fields_ = [("kind", C.c_int), ("W", C.c_double), ("q0", C.c_double * 5),
                ("nu", C.c_double * 3)]


class _Geometry(C.Structure):
    _fields_ = [("N", C.c_int64), ("sim", C.POINTER(C.c_uint8)),
                ("rec_index", C.POINTER(C.c_int32)),
                ("recs", C.POINTER(_Anchor)), ("nrec", C.c_int64)]


class _FireParams(C.Structure):
    _fields_ = [("dt0", C.c_double), ("dt_max", C.c_double), ("alpha0", C.c_double),
                ("f_alpha", C.c_double), ("f_inc", C.c_double), ("f_dec", C.c_double),
                ("n_min", C.c_int), ("max_iter", C.c_int64), ("force_tol", C.c_double)]


class _FireState(C.Structure):
    _fields_ = [("dt", C.c_double), ("alpha", C.c_double),
                ("npos", C.c_int64), ("iter", C.c_int64),
                ("initialized", C.c_int), ("status", C.c_int),
                ("P", C.c_double), ("normF", C.c_double), ("normv", C.c_double),
                ("rmax", C.c_double)]


_lib = None


class _DescentState(C.Structure):
    _fields_ = [("iter", C.c_int64), ("initialized", C.c_int), ("status", C.c_int),
                ("normF", C.c_double), ("rmax", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, p, i64 = C.c_double, C.c_void_p, C.c_int64
        _lib.orc_uniaxial_s0.restype = d
        _lib.orc_uniaxial_s0.argtypes = [d, d, d]
        _lib.orc_build_geometry.argtypes = [C.POINTER(_Model), C.POINTER(_Object), C.c_int,
                                            C.POINTER(_Geometry)]
        _lib.orc_free_geometry.argtypes = [C.POINTER(_Geometry)]
        _lib.orc_site_energy.argtypes = [C.POINTER(_Model), C.POINTER(_Geometry), p, i64, p]
        _lib.orc_energy.restype = d
        _lib.orc_energy.argtypes = [C.POINTER(_Model), C.POINTER(_Geometry), p, p]
        _lib.orc_force.argtypes = [C.POINTER(_Model), C.POINTER(_Geometry), p, p]
        _lib.orc_force_sites.argtypes = [C.POINTER(_Model), C.POINTER(_Geometry), p, i64, p, p]
        _lib.orc_fire_scalars.argtypes = [C.POINTER(_FireParams), C.POINTER(_FireState),
                                          d, d, d, C.POINTER(d), C.POINTER(d)]
        _lib.orc_fire_run.restype = C.c_int
        _lib.orc_fire_run.argtypes = [C.POINTER(_Model), C.POINTER(_Geometry),
                                      C.POINTER(_FireParams), p, p, p,
                                      C.POINTER(_FireState), i64]
        _lib.orc_descent_run.restype = C.c_int
        _lib.orc_descent_run.argtypes = [C.POINTER(_Model), C.POINTER(_Geometry), C.c_int, d, d,
                                         i64, d, p, p, p, p, C.POINTER(_DescentState), i64]
        _lib.orc_eig_sym3.argtypes = [p, p, p]
        _lib.orc_order_field.argtypes = [C.POINTER(_Geometry), p, i64, p]
        _lib.orc_num_threads.restype = C.c_int
        _lib.orc_set_num_threads.restype = C.c_int
        _lib.orc_set_num_threads.argtypes = [C.c_int]
        _lib.orc_distortion_density.restype = d
        _lib.orc_distortion_density.argtypes = [C.POINTER(_Model), p, p]
    return _lib


def uniaxial_s0(A: float, B: float, C_: float) -> float:
    """Degree of order of the bulk minimum, Eq. (S0def)."""
    return lib().orc_uniaxial_s0(A, B, C_)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> int:
    """Threads of the oracle's parallel loops from now on; returns the count
    in effect."""
    return lib().orc_set_num_threads(int(n))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One lattice + material + object list, resolved into the oracle's own
    geometry (object sites, boundary records).

    ``objects`` is a list of dicts, in the order the objects were added:
      {"type": "wall", "axis": k, "plane": p, "anchor": (kind, W, dir)}
      {"type": "sphere", "c": (x, y, z), "R": r, "anchor": (kind, W, dir)}
      {"type": "droplet", "c": (x, y, z), "R": r, "anchor": ...}   (fills the ball)
      {"type": "spherocylinder", "c": p0, "c2": p1, "R": r, "anchor": ...}
      {"type": "sites", "xyz": int array (n, 3), "anchor": (kind, W, dir)}
      {"type": "anchored", "xyz": int array (n, 3), "kinds": (n,), "W": (n,), "dirs": (n, 3)}
    ``S0`` defaults to Eq. (S0def) of the bulk constants.
    """

    def __init__(self, shape, A, B, C_, L1, L2=0.0, L3=0.0, periodic=(1, 1, 1),
                 objects=(), S0=None, L4=0.0, L6=0.0, H=(0.0, 0.0, 0.0), mu0_dchi=0.0,
                 E=(0.0, 0.0, 0.0), eps0_deps=0.0):
        self.nx, self.ny, self.nz = (int(s) for s in shape)
        self.shape = (self.nx, self.ny, self.nz)
        self.periodic = tuple(int(bool(p)) for p in periodic)
        self.N = self.nx * self.ny * self.nz
        self.S0 = uniaxial_s0(A, B, C_) if S0 is None else float(S0)
        self.model = _Model(self.nx, self.ny, self.nz, (C.c_int * 3)(*periodic),
                            A, B, C_, L1, L2, L3, self.S0, L4, L6, (C.c_double * 3)(*H),
                            mu0_dchi, (C.c_double * 3)(*E), eps0_deps)
        self._keep = []
        objs = (_Object * max(1, len(objects)))()
        for o, spec in zip(objs, objects):
            t = spec["type"]
            if t in ("wall", "sphere", "sites", "droplet", "spherocylinder"):
                kind, W, dr = spec.get("anchor", (ND_HOMEOTROPIC, 0.0, (0, 0, 1)))
                o.anch = _AnchorSpec(kind, W, (C.c_double * 3)(*dr))
            if t == "wall":
                o.type, o.axis, o.plane = WALL, spec["axis"], spec["plane"]
            elif t == "sphere":
                o.type, o.R = SPHERE, spec["R"]
                o.c = (C.c_double * 3)(*spec["c"])
            elif t == "droplet":
                o.type, o.R = DROPLET, spec["R"]
                o.c = (C.c_double * 3)(*spec["c"])
            elif t == "spherocylinder":
                o.type, o.R = SPHEROCYLINDER, spec["R"]
                o.c = (C.c_double * 3)(*spec["c"])
                o.c2 = (C.c_double * 3)(*spec["c2"])
            elif t in ("sites", "anchored"):
                xyz = np.ascontiguousarray(spec["xyz"], dtype=np.int32).reshape(-1, 3)
                self._keep.append(xyz)
                o.type = SITES if t == "sites" else ANCHORED
                o.n = xyz.shape[0]
                o.xyz = xyz.ctypes.data_as(C.POINTER(C.c_int32))
                if t == "anchored":
                    per = (_AnchorSpec * max(1, o.n))()
                    for s in range(o.n):
                        per[s] = _AnchorSpec(int(spec["kinds"][s]), float(spec["W"][s]),
                                             (C.c_double * 3)(*spec["dirs"][s]))
                    self._keep.append(per)
                    o.per_site = C.cast(per, C.POINTER(_AnchorSpec))
            else:
                raise ValueError(t)
        self.geom = _Geometry()
        if lib().orc_build_geometry(C.byref(self.model), objs, len(objects),
                                    C.byref(self.geom)) != 0:
            raise MemoryError("oracle geometry")
        self._keep.clear()

    def __del__(self):
        try:
            lib().orc_free_geometry(C.byref(self.geom))
        except Exception:
            pass

    # ---- geometry readback -------------------------------------------------
    def simulated(self) -> np.ndarray:
        return np.ctypeslib.as_array(self.geom.sim, shape=(self.N,)).astype(bool).copy()

    def records(self):
        """(site index array, kind, W, q0 (n,5), nu (n,3)) of the anchored sites."""
        ri = np.ctypeslib.as_array(self.geom.rec_index, shape=(self.N,)).copy()
        sites = np.nonzero(ri >= 0)[0]
        n = int(self.geom.nrec)
        kind = np.array([self.geom.recs[ri[s]].kind for s in sites], dtype=np.int32)
        W = np.array([self.geom.recs[ri[s]].W for s in sites])
        q0 = np.array([list(self.geom.recs[ri[s]].q0) for s in sites]).reshape(-1, 5)
        nu = np.array([list(self.geom.recs[ri[s]].nu) for s in sites]).reshape(-1, 3)
        assert len(sites) == n
        return sites, kind, W, q0, nu

    def distortion_density(self, Q, d):
        """Eq. (fdistortionFull) with this oracle's constants at one point:
        Q (3, 3) and d (3, 3, 3), d[i, j, k] = dQ_ij/dx_k."""
        Q = np.ascontiguousarray(Q, dtype=np.float64).reshape(9)
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(27)
        return lib().orc_distortion_density(C.byref(self.model), _ptr(Q), _ptr(d))

    # ---- energy and force --------------------------------------------------
    def _q(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(5, self.N)
        return q

    def energy(self, q):
        """Total energy and its (bulk, distortion, anchoring) parts."""
        q = self._q(q)
        parts = np.zeros(3)
        tot = lib().orc_energy(C.byref(self.model), C.byref(self.geom), _ptr(q), _ptr(parts))
        return tot, parts

    def site_energy(self, q, site):
        q = self._q(q)
        parts = np.zeros(3)
        lib().orc_site_energy(C.byref(self.model), C.byref(self.geom), _ptr(q),
                              int(site), _ptr(parts))
        return parts

    def force(self, q):
        q = self._q(q)
        F = np.zeros((5, self.N))
        lib().orc_force(C.byref(self.model), C.byref(self.geom), _ptr(q), _ptr(F))
        return F

    def force_sites(self, q, sites):
        q = self._q(q)
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        F = np.zeros((5, sites.size))
        lib().orc_force_sites(C.byref(self.model), C.byref(self.geom), _ptr(q),
                              sites.size, _ptr(sites), _ptr(F))
        return F

    def order_field(self, q):
        q = self._q(q)
        S = np.zeros(self.N)
        lib().orc_order_field(C.byref(self.geom), _ptr(q), self.N, _ptr(S))
        return S

    # ---- FIRE -------------------------------------------------------------
    def fire(self, q, params, max_steps, state=None, v=None, F=None):
        """Run up to ``max_steps`` FIRE iterations (Algorithm 1).  Returns
        (q, v, F, state) with ``state`` a dict; pass it back to continue."""
        q = self._q(q).copy()
        v = np.zeros((5, self.N)) if v is None else np.ascontiguousarray(v, dtype=np.float64).copy()
        F = np.zeros((5, self.N)) if F is None else np.ascontiguousarray(F, dtype=np.float64).copy()
        st = _FireState()
        if state is not None:
            for k, val in state.items():
                setattr(st, k, val)
        p = fire_params(**params)
        lib().orc_fire_run(C.byref(self.model), C.byref(self.geom), C.byref(p),
                           _ptr(q), _ptr(v), _ptr(F), C.byref(st), int(max_steps))
        out = {k: getattr(st, k) for k, _ in _FireState._fields_}
        return q, v, F, out

    def descent(self, x, method, eta, mu=0.0, max_iter=10 ** 9, force_tol=1e-9, max_steps=1,
                state=None):
        """Run up to ``max_steps`` iterations of gradient descent (method GD)
        or Nesterov's accelerated gradient (NESTEROV).  ``state`` is None
        (start from ``x``) or the dict returned by a previous call.  Returns
        a dict with x, xprev, y (where F is evaluated), F and the scalars."""
        st = _DescentState()
        if state is None:
            x = self._q(x).copy()
            xprev, y, F = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
        else:
            x, xprev, y, F = (state[k].copy() for k in ("x", "xprev", "y", "F"))
            for k, _ in _DescentState._fields_:
                setattr(st, k, state[k])
        lib().orc_descent_run(C.byref(self.model), C.byref(self.geom), int(method), float(eta),
                              float(mu), int(max_iter), float(force_tol), _ptr(x), _ptr(xprev),
                              _ptr(y), _ptr(F), C.byref(st), int(max_steps))
        out = {k: getattr(st, k) for k, _ in _DescentState._fields_}
        out.update(x=x, xprev=xprev, y=y, F=F)
        return out


GD, NESTEROV = 1, 2


def frank_to_landau(K1, K2, K3, K24, q0, S):
    """Distortion constants of Eq. (fdistortionFull) that reproduce the
    Frank-Oseen density Eq. (FOfull) in the uniaxial limit at order S
    (section II, the identifications after Mori et al. 1999): L1 from the
    splay, twist and bend constants, L2 and L3 from splay, twist and
    saddle-splay, L4 from the chiral wavenumber q0 with the twist constant,
    L6 from bend minus splay."""
    return dict(L1=2.0 / (27.0 * S * S) * (K3 - K1 + 3.0 * K2),
                L2=4.0 / (9.0 * S * S) * (K1 - K24),
                L3=4.0 / (9.0 * S * S) * (K24 - K2),
                L4=-8.0 / (9.0 * S * S) * q0 * K2,
                L6=4.0 / (27.0 * S ** 3) * (K3 - K1))


def dipolar_director(u, axis, rd):
    """Director of the dipolar configuration about a homeotropic colloid
    (section IV.A, the dipolar start after Lubensky et al.), at offsets u
    (m, 3) from the colloid centre: a radial hedgehog at the centre and a
    hyperbolic hedgehog at h = rd a on the axis a.  With theta_c and
    theta_h the polar angles (about a) of the point seen from the centre
    and from h, the director is tilted from a by psi = theta_c - theta_h
    toward the point's radial direction away from the axis:
    n = cos(psi) a + sin(psi) e_rho.  Far away theta_c ~ theta_h and n -> a;
    near the centre n ~ u/|u| (radial); near h, n is the hyperbolic
    hedgehog's reflection of w/|w| through the axis."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    w = u - rd * a[None, :]
    ua, wa = u @ a, w @ a
    perp = u - ua[:, None] * a[None, :]
    rho = np.linalg.norm(perp, axis=1)
    theta_c = np.arctan2(rho, ua)
    theta_h = np.arctan2(rho, wa)
    psi = theta_c - theta_h
    e_rho = np.zeros_like(perp)
    nz = rho > 0
    e_rho[nz] = perp[nz] / rho[nz, None]
    return np.cos(psi)[:, None] * a[None, :] + np.sin(psi)[:, None] * e_rho


def dipolar_q(oracle, c, axis, rd, S):
    """Q = 3/2 S (n n - I/3) of ``dipolar_director`` on the oracle's
    simulated sites (offsets by the minimum image along periodic axes),
    zero on object sites; (5, N) like every Q field here."""
    nx, ny, nz = oracle.shape
    i = np.arange(oracle.N)
    xyz = np.stack([i % nx, (i // nx) % ny, i // (nx * ny)], axis=1).astype(np.float64)
    u = xyz - np.asarray(c, dtype=np.float64)[None, :]
    for k, n in enumerate((nx, ny, nz)):
        if oracle.periodic[k]:
            u[:, k] -= n * np.floor(u[:, k] / n + 0.5)
    d = dipolar_director(u, axis, rd)
    q = np.stack([1.5 * S * (d[:, 0] * d[:, 0] - 1.0 / 3.0), 1.5 * S * d[:, 0] * d[:, 1],
                  1.5 * S * d[:, 0] * d[:, 2], 1.5 * S * (d[:, 1] * d[:, 1] - 1.0 / 3.0),
                  1.5 * S * d[:, 1] * d[:, 2]])
    q[:, ~oracle.simulated()] = 0.0
    return q


def fire_params(dt0=1e-3, dt_max=1e-2, alpha0=0.99, f_alpha=0.99, f_inc=1.1, f_dec=0.5,
                n_min=5, max_iter=10**9, force_tol=1e-9):
    return _FireParams(dt0, dt_max, alpha0, f_alpha, f_inc, f_dec, n_min, max_iter, force_tol)


def fire_scalars(params: dict, state: dict, P, normF, normv):
    """One application of the FIRE scalar rules; returns (a, b, new state)."""
    p = fire_params(**params)
    st = _FireState()
    for k, val in state.items():
        setattr(st, k, val)
    a, b = C.c_double(), C.c_double()
    lib().orc_fire_scalars(C.byref(p), C.byref(st), P, normF, normv, C.byref(a), C.byref(b))
    return a.value, b.value, {k: getattr(st, k) for k, _ in _FireState._fields_}


def eig_sym3(q5):
    q5 = np.ascontiguousarray(q5, dtype=np.float64)
    ev = np.zeros(3)
    vec = np.zeros(9)
    lib().orc_eig_sym3(_ptr(q5), _ptr(ev), _ptr(vec))
    return ev, vec.reshape(3, 3)
