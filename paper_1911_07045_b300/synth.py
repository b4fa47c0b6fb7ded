"""Seeded synthetic inputs: initial Q fields, object layouts, batches and
request streams shaped like the paper's workloads.

This module holds no part of the method's arithmetic (no energy, force or
minimiser step).  It only produces inputs, and both the CUDA path and the
CPU oracle receive exactly the arrays and object lists it returns.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014),
keyed on (seed, counter): the k-th output of a SplitMix64 stream started at
``seed`` is ``mix(seed + k * GAMMA)``.  A uniform double in [0, 1) takes the
top 53 bits.  Random directors are uniform on the sphere
(z = 2 u1 - 1, phi = 2 pi u2) and the initial Q is the uniaxial tensor
3/2 S (n n - I/3) of Eq. (Qtensor) (paper section II), which is how the
paper's GUI starts a bulk minimisation from random directors (section V).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# anchoring kinds (the numbering of the C interface)
ND_HOMEOTROPIC, ND_ORIENTED, FG_PLANAR = 0, 1, 2

# 5CB constants in lattice units (A, B, C) and the one-constant L1 of
# section III.B; L2, L3 of the three-constant workloads
A_5CB, B_5CB, C_5CB = -0.172, -2.12, 1.73
L1_5CB = 2.32
L2_3C, L3_3C = 0.5, 0.3
W_HOMEOTROPIC = 5.3
W_PLANAR = 1.0

FIRE_DEFAULTS = dict(dt0=1e-3, dt_max=1e-2, alpha0=0.99, f_alpha=0.99, f_inc=1.1,
                     f_dec=0.5, n_min=5)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output number ``counter`` (1-based) of the stream ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + counter.astype(np.uint64) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counter: np.ndarray) -> np.ndarray:
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def random_directors(n_sites: int, seed: int) -> np.ndarray:
    """(3, n) unit vectors, uniform on the sphere; site i uses stream
    outputs 2i+1 (for z) and 2i+2 (for phi)."""
    i = np.arange(n_sites, dtype=np.uint64)
    u1 = uniform01(seed, np.uint64(2) * i + np.uint64(1))
    u2 = uniform01(seed, np.uint64(2) * i + np.uint64(2))
    z = 2.0 * u1 - 1.0
    phi = 2.0 * math.pi * u2
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z])


def uniaxial_q(n: np.ndarray, S) -> np.ndarray:
    """(5, N) components (Qxx, Qxy, Qxz, Qyy, Qyz) of 3/2 S (n n - I/3)."""
    S = np.asarray(S, dtype=np.float64)
    return np.stack([1.5 * S * (n[0] * n[0] - 1.0 / 3.0), 1.5 * S * n[0] * n[1],
                     1.5 * S * n[0] * n[2], 1.5 * S * (n[1] * n[1] - 1.0 / 3.0),
                     1.5 * S * n[1] * n[2]])


def s0_closed_form(A: float, B: float, C: float) -> float:
    """The amplitude of the generated start states: the workloads start
    uniaxial at the closed-form S0 of Eq. (S0def) for their A, B, C.  Only
    the inputs use it; the CUDA path and the oracle each compute S0 for their
    own arithmetic (anchoring targets, random starts) independently."""
    return (-B + math.sqrt(B * B - 24.0 * A * C)) / (6.0 * C)


def random_uniaxial_q(shape, seed: int, S=None, A=A_5CB, B=B_5CB, C=C_5CB) -> np.ndarray:
    nx, ny, nz = shape
    S = s0_closed_form(A, B, C) if S is None else S
    return uniaxial_q(random_directors(nx * ny * nz, seed), S)


def texture_q(shape, kind: str, m: int = 1, S=None, A=A_5CB, B=B_5CB, C=C_5CB):
    """Smooth 1-D textures along z with wavenumber k = pi m / nz:
    'twist' n = (cos kz, sin kz, 0); 'splaybend' n = (sin kz, 0, cos kz)."""
    nx, ny, nz = shape
    S = s0_closed_form(A, B, C) if S is None else S
    z = np.repeat(np.arange(nz), nx * ny).astype(np.float64)
    k = math.pi * m / nz
    if kind == "twist":
        n = np.stack([np.cos(k * z), np.sin(k * z), np.zeros_like(z)])
    elif kind == "splaybend":
        n = np.stack([np.sin(k * z), np.zeros_like(z), np.cos(k * z)])
    else:
        raise ValueError(kind)
    return uniaxial_q(n, S)


# ---- object layouts of the paper's workloads ------------------------------

def _rng_stream(seed: int):
    """Endless uniform stream from SplitMix64 (counter 1, 2, ...)."""
    k = 0
    while True:
        k += 1
        yield float(uniform01(seed, np.array([k], dtype=np.uint64))[0])


def place_spheres(L: int, count: int, r_lo: float, r_hi: float, seed: int,
                  walls: bool = True, gap: int = 3, r_clamp=None):
    """Non-overlapping spheres with radius uniform in [r_lo, r_hi] (clamped to
    r_clamp), centres on lattice sites.  Surfaces stay ``gap`` sites apart
    (minimum-image distance: the box is periodic along x and y, and along z
    too when ``walls`` is False); with ``walls`` the spheres also stay
    ``gap`` sites clear of the z = 0 and z = L-1 wall planes.  A draw that
    cannot be placed after many tries is redrawn with its radius scaled by
    0.9 (only small boxes ever need this)."""
    u = _rng_stream(seed)
    out = []
    shrink = 1.0
    tries = 0
    while len(out) < count:
        tries += 1
        if tries % 2000 == 0:
            shrink *= 0.9
        if tries > 200000:
            raise RuntimeError("could not place spheres")
        R = (r_lo + (r_hi - r_lo) * next(u)) * shrink
        if r_clamp is not None:
            R = min(R, r_clamp)
        c = [int(L * next(u)) % L for _ in range(3)]
        if walls:
            lo = int(math.ceil(R)) + gap + 1
            hi = L - 1 - lo
            if hi < lo:
                continue
            c[2] = lo + int((hi - lo + 1) * next(u))
        ok = True
        for (c2, R2) in out:
            d2 = 0.0
            for k in range(3):
                dk = abs(c[k] - c2[k])
                if k < 2 or not walls:
                    dk = min(dk, L - dk)
                d2 += dk * dk
            if math.sqrt(d2) < R + R2 + gap:
                ok = False
                break
        if ok:
            out.append((tuple(float(v) for v in c), R))
    return out


def config_small_periodic():
    """32^3 periodic bulk, one-constant, random uniaxial start (seed 1)."""
    return dict(shape=(32, 32, 32), L1=L1_5CB, L2=0.0, L3=0.0, objects=[], seed=1,
                tol=1e-9)


def config_colloid_slab():
    """128^3: homeotropic walls at z = 0 and z = 127, one homeotropic colloid
    of radius 20 at the centre, three-constant elasticity (seed 2)."""
    hom = (ND_HOMEOTROPIC, W_HOMEOTROPIC, (0.0, 0.0, 1.0))
    objs = [dict(type="wall", axis=2, plane=0, anchor=hom),
            dict(type="wall", axis=2, plane=127, anchor=hom),
            dict(type="sphere", c=(64.0, 64.0, 64.0), R=20.0, anchor=hom)]
    return dict(shape=(128, 128, 128), L1=L1_5CB, L2=L2_3C, L3=L3_3C, objects=objs,
                seed=2, tol=1e-8)


def config_large(L: int = 512, seed: int = 3):
    """L^3 (512^3 by default): planar-degenerate walls at z = 0, L-1 (W = 1)
    and four homeotropic colloids of radius U[12, 24] (W = 5.3) at seeded
    non-overlapping positions; three-constant elasticity."""
    pla = (FG_PLANAR, W_PLANAR, (0.0, 0.0, 1.0))
    hom = (ND_HOMEOTROPIC, W_HOMEOTROPIC, (0.0, 0.0, 1.0))
    objs = [dict(type="wall", axis=2, plane=0, anchor=pla),
            dict(type="wall", axis=2, plane=L - 1, anchor=pla)]
    scale = L / 512.0
    for c, R in place_spheres(L, 4, 12 * scale, 24 * scale, seed, walls=True,
                              r_clamp=max(2.0, 0.2 * L)):
        objs.append(dict(type="sphere", c=c, R=R, anchor=hom))
    return dict(shape=(L, L, L), L1=L1_5CB, L2=L2_3C, L3=L3_3C, objects=objs, seed=seed,
                tol=1e-8)


def config_fig3(L: int = 250):
    """The three geometries of Fig. 3 at L^3, one-constant elasticity,
    periodic box with plates at z = 0 and z = L-1 where present (sizes are
    not printed in the paper: colloid radius L/10, droplet radius 0.48 L,
    spherocylinder of radius L/12 and axis length 0.4 L along x):
      two_colloids  two homeotropic colloids between homeotropic plates;
      droplet       the interior of a homeotropic droplet;
      rod_plates    a homeotropic spherocylinder between planar-degenerate
                    plates."""
    hom = (ND_HOMEOTROPIC, W_HOMEOTROPIC, (0.0, 0.0, 1.0))
    pla = (FG_PLANAR, W_PLANAR, (0.0, 0.0, 1.0))
    h = (L - 1) / 2.0
    walls = lambda a: [dict(type="wall", axis=2, plane=0, anchor=a),
                       dict(type="wall", axis=2, plane=L - 1, anchor=a)]
    R = L / 10.0
    return {
        "two_colloids": dict(shape=(L, L, L), L1=L1_5CB, L2=0.0, L3=0.0,
                             objects=walls(hom) + [
                                 dict(type="sphere", c=(h - 1.6 * R, h, h), R=R, anchor=hom),
                                 dict(type="sphere", c=(h + 1.6 * R, h, h), R=R, anchor=hom)]),
        "droplet": dict(shape=(L, L, L), L1=L1_5CB, L2=0.0, L3=0.0,
                        objects=[dict(type="droplet", c=(h, h, h), R=0.48 * L, anchor=hom)]),
        "rod_plates": dict(shape=(L, L, L), L1=L1_5CB, L2=0.0, L3=0.0,
                           objects=walls(pla) + [
                               dict(type="spherocylinder", c=(h - 0.2 * L, h, h),
                                    c2=(h + 0.2 * L, h, h), R=L / 12.0, anchor=hom)]),
    }


def config_batch(seed: int = 4, count: int = 64):
    """Independent cubic lattices, edge uniform in {32, 48, 64, 96, 128}, each
    with 0-3 homeotropic colloids of radius U[6, 16] (periodic box, no walls),
    one-constant elasticity, random uniaxial starts."""
    u = _rng_stream(seed)
    edges = (32, 48, 64, 96, 128)
    out = []
    for b in range(count):
        L = edges[min(4, int(5 * next(u)))]
        nsph = min(3, int(4 * next(u)))
        hom = (ND_HOMEOTROPIC, W_HOMEOTROPIC, (0.0, 0.0, 1.0))
        # radii clamped to L/5 so that three colloids fit the smallest boxes
        objs = [dict(type="sphere", c=c, R=R, anchor=hom)
                for c, R in place_spheres(L, nsph, 6.0, 16.0, seed * 1000 + b + 1,
                                          walls=False, r_clamp=0.2 * L)]
        out.append(dict(shape=(L, L, L), L1=L1_5CB, L2=0.0, L3=0.0, objects=objs,
                        seed=seed * 1000 + 500 + b))
    return out


def patterned_directors(L: int, d: int) -> np.ndarray:
    """In-plane director angle field of a square array of alternating +-1
    surface defects with period d: phi = arg(sin(pi(x+1/2)/d) + i sin(pi(y+1/2)/d));
    returns (L*L, 3) directors for the sites of one z plane (x fastest)."""
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    phi = np.arctan2(np.sin(math.pi * (y + 0.5) / d), np.sin(math.pi * (x + 0.5) / d))
    return np.stack([np.cos(phi), np.sin(phi), np.zeros_like(phi)], axis=-1).reshape(-1, 3)


def serving_requests(seed: int = 5, count: int = 2000, rate: float = 20.0):
    """Poisson arrivals (mean ``rate`` per second) of minimisations with cubic
    edge uniform in {48, 64, ..., 192}; half with a patterned bottom wall
    (alternating +-1 surface defects, period drawn from [16, 48] among values
    with L divisible by 2d) and a homeotropic top wall, half with 1-2
    homeotropic colloids."""
    return list(iter_serving_requests(seed, count, rate))


def iter_serving_requests(seed: int = 5, count: int = 2000, rate: float = 20.0):
    """The requests of ``serving_requests`` one at a time (the same stream),
    so that a long stream never sits in memory at once."""
    u = _rng_stream(seed)
    t = 0.0
    edges = list(range(48, 193, 16))
    hom = (ND_HOMEOTROPIC, W_HOMEOTROPIC, (0.0, 0.0, 1.0))
    for r in range(count):
        t += -math.log(1.0 - next(u)) / rate
        L = edges[min(len(edges) - 1, int(len(edges) * next(u)))]
        if next(u) < 0.5:
            periods = [d for d in range(16, 49) if L % (2 * d) == 0] or [L // 2]
            d = periods[min(len(periods) - 1, int(len(periods) * next(u)))]
            dirs = patterned_directors(L, d)
            xy = np.stack(np.meshgrid(np.arange(L), np.arange(L), indexing="xy"), -1).reshape(-1, 2)
            xyz = np.concatenate([xy, np.ones((xy.shape[0], 1), dtype=np.int64)], axis=1)
            # the explicit records come first so that they win over the
            # bottom wall's own anchoring on the z = 1 sites
            objs = [dict(type="anchored", xyz=xyz, kinds=np.full(len(xyz), ND_ORIENTED),
                         W=np.full(len(xyz), W_HOMEOTROPIC), dirs=dirs),
                    dict(type="wall", axis=2, plane=0, anchor=hom),
                    dict(type="wall", axis=2, plane=L - 1, anchor=hom)]
            kind = "patterned"
        else:
            nsph = 1 + int(2 * next(u)) % 2
            objs = [dict(type="sphere", c=c, R=R, anchor=hom)
                    for c, R in place_spheres(L, nsph, 12.0, 24.0, seed * 100000 + r + 1,
                                              walls=False, r_clamp=math.floor(0.2 * L))]
            kind = "colloids"
        yield dict(t_arrival=t, shape=(L, L, L), L1=L1_5CB, L2=0.0, L3=0.0,
                   objects=objs, seed=seed * 100000 + 50000 + r, kind=kind, tol=1e-6)
