"""CPU-side checks: the C-ABI library builds and exports every symbol the
header declares (no compute calls), and the seeded input generators follow
their published definitions."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1911_07045_b300 import build, lqmin, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lqmin.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lq_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = build.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib], text=True)
    exported = set(re.findall(r"\bT (lq_[a-z0-9_]+)", out))
    decl = declared_symbols()
    assert decl, "no declarations parsed"
    missing = [s for s in decl if s not in exported]
    assert not missing, missing
    assert sorted(lqmin.EXPORTS) == decl
    # loads without a GPU (no call is made)
    ctypes.CDLL(lib)


def test_binding_refuses_to_run_without_library(tmp_path):
    saved = lqmin._lib
    lqmin._lib = None
    try:
        with pytest.raises(RuntimeError):
            lqmin.load(str(tmp_path / "missing.so"))
    finally:
        lqmin._lib = saved


def test_splitmix64_published_outputs():
    # reference outputs of SplitMix64 (Steele, Lea, Flood 2014) seeded 1234567
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    got = synth.splitmix64(1234567, np.arange(1, 6, dtype=np.uint64))
    assert [int(v) for v in got] == want


def test_random_directors_are_unit_and_uniform():
    n = synth.random_directors(200000, 9)
    assert np.abs((n * n).sum(0) - 1).max() < 1e-14
    # uniform on the sphere: each Cartesian component is uniform on [-1, 1]
    for k in range(3):
        h, _ = np.histogram(n[k], bins=10, range=(-1, 1))
        assert np.abs(h / 20000.0 - 1).max() < 0.05
    q = synth.uniaxial_q(n[:, :5], 0.5)
    Q = np.zeros((5, 3, 3))
    for t in range(5):
        a, b, c, d, e = q[:, t]
        Q[t] = [[a, b, c], [b, d, e], [c, e, -a - d]]
        ev = np.linalg.eigvalsh(Q[t])
        assert np.allclose(ev, [-0.25, -0.25, 0.5], atol=1e-15)


def test_workload_layouts():
    c3 = synth.config_large()
    sph = [o for o in c3["objects"] if o["type"] == "sphere"]
    assert len(sph) == 4 and all(12 <= o["R"] <= 24 for o in sph)
    for i, a in enumerate(sph):
        assert a["c"][2] - a["R"] >= 3 and 511 - (a["c"][2] + a["R"]) >= 3
        for b in sph[i + 1:]:
            d = np.abs(np.subtract(a["c"], b["c"]))
            d[:2] = np.minimum(d[:2], 512 - d[:2])
            assert np.linalg.norm(d) >= a["R"] + b["R"] + 3
    batch = synth.config_batch()
    assert len(batch) == 64
    assert {b["shape"][0] for b in batch} <= {32, 48, 64, 96, 128}
    reqs = synth.serving_requests(count=50)
    assert all(48 <= r["shape"][0] <= 192 and r["shape"][0] % 16 == 0 for r in reqs)
    assert all(b["t_arrival"] > a["t_arrival"] for a, b in zip(reqs, reqs[1:]))


def test_frank_helper_equals_the_oracle_mapping(oracle_mod):
    """lq_frank_to_landau (host arithmetic, callable without a GPU) gives the
    oracle's identifications of section II."""
    for K in [(1.3, 0.7, 1.9, 0.45, 0.21, 0.6), (6.0, 3.0, 8.0, 1.0, -0.1, 0.53),
              (1.0, 1.0, 1.0, 1.0, 0.0, 0.5)]:
        got = lqmin.frank_to_landau(*K)
        want = oracle_mod.frank_to_landau(*K)
        for k in ("L1", "L2", "L3", "L4", "L6"):
            assert got[k] == pytest.approx(want[k], rel=1e-15, abs=1e-300)
    for bad in [(1, 1, 1, 1, 0, 0.0), (1, 1, 1, 1, 0, -0.5), (1, float("nan"), 1, 1, 0, 0.5)]:
        with pytest.raises(lqmin.LqError):
            lqmin.frank_to_landau(*bad)
