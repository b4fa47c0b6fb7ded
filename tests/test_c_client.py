"""The C interface used from plain C: a client that includes only
include/lqmin.h compiles as C99 with warnings as errors and links against
the library (CPU); on a GPU it minimises a colloid slab and its energy
matches the Python binding's result for the same calls."""
import os
import subprocess

import pytest

from paper_1911_07045_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "minimize_slab.c")


def _compile(out):
    lib = build.build()
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), SRC, "-o", out,
                           lib, "-Wl,-rpath," + os.path.dirname(lib), "-lm"])


def test_c_client_compiles_and_links(tmp_path):
    _compile(str(tmp_path / "minimize_slab"))
    assert os.path.exists(tmp_path / "minimize_slab")


@pytest.mark.gpu
def test_c_client_minimises_like_the_binding(tmp_path):
    from _helpers import need_gpu
    need_gpu()
    exe = str(tmp_path / "minimize_slab")
    _compile(exe)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    fields = r.stdout.split()
    energy = float(fields[fields.index("energy") + 1])
    from paper_1911_07045_b300 import lqmin, synth
    s = lqmin.Solver((32, 32, 24), synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, 0.5, 0.3)
    hom = (lqmin.ND_HOMEOTROPIC, 5.3, (0.0, 0.0, 1.0))
    s.add_wall(2, 0, *hom)
    s.add_wall(2, 23, *hom)
    s.add_sphere((16.0, 16.0, 12.0), 5.0, *hom)
    s.init_random_uniaxial(7)
    st, res = s.minimize(lqmin.fire_params(max_iter=200000, force_tol=1e-6))
    assert res.fire_status == lqmin.FIRE_CONVERGED
    assert res.energy == pytest.approx(energy, rel=1e-12)
