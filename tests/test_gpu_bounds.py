"""The bounds-checked build (every shared-memory slot, tile and ring index
and every global element index of the step kernels checked and counted)
run over the parity geometries: forces and FIRE steps against the oracle,
a batch, the wide one-constant tiles and the 64-bit index path, with no
index out of range.  It runs in a child process, which loads that variant
of the library instead of the release one."""
import os
import subprocess
import sys

import pytest

from _helpers import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np
from paper_1911_07045_b300 import build, lqmin, synth
lqmin.load(build.build(bounds_check=True))
import oracle
from _helpers import CASES, force_rel_err, make_pair, rand_q
import ctypes as C
hits = C.c_uint32()
assert lqmin.load().lq_bounds_check_hits(C.byref(hits)) == 0 and hits.value == 0
fp = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=1e-14)
p = lqmin.fire_params(**fp)
for name, c in sorted(CASES.items()):
    per = c.get("periodic", (1, 1, 1))
    for prec in (0, 1):
        for idx64 in (False, True):
            s, o = make_pair(oracle, c["shape"], c["L"], c["objects"], per, precision=prec)
            if idx64:
                s.set_index_width(64)
            q = np.round(rand_q(o.N, 3) * 2.0 ** 28) / 2.0 ** 28
            s.set_q(q)
            err = force_rel_err(s.force(), o.force(q), o.simulated())
            assert err < (1e-10 if prec == 0 else 5e-5), (name, prec, err)
            s.step(p, 7)
            s.close()
# a batch (persistent kernel, both tile heights) and a wide one-constant lattice
for ty in (4, 8):
    ss = [lqmin.Solver((40, 24, 18), synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, precision=1),
          lqmin.Solver((33, 17, 9), synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, precision=1)]
    ss[0].add_objects([dict(type="sphere", c=(20.0, 12.0, 9.0), R=5.0, anchor=(0, 5.3, (0, 0, 1)))])
    for k, s in enumerate(ss):
        s.init_random_uniaxial(k + 1)
    b = lqmin.Batch(ss)
    b.set_tiling(ty, 8)
    b.step(p, 9)
    b.close()
w = lqmin.Solver((260, 12, 10), synth.A_5CB, synth.B_5CB, synth.C_5CB, 2.32, precision=1)
w.init_random_uniaxial(5)
w.step(p, 9)
assert lqmin.load().lq_bounds_check_hits(C.byref(hits)) == 0, "query"
print("HITS", hits.value)
assert hits.value == 0
'''


def test_bounds_checked_build_sees_no_index_out_of_range():
    need_gpu()
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "HITS 0" in r.stdout
