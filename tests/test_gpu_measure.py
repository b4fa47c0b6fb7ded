"""The measurement call behind the FP64 form's roofline: lq_fp64_fma_rate
returns a finite, repeatable rate of FP64 fused multiply-adds, and rejects
bad arguments without running anything."""
import ctypes as C

import pytest

from _helpers import need_gpu
from paper_1911_07045_b300 import lqmin

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_finite_and_repeatable():
    need_gpu()
    a = lqmin.fp64_fma_rate(1 << 14)
    b = lqmin.fp64_fma_rate(1 << 14)
    # between 10 G and 100 T FMA/s on any current GPU; two calls within 25%
    assert 1e10 < a < 1e14 and 1e10 < b < 1e14
    assert abs(a - b) <= 0.25 * max(a, b)
    lib = lqmin.load()
    out = C.c_double(-1.0)
    assert lib.lq_fp64_fma_rate(0, C.byref(out)) == lqmin.LQ_EINVAL
    assert lib.lq_fp64_fma_rate(16, None) == lqmin.LQ_EINVAL
    assert out.value == -1.0
