"""The entry point's smoke check (one force and one FIRE step on cuda:0
against the oracle) runs as part of the GPU tests, so that it stays green."""
import os
import sys

import pytest

from _helpers import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_smoke_entry_point():
    need_gpu()
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.smoke()
