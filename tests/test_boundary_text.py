"""The custom boundary text format (section VI: objects made of arbitrary
site sets, each boundary site with its own homeotropic or planar anchoring,
read from a prepared text file).  Parsing runs on the host without a
solver, so these checks need no GPU; the GPU tests compare geometry built
from text with the same objects built through the in-memory calls."""
import pytest

from paper_1911_07045_b300 import lqmin

EXAMPLE = """
# a pyramid-like colloid above a patterned substrate
object homeotropic 2.5            # object sites, homeotropic on their neighbours
  10 10 10
  11 10 10
  10 11 10
  10 10 11
end

object planar 1.0 0 0 1           # planar-degenerate, normal +z
  3 4 5
end

boundary                          # per-site anchoring records
  0 0 1  oriented 3.0  0.0 1.0 0.0
  1 0 1  planar 1.5  0 0 1
  2 0 1  homeotropic 0.5  0 0 1
  5 5 5  1 2e-1 1 1 0
end
"""


def test_example_parses_into_blocks_and_sites():
    assert lqmin.boundary_check(EXAMPLE) == (3, 9)
    assert lqmin.boundary_check("") == (0, 0)
    assert lqmin.boundary_check("# only a comment\n\n   \n") == (0, 0)
    # no trailing newline, tabs as separators, an empty block
    assert lqmin.boundary_check("object\t0\t1.0\n1\t2\t3\nend") == (1, 1)
    assert lqmin.boundary_check("boundary\nend\n") == (1, 0)


@pytest.mark.parametrize("text, line, what", [
    ("thing 1 2\n", 1, "expected 'object' or 'boundary'"),
    ("object homeotropic 1\n1 2 3\n", 1, "not closed"),
    ("\n\nobject homeotropic\n", 3, "object takes"),
    ("object sideways 1\nend\n", 1, "unknown anchoring"),
    ("object planar -1\nend\n", 1, "strength"),
    ("object planar 1 0 0\nend\n", 1, "object takes"),
    ("object planar 1\n1 2\nend\n", 2, "object site takes"),
    ("object planar 1\n1 2 3.5\nend\n", 2, "coordinate"),
    ("object planar 1\n1 2 99999999999\nend\n", 2, "coordinate"),
    ("boundary\n1 2 3 planar 1 0 0\nend\n", 2, "boundary site takes"),
    ("boundary\n1 2 3 planar nan 0 0 1\nend\n", 2, "strength"),
    ("boundary\n1 2 3 planar 1 0 x 1\nend\n", 2, "direction"),
    ("boundary extra\nend\n", 1, "no arguments"),
    ("end\n", 1, "expected 'object' or 'boundary'"),
    ("object planar 1\nobject planar 1\nend\n", 2, "not closed"),
    ("boundary\n1 2 3 planar 1 0 0 1\nboundary\nend\n", 3, "not closed"),
    ("boundary\nend now\n", 2, "end takes no arguments"),
])
def test_errors_name_the_line(text, line, what):
    with pytest.raises(lqmin.LqError) as e:
        lqmin.boundary_check(text)
    msg = str(e.value)
    assert f"line {line}:" in msg and what in msg
