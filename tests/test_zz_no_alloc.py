"""lbm_get_wall_loads_noalloc (wall loads computed with a static device
scratch, for callers that cannot allocate device memory) against
lbm_get_wall_loads, on two calls in a row.  Kept in its own file that
collects last."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _close(a, b, rtol=1e-12):
    scale = max(1e-300, np.max(np.abs(b)))
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) <= rtol * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_wall_loads_match(precision):
    case = C.cylinder_c1()
    _, geo = C.make_oracle(case)
    g = C.make_gpu(case, precision, geo)
    for _ in range(2):
        g.step(7)
        ref = g.wall_loads()
        got = g.wall_loads_noalloc()
        assert _close(got["force"], ref["force"])
        assert _close([got["heat"]], [ref["heat"]])
        assert _close([got["work"]], [ref["work"]])
    g.close()


def test_noalloc_sphere_many_points():
    """3D body with more points than one reduction block (1000+ points)."""
    case = C.small_sphere()
    case["shape"] = (40, 36, 36)
    from paper_2607_07432_b300 import inputs
    case["geo"] = lambda th: inputs.icosphere((18.3, 18.1, 17.8), 20.0, 12, tbc=0, t_value=1.05 * th)
    _, geo = C.make_oracle(case)
    g = C.make_gpu(case, "fp32", geo)
    assert g.NL > 256
    for _ in range(2):
        g.step(3)
        ref = g.wall_loads()
        got = g.wall_loads_noalloc()
        assert _close(got["force"], ref["force"])
        assert _close([got["heat"]], [ref["heat"]])
    g.close()
