"""Checkpoints: lbm_save_state / lbm_load_state resume a run bit for bit
(FP32 and FP16 storage, 2D and 3D), and a file from another grid is
rejected without touching the handle."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _solver(case, precision):
    from paper_2607_07432_b300 import lbmib
    s = lbmib.Solver(case["lattice"], precision, case["shape"], mach=case["mach"], reynolds=case["reynolds"],
                     ref_length=case["ref_length"], method=case["method"], bc=case["bc"])
    s.set_geometry(case["geo"](s.constants()["theta_inf"]))
    return s


@pytest.mark.parametrize("case_fn,precision", [(C.cylinder_c1, "fp32"), (C.small_sphere, "fp32"),
                                               (C.cylinder_c1, "fp16")])
def test_checkpoint_resumes_bit_for_bit(case_fn, precision, tmp_path):
    case = case_fn()
    path = tmp_path / "state.bin"
    a = _solver(case, precision)
    a.step(7)
    a.save_state(path)
    a.step(9)
    fa, Ea = a.state()
    la = a.wall_loads()
    b = _solver(case, precision)
    b.step(3)            # a different state (and buffer parity) before loading
    b.load_state(path)
    b.step(9)
    fb, Eb = b.state()
    lb = b.wall_loads()
    assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb)
    assert np.array_equal(la["force"], lb["force"])
    a.close()
    b.close()


def test_checkpoint_of_another_grid_is_rejected(tmp_path):
    from paper_2607_07432_b300 import lbmib
    case = C.cylinder_c1()
    path = tmp_path / "state.bin"
    a = _solver(case, "fp32")
    a.step(2)
    a.save_state(path)
    other = dict(case, shape=(120, 100))
    b = lbmib.Solver("D2Q9", "fp32", other["shape"], mach=case["mach"], reynolds=case["reynolds"],
                     ref_length=case["ref_length"], bc=case["bc"])
    f0, E0 = b.state()
    with pytest.raises(lbmib.LBMError) as e:
        b.load_state(path)
    assert e.value.status == 7  # LBM_ESTATE
    f1, E1 = b.state()
    assert np.array_equal(f0, f1) and np.array_equal(E0, E1)
    with pytest.raises(lbmib.LBMError):
        b.load_state(tmp_path / "missing.bin")
    a.close()
    b.close()
