"""One case split into z slabs on one GPU through the exchange path
(lbm_create_slab, lbm_slab_pack / unpack after every step): the owned
planes equal the unsplit case bit for bit in FP64, the slabs' wall loads
add up to the unsplit loads, and FP32 agrees to rounding."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu

SHAPE = (24, 20, 48)
BC = [C.BC_IN, C.BC_OUT, C.BC_FF, C.BC_FF, C.BC_FF, C.BC_FF]


def _geo(th):
    from paper_2607_07432_b300 import inputs
    return inputs.icosphere((9.3, 10.1, 24.3), 8.0, 4, tbc=0, t_value=1.05 * th)


def _solver(precision, slab=None):
    from paper_2607_07432_b300 import lbmib
    s = lbmib.Solver("D3Q19", precision, SHAPE, mach=0.2, reynolds=20.0, ref_length=8.0, bc=BC, slab=slab)
    s.set_geometry(_geo(s.constants()["theta_inf"]))
    return s


def _run_split(precision, n_slabs, steps, halo=10):
    import torch
    from paper_2607_07432_b300 import slab
    plan = slab.plan(SHAPE[2], n_slabs, halo)
    ss = [_solver(precision, (p["z0"], p["z1"], halo)) for p in plan]
    bufs = [slab.Buffers(s, "cuda") for s in ss]
    for _ in range(steps):
        for s in ss:
            s.step(1)
        slab.exchange_local(ss, bufs)
    torch.cuda.synchronize()
    return plan, ss


@pytest.mark.parametrize("n_slabs", [2, 4])
def test_fp64_slabs_equal_unsplit_bitwise(n_slabs):
    from paper_2607_07432_b300 import slab
    steps = 24
    ref = _solver("fp64")
    ref.step(steps)
    f_ref, E_ref = ref.state()
    L_ref = ref.wall_loads()
    plan, ss = _run_split("fp64", n_slabs, steps)
    parts = []
    for p, s in zip(plan, ss):
        f, E = s.state()
        zg = slice(p["z0"], p["z1"])
        assert np.array_equal(slab.owned(f, p), f_ref[:, zg]), p
        assert np.array_equal(slab.owned(E, p), E_ref[zg]), p
        parts.append(s.wall_loads())
        s.close()
    L = slab.reduce_loads(parts)
    assert np.allclose(L["force"], L_ref["force"], rtol=1e-12, atol=1e-15)
    assert abs(L["heat"] - L_ref["heat"]) <= 1e-12 * abs(L_ref["heat"])
    ref.close()


def test_fp32_slabs_match_unsplit():
    """FP32: the fused step's z chunks start at other planes in a slab, and
    one inline function can contract its multiply-adds differently at two
    call sites, so the owned planes agree to rounding (relative L2 1e-6)."""
    from paper_2607_07432_b300 import slab
    steps = 24
    ref = _solver("fp32")
    ref.step(steps)
    f_ref, _ = ref.state()
    plan, ss = _run_split("fp32", 2, steps)
    for p, s in zip(plan, ss):
        f, _ = s.state()
        a, b = slab.owned(f, p), f_ref[:, p["z0"]:p["z1"]]
        assert np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()) < 1e-6
        s.close()
    ref.close()


def test_slab_without_exchange_diverges():
    """Control: without the exchange the ghost planes go stale and the owned
    planes next to the cut leave the unsplit solution."""
    from paper_2607_07432_b300 import slab
    ref = _solver("fp64")
    ref.step(24)
    f_ref, _ = ref.state()
    p = slab.plan(SHAPE[2], 2, 10)[0]
    s = _solver("fp64", (p["z0"], p["z1"], 10))
    s.step(24)
    f, _ = s.state()
    assert not np.array_equal(slab.owned(f, p), f_ref[:, p["z0"]:p["z1"]])
    s.close()
    ref.close()
