"""Edge cases of the CUDA path against the FP64 oracle and the C ABI's
error behaviour: grids smaller than one tile, grids that leave ragged tiles
in every direction, cases without an immersed body, x extents too short for
the in-kernel x faces, and invalid configurations and geometries."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _maxrel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


CASES = {
    # smaller than one tile, periodic, no body
    "d2_tiny_periodic": dict(lattice="D2Q9", shape=(5, 4), mach=0.2, reynolds=20.0, ref_length=4.0,
                             bc=[C.BC_P] * 4, method=2),
    "d3_tiny_periodic": dict(lattice="D3Q19", shape=(6, 5, 4), mach=0.2, reynolds=20.0, ref_length=4.0,
                             bc=[C.BC_P] * 6, method=2),
    # ragged tiles in x and y, far-field boundaries, a small cylinder
    "d2_ragged_body": dict(lattice="D2Q9", shape=(37, 23), mach=0.2, reynolds=30.0, ref_length=8.0,
                           bc=[C.BC_IN, C.BC_OUT, C.BC_FF, C.BC_FF], method=2,
                           geo=lambda th: C.inputs.cylinder((12.3, 11.6), 8.0, 26, tbc=0, t_value=1.05 * th)),
    # ragged in x, y and z (z chunking), boundaries on every face, no body
    "d3_ragged_bc": dict(lattice="D3Q19", shape=(33, 17, 11), mach=0.2, reynolds=40.0, ref_length=6.0,
                         bc=[C.BC_IN, C.BC_OUT, C.BC_FF, C.BC_FF, C.BC_FF, C.BC_FF], method=2),
    # x extent of three nodes: the x faces go to the boundary kernel
    "d2_short_x": dict(lattice="D2Q9", shape=(3, 16), mach=0.2, reynolds=20.0, ref_length=4.0,
                       bc=[C.BC_IN, C.BC_OUT, C.BC_P, C.BC_P], method=2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_parity_on_edge_grids(name):
    case = CASES[name]
    sim, geo = C.make_oracle(case)
    C.perturb(sim, seed=5)
    g = C.make_gpu(case, "fp64", geo)
    g.set_state(sim.f, sim.E)
    sim.run(12)
    g.step(12)
    f, E = g.state()
    assert _maxrel(f, sim.f) < 1e-12
    assert _maxrel(E, sim.E) < 1e-12
    g.close()


def test_uniform_flow_without_body_stays_uniform():
    from paper_2607_07432_b300 import lbmib
    s = lbmib.Solver("D3Q19", "fp64", (20, 12, 10), mach=0.3, reynolds=100.0, ref_length=8.0,
                     bc=[C.BC_P] * 6)
    rho0, u0, T0, _ = s.fields()
    s.step(30)
    rho, u, T, _ = s.fields()
    assert np.max(np.abs(rho - rho0)) < 1e-13
    assert np.max(np.abs(u - u0)) < 1e-13
    assert np.max(np.abs(T - T0)) < 1e-13
    s.close()


def test_invalid_configuration_and_geometry_are_rejected():
    from paper_2607_07432_b300 import inputs, lbmib
    with pytest.raises(lbmib.LBMError) as e:
        lbmib.Solver("D2Q9", "fp32", (0, 16))
    assert e.value.status == 1  # LBM_EINVAL
    s = lbmib.Solver("D2Q9", "fp32", (32, 32), bc=[C.BC_IN, C.BC_OUT, C.BC_FF, C.BC_FF])
    # a body whose stencils leave the domain
    geo = inputs.cylinder((1.0, 16.0), 6.0, 20, tbc=0, t_value=1.0)
    with pytest.raises(lbmib.LBMError) as e:
        s.set_geometry(geo)
    assert e.value.status == 4  # LBM_EGEOM
    # the handle stays usable after the rejected geometry
    s.step(3)
    s.check()
    s.close()
