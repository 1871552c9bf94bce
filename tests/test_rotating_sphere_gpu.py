"""Rotating sphere (moving-wall targets u^t = omega x r on a 3D body,
adiabatic wall; the Sec. 3.9 case): FP64 parity with the oracle, and the
FP32 path's lift points to the side where the surface moves with the
stream (the Magnus direction) with |C_l| growing with the rotation rate."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _maxrel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def test_rotating_sphere_fp64_parity():
    """D3Q19 sphere turning about z at Omega* = omega D / (2 u_inf) = 0.6,
    Neumann (adiabatic) wall: populations, rho E and the per-point forces
    equal the oracle's to 1e-12 after 30 steps."""
    from paper_2607_07432_b300 import inputs
    case = C.small_sphere()
    ctr = (9.3, 10.1, 9.8)

    def geo(th):
        g = inputs.icosphere(ctr, 8.0, 4, tbc=1, t_value=0.0)
        return g
    case["geo"] = geo
    sim, g0 = C.make_oracle(case)
    u_inf = sim.prm.u_mag
    omega = 2.0 * 0.6 * u_inf / 8.0
    g0 = inputs.rotating(g0, ctr, (0.0, 0.0, omega))
    from oracle import lbm
    sim = lbm.Sim(sim.prm, g0)
    g = C.make_gpu(case, "fp64", g0)
    sim.run(30)
    g.step(30)
    f, E = g.state()
    assert _maxrel(f, sim.f) < 1e-12
    assert _maxrel(E, sim.E) < 1e-12
    wl = g.wall_loads(per_point=True)
    assert np.max(np.abs(wl["F"] - sim.last_loads["F"])) < 1e-12 * max(1.0, np.abs(sim.last_loads["F"]).max())
    g.close()


def test_rotating_sphere_magnus_direction():
    """FP32, 64x48x48, D = 12, Ma 0.3, Re 100, rotation about +z with the
    stream along +x: the surface at -y moves with the stream, so the
    time-averaged lift points to -y; it grows from Omega* = 0.3 to 0.6 and
    vanishes without rotation (to the symmetric-flow level)."""
    from paper_2607_07432_b300 import inputs, lbmib
    ctr = (20.0, 24.0, 24.0)
    out = {}
    for om in (0.0, 0.3, 0.6):
        s = lbmib.Solver("D3Q19", "fp32", (64, 48, 48), mach=0.3, reynolds=100.0, ref_length=12.0,
                         bc=[lbmib.BC_INLET, lbmib.BC_OUTLET] + [lbmib.BC_FARFIELD] * 4)
        u_inf = s.constants()["u_mag"]
        geo = inputs.rotating(inputs.icosphere(ctr, 12.0, 6, tbc=1, t_value=0.0), ctr,
                              (0.0, 0.0, 2.0 * om * u_inf / 12.0))
        s.set_geometry(geo)
        s.step(1500)
        cl = []
        for _ in range(10):
            s.step(50)
            cl.append(s.wall_diagnostics(per_point=False)["Cl"])
        s.check()
        out[om] = float(np.mean(cl))
        s.close()
    # C_l is along e_d rotated towards +y: -y lift is a negative C_l
    assert out[0.3] < 0.0 and out[0.6] < out[0.3]
    assert abs(out[0.0]) < 0.1 * abs(out[0.6])
