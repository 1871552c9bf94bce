"""Characteristic far-field faces (LBM_BC_CHARACTERISTIC) through the C ABI
against the oracle: FP64 bit-level parity with a body, in 2D and 3D, and the
acoustic absorption of the oracle's pin reproduced by the FP32 path."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu
BC_CHAR = 5


def _maxrel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _cyl():
    case = C.small_cylinder_periodic()
    case.update(shape=(48, 40), bc=[C.BC_IN, BC_CHAR, BC_CHAR, BC_CHAR])
    return case


def _sph():
    return C.small_sphere(bc=[C.BC_IN] + [BC_CHAR] * 5)


@pytest.mark.parametrize("case_fn,steps", [(_cyl, 40), (_sph, 12)])
def test_characteristic_faces_fp64_parity(case_fn, steps):
    """From a seeded perturbed state with the body: populations and rho E
    equal the oracle's to 1e-12 (FP64), edges between characteristic faces
    and corners with the inlet included."""
    case = case_fn()
    sim, geo = C.make_oracle(case)
    C.perturb(sim, seed=5)
    g = C.make_gpu(case, "fp64", geo)
    g.set_state(sim.f, sim.E)
    sim.run(steps)
    g.step(steps)
    f, E = g.state()
    assert _maxrel(f, sim.f) < 1e-12
    assert _maxrel(E, sim.E) < 1e-12
    g.close()


def test_characteristic_face_absorbs_pulse_fp32():
    """An acoustic pulse leaves through characteristic x faces of the FP32
    path with under 2% of it left in the domain (the oracle pin's bar)."""
    from paper_2607_07432_b300 import lbmib
    nx, A = 160, 1e-4
    s = lbmib.Solver("D2Q9", "fp32", (nx, 4), mach=0.1, reynolds=1.0, ref_length=1.0, theta_inf=1.0,
                     bc=[BC_CHAR, BC_CHAR, C.BC_P, C.BC_P], inflow_dir=(1.0, 0.0, 0.0))
    k = s.constants()
    c = np.sqrt(1.4 / 3.0)
    U = k["u_mag"]
    x = np.arange(nx)
    g1 = A * np.exp(-((x - nx / 2) / 6.0) ** 2)
    rho = np.broadcast_to(1.0 + g1, (4, nx)).ravel().copy()
    u = np.concatenate([np.broadcast_to(U + c * g1, (4, nx)).ravel(), np.zeros(4 * nx)])
    T = np.broadcast_to(1.0 + 0.4 * g1, (4, nx)).ravel().copy()
    s.set_fields(rho, u, T)
    t_hit = int((nx / 2) / (c + U))
    inc = left = 0.0
    for kk in range(int(1.6 * t_hit)):
        s.step(1)
        if kk == int(0.3 * t_hit) or kk > 1.3 * t_hit:
            p = s.fields()[3].reshape(4, nx)[0]
            p = p - p.mean()
            if kk == int(0.3 * t_hit):
                inc = np.abs(p).max()
            else:
                left = max(left, np.abs(p[: nx - 20]).max())
    assert left / inc < 0.02
    s.close()
