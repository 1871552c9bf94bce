"""Wall diagnostics through the C ABI (lbm_get_wall_diagnostics) against the
oracle's (Sec. 3.1-3.2, reading Q26): body coefficients C_d, C_l, Nu and,
per Lagrangian point, C_p, tau_w, u^s, T^s and (dT/dn)^s of the updated
field.  FP64 path: the same values to round-off."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu

KEYS = ("Cp", "tau_w", "u_s", "T_s", "dTdn", "CpP")


def _check(gd, coeffs, per, atol):
    for k in ("Cd", "Cl", "Cl2", "Nu"):
        assert abs(gd[k] - coeffs[k]) <= atol * max(1.0, abs(coeffs[k])), (k, gd[k], coeffs[k])
    for k in KEYS:
        ref = np.asarray(per[k])
        err = np.max(np.abs(gd[k] - ref))
        assert err <= atol * max(1.0, np.abs(ref).max()), (k, err)


@pytest.mark.parametrize("case_fn,steps", [(C.small_cylinder_periodic, 40), (C.cylinder_c1, 300),
                                           (C.small_sphere, 12)])
def test_wall_diagnostics_fp64_parity(case_fn, steps):
    """FP64: C_d, C_l, Nu and every per-point quantity equal the oracle's to
    1e-11 (C_p amplifies the pressure difference by 1/q_inf)."""
    case = case_fn()
    sim, geo = C.make_oracle(case)
    g = C.make_gpu(case, "fp64", geo)
    sim.run(steps)
    g.step(steps)
    coeffs, per = sim.wall_diagnostics()
    _check(g.wall_diagnostics(), coeffs, per, 1e-11)
    g.close()


def test_wall_diagnostics_naca_inflow_angle():
    """The airfoil downscale at 2 degrees (adiabatic wall: Nu = 0, heat-flux
    diagnostics read (dT/dn)^s ~ 0): lift and drag axes follow the inflow
    direction, C_p and tau_w match the oracle."""
    case = C.naca_downscale()
    sim, geo = C.make_oracle(case)
    g = C.make_gpu(case, "fp64", geo)
    sim.run(5)
    g.step(5)
    coeffs, per = sim.wall_diagnostics()
    gd = g.wall_diagnostics()
    _check(gd, coeffs, per, 1e-11)
    assert gd["Nu"] == 0.0
    g.close()


def test_wall_diagnostics_fp32_close_to_fp64():
    """FP32 diagnostics of the small cylinder after 200 steps are close to the
    FP64 path's: per-point values within 1e-4 of the largest magnitude, C_d
    and C_l within 1e-4, Nu within 1e-3 (the heat of Eq. qib2 is
    C_v rho (T^t - T*), a difference of temperatures equal to about 1e-3
    near the wall, so FP32 rounding of T (1e-7) enters it at about 1e-4)."""
    case = C.small_cylinder_periodic()
    _, geo = C.make_oracle(case)
    out = []
    for prec in ("fp64", "fp32"):
        g = C.make_gpu(case, prec, geo)
        g.step(200)
        out.append(g.wall_diagnostics())
        g.close()
    a, b = out
    for k, tol in (("Cd", 1e-4), ("Cl", 1e-4), ("Nu", 1e-3)):
        assert abs(a[k] - b[k]) <= tol * max(1.0, abs(a[k])), k
    for k in KEYS:
        assert np.max(np.abs(a[k] - b[k])) <= 1e-4 * max(1e-3, np.abs(a[k]).max()), k
