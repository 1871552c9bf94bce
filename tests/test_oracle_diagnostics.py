"""Pins of the oracle's wall diagnostics (Sec. 3.1-3.2 and reading Q26):
C_p, u^s, T^s by Eq. int1 at d = 2 over Omega, tau_w and (dT/dn)^s from the
projection point (Eq. int1, d = 1).  CPU only."""
import math

import numpy as np

from oracle import ib, lbm


def _wall_case(a=0.3):
    """Periodic channel 16 x 24 with a flat wall at y = 10 + a (one point per
    column, points at x + 0.3), normals +y, fluid above."""
    nx, ny = 16, 24
    X = np.stack([np.arange(nx, dtype=float) + 0.3, np.full(nx, 10.0 + a)], axis=1)
    N = np.tile([0.0, 1.0], (nx, 1))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    geo = dict(X=X, normals=N, shape=dict(kind="mask", mask=yy < 10.0 + a), tbc=np.zeros(nx, int),
               t_value=np.ones(nx), u_target=np.tile([0.02, 0.0], (nx, 1)))
    prm = lbm.Params("D2Q9", (nx, ny), mach=0.2, reynolds=40, ref_length=10, method=ib.FODIBM_R,
                     bc=[lbm.BC_PERIODIC] * 4)
    return prm, ib.Setup(prm, lbm.Grid(prm), geo), (yy, xx)


def _m1(a):
    return 0.25 * ((2 - 4 * a) + 2 * math.sin(math.pi * a / 2) - 2 * math.cos(math.pi * a / 2))


def test_uniform_field_is_read_exactly():
    """A uniform field is read back exactly at every point (partition of
    unity of the two-sided d = 2 and d = 1 stencils): C_p of the free-stream
    pressure is 0, of a pressure raised by dp is dp/q_inf; u^s = u, T^s = T,
    (dT/dn)^s = 0 and tau_w = mu (u - u^B)_t / d_n."""
    prm, S, (yy, xx) = _wall_case()
    rho = np.full(yy.shape, 1.0)
    T = np.full(yy.shape, prm.theta_inf)
    u = np.stack([np.full(yy.shape, 0.05), np.full(yy.shape, -0.01)])
    d = S.diagnostics(rho, u, T)
    assert np.abs(d["Cp"]).max() < 1e-13
    assert np.abs(d["u_s"] - [0.05, -0.01]).max() < 1e-15
    assert np.abs(d["T_s"] - prm.theta_inf).max() < 1e-15
    assert np.abs(d["dTdn"]).max() < 1e-13
    assert np.allclose(d["tau_w"][:, 0], prm.mu * (0.05 - 0.02) / prm.d_n, rtol=1e-13)
    assert np.abs(d["tau_w"][:, 1]).max() < 1e-16          # the normal part is removed
    q_inf = 0.5 * prm.rho_inf * prm.u_mag ** 2
    d2 = S.diagnostics(rho * 1.01, u, T)
    assert np.allclose(d2["Cp"], 0.01 * prm.R * prm.theta_inf / q_inf, rtol=1e-12)
    assert np.allclose(d2["CpP"], 0.01 * prm.R * prm.theta_inf / q_inf, rtol=1e-12)


def test_linear_field_error_is_the_kernel_first_moment():
    """A field linear in y is read at X_l with the error slope * M1(frac(Y))
    of the d = 2 kernel's closed-form first moment (two-sided stencil: the
    body does not cut it)."""
    a = 0.3
    prm, S, (yy, xx) = _wall_case(a)
    s = 1e-3
    T = prm.theta_inf + s * yy
    d = S.diagnostics(np.ones(yy.shape), np.zeros((2,) + yy.shape), T)
    exact = prm.theta_inf + s * (10.0 + a)
    assert np.allclose(d["T_s"] - exact, s * _m1(a), atol=1e-15)


def test_shear_and_normal_gradient_with_projection_on_nodes():
    """With the projection point on a node (wall at y = 3.5 + offset with
    d_n = 1.5 puts P at y = 5), Eq. int1 at d = 1 reads that node exactly:
    for u_x = g y, tau_w = mu (5 g - u^B_x) / d_n; for T = T0 + h y,
    (dT/dn)^s = (T(5) - T^s) / d_n with T^s = T0 + h (3.5 + M1(0.5))."""
    nx, ny = 12, 16
    X = np.stack([np.arange(nx, dtype=float), np.full(nx, 3.5)], axis=1)
    N = np.tile([0.0, 1.0], (nx, 1))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    geo = dict(X=X, normals=N, shape=dict(kind="mask", mask=yy < 3.5), tbc=np.zeros(nx, int),
               t_value=np.ones(nx), u_target=np.zeros((nx, 2)))
    prm = lbm.Params("D2Q9", (nx, ny), mach=0.2, reynolds=40, ref_length=10, bc=[lbm.BC_PERIODIC] * 4)
    S = ib.Setup(prm, lbm.Grid(prm), geo)
    g, h, T0 = 2e-3, 1e-3, 0.8
    u = np.stack([g * yy, np.zeros(yy.shape)])
    d = S.diagnostics(np.ones(yy.shape), u, T0 + h * yy)
    assert np.allclose(d["tau_w"][:, 0], prm.mu * 5 * g / 1.5, rtol=1e-13)
    Ts = T0 + h * (3.5 + _m1(0.5))
    assert np.allclose(d["T_s"], Ts, atol=1e-15)
    assert np.allclose(d["dTdn"], (T0 + 5 * h - Ts) / 1.5, atol=1e-14)


def test_body_coefficients_from_loads():
    """C_d, C_l and Nu follow from the last step's Lagrangian loads: for a
    cylinder in a flow at 30 degrees the force projected on the inflow axis
    and its normal reproduces the force vector, and Nu has the sign of
    T_w - T_inf times the heat into the fluid."""
    from paper_2607_07432_b300 import inputs
    ang = np.deg2rad(30.0)
    geo = inputs.cylinder((16.3, 15.6), 10.0, 32, tbc=0, t_value=1.05)
    prm = lbm.Params("D2Q9", (36, 32), mach=0.2, reynolds=30, ref_length=10, method=ib.FODIBM_R,
                     inflow_dir=(math.cos(ang), math.sin(ang), 0.0))
    sim = lbm.Sim(prm, geo)
    sim.run(3)
    c, per = sim.wall_diagnostics()
    q = 0.5 * prm.rho_inf * prm.u_mag ** 2 * prm.ref_length
    F = c["Cd"] * q * np.array([math.cos(ang), math.sin(ang)]) + c["Cl"] * q * np.array([-math.sin(ang), math.cos(ang)])
    assert np.allclose(F, sim.last_loads["force"], rtol=1e-12)
    assert c["Nu"] * (1.05 - prm.theta_inf) * sim.last_loads["heat"] >= 0
    assert per["Cp"].shape == (32,) and per["tau_w"].shape == (32, 2)
