"""Couette pin of the oracle's immersed-boundary step: two flat immersed
walls (Lagrangian points along y = y0 and y = y1, solid outside the
channel), the lower one at rest and the upper one moving with the
free-stream speed U, fluid starting at U everywhere.  The start-up has the
closed form u(eta, t) = U eta + sum_n 2U/(n pi) sin(n pi eta)
exp(-(n pi)^2 nu t / H^2), eta = (y - y0)/H, and the steady state is the
linear profile.  A diffuse interface places the effective walls within a
fraction of a cell of the points, so the bars are a few percent of U, the
target-value reconstruction (FODIBM-R, Sec. 2.4) must beat the plain
direct-forcing method (DIBM), and the steady profile must be a straight
line whatever the wall offset."""
import numpy as np
import pytest

from oracle import ib as IB
from oracle import lbm

NX, NY, Y0, Y1, MU = 4, 32, 8.3, 23.7, 0.08
H = Y1 - Y0


MACH, THETA = 0.1, 0.25              # T_inf = T_ref / 4 keeps the explicit conduction stable at this mu
U_MAG = MACH * np.sqrt(1.4 / 3.0 * THETA)   # Ma c_inf
REYNOLDS = U_MAG * H / MU                   # gives mu = MU


def config():
    """Solver parameters shared with the GPU parity test."""
    return dict(mach=MACH, reynolds=REYNOLDS, ref_length=H, theta_inf=THETA)


def geometry(U, th):
    X = np.array([[x + 0.5, Y0] for x in range(NX)] + [[x + 0.5, Y1] for x in range(NX)])
    N = np.array([[0.0, 1.0]] * NX + [[0.0, -1.0]] * NX)
    ut = np.array([[0.0, 0.0]] * NX + [[U, 0.0]] * NX)
    yy = np.arange(NY)[:, None] * np.ones((1, NX))
    mask = ((yy < Y0) | (yy > Y1)).astype(np.uint8)
    return dict(X=X, normals=N, shape=dict(kind="mask", mask=mask), tbc=np.zeros(2 * NX, dtype=np.int64),
                t_value=np.full(2 * NX, th), u_target=ut)


def _sim(method):
    prm = lbm.Params("D2Q9", (NX, NY), method=method, **config())
    assert abs(prm.mu - MU) < 1e-15
    return lbm.Sim(prm, geometry(prm.u_mag, prm.theta_inf)), prm.u_mag


def _exact(eta, t, U):
    s = U * eta
    for n in range(1, 400):
        s = s + 2 * U / (n * np.pi) * np.sin(n * np.pi * eta) * np.exp(-(n * np.pi) ** 2 * MU * t / H ** 2)
    return s


def _profile(sim):
    _, u, _, _ = sim.fields()
    return u[0][:, 1]


YS = np.arange(NY)
INNER = (YS > Y0 + 1) & (YS < Y1 - 1)
ETA = (YS - Y0) / H


def test_startup_error_and_method_ordering():
    t = int(0.2 * H * H / MU)
    errs = {}
    for m in (IB.FODIBM_R, IB.DIBM):
        sim, U = _sim(m)
        sim.run(t)
        errs[m] = np.abs(_profile(sim) - _exact(ETA, t, U))[INNER].max() / U
    assert errs[IB.FODIBM_R] < 0.05
    assert errs[IB.FODIBM_R] < 0.7 * errs[IB.DIBM]


@pytest.mark.timeout(300)
def test_steady_profile_is_linear():
    sim, U = _sim(IB.FODIBM_R)
    t = int(1.5 * H * H / MU)
    sim.run(t)
    u = _profile(sim)
    assert np.abs(u - _exact(ETA, t, U))[INNER].max() < 0.035 * U
    # a straight line through the interior, whatever the effective wall offsets
    c = np.polyfit(YS[INNER], u[INNER], 1)
    assert np.abs(np.polyval(c, YS[INNER]) - u[INNER]).max() < 0.005 * U
    # and its slope is U over a channel within a cell of the nominal height
    assert abs(U / c[0] - H) < 1.0


@pytest.mark.timeout(300)
def test_viscous_heating_profile():
    """Couette flow with viscous heating (both walls isothermal at T_w, the
    upper one moving at Ma 0.3): the steady temperature is the parabola
    T_w + (mu U^2 / 2 lambda) eta (1 - eta).  Checked locally, where the
    diffuse walls do not enter: the interior profile is a parabola (fit
    residual below 1e-4 of the rise) whose curvature balances the viscous
    work, lambda T'' = -mu (du/dy)^2, with the measured shear rate (within
    0.5%; measured 3e-5); the peak rise is mu U^2 / (8 lambda) within 10%
    (the effective walls sit about half a cell inside the points, which
    raises the shear rate by 6%).  This pins the viscous work carried into
    the energy equation by the LB momentum fluxes of Eq. energy and the
    conductivity lambda = mu C_p / Pr."""
    mach = 0.3
    U = mach * np.sqrt(1.4 / 3.0 * THETA)
    prm = lbm.Params("D2Q9", (NX, NY), method=IB.FODIBM_R, mach=mach, reynolds=U * H / MU, ref_length=H,
                     theta_inf=THETA)
    sim = lbm.Sim(prm, geometry(prm.u_mag, prm.theta_inf))
    sim.run(4000)
    _, u, T, _ = sim.fields()
    ux, Ty = u[0][:, 1], T[:, 1]
    Y = YS[INNER]
    cu = np.polyfit(Y, ux[INNER], 1)
    cT = np.polyfit(Y, Ty[INNER], 2)
    rise = Ty[INNER].max() - THETA
    assert np.abs(np.polyval(cT, Y) - Ty[INNER]).max() < 1e-4 * rise
    assert abs(2 * cT[0] / (-prm.mu * cu[0] ** 2 / prm.lam) - 1.0) < 5e-3
    assert abs(rise / (prm.mu * prm.u_mag ** 2 / (8 * prm.lam)) - 1.0) < 0.10
