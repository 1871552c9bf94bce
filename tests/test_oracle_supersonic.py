"""Pins of the a^C stencil readings (Eq. af2, reading Q6) on what the
mathematics fixes: the linear stability of one oracle step around a uniform
stream (spectrum of its Jacobian on a small periodic grid), and the order
and leading error of the differences against analytic derivatives."""
import numpy as np
import pytest
import sympy as sp

from oracle import lbm


def _sim(mach, theta, use_ac, nx=8, ny=4, angle_deg=0.0, ref_length=20.0):
    a = np.radians(angle_deg)
    prm = lbm.Params("D2Q9", (nx, ny), mach, 300.0, ref_length, theta_inf=theta,
                     inflow_dir=(np.cos(a), np.sin(a), 0.0), use_ac=use_ac)
    return lbm.Sim(prm)


def _pack(sim):
    dev = sim.devAF_prev
    return np.concatenate([sim.f.ravel(), sim.E.ravel(), sim.P_prev.ravel(), dev[0][0].ravel(), dev[0][1].ravel()])


def _unpack(sim, x):
    Q, zyx, N = sim.prm.lat.Q, sim.zyx, sim.E.size
    sim.f = x[:Q * N].reshape((Q,) + zyx).copy()
    o = Q * N
    sim.E = x[o:o + N].reshape(zyx).copy()
    sim.P_prev = x[o + N:o + 2 * N].reshape(zyx).copy()
    d00 = x[o + 2 * N:o + 3 * N].reshape(zyx).copy()
    d01 = x[o + 3 * N:o + 4 * N].reshape(zyx).copy()
    # the carried deviator is symmetric and traceless (reading Q8)
    sim.devAF_prev = [[d00, d01], [d01.copy(), -d00]]


def _spectrum(sim, eps=1e-7):
    """Eigenvalues and eigenvectors of the Jacobian of one step (populations,
    rho E, rho(1-theta) and the deviator of a^F carried to the next step),
    by central differences around the free-stream state."""
    x0 = _pack(sim)
    J = np.empty((x0.size, x0.size))
    for k in range(x0.size):
        h = eps * max(1.0, abs(x0[k]))
        out = []
        for s in (+1.0, -1.0):
            x = x0.copy()
            x[k] += s * h
            _unpack(sim, x)
            sim.step()
            out.append(_pack(sim))
        J[:, k] = (out[0] - out[1]) / (2.0 * h)
    return np.linalg.eig(J)


def test_central_stencil_odd_even_instability_above_sound_speed():
    """Central differences vanish on the odd-even mode along the stream; the
    step then amplifies it once the stream is faster than the sound speed
    (a real eigenvalue above 1 whose density pattern alternates in x and is
    uniform in y), and leaves it bounded below."""
    ev, V = _spectrum(_sim(1.2, 0.1, lbm.AC_FULL))
    i = int(np.argmax(np.abs(ev)))
    assert abs(ev[i]) > 1.05
    assert abs(ev[i].imag) < 1e-9 and ev[i].real > 0
    nx, ny, Q = 8, 4, 9
    rho = V[:Q * nx * ny, i].reshape(Q, ny, nx).sum(axis=0)
    spec = np.abs(np.fft.fft2(rho))
    assert np.unravel_index(np.argmax(spec), spec.shape) == (0, nx // 2)
    ev, _ = _spectrum(_sim(0.8, 0.1, lbm.AC_FULL))
    assert np.max(np.abs(ev)) <= 1.0 + 1e-7


def _sim16(mach, theta, angle_deg):
    a = np.radians(angle_deg)
    prm = lbm.Params("D2Q9", (16, 8), mach, 300.0, 16.0, theta_inf=theta, mu=0.01,
                     inflow_dir=(np.cos(a), np.sin(a), 0.0), use_ac=lbm.AC_UPWIND)
    return lbm.Sim(prm)


@pytest.mark.parametrize("mach,theta,angle", [(1.2, 0.1, 0.0), (2.0, 0.02, 0.0), (2.0, 0.05, 30.0), (0.5, 0.3, 0.0)])
def test_upstream_stencil_keeps_supersonic_streams_stable(mach, theta, angle):
    """With the a^C differences biased to the upstream side by the local
    Mach number (AC_UPWIND) no mode of a uniform stream grows, at Mach 1.2
    and 2 along an axis and obliquely, and below the sound speed."""
    ev, _ = _spectrum(_sim(mach, theta, lbm.AC_UPWIND, angle_deg=angle))
    assert np.max(np.abs(ev)) <= 1.0 + 1e-7


@pytest.mark.parametrize("mach,theta,angle", [(3.0, 0.02, 0.0), (4.0, 0.01, 30.0)])
def test_mach_weighted_stencil_stable_to_mach_4(mach, theta, angle):
    """Up to Mach 4 the Mach-weighted bias leaves no growing mode on a
    16 x 8 grid, which holds the slowly varying oblique modes that grow
    when the plain one-sided difference (the one-sided bias for every
    moving component, whatever its speed) is used instead."""
    ev, _ = _spectrum(_sim16(mach, theta, angle))
    assert np.max(np.abs(ev)) <= 1.0 + 1e-7
    saved = lbm.AC_UPWIND_CAP
    try:
        lbm.AC_UPWIND_CAP = 1.0
        sim = _sim16(mach, theta, angle)
        sim.prm.gamma = sim.prm.gamma * 1e-12   # u_b / c far beyond the cap: full one-sided bias
        ev2, _ = _spectrum(sim)
    finally:
        lbm.AC_UPWIND_CAP = saved
    assert np.max(np.abs(ev2)) > 1.0 + 1e-3


def _sym_fields(N):
    """Smooth periodic rho, u, theta on an N x N grid (wavelength N cells)."""
    X, Y = sp.symbols("X Y")
    k = 2 * sp.pi / N
    rho = 1 + sp.Rational(1, 10) * sp.sin(k * X + sp.Rational(3, 10)) * sp.cos(k * Y)
    ux = sp.Rational(3, 10) + sp.Rational(1, 10) * sp.sin(k * Y + 1) * sp.cos(k * X)
    uy = -sp.Rational(1, 5) + sp.Rational(1, 10) * sp.cos(k * X - sp.Rational(1, 2))
    th = sp.Rational(1, 2) + sp.Rational(1, 10) * sp.cos(k * X + k * Y)
    return (X, Y), rho, [ux, uy], th


def _on_grid(N, e, var):
    x = np.arange(N, dtype=np.float64)
    XX, YY = np.meshgrid(x, x, indexing="xy")   # arrays indexed [y, x]
    return np.broadcast_to(sp.lambdify(var, e, "numpy")(XX, YY), XX.shape).astype(np.float64)


def _derivative_parts(N, n):
    """n-th derivatives of P = rho(1-theta) along x and y and of rho u_a^3
    along a (n = 1 builds the analytic a^C), and u itself, on the grid."""
    var, rho, u, th = _sym_fields(N)
    P = rho * (1 - th)
    cs2 = sp.Rational(1, 3)
    dP = [_on_grid(N, sp.diff(P, var[b], n), var) for b in range(2)]
    cub = [_on_grid(N, sp.diff(rho * u[a] ** 3, var[a], n), var) for a in range(2)]
    un = [_on_grid(N, u[a], var) for a in range(2)]
    return dP, cub, un, float(cs2)


@pytest.mark.parametrize("N", [32, 64])
def test_lattice_correction_leading_errors(N):
    """a^C against its analytic value: the central form errs by the third
    derivatives / 6 (second order); the upstream-biased form adds -alpha_b/2
    of the second derivatives (first order, alpha_b the node's Mach number
    along b), so a bias to the wrong side, a dropped term or a swapped index
    leaves a residual of the size of the error itself here."""
    var, rho, u, th = _sym_fields(N)
    num = dict(rho=_on_grid(N, rho, var), u=np.stack([_on_grid(N, u[a], var) for a in range(2)]),
               th=_on_grid(N, th, var))
    dP1, cub1, un, cs2 = _derivative_parts(N, 1)
    dP2, cub2, _, _ = _derivative_parts(N, 2)
    dP3, cub3, _, _ = _derivative_parts(N, 3)

    def combine(dP, cub, wP=None, wc=None):
        out = [[None, None], [None, None]]
        for a in range(2):
            for b in range(2):
                tb = dP[b] * (1.0 if wP is None else wP[b])
                ta = dP[a] * (1.0 if wP is None else wP[a])
                v = cs2 * (un[a] * tb + un[b] * ta)
                if a == b:
                    v = v - cub[a] * (1.0 if wc is None else wc[a])
                out[a][b] = v
        return out

    exact = combine(dP1, cub1)
    # AC_UPWIND: D_b g = g_b + g_bbb / 6 - (alpha_b / 2) g_bb + O(1/N^4),
    # alpha_b = clip(u_b / sqrt(gamma R theta), -cap, cap)
    c = np.sqrt(1.4 * cs2 * num["th"])
    alpha = [np.clip(un[b] / c, -lbm.AC_UPWIND_CAP, lbm.AC_UPWIND_CAP) for b in range(2)]
    third = combine(dP3, cub3, [1.0 / 6.0] * 2, [1.0 / 6.0] * 2)
    bias = combine(dP2, cub2, [-0.5 * alpha[b] for b in range(2)], [-0.5 * alpha[b] for b in range(2)])
    pred = {lbm.AC_FULL: third,
            lbm.AC_UPWIND: [[third[a][b] + bias[a][b] for b in range(2)] for a in range(2)]}
    scale = max(np.abs(exact[a][b]).max() for a in range(2) for b in range(2))
    sim = _sim(0.3, 0.5, lbm.AC_FULL, nx=N, ny=N)
    for mode in (lbm.AC_FULL, lbm.AC_UPWIND):
        sim.prm.use_ac = mode
        aC = lbm.lattice_correction(sim.prm, sim.grid, num["rho"], num["u"], num["th"])
        for a in range(2):
            for b in range(2):
                err = aC[a][b] - exact[a][b]
                rest = err - pred[mode][a][b]
                assert np.abs(err).max() > 10 * np.abs(rest).max()
                if mode == lbm.AC_UPWIND:
                    assert np.abs(err).max() > 0.05 * scale / N
