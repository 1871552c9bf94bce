"""Hybrid compressible LBM time step, plain numpy FP64 (oracle).

Implements, in the paper's order and notation:
  * Eq. LB   pull-form lattice Boltzmann update with the shifted variable f-bar
  * Eq. fi   Guo-type force populations with the Hermite force moment a^{F,(2)}
  * Eq. feq  thermal equilibrium with the (w_i - delta_0i) rho (theta-1) term
  * Eq. fneq / pi2 / pi3   hybrid recursive regularized off-equilibrium
  * Eq. energy / deltata / fluxx-z / linear   total-energy equation with
    LB-consistent mass and momentum fluxes and MUSCL-Hancock face values
  * Sec. 2.5 steps 1-5 (IB forcing from oracle.ib, then LBM + energy)

Arrays are stored with the x axis last: a field has shape (ny, nx) in 2D and
(nz, ny, nx) in 3D; populations have a leading Q axis, vectors a leading D
axis.  Lattice units dx = dt = 1, c_s^2 = 1/3, T_ref = 1 (so theta = T and
R = c_s^2).

Readings where the paper is silent or garbled (each also listed in the
design notes of the repository):
  Q3  third-order Hermite terms use the orthogonal projection 1/N_k with
      N_k = sum_i w_i H3r_k,i^2 (2 c_s^6 for the '+' and 6 c_s^6 for the '-'
      D3Q19 combinations) in place of the printed single 1/(6 c_s^6).
  Q4  the trace projection in Eq. pi2 uses delta/D (delta/3 in 3D as printed).
  Q6  a^C (Eq. af2, only cited as the lattice-dependent component) is the
      second-order Hermite force moment that cancels, in the Chapman-Enskog
      expansion, the part of the momentum-flux relaxation the lattice gets
      wrong.  With the equilibrium of Eq. feq the lattice's third moment is
      c_s^2 rho (u_a d_bg + u_b d_ag + u_g d_ab) plus the off-diagonal
      rho u u u terms, not the Maxwellian's p/rho = c_s^2 theta form and not
      the diagonal rho u_a^3.  Expanding d_t Pi^(0) + d_g Q^(0) with the
      Euler equations then leaves, besides rho c_s^2 (grad u + grad u^T)
      (which with the literal tau_LB = nu/c_s^2 is the right shear stress
      at any theta), the trace terms Eq. af2 already carries explicitly
      ((2/D) rho c_s^2 div u, -c_s^2 d_t[rho(1-theta)]) and two terms a^C
      must remove:
          a^C_ab = c_s^2 (u_a d_b P + u_b d_a P) - d_ab d_a(rho u_a^3),
      P = rho(1-theta) (central differences, Q7).  The first part is the
      advective remainder of the theta defect (zero at theta = 1 up to the
      perturbation of theta), the second the diagonal cubic defect.
      PARITY UNPINNED against the paper (only cited); pinned by physics
      tests: sound attenuation equal at rest and in frames moving along and
      against the wave at theta = 1, 0.5 and 0.25 (D2Q9, D3Q19), no
      transverse velocity generated by a sound wave in a frame moving
      across it (the off-diagonal part), shear viscosity mu at any theta
      and frame, linear stability at low theta.  use_ac: AC_FULL (default),
      AC_CUBIC (the cubic term only: frame-dependent attenuation at
      theta != 1), AC_OFF, and AC_UPWIND: the AC_FULL terms with each
      difference along b biased to the upstream side in proportion to the
      node's Mach number along b (central for a slow component, one-sided at
      Mach 1, capped at 1.5 times the one-sided bias; lattice_correction).
      The paper gives no stencil for a^C.  With central differences a
      uniform stream faster than the sound speed is linearly unstable: on the
      odd-even mode along the stream every central difference vanishes, and
      what is left of the lattice part feeds a density perturbation back
      through its momentum flux (c^2 - u^2) d rho, whose sign turns at u = c
      (for a D1Q3 stream at temperature theta the mode's eigenvalues solve
      l^2 - w(1 - 2a) l - (1 - w) = 0, a = theta/3 - u^2, w = 1/tau-bar: a
      root above 1 exactly when a < 0).  Upstream-biased differences see the
      mode.  The Mach weighting with the cap 1.5 leaves uniform streams,
      along an axis and oblique, without growing modes up to Mach 4 while
      the lattice speed stays below about 0.35 (Mach 3 at theta 0.02, 2.5 at
      0.05, 4 at 0.01 and below), where a plain one-sided difference lets
      slowly varying oblique modes grow from Mach 2.5 (caps 1 and 1.25 from
      Mach 2.5-3, cap 2 from Mach 2 at theta 0.05); pinned by the Jacobian
      spectrum of one step.
  Q7  spatial derivatives are 2nd-order central (those of a^C upstream-
      biased under AC_UPWIND, Q6); time derivative of
      rho(1-theta) is the backward difference with the stored previous value.
  Q8  the F_i(t - dt) term of Eq. pi2 enters through its traceless second
      moment, the stored deviator of a^F of the previous step.
  Q9  tau_LB = nu / c_s^2 with nu = mu / rho (Eq. LB, default); a theta-scaled
      variant mu / (rho c_s^2 theta) is kept as an option, with the
      finite-difference part of Eq. pi2 scaled the same way.  The
      theta-scaled variant needs a theta correction in a^C that is an
      explicit anti-diffusion and is unstable for theta < 1; it is not the
      paper's scheme.
  Q12 face values of h, k and u_beta in the energy flux are the arithmetic
      mean of the two cells sharing the face.
  Q14 no limiter; sign(0) = 0; u_alpha ~ = 0 takes the '+' branch; the
      velocity in the face value and in eta is the reconstructing cell's.
  Q15 the IB energy forcing f_E = w + q is added once to rho E before the
      fluxes are formed.
  Q29 artificial bulk viscosity: the paper runs its shock cases with a low
      artificial bulk viscosity defined in its cited prior work; here a
      constant mu_b = bulk_ratio mu (default 0) enters the trace of Eq. af2
      as -2 mu_b div u (central differences), which adds mu_b to the zero
      bulk viscosity the trace terms give (pinned by sound attenuation).
  Q24 far field: inlet and far-field faces are reset to the free-stream
      equilibrium, the outlet is a zero-gradient copy; stencil reads
      outside a non-periodic axis are clamped to the edge node.
"""
import numpy as np

from . import lattice as L
from . import ib as IB

CS2 = L.CS2

BC_PERIODIC, BC_INLET, BC_OUTLET, BC_FARFIELD, BC_GHOST, BC_CHAR = 0, 1, 2, 3, 4, 5
TAU_THETA, TAU_LITERAL = 0, 1
# a^C readings (Q6): off, the diagonal cubic defect only, full (default)
AC_OFF, AC_CUBIC, AC_FULL, AC_UPWIND = 0, 1, 2, 3
# largest upstream weight of the AC_UPWIND differences (reading Q6)
AC_UPWIND_CAP = 1.5


def theta_inf_rule(mach, gamma, reynolds, ref_length, prandtl, dim):
    """Q11: T_ref is free (App. A: it sets the CFL number); theta_inf = T_inf/T_ref
    is the largest value <= 1 that keeps (a) u_inf = Ma sqrt(gamma c_s^2 theta)
    <= U_MAX and (b) the explicit conduction number kappa = lambda/(rho C_v)
    = mu gamma / Pr <= KAPPA_MAX[dim] (mu = u_inf L / Re scales with sqrt(theta))."""
    u1 = mach * np.sqrt(gamma * CS2)
    k1 = (u1 * ref_length / reynolds) * gamma / prandtl
    th = 1.0
    if u1 > U_MAX:
        th = min(th, (U_MAX / u1) ** 2)
    if k1 > KAPPA_MAX[dim]:
        th = min(th, (KAPPA_MAX[dim] / k1) ** 2)
    return th


U_MAX = 0.15
KAPPA_MAX = {2: 0.10, 3: 0.0667}


class Params:
    """Physical and numerical parameters, derived as in Sec. 3 / Q10-Q11.

    Re = rho_inf u_inf L / mu (Sec. 2.4), Ma = u_inf / c_inf with
    c_inf = sqrt(gamma R T_inf); Pr fixes lambda = mu C_p / Pr; C_v = R/(gamma-1).
    """

    def __init__(self, lattice, shape, mach, reynolds, ref_length, prandtl=0.71,
                 gamma=1.4, theta_inf=0.0, inflow_dir=(1.0, 0.0, 0.0), sigma=0.98,
                 d_n=1.5, method=IB.FODIBM_R, bc=None, tau_mode=TAU_LITERAL, use_ac=AC_FULL, mu=None, zoff=0,
                 bulk_ratio=0.0):
        self.lat = L.get(lattice)
        D = self.lat.D
        self.shape = tuple(int(s) for s in shape)  # (nx, ny[, nz])
        assert len(self.shape) == D
        self.gamma = gamma
        self.R = CS2
        self.Cv = self.R / (gamma - 1.0)
        self.Cp = gamma * self.R / (gamma - 1.0)
        self.theta_inf = (theta_inf if theta_inf > 0 else
                          theta_inf_rule(mach, gamma, reynolds, ref_length, prandtl, D))
        self.rho_inf = 1.0
        c_inf = np.sqrt(gamma * self.R * self.theta_inf)
        self.u_mag = mach * c_inf
        d = np.array(inflow_dir[:D], dtype=np.float64)
        d = d / np.sqrt((d * d).sum())
        self.u_inf = self.u_mag * d
        self.mu = self.rho_inf * self.u_mag * ref_length / reynolds if mu is None else float(mu)
        self.lam = self.mu * self.Cp / prandtl
        # artificial bulk viscosity (reading Q29): mu_b = bulk_ratio mu
        self.mu_b = float(bulk_ratio) * self.mu
        self.sigma = sigma
        self.d_n = d_n
        self.method = method
        self.tau_mode = tau_mode
        self.use_ac = use_ac
        if bc is None:
            bc = [BC_PERIODIC] * (2 * D)
        self.bc = list(bc)[: 2 * D]
        self.ref_length = ref_length
        # a z slab of a larger grid: global z of plane 0 (its faces towards
        # neighbour slabs have bc BC_GHOST: no boundary condition, edge reads
        # clamped, the planes refreshed from the neighbours between steps)
        self.zoff = int(zoff)


# --------------------------------------------------------------------------
# neighbour access with periodic wrap or edge clamping per axis
# --------------------------------------------------------------------------
class Grid:
    def __init__(self, prm):
        self.D = prm.lat.D
        self.n = prm.shape  # (nx, ny, nz)
        self.periodic = [prm.bc[2 * a] == BC_PERIODIC for a in range(self.D)]

    def idx(self, a, off):
        n = self.n[a]
        i = np.arange(n) + off
        if self.periodic[a]:
            return np.mod(i, n)
        return np.clip(i, 0, n - 1)

    def at(self, field, off):
        """field evaluated at x + off (off = (dx, dy[, dz])); field has the
        grid as its trailing axes (x last)."""
        D = self.D
        out = field
        for a in range(D):
            if off[a] == 0:
                continue
            out = np.take(out, self.idx(a, off[a]), axis=out.ndim - 1 - a)
        return out

    def unit(self, a, s=1):
        o = [0] * self.D
        o[a] = s
        return tuple(o)


# --------------------------------------------------------------------------
# equilibrium, forcing, regularized collision
# --------------------------------------------------------------------------
def equilibrium(lat, rho, u, theta):
    """Eq. feq: f^eq_i = w_i [rho + (w_i - d_0i)/w_i rho (theta - 1)
    + H1.rho u / c_s^2 + H2:rho u u / (2 c_s^4) + sum_k H3r_k A_k / N_k],
    with A_k the H3r combinations of rho u_a u_b u_g (reading Q3)."""
    D, Q = lat.D, lat.Q
    c = lat.c.astype(np.float64)
    feq = np.empty((Q,) + rho.shape)
    T3 = [[[rho * u[a] * u[b] * u[g] for g in range(D)] for b in range(D)] for a in range(D)]
    A = lat.combo3(T3)
    for i in range(Q):
        wi = lat.w[i]
        t0 = rho
        tth = ((wi - (1.0 if i == 0 else 0.0)) / wi) * rho * (theta - 1.0)
        t1 = sum(c[i, a] * rho * u[a] for a in range(D)) / CS2
        t2 = 0.0
        for a in range(D):
            for b in range(D):
                t2 = t2 + lat.H2(a, b)[i] * rho * u[a] * u[b]
        t2 = t2 / (2.0 * CS2 * CS2)
        t3 = 0.0
        for k in range(len(A)):
            t3 = t3 + lat.H3r[k, i] * A[k] / lat.N3r[k]
        feq[i] = wi * (t0 + tth + t1 + t2 + t3)
    return feq


def force_populations(lat, fu, aF):
    """Eq. fi: F_i = w_i [H1_a f_u,a / c_s^2 + H2_ab a^F_ab / (2 c_s^4)]."""
    D, Q = lat.D, lat.Q
    c = lat.c.astype(np.float64)
    F = np.empty((Q,) + fu.shape[1:])
    for i in range(Q):
        t1 = sum(c[i, a] * fu[a] for a in range(D)) / CS2
        t2 = 0.0
        for a in range(D):
            for b in range(D):
                t2 = t2 + lat.H2(a, b)[i] * aF[a][b]
        F[i] = lat.w[i] * (t1 + t2 / (2.0 * CS2 * CS2))
    return F


def regularized_neq(lat, u, Pi):
    """Eq. fneq with Eq. pi3: f-bar^neq_i = w_i [H2:Pi/(2 c_s^4)
    + sum_k H3r_k A_k^neq / N_k], A^neq = combos of
    Pi3_abg = u_a Pi_bg + u_b Pi_ga + u_g Pi_ab."""
    D, Q = lat.D, lat.Q
    T3 = [[[u[a] * Pi[b][g] + u[b] * Pi[g][a] + u[g] * Pi[a][b] for g in range(D)]
           for b in range(D)] for a in range(D)]
    A = lat.combo3(T3)
    out = np.empty((Q,) + u.shape[1:])
    for i in range(Q):
        t2 = 0.0
        for a in range(D):
            for b in range(D):
                t2 = t2 + lat.H2(a, b)[i] * Pi[a][b]
        t2 = t2 / (2.0 * CS2 * CS2)
        t3 = 0.0
        for k in range(len(A)):
            t3 = t3 + lat.H3r[k, i] * A[k] / lat.N3r[k]
        out[i] = lat.w[i] * (t2 + t3)
    return out


def deviator(lat, T):
    """Traceless part of a symmetric tensor, as carried between steps
    (reading Q8): its independent components T_ab - delta_ab tr/D (a <= b;
    the lower triangle mirrors the upper one, so the carried tensor is
    exactly symmetric), and the last diagonal component from the traceless
    condition (minus the sum of the other diagonal components), so that it
    is exactly traceless."""
    D = lat.D
    tr = sum(T[a][a] for a in range(D))
    out = [[T[a][b] - (tr / D if a == b else 0.0) for b in range(D)] for a in range(D)]
    for a in range(D):
        for b in range(a):
            out[a][b] = out[b][a]
    last = -out[0][0]
    for a in range(1, D - 1):
        last = last - out[a][a]
    out[D - 1][D - 1] = last
    return out


def lattice_correction(prm, grid, rho, u, theta):
    """a^C of Eq. af2 (reading Q6): c_s^2 (u_a d_b P + u_b d_a P)
    - d_ab d_a(rho u_a^3), P = rho(1-theta).  Central differences; under
    AC_UPWIND each difference along b adds an upstream-biased share of the
    second difference, D_b g = (g+ - g-)/2 - (alpha_b/2)(g+ - 2g + g-),
    weighted by the node's Mach number along b,
    alpha_b = clip(u_b / c, -AC_UPWIND_CAP, AC_UPWIND_CAP), c = sqrt(gamma R T):
    central where the component is slow, the one-sided difference at
    alpha = 1, more upstream weight beyond."""
    D = prm.lat.D
    aC = [[np.zeros_like(rho) for _ in range(D)] for _ in range(D)]
    if not prm.use_ac:
        return aC
    if prm.use_ac == AC_UPWIND:
        c = np.sqrt(prm.gamma * CS2 * theta)

    def diff(g, b):
        gp = grid.at(g, grid.unit(b, +1))
        gm = grid.at(g, grid.unit(b, -1))
        if prm.use_ac == AC_UPWIND:
            alpha = np.clip(u[b] / c, -AC_UPWIND_CAP, AC_UPWIND_CAP)
            return 0.5 * (gp - gm) - 0.5 * alpha * (gp - 2.0 * g + gm)
        return (gp - gm) * 0.5

    for a in range(D):
        aC[a][a] = -diff(rho * (u[a] * u[a] * u[a]), a)
    if prm.use_ac in (AC_FULL, AC_UPWIND):
        dP = [diff(rho * (1.0 - theta), b) for b in range(D)]
        for a in range(D):
            for b in range(D):
                aC[a][b] = aC[a][b] + CS2 * (u[a] * dP[b] + u[b] * dP[a])
    return aC


def collide(prm, grid, f, rho, u, theta, fu, P_prev, devAF_prev):
    """Sec. 2.2 / App. A collision at every node.

    Returns f^col = f^eq + (1 - 1/tau-bar) f-bar^neq + F/2 (Eq. LB with
    dt = 1), the new rho(1-theta) and the deviator of a^F (stored for the
    F(t - dt) term of the next step, reading Q8).
    """
    lat = prm.lat
    D = lat.D
    c = lat.c.astype(np.float64)
    # velocity gradient, central differences (Q7): du[a][b] = d u_a / d x_b
    du = [[(grid.at(u[a], grid.unit(b, +1)) - grid.at(u[a], grid.unit(b, -1))) * 0.5
           for b in range(D)] for a in range(D)]
    div = sum(du[a][a] for a in range(D))
    P = rho * (1.0 - theta)
    dPdt = P - P_prev
    aC = lattice_correction(prm, grid, rho, u, theta)
    # Eq. af2
    aF = [[None] * D for _ in range(D)]
    for a in range(D):
        for b in range(D):
            v = aC[a][b] + fu[a] * u[b] + fu[b] * u[a]
            if a == b:
                v = v + (2.0 / D) * rho * CS2 * div - CS2 * dPdt - (2.0 * prm.mu_b) * div
            aF[a][b] = v
    feq = equilibrium(lat, rho, u, theta)
    # relaxation time (Eq. LB, reading Q9)
    th_m = theta if prm.tau_mode == TAU_THETA else 1.0
    tau_lb = prm.mu / (rho * CS2 * th_m)
    tau_bar = tau_lb + 0.5
    # Eq. pi2 (HRR), traceless projection with delta/D (Q4)
    sig = prm.sigma
    Pi = [[None] * D for _ in range(D)]
    c2 = (c * c).sum(axis=1)
    for a in range(D):
        for b in range(D):
            proj = c[:, a] * c[:, b] - (c2 / D if a == b else 0.0)
            s = 0.0
            for i in range(lat.Q):
                s = s + proj[i] * (f[i] - feq[i])
            s = s + 0.5 * devAF_prev[a][b]
            S = du[a][b] + du[b][a] - ((2.0 / D) * div if a == b else 0.0)
            Pi[a][b] = sig * s - (1.0 - sig) * rho * CS2 * th_m * tau_bar * S
    fneq = regularized_neq(lat, u, Pi)
    F = force_populations(lat, fu, aF)
    fcol = feq + (1.0 - 1.0 / tau_bar) * fneq + 0.5 * F
    return fcol, P, deviator(lat, aF)


# --------------------------------------------------------------------------
# energy equation (Eq. energy, App. A)
# --------------------------------------------------------------------------
def lb_face_fluxes(prm, grid, fcol, axis):
    """Eqs. fluxx-z and the momentum rule below them: mass flux F^rho and
    momentum fluxes F^{rho u_b} through the face x + e_axis/2."""
    lat = prm.lat
    D = lat.D
    Frho = 0.0
    Fm = [0.0] * D
    for (i, off, coef) in lat.flux_table(axis):
        v = coef * grid.at(fcol[i], off)
        Frho = Frho + v
        for b in range(D):
            if lat.c[i, b] != 0:
                Fm[b] = Fm[b] + float(lat.c[i, b]) * v
    return Frho, Fm


def muscl_face(grid, phi, ua, axis):
    """Eq. linear: MUSCL-Hancock face value F*_{+axis/2}(phi) at x + e/2.

    Slope Delta = 1/2 {(1+eta)(phi - phi_{-1}) + (1-eta)(phi_{+1} - phi)},
    eta = (2u - sign(u))/3; phi_+- = phi +- Delta/2;
    phibar_+- = phi_+- + (u/2)(phi_- - phi_+); upwind on
    u~ = (u(x) + u(x+e))/2 >= 0.
    """
    e = grid.unit(axis, +1)
    m = grid.unit(axis, -1)
    eta = (2.0 * ua - np.sign(ua)) / 3.0
    delta = 0.5 * ((1.0 + eta) * (phi - grid.at(phi, m)) + (1.0 - eta) * (grid.at(phi, e) - phi))
    phi_p = phi + 0.5 * delta
    phi_m = phi - 0.5 * delta
    bar_p = phi_p + 0.5 * ua * (phi_m - phi_p)
    bar_m = phi_m + 0.5 * ua * (phi_m - phi_p)
    ut = 0.5 * (ua + grid.at(ua, e))
    return np.where(ut >= 0.0, bar_p, grid.at(bar_m, e))


def energy_update(prm, grid, fcol, rho, u, theta, E):
    """Eq. energy: (rho E)^{n+1} = (rho E) - sum_a delta_a F^{rho E}_{+a/2},
    with F^{rho E} = F*(rho H u_a) + (h - k)[F^rho - F*(rho u_a)]
    + u_b [F^{rho u_b} - F*(rho u_a u_b + p d_ab)] - lambda delta_a T(x + e_a).
    E here already contains the IB energy forcing (Q15)."""
    D = prm.lat.D
    p = rho * CS2 * theta
    h = prm.Cp * theta            # gamma R T / (gamma - 1), T = theta
    k = 0.5 * sum(u[b] * u[b] for b in range(D))
    Enew = E.copy()
    for a in range(D):
        e = grid.unit(a, +1)
        m = grid.unit(a, -1)
        Frho, Fm = lb_face_fluxes(prm, grid, fcol, a)
        ua = u[a]
        FH = muscl_face(grid, (E + p) * ua, ua, a)
        Fr = muscl_face(grid, rho * ua, ua, a)
        hk = 0.5 * ((h - k) + grid.at(h - k, e))
        FE = FH + hk * (Frho - Fr)
        for b in range(D):
            phib = rho * ua * u[b] + (p if a == b else 0.0)
            Fb = muscl_face(grid, phib, ua, a)
            ub = 0.5 * (u[b] + grid.at(u[b], e))
            FE = FE + ub * (Fm[b] - Fb)
        FE = FE - prm.lam * (grid.at(theta, e) - theta)
        Enew = Enew - (FE - grid.at(FE, m))
    return Enew


def stream(prm, grid, fcol):
    """Eq. LB pull form: f-bar_i(x, t+1) = f^col_i(x - c_i)."""
    lat = prm.lat
    out = np.empty_like(fcol)
    for i in range(lat.Q):
        out[i] = grid.at(fcol[i], tuple(-int(v) for v in lat.c[i]))
    return out


def freestream(prm, shape_zyx):
    lat = prm.lat
    D = lat.D
    rho = np.full(shape_zyx, prm.rho_inf)
    u = np.stack([np.full(shape_zyx, prm.u_inf[a]) for a in range(D)])
    th = np.full(shape_zyx, prm.theta_inf)
    f = equilibrium(lat, rho, u, th)
    E = rho * (0.5 * sum(u[a] ** 2 for a in range(D)) + prm.Cv * th)
    return f, E


def characteristic_face(prm, f, E, a, side):
    """Characteristic far field on the face (axis a, side) (Sec. 3.2;
    the paper cites characteristic boundaries without giving them): the face
    nodes take the equilibrium of the state built from the linearized
    one-dimensional Riemann invariants normal to the face,
        W+ = p + rho c u_n, W- = p - rho c u_n, W0 = rho - p / c^2, u_t,
    each taken from the interior neighbour when its characteristic leaves
    the domain (speed u_n + c, u_n - c, u_n, u_n > 0 with u_n along the
    outward normal) and from the free stream when it enters; rho c and c^2
    are the neighbour's.  Returns the face populations and rho E."""
    lat = prm.lat
    D = lat.D
    zyx = f.shape[1:]
    ax = len(zyx) - 1 - a
    n = zyx[ax]
    sl = [slice(None)] * len(zyx)
    sl[ax] = 1 if side == 0 else n - 2
    fi = f[(slice(None),) + tuple(sl)]
    Ei = E[tuple(sl)]
    c = lat.c.astype(np.float64)
    rho = np.zeros(fi.shape[1:])
    j = np.zeros((D,) + fi.shape[1:])
    for i in range(lat.Q):
        rho = rho + fi[i]
        for b in range(D):
            if c[i, b] != 0:
                j[b] = j[b] + c[i, b] * fi[i]
    u = j / rho
    th = (Ei / rho - 0.5 * (u * u).sum(axis=0)) / prm.Cv
    p = rho * prm.R * th
    cs = np.sqrt(prm.gamma * prm.R * th)
    sgn = -1.0 if side == 0 else 1.0
    un = sgn * u[a]
    un_inf = sgn * prm.u_inf[a]
    p_inf = prm.rho_inf * prm.R * prm.theta_inf
    rc = rho * cs
    c2 = cs * cs
    Wp = np.where(un + cs > 0.0, p + rc * un, p_inf + rc * un_inf)
    Wm = np.where(un - cs < 0.0, p_inf - rc * un_inf, p - rc * un)
    out = un > 0.0
    W0 = np.where(out, rho - p / c2, prm.rho_inf - p_inf / c2)
    pb = 0.5 * (Wp + Wm)
    unb = (Wp - Wm) / (2.0 * rc)
    rb = W0 + pb / c2
    ub = np.empty_like(u)
    for b in range(D):
        ub[b] = sgn * unb if b == a else np.where(out, u[b], prm.u_inf[b])
    thb = pb / (rb * prm.R)
    fb = equilibrium(lat, rb, ub, thb)
    Eb = rb * (0.5 * (ub * ub).sum(axis=0) + prm.Cv * thb)
    return fb, Eb


def apply_bc(prm, f, E):
    """Q24 far field on the outermost nodes of non-periodic axes: outlet faces
    copy the neighbouring inner plane first, then characteristic faces take
    the state of their Riemann invariants (computed from the state before
    any face is set), then inlet / far-field faces are set to the free-stream
    equilibrium (so edges and corners with them are free-stream); a node on
    two or more characteristic faces (an edge between them) is set to the
    free-stream equilibrium too."""
    D = prm.lat.D
    zyx = f.shape[1:]
    feq1, E1 = freestream(prm, ())
    chars = [(a, side) for a in range(D) for side in (0, 1) if prm.bc[2 * a + side] == BC_CHAR]
    assert not (chars and BC_OUTLET in prm.bc[:2 * D]), "characteristic faces are not combined with outlets"
    cvals = [characteristic_face(prm, f, E, a, side) for (a, side) in chars]
    for a in range(D):
        ax = len(zyx) - 1 - a
        for side in (0, 1):
            if prm.bc[2 * a + side] != BC_OUTLET:
                continue
            n = zyx[ax]
            sl_d = [slice(None)] * len(zyx)
            sl_s = [slice(None)] * len(zyx)
            sl_d[ax] = 0 if side == 0 else n - 1
            sl_s[ax] = 1 if side == 0 else n - 2
            f[(slice(None),) + tuple(sl_d)] = f[(slice(None),) + tuple(sl_s)]
            E[tuple(sl_d)] = E[tuple(sl_s)]
    for (a, side), (fb, Eb) in zip(chars, cvals):
        ax = len(zyx) - 1 - a
        sl = [slice(None)] * len(zyx)
        sl[ax] = 0 if side == 0 else zyx[ax] - 1
        f[(slice(None),) + tuple(sl)] = fb
        E[tuple(sl)] = Eb
    if len(chars) > 1:
        # edges between characteristic faces
        count = np.zeros(zyx, dtype=int)
        for (a, side) in chars:
            ax = len(zyx) - 1 - a
            sl = [slice(None)] * len(zyx)
            sl[ax] = 0 if side == 0 else zyx[ax] - 1
            count[tuple(sl)] += 1
        edge = count >= 2
        for i in range(prm.lat.Q):
            f[i][edge] = feq1[i]
        E[edge] = E1
    for a in range(D):
        ax = len(zyx) - 1 - a
        for side in (0, 1):
            if prm.bc[2 * a + side] not in (BC_INLET, BC_FARFIELD):
                continue
            n = zyx[ax]
            sl = [slice(None)] * len(zyx)
            sl[ax] = 0 if side == 0 else n - 1
            f[(slice(None),) + tuple(sl)] = feq1.reshape((prm.lat.Q,) + (1,) * (len(zyx) - 1))
            E[tuple(sl)] = E1


def lift_axes(ed, D):
    """Drag direction e_d (unit inflow direction) and the lift directions:
    2D e_d rotated by +90 degrees; 3D the y axis made orthogonal to e_d,
    then e_d x e_l1."""
    ed = np.asarray(ed, dtype=np.float64)[:D]
    if D == 2:
        return ed, np.array([-ed[1], ed[0]]), np.zeros(2)
    ey = np.array([0.0, 1.0, 0.0])
    l1 = ey - (ey @ ed) * ed
    l1 = l1 / np.sqrt(l1 @ l1)
    return ed, l1, np.cross(ed, l1)


class Sim:
    """Oracle state and the Sec. 2.5 time step.

    State: f (post-stream f-bar), E (rho E without the current IB forcing),
    P_prev (rho(1-theta) of the previous step), devAF_prev (deviator of
    a^F of the previous step), step counter.
    """

    def __init__(self, prm, geometry=None):
        self.prm = prm
        self.grid = Grid(prm)
        D = prm.lat.D
        self.zyx = tuple(reversed(prm.shape))
        self.f, self.E = freestream(prm, self.zyx)
        # Q25: the previous-step auxiliaries of the first step are those of
        # the initial state, rho(1 - theta) from its own moments
        self.reset_aux()
        self.devAF_prev = [[np.zeros(self.zyx) for _ in range(D)] for _ in range(D)]
        self.ib = None
        if geometry is not None:
            self.ib = IB.Setup(prm, self.grid, geometry)
        self.last_loads = None
        self.nstep = 0

    def reset_aux(self):
        """rho(1 - theta) of the current state as the previous-step value
        (a fresh start, reading Q25)."""
        rho, _, _, T = self.predicted()
        self.P_prev = rho * (1.0 - T)

    # Sec. 2.2: rho = sum f-bar, j = sum c f-bar (moments before forcing)
    def moments(self):
        """Sums in population order i = 0..Q-1 (no library reduction), so
        that near-zero momenta (far-field faces, symmetry lines) carry the
        same rounding as any other in-order evaluation; the sign of u enters
        the MUSCL slope (Eq. linear) discontinuously."""
        lat = self.prm.lat
        c = lat.c.astype(np.float64)
        rho = np.zeros(self.zyx)
        j = np.zeros((lat.D,) + self.zyx)
        for i in range(lat.Q):
            rho = rho + self.f[i]
            for a in range(lat.D):
                if c[i, a] != 0:
                    j[a] = j[a] + c[i, a] * self.f[i]
        return rho, j

    def predicted(self):
        """Predicted (pre-forcing) rho, rho u, u, T (Sec. 2.5 step 1)."""
        prm = self.prm
        rho, j = self.moments()
        u = j / rho
        T = (self.E / rho - 0.5 * (u * u).sum(axis=0)) / prm.Cv
        return rho, j, u, T

    def step(self):
        prm, grid = self.prm, self.grid
        D = prm.lat.D
        rho, j, ustar, Tstar = self.predicted()
        # Sec. 2.5 steps 1-4: interpolation, projection points, forces, spreading
        fu = np.zeros((D,) + self.zyx)
        wq = np.zeros(self.zyx)
        if self.ib is not None:
            fu, wq, self.last_loads = self.ib.force(rho, j, ustar, Tstar)
        # corrected macroscopic quantities (Sec. 2.2, Q15)
        u = (j + 0.5 * fu) / rho
        E = self.E + wq
        theta = (E / rho - 0.5 * (u * u).sum(axis=0)) / prm.Cv
        # Sec. 2.5 step 5: collision, energy fluxes, streaming, boundaries
        fcol, P, devAF = collide(prm, grid, self.f, rho, u, theta, fu, self.P_prev, self.devAF_prev)
        Enew = energy_update(prm, grid, fcol, rho, u, theta, E)
        fnew = stream(prm, grid, fcol)
        apply_bc(prm, fnew, Enew)
        self.f, self.E = fnew, Enew
        self.P_prev, self.devAF_prev = P, devAF
        self.nstep += 1

    def run(self, n):
        for _ in range(n):
            self.step()

    def wall_diagnostics(self):
        """Wall diagnostics of the current (updated) field (reading Q26):
        per point C_p, tau_w, u^s, T^s, (dT/dn)^s (oracle.ib), and the body
        coefficients C_d, C_l (and C_l2 in 3D) from the last step's loads
        and the Nusselt number from the heat into the fluid,
          C_d = F.e_d / (q_inf A),  A = L (2D) or pi L^2/4 (3D),
          Nu = heat L / (lambda (T_w - T_inf) S),  S = pi L (2D) or pi L^2 (3D),
        e_d the inflow direction, T_w the mean Dirichlet wall target, L the
        reference length (the diameter of a circle or sphere)."""
        prm = self.prm
        D = prm.lat.D
        rho, u, T, _ = self.fields()
        per = self.ib.diagnostics(rho, u, T)
        L = self.last_loads
        Lr = prm.ref_length
        q_inf = 0.5 * prm.rho_inf * prm.u_mag * prm.u_mag
        A = Lr if D == 2 else np.pi * Lr * Lr / 4.0
        S = np.pi * Lr if D == 2 else np.pi * Lr * Lr
        ed, el1, el2 = lift_axes(prm.u_inf / prm.u_mag, D)
        F = L["force"]
        coeffs = {"Cd": float(F @ ed) / (q_inf * A), "Cl": float(F @ el1) / (q_inf * A),
                  "Cl2": float(F @ el2) / (q_inf * A) if D == 3 else 0.0}
        dir_ = self.ib.tbc == IB.TBC_DIRICHLET
        if dir_.any():
            Tw = float(self.ib.tB[dir_].mean())
            coeffs["Nu"] = L["heat"] * Lr / (prm.lam * (Tw - prm.theta_inf) * S) if Tw != prm.theta_inf else 0.0
        else:
            coeffs["Nu"] = 0.0
        return coeffs, per

    def fields(self):
        """rho, u, T, p from the current state (predicted moments)."""
        rho, j, u, T = self.predicted()
        return rho, u, T, rho * self.prm.R * T
