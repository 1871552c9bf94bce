"""Two-level static refinement of the hybrid LBM step, plain numpy FP64
(oracle; test infrastructure, imported only by the tests and the
benchmark's CPU baseline).

The paper runs every case on locally refined meshes (Secs. 3.2-3.9: a box
around the body with the minimum spacing, coarser cells outside) but gives
no refinement algorithm.  This module is the reading adopted here, written
as plainly as the rest of the oracle:

  * Levels.  Level 0 covers the domain with spacing 1.  Level 1 refines the
    box of level-0 nodes [lo_a, hi_a] by 2: its node k along axis a sits at
    level-0 coordinate lo_a + (k - G)/2, so every other level-1 node
    coincides with a level-0 node.  Level 1 carries G ghost nodes beyond the
    box on every side (its faces have no boundary condition: edge reads
    are clamped, as on the ghost faces of a z slab).
  * Units (acoustic scaling).  dt_1 = dt_0 / 2, so lattice velocities, theta
    and the density are the same numbers on both levels, while mu and
    lambda in lattice units double on level 1 (its Reynolds number is taken
    on 2 L cells).  One step of level 0 is two steps of level 1.
  * Level 0 -> level-1 ghost nodes (space).  A ghost node takes the mean of
    the level-0 nodes around it: one node (both indices even), two (one odd)
    or four / eight (averages taken along x, then y, then z).  Averaged are
    the predicted moments rho, rho u, rho E and the off-equilibrium part
    f-bar_i - f^eq_i of every population; the populations are rebuilt as
    f^eq(rho, u, theta) + s_01 (f-bar - f^eq) with s_01 = tau-bar_1 /
    (2 tau-bar_0): the off-equilibrium part scales with tau-bar times the
    velocity gradient, whose lattice value halves on the finer level
    (tau-bar = mu / (rho c_s^2) + 1/2 on each level, Eq. LB with reading Q9).
  * Time.  The ghost state of the first level-1 step is level 0 at time n;
    that of the second step the mean of level 0 at n and n+1.  The stored
    previous-step values the level-1 step needs (rho(1-theta) of Eq. af2's
    backward difference, the deviator of a^F of Eq. pi2, reading Q8) come
    from level 0's own: rho(1-theta) at n - 1/2 as the mean of level 0's at
    n-1 and n, at n as level 0's at n; the a^F deviator, a velocity-gradient
    quantity, halved (its independent components averaged, the lower
    triangle mirrored and the last diagonal minus the others, as carried).
  * Level 1 -> level 0 (restriction).  Level-0 nodes at least R nodes inside
    the box take the coinciding level-1 node's state after its second step:
    populations f^eq + s_10 (f-bar - f^eq) with s_10 = 2 tau-bar_0 /
    tau-bar_1 from that node's predicted moments, rho E as is, and its
    rho(1-theta) and a^F deviator (doubled) at level-1 time n, which are
    level 0's previous-step values for its next step.
  * The energy equation is coupled through the same ghost and restriction
    values (no refluxing of face fluxes), and the body lives on level 1.

Every choice above is a reading (the paper is silent); the pins in
tests/test_oracle_refine.py check it against properties that hold
independently of it: a uniform stream is a fixed point, a decaying shear
wave across the interface decays at the viscous rate, and the two-level
solution of a smooth problem lies between the level-0-only and
level-1-only solutions.
"""
import numpy as np

from . import lbm

G = 4   # level-1 ghost nodes beyond the box on each side
R = 2   # restriction margin: level-0 nodes at least R nodes inside the box


def _tau_bar(prm, rho):
    th_m = 1.0  # reading Q9: tau_LB = nu / c_s^2
    return prm.mu / (rho * lbm.CS2 * th_m) + 0.5


class Refined:
    """Level 0 (the whole domain with its boundary conditions) and level 1
    (the box [lo, hi] of level-0 nodes refined by 2, G ghost nodes), built
    from the same case arguments as oracle.lbm.Params (Reynolds number and
    ref_length in level-0 cells).  theta_inf <= 0 applies reading Q11 to
    level 1 (ref_length 2 L there: its conduction number is the larger one)
    and both levels take that value."""

    def __init__(self, lattice, shape0, lo, hi, mach, reynolds, ref_length, prandtl=0.71, gamma=1.4,
                 theta_inf=0.0, inflow_dir=(1.0, 0.0, 0.0), sigma=0.98, d_n=1.5, method=lbm.IB.FODIBM_R,
                 bc=None, use_ac=lbm.AC_FULL, geometry1=None):
        D = 2 if lattice in ("D2Q9", 2) else 3
        self.D = D
        self.lo = [int(v) for v in lo[:D]]
        self.hi = [int(v) for v in hi[:D]]
        for a in range(D):
            assert self.lo[a] - G // 2 - 1 >= 0 and self.hi[a] + G // 2 + 1 <= shape0[a] - 1, \
                "the box and its ghost sources must lie inside level 0"
            assert self.hi[a] - self.lo[a] > 2 * R, "box too small"
        if theta_inf <= 0:
            theta_inf = lbm.theta_inf_rule(mach, gamma, reynolds, 2.0 * ref_length, prandtl, D)
        shape1 = tuple(2 * (self.hi[a] - self.lo[a]) + 1 + 2 * G for a in range(D))
        common = dict(mach=mach, reynolds=reynolds, prandtl=prandtl, gamma=gamma, theta_inf=theta_inf,
                      inflow_dir=inflow_dir, sigma=sigma, d_n=d_n, method=method, use_ac=use_ac)
        self.prm0 = lbm.Params(lattice, shape0, ref_length=ref_length, bc=bc, **common)
        self.prm1 = lbm.Params(lattice, shape1, ref_length=2.0 * ref_length, bc=[lbm.BC_GHOST] * (2 * D),
                               **common)
        self.s0 = lbm.Sim(self.prm0)
        self.s1 = lbm.Sim(self.prm1, geometry1)
        # level-1 ghost nodes (index arrays, x first) and the level-0 nodes
        # that coincide with the restricted level-1 nodes
        n1 = shape1
        grids = np.meshgrid(*[np.arange(n1[a]) for a in range(D)], indexing="ij")
        ghost = np.zeros(grids[0].shape, dtype=bool)
        for a in range(D):
            ghost |= (grids[a] < G) | (grids[a] >= n1[a] - G)
        self.gk = [grids[a][ghost] for a in range(D)]      # level-1 indices per axis
        rk = [np.arange(self.lo[a] + R, self.hi[a] - R + 1) for a in range(D)]
        rg = np.meshgrid(*rk, indexing="ij")
        self.rc = [rg[a].ravel() for a in range(D)]         # level-0 indices
        self.rf = [G + 2 * (self.rc[a] - self.lo[a]) for a in range(D)]
        self.nstep = 0

    def init_fields(self, fields):
        """Start both levels from the equilibrium of given fields:
        fields(X) -> (rho, u, theta) at level-0 coordinates X (a list of D
        arrays); level-1 node k sits at lo + (k - G)/2.  The previous-step
        rho(1-theta) is that of the start (reading Q25) and the a^F deviator
        zero."""
        D = self.D
        for sim, coords in ((self.s0, [np.arange(self.prm0.shape[a], dtype=np.float64) for a in range(D)]),
                            (self.s1, [self.lo[a] + (np.arange(self.prm1.shape[a]) - G) / 2.0
                                       for a in range(D)])):
            X = list(reversed(np.meshgrid(*reversed(coords), indexing="ij")))
            rho, u, th = fields(X)
            prm = sim.prm
            sim.f = lbm.equilibrium(prm.lat, rho, u, th)
            sim.E = rho * (0.5 * (u * u).sum(0) + prm.Cv * th)
            sim.P_prev = rho * (1.0 - th)
            sim.devAF_prev = [[np.zeros_like(rho) for _ in range(D)] for _ in range(D)]

    # ---------------------------------------------------------------- helpers
    def _zyx(self, idx):
        """numpy index tuple (z, y, x order) of per-axis index arrays."""
        return tuple(reversed(idx))

    def _interp(self, c):
        """Level-0 field c (zyx) at the level-1 ghost nodes: nested means
        along x, then y, then z."""
        D = self.D
        base, odd = [], []
        for a in range(D):
            v = self.gk[a] - G
            odd.append((v & 1) == 1)
            base.append(self.lo[a] + (v - (v & 1)) // 2)

        def val(off):
            return c[self._zyx([base[a] + off[a] for a in range(D)])]

        def along(a, off):
            # mean over axes < a+1 with the offsets of higher axes fixed
            if a < 0:
                return val(off)
            o0 = list(off)
            o1 = list(off)
            o1[a] = 1
            v0 = along(a - 1, o0)
            v1 = along(a - 1, o1)
            return np.where(odd[a], 0.5 * (v0 + v1), v0)

        return along(D - 1, [0] * D)

    def _neq_parts(self, sim):
        """Predicted moments and f-bar - f^eq of every node of a level."""
        rho, j, u, T = sim.predicted()
        feq = lbm.equilibrium(sim.prm.lat, rho, u, T)
        return rho, j, sim.E, sim.f - feq

    def _dev_components(self):
        D = self.D
        return [(a, b) for a in range(D) for b in range(a, D) if not (a == b == D - 1)]

    def _expand(self, comp):
        """Carried deviator from its independent components (reading Q8:
        lower triangle mirrored, last diagonal minus the other ones)."""
        D = self.D
        T = [[None] * D for _ in range(D)]
        for (a, b), v in comp.items():
            T[a][b] = v
            T[b][a] = v
        last = -T[0][0]
        for a in range(1, D - 1):
            last = last - T[a][a]
        T[D - 1][D - 1] = last
        return T

    # ------------------------------------------------------------ transfers
    def ghost_state(self):
        """Level-1 ghost populations and rho E from level 0's current state."""
        prm0, prm1 = self.prm0, self.prm1
        lat = prm0.lat
        D = self.D
        rho0, j0, E0, neq0 = self._neq_parts(self.s0)
        rho = self._interp(rho0)
        j = np.stack([self._interp(j0[a]) for a in range(D)])
        E = self._interp(E0)
        u = j / rho
        T = (E / rho - 0.5 * (u * u).sum(axis=0)) / prm0.Cv
        feq = lbm.equilibrium(lat, rho, u, T)
        s01 = _tau_bar(prm1, rho) / (2.0 * _tau_bar(prm0, rho))
        f = np.stack([feq[i] + s01 * self._interp(neq0[i]) for i in range(lat.Q)])
        return f, E

    def fill(self, f, E, P_prev, A_comp):
        """Write a ghost state into level 1."""
        idx = self._zyx(self.gk)
        s1 = self.s1
        for i in range(self.prm1.lat.Q):
            s1.f[i][idx] = f[i]
        s1.E[idx] = E
        s1.P_prev[idx] = P_prev
        T = self._expand(A_comp)
        for a in range(self.D):
            for b in range(self.D):
                s1.devAF_prev[a][b][idx] = T[a][b]

    def restrict(self, P1, A1):
        """Level-1 state at the restricted nodes into level 0 (P1, A1: level
        1's rho(1-theta) and a^F deviator components at level-1 time n)."""
        prm0, prm1 = self.prm0, self.prm1
        lat = prm0.lat
        D = self.D
        fi = self._zyx(self.rf)
        ci = self._zyx(self.rc)
        rho, j, u, T = self.s1.predicted()
        rho, u, T = rho[fi], np.stack([u[a][fi] for a in range(D)]), T[fi]
        feq = lbm.equilibrium(lat, rho, u, T)
        s10 = 2.0 * _tau_bar(prm0, rho) / _tau_bar(prm1, rho)
        for i in range(lat.Q):
            self.s0.f[i][ci] = feq[i] + s10 * (self.s1.f[i][fi] - feq[i])
        self.s0.E[ci] = self.s1.E[fi]
        self.s0.P_prev[ci] = P1
        T0 = self._expand({k: 2.0 * v for k, v in A1.items()})
        for a in range(D):
            for b in range(D):
                self.s0.devAF_prev[a][b][ci] = T0[a][b]

    # ------------------------------------------------------------------ step
    def step(self):
        """One level-0 step (two level-1 steps)."""
        D = self.D
        comps = self._dev_components()
        s0, s1 = self.s0, self.s1
        P_old = s0.P_prev.copy()
        A_old = {k: s0.devAF_prev[k[0]][k[1]].copy() for k in comps}
        fa, Ea = self.ghost_state()                       # level 0 at n
        s0.step()                                         # level 0: n -> n+1
        P_new = s0.P_prev
        A_new = {k: s0.devAF_prev[k[0]][k[1]] for k in comps}
        # first level-1 step (n -> n + 1/2): previous values at n - 1/2
        P1 = 0.5 * (self._interp(P_old) + self._interp(P_new))
        A1 = {k: 0.25 * (self._interp(A_old[k]) + self._interp(A_new[k])) for k in comps}
        self.fill(fa, Ea, P1, A1)
        s1.step()
        fi = self._zyx(self.rf)
        P1n = s1.P_prev[fi].copy()
        A1n = {k: s1.devAF_prev[k[0]][k[1]][fi].copy() for k in comps}
        # second level-1 step (n + 1/2 -> n + 1): ghost state at n + 1/2
        fb, Eb = self.ghost_state()                       # level 0 at n+1
        P2 = self._interp(P_new)
        A2 = {k: 0.5 * self._interp(A_new[k]) for k in comps}
        self.fill(0.5 * (fa + fb), 0.5 * (Ea + Eb), P2, A2)
        s1.step()
        self.restrict(P1n, A1n)
        self.nstep += 1

    def run(self, n):
        for _ in range(n):
            self.step()

