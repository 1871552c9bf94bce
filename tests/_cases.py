"""Shared case builders for the parity tests: the same seeded inputs go to
the CUDA path (through the C ABI binding) and to the CPU oracle."""
import numpy as np

from paper_2607_07432_b300 import inputs

BC_P, BC_IN, BC_OUT, BC_FF = 0, 1, 2, 3


def cylinder_c1(n_points=64, tw=None, method=2):
    """2D cylinder: grid 200x100, D = 20 at (60, 50), 64 points, Ma 0.2, Re 40,
    isothermal wall at 1.1 T_inf (T_inf from the theta rule), inlet/outlet
    in x, far field in y."""
    return dict(lattice="D2Q9", shape=(200, 100), mach=0.2, reynolds=40.0, ref_length=20.0,
                bc=[BC_IN, BC_OUT, BC_FF, BC_FF], method=method,
                geo=lambda th: inputs.cylinder((60.0, 50.0), 20.0, n_points, tbc=0,
                                               t_value=1.1 * th if tw is None else tw))


def small_cylinder_periodic(method=2):
    return dict(lattice="D2Q9", shape=(40, 32), mach=0.2, reynolds=30.0, ref_length=10.0,
                bc=[BC_P] * 4, method=method,
                geo=lambda th: inputs.cylinder((15.3, 16.4), 10.0, 32, tbc=0, t_value=1.05 * th))


def ellipse_case(method=2):
    """Rotated ellipse (aspect 2.5) on a 96x64 grid: exercises the ellipse
    classification predicate."""
    return dict(lattice="D2Q9", shape=(96, 64), mach=0.3, reynolds=60.0, ref_length=30.0,
                bc=[BC_IN, BC_OUT, BC_FF, BC_FF], method=method,
                geo=lambda th: inputs.ellipse((40.3, 31.7), 15.0, 6.0, 0.6, 80, tbc=0, t_value=1.05 * th))


def small_sphere(method=2, bc=None):
    return dict(lattice="D3Q19", shape=(24, 20, 20), mach=0.2, reynolds=20.0, ref_length=8.0,
                bc=bc or [BC_IN, BC_OUT, BC_FF, BC_FF, BC_FF, BC_FF], method=method,
                geo=lambda th: inputs.icosphere((9.3, 10.1, 9.8), 8.0, 4, tbc=0, t_value=1.05 * th))


def naca_downscale(method=2, aoa_deg=2.0):
    """NACA0012 at the 512x256 downscale of the airfoil case: chord 100,
    256 points, Ma 0.5, Re 5000, adiabatic wall."""
    a = np.deg2rad(aoa_deg)
    return dict(lattice="D2Q9", shape=(512, 256), mach=0.5, reynolds=5000.0, ref_length=100.0,
                bc=[BC_IN, BC_OUT, BC_FF, BC_FF], method=method, inflow_dir=(np.cos(a), np.sin(a), 0.0),
                geo=lambda th: inputs.naca0012((128.0, 128.0), 100.0, 256, tbc=1, t_value=0.0))


def make_oracle(case):
    from oracle import lbm
    prm = lbm.Params(case["lattice"], case["shape"], mach=case["mach"], reynolds=case["reynolds"],
                     ref_length=case["ref_length"], method=case["method"], bc=case["bc"],
                     inflow_dir=case.get("inflow_dir", (1.0, 0.0, 0.0)))
    geo = case["geo"](prm.theta_inf) if case.get("geo") else None
    return lbm.Sim(prm, geo), geo


def make_gpu(case, precision, geo):
    from paper_2607_07432_b300 import lbmib
    s = lbmib.Solver(case["lattice"], precision, case["shape"], mach=case["mach"], reynolds=case["reynolds"],
                     ref_length=case["ref_length"], method=case["method"], bc=case["bc"],
                     inflow_dir=case.get("inflow_dir", (1.0, 0.0, 0.0)))
    if geo is not None:
        s.set_geometry(geo)
    return s


def perturb(sim, seed, amp=2e-3):
    """Seeded smooth-ish perturbation of the oracle's populations and energy
    (same arrays then go to the GPU through lbm_set_state)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sim.f = sim.f * (1.0 + amp * rng.standard_normal(sim.f.shape))
    sim.E = sim.E * (1.0 + amp * rng.standard_normal(sim.E.shape))
    rho, j, u, T = sim.predicted()
    sim.P_prev = rho * (1.0 - T)
