"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 path max relative error <= 1e-12 (populations, rho E);
FP32 path relative L2 of velocity and temperature <= 1e-5; immersed
boundary classification and CSR structure bit-exact."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _maxrel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.mark.parametrize("case_fn", [C.cylinder_c1, C.small_cylinder_periodic, C.small_sphere,
                                     C.naca_downscale, lambda: C.small_cylinder_periodic(method=0),
                                     C.ellipse_case])
def test_ib_setup_parity(case_fn):
    """Classification, spreading CSR, phi, W, X*, d_BV and CSR weights
    bit-exact."""
    case = case_fn()
    sim, geo = C.make_oracle(case)
    g = C.make_gpu(case, "fp64", geo)
    st = g.ib_setup()
    S = sim.ib
    assert np.array_equal(st["inside"], S.inside)
    assert np.array_equal(st["cell_id"], S.cell_id)
    assert np.array_equal(st["row_ptr"], S.row_ptr)
    assert np.array_equal(st["col"], S.col)
    # kernel weights use the correctly rounded cosine on both sides and the
    # sums run in the same order: the FP64 setup agrees bit for bit
    assert np.array_equal(st["phi"], S.phi)
    assert np.array_equal(st["W"], S.W)
    assert np.array_equal(st["Xstar"], S.Xstar)
    assert np.array_equal(st["dBV"], S.dBV)
    assert np.array_equal(st["wt"], S.wt)
    g.close()


@pytest.mark.parametrize("case_fn,steps,method", [(C.small_cylinder_periodic, 1, 2), (C.small_cylinder_periodic, 30, 2),
                                                  (C.small_cylinder_periodic, 30, 1), (C.small_cylinder_periodic, 30, 0),
                                                  (C.small_sphere, 1, 2), (C.small_sphere, 10, 2),
                                                  (C.small_sphere, 10, 0)])
def test_fp64_step_parity_perturbed(case_fn, steps, method):
    """FP64 path vs oracle from a seeded perturbed state, with the body, for
    FODIBM-R (2), FODIBM (1) and DIBM (0): max relative error of populations
    and rho E <= 1e-12."""
    case = case_fn(method=method)
    sim, geo = C.make_oracle(case)
    C.perturb(sim, seed=11)
    g = C.make_gpu(case, "fp64", geo)
    g.set_state(sim.f, sim.E)
    sim.run(steps)
    g.step(steps)
    f, E = g.state()
    assert _maxrel(f, sim.f) < 1e-12
    assert _maxrel(E, sim.E) < 1e-12
    wl = g.wall_loads(per_point=True)
    L = sim.last_loads
    assert np.max(np.abs(wl["F"] - L["F"])) < 1e-12 * max(1.0, np.abs(L["F"]).max())
    assert np.max(np.abs(wl["force"] - L["force"])) < 1e-11 * max(1.0, np.abs(L["force"]).max())
    g.close()


def test_fp64_cylinder_1000_steps():
    """The 2D cylinder case (200x100, D = 20, 64 points, Ma 0.2, Re 40,
    isothermal wall, uniform start), FP64: max relative error <= 1e-12
    after 1000 steps, wall loads to the same accuracy."""
    case = C.cylinder_c1()
    sim, geo = C.make_oracle(case)
    g = C.make_gpu(case, "fp64", geo)
    sim.run(1000)
    g.step(1000)
    f, E = g.state()
    assert _maxrel(f, sim.f) < 1e-12
    assert _maxrel(E, sim.E) < 1e-12
    wl = g.wall_loads()
    assert np.max(np.abs(wl["force"] - sim.last_loads["force"])) < 1e-12 * np.abs(sim.last_loads["force"]).max() * 10
    g.close()


@pytest.mark.parametrize("case_fn,steps", [(C.cylinder_c1, 300), (C.small_sphere, 50)])
def test_fp32_against_oracle(case_fn, steps):
    """FP32 path vs FP64 oracle: relative L2 of velocity and temperature
    <= 1e-5."""
    case = case_fn()
    sim, geo = C.make_oracle(case)
    g = C.make_gpu(case, "fp32", geo)
    sim.run(steps)
    g.step(steps)
    rho, u, T, p = g.fields()
    r0, u0, T0, p0 = sim.fields()
    assert _rel_l2(u, u0) < 1e-5
    assert _rel_l2(T, T0) < 1e-5
    assert _rel_l2(rho, r0) < 1e-5
    g.close()


def test_determinism():
    """Two runs of the same case are bit-identical (no float atomics)."""
    case = C.small_cylinder_periodic()
    sim, geo = C.make_oracle(case)
    a = C.make_gpu(case, "fp32", geo)
    b = C.make_gpu(case, "fp32", geo)
    a.step(50)
    b.step(50)
    fa, Ea = a.state()
    fb, Eb = b.state()
    assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb)


@pytest.mark.parametrize("lattice,precision", [("D2Q9", "fp32"), ("D3Q19", "fp32"), ("D3Q19", "fp64")])
def test_boundaries_in_kernel_match_separate_kernel(lattice, precision, monkeypatch):
    """The fused kernel's in-place far-field faces (equilibrium on inlet and
    far-field faces, the outlet written as a copy by its inner neighbour)
    equal the separate boundary kernel bit for bit."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    if lattice == "D2Q9":
        case = C.cylinder_c1()
    else:
        case = dict(lattice="D3Q19", shape=(40, 24, 24), mach=0.3, reynolds=100.0, ref_length=8.0,
                    bc=[C.BC_IN, C.BC_OUT, C.BC_FF, C.BC_FF, C.BC_FF, C.BC_FF], method=2,
                    geo=lambda th: inputs.icosphere((12.3, 12.1, 11.8), 8.0, 4, tbc=0, t_value=1.05 * th))
    out = []
    for sep in ("0", "1"):
        monkeypatch.setenv("LBMIB_BC_SEPARATE", sep)
        s = lbmib.Solver(case["lattice"], precision, case["shape"], mach=case["mach"], reynolds=case["reynolds"],
                         ref_length=case["ref_length"], method=case["method"], bc=case["bc"])
        s.set_geometry(case["geo"](s.constants()["theta_inf"]))
        s.step(25)
        s.check()
        out.append(s.state())
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_naca_downscale_fp32_against_oracle():
    """Airfoil case at its 512x256 downscale (NACA0012, chord 100, 256
    points, Ma 0.5, Re 5000, adiabatic wall, 2 degrees): FP32 path vs FP64
    oracle after 60 steps.  Fields: relative L2 of velocity and temperature
    <= 1e-5.  Wall distributions: the per-point Lagrangian force split into
    its normal part (wall pressure) and tangential part (skin friction),
    relative L2 <= 1e-4 each."""
    case = C.naca_downscale()
    sim, geo = C.make_oracle(case)
    g = C.make_gpu(case, "fp32", geo)
    sim.run(60)
    g.step(60)
    g.check()
    rho, u, T, p = g.fields()
    r0, u0, T0, p0 = sim.fields()
    assert _rel_l2(u, u0) < 1e-5
    assert _rel_l2(T, T0) < 1e-5
    wl = g.wall_loads(per_point=True)
    F, F0 = wl["F"], sim.last_loads["F"]
    n = np.asarray(geo["normals"])
    t = np.stack([-n[:, 1], n[:, 0]], axis=1)
    fn, fn0 = np.sum(F * n, axis=1), np.sum(F0 * n, axis=1)
    ft, ft0 = np.sum(F * t, axis=1), np.sum(F0 * t, axis=1)
    assert _rel_l2(fn, fn0) < 1e-4
    assert _rel_l2(ft, ft0) < 1e-4
    g.close()


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_step_graph_matches_eager_steps(lattice, monkeypatch):
    """lbm_step replays captured CUDA graphs (two steps, or one step from
    either buffer parity); the state equals eager stepping (LBMIB_NO_GRAPH=1)
    bit for bit, for even and odd step counts, single steps in a row and
    after the geometry is replaced.  The loads queued by
    lbm_get_wall_loads_async after each single step equal the synchronous
    lbm_get_wall_loads of that step."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    if lattice == "D2Q9":
        case = C.cylinder_c1()
    else:
        case = dict(lattice="D3Q19", shape=(40, 24, 24), mach=0.3, reynolds=100.0, ref_length=8.0,
                    bc=[C.BC_IN, C.BC_OUT, C.BC_FF, C.BC_FF, C.BC_FF, C.BC_FF], method=2,
                    geo=lambda th: inputs.icosphere((12.3, 12.1, 11.8), 8.0, 4, tbc=0, t_value=1.05 * th))
    out = []
    for off in ("0", "1"):
        monkeypatch.setenv("LBMIB_NO_GRAPH", off)
        s = lbmib.Solver(case["lattice"], "fp32", case["shape"], mach=case["mach"], reynolds=case["reynolds"],
                         ref_length=case["ref_length"], method=case["method"], bc=case["bc"])
        th = s.constants()["theta_inf"]
        s.set_geometry(case["geo"](th))
        s.step(7)
        s.step(4)
        rows = torch.zeros((5, 5), dtype=torch.float64).pin_memory()
        sync_loads = []
        for k in range(5):
            s.step(1)
            s.wall_loads_async(rows[k])
            wl = s.wall_loads()
            sync_loads.append(list(wl["force"]) + [0.0] * (3 - s.D) + [wl["heat"], wl["work"]])
        s.sync()
        assert np.array_equal(rows.numpy(), np.array(sync_loads))
        s.set_geometry(case["geo"](th))
        s.step(5)
        s.check()
        out.append(s.state())
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_moving_wall_couette_fp64_parity():
    """Two immersed flat walls, the upper one moving (non-zero velocity
    targets): FP64 path vs oracle after 300 steps, max relative error
    <= 1e-12."""
    from tests import test_oracle_couette as K
    from paper_2607_07432_b300 import lbmib
    sim, U = K._sim(2)
    g = lbmib.Solver("D2Q9", "fp64", (K.NX, K.NY), bc=[C.BC_P] * 4, **K.config())
    assert abs(g.constants()["u_mag"] - U) < 1e-15
    g.set_geometry(K.geometry(U, g.constants()["theta_inf"]))
    sim.run(300)
    g.step(300)
    f, E = g.state()
    assert _maxrel(f, sim.f) < 1e-12
    assert _maxrel(E, sim.E) < 1e-12
    g.close()


def test_rotating_cylinder_with_heat_flux_fp64_parity():
    """Rotating wall (velocity targets omega x r on every Lagrangian point)
    and a non-zero Neumann temperature condition (prescribed wall-normal
    gradient, Eq. virtualneu): FP64 path vs oracle after 200 steps, max
    relative error <= 1e-12."""
    from paper_2607_07432_b300 import inputs
    case = C.small_cylinder_periodic()

    def geo(th):
        g = inputs.cylinder((15.3, 16.4), 10.0, 32, tbc=1, t_value=0.004)
        r = g["X"] - np.array([15.3, 16.4])
        omega = 0.01
        g["u_target"] = np.stack([-omega * r[:, 1], omega * r[:, 0]], axis=1)
        return g
    case["geo"] = geo
    sim, g0 = C.make_oracle(case)
    g = C.make_gpu(case, "fp64", g0)
    sim.run(200)
    g.step(200)
    f, E = g.state()
    assert _maxrel(f, sim.f) < 1e-12
    assert _maxrel(E, sim.E) < 1e-12
    wl = g.wall_loads(per_point=True)
    assert np.max(np.abs(wl["F"] - sim.last_loads["F"])) < 1e-12 * max(1.0, np.abs(sim.last_loads["F"]).max())
    g.close()


@pytest.mark.parametrize("zc", ["4", "7", "13"])
def test_z_chunk_length_does_not_change_the_state(zc, monkeypatch):
    """The planes per CTA of the 3D fused step (LBMIB_ZCHUNK; chosen from
    the grid and SM count otherwise) only partition the work: every chunk
    length, including ones that leave a ragged last chunk, gives the default
    state bit for bit (body, far-field boundaries, FP32)."""
    from paper_2607_07432_b300 import inputs, lbmib
    out = []
    for val in (None, zc):
        if val is None:
            monkeypatch.delenv("LBMIB_ZCHUNK", raising=False)
        else:
            monkeypatch.setenv("LBMIB_ZCHUNK", val)
        s = lbmib.Solver("D3Q19", "fp32", (40, 24, 30), mach=0.3, reynolds=100.0, ref_length=8.0,
                         bc=[C.BC_IN, C.BC_OUT, C.BC_FF, C.BC_FF, C.BC_FF, C.BC_FF])
        th = s.constants()["theta_inf"]
        s.set_geometry(inputs.icosphere((12.3, 12.1, 14.8), 8.0, 4, tbc=0, t_value=1.05 * th))
        s.step(9)
        out.append(s.state())
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
