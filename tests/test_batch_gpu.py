"""Batched stepping (several uneven cases in one persistent launch or in one
launch per phase, graph replay) gives the same states bit for bit as
stepping each case alone; the autotuner leaves the state unchanged."""
import numpy as np
import pytest

from paper_2607_07432_b300 import inputs

pytestmark = pytest.mark.gpu

BC = [1, 2, 3, 3]


def _cases():
    specs = inputs.batch_cases(4, seed=20260001)
    cases, geos = [], []
    for k, c in enumerate(specs):
        nx, ny = min(c["nx"], 384), min(c["ny"], 192)
        cases.append(dict(shape=(nx, ny), mach=c["mach"], reynolds=c["reynolds"], ref_length=c["ref_length"],
                          bc=BC))
        geos.append(c)
    return cases, geos


def _geometry(c, spec, theta):
    nx, ny = c["shape"]
    center = (nx / 4.0 + 0.37, ny / 2.0 + 0.21)
    if spec["ellipse"]:
        return inputs.ellipse(center, spec["a"], spec["b"], spec["angle"], spec["n_points"], tbc=0,
                              t_value=1.05 * theta)
    return inputs.cylinder(center, 2 * spec["a"], spec["n_points"], tbc=0, t_value=1.05 * theta)


@pytest.mark.parametrize("form", [1, 0])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_equals_individual(precision, form):
    from paper_2607_07432_b300 import lbmib
    cases, specs = _cases()
    b = lbmib.Batch("D2Q9", precision, cases)
    assert b.launch_form() == 1    # 2D default: one persistent launch
    b.set_launch_form(form)
    solo = []
    for k, c in enumerate(cases):
        s = lbmib.Solver("D2Q9", precision, c["shape"], mach=c["mach"], reynolds=c["reynolds"],
                         ref_length=c["ref_length"], bc=BC)
        th = s.constants()["theta_inf"]
        geo = _geometry(c, specs[k], th)
        s.set_geometry(geo)
        b.case(k).set_geometry(geo)
        solo.append(s)
    for tile_rows, sched in [(0, 0), (16, 1), (0, 2), (32, 2)] if precision == "fp32" else [(0, 0)]:
        b.set_plan(tile_rows, sched)
        b.step(5)   # graph path (2 + 2) and one eager step
        for s in solo:
            s.step(5)
        b.sync()
        for k, s in enumerate(solo):
            fa, Ea = b.case(k).state()
            fb, Eb = s.state()
            assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb)
    b.step_sequential(3)
    for s in solo:
        s.step(3)
    for k, s in enumerate(solo):
        fa, Ea = b.case(k).state()
        fb, Eb = s.state()
        assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb)
    b.close()


def test_autotune_restores_state(tmp_path):
    from paper_2607_07432_b300 import lbmib
    cases, specs = _cases()
    b = lbmib.Batch("D2Q9", "fp32", cases)
    for k, c in enumerate(cases):
        th = b.case(k).constants()["theta_inf"]
        b.case(k).set_geometry(_geometry(c, specs[k], th))
    b.step(3)
    before = [b.case(k).state() for k in range(len(cases))]
    cache = str(tmp_path / "plans.txt")
    (plan, ms) = b.autotune(steps=4, cache_path=cache)
    assert ms > 0 and plan[0] in (0, 16) and plan[1] in (0, 1, 2)
    after = [b.case(k).state() for k in range(len(cases))]
    for (fa, Ea), (fb, Eb) in zip(before, after):
        assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb)
    # second call is served from the cache file
    plan2, _ = b.autotune(steps=4, cache_path=cache)
    assert plan2 == plan
    b.close()


def test_batched_3d_equals_individual():
    """Two uneven 3D sphere cases (different grids, points and Mach numbers)
    stepped together equal the same cases stepped alone, bit for bit."""
    from paper_2607_07432_b300 import lbmib
    bc3 = [1, 2, 3, 3, 3, 3]
    cases = [dict(shape=(40, 24, 24), mach=0.3, reynolds=100.0, ref_length=8.0, bc=bc3),
             dict(shape=(32, 20, 28), mach=0.2, reynolds=80.0, ref_length=7.0, bc=bc3)]
    geos = [lambda th: inputs.icosphere((12.3, 12.1, 11.8), 8.0, 4, tbc=0, t_value=1.05 * th),
            lambda th: inputs.icosphere((10.2, 9.7, 14.1), 7.0, 3, tbc=0, t_value=1.05 * th)]
    b = lbmib.Batch("D3Q19", "fp32", cases)
    assert b.launch_form() == 0
    with pytest.raises(lbmib.LBMError):
        b.set_launch_form(1)
    solo = []
    for k, c in enumerate(cases):
        s = lbmib.Solver("D3Q19", "fp32", c["shape"], mach=c["mach"], reynolds=c["reynolds"],
                         ref_length=c["ref_length"], bc=bc3)
        geo = geos[k](s.constants()["theta_inf"])
        s.set_geometry(geo)
        b.case(k).set_geometry(geo)
        solo.append(s)
    b.step(5)
    for s in solo:
        s.step(5)
    b.sync()
    for k, s in enumerate(solo):
        fa, Ea = b.case(k).state()
        fb, Eb = s.state()
        assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb)
        s.close()
    b.close()


def test_batched_full_grid_range_equals_individual():
    """The two ends of the sweep's grid range in one batch, 256x128 and
    1024x512 (FP32, characteristic far field on the outflow and lateral
    faces as well as the equilibrium far field), bit for bit against each
    case stepped alone."""
    from paper_2607_07432_b300 import lbmib
    specs = inputs.batch_cases(2, seed=20260001)
    cases = [dict(shape=(256, 128), mach=0.3, reynolds=80.0, ref_length=20.0, bc=BC),
             dict(shape=(1024, 512), mach=0.2, reynolds=150.0, ref_length=60.0, bc=[1, 5, 5, 5])]
    b = lbmib.Batch("D2Q9", "fp32", cases)
    solo = []
    for k, c in enumerate(cases):
        s = lbmib.Solver("D2Q9", "fp32", c["shape"], mach=c["mach"], reynolds=c["reynolds"],
                         ref_length=c["ref_length"], bc=c["bc"])
        th = s.constants()["theta_inf"]
        geo = _geometry(c, specs[k], th)
        s.set_geometry(geo)
        b.case(k).set_geometry(geo)
        solo.append(s)
    b.step(6)
    for s in solo:
        s.step(6)
    b.sync()
    for k, s in enumerate(solo):
        fa, Ea = b.case(k).state()
        fb, Eb = s.state()
        assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb)
        s.close()
    b.close()


def test_batched_mixed_stencils_equal_individual():
    """A batch whose cases differ in the a^C stencil and bulk viscosity (a
    cylinder with the central stencil; a seeded Mach 1.4 periodic stream
    with the Mach-weighted upstream stencil and mu_b = 2 mu) steps each case
    exactly as it steps alone."""
    from paper_2607_07432_b300 import lbmib
    bc = [1, 5, 5, 5]
    cases = [dict(shape=(96, 64), mach=0.3, reynolds=80.0, ref_length=16.0, bc=bc),
             dict(shape=(128, 64), mach=1.4, reynolds=200.0, ref_length=12.0, bc=[0] * 4, theta_inf=0.03,
                  use_ac=lbmib.AC_UPWIND, bulk_ratio=2.0)]
    b = lbmib.Batch("D2Q9", "fp32", cases)
    solo = []
    for k, c in enumerate(cases):
        s = lbmib.Solver("D2Q9", "fp32", c["shape"], mach=c["mach"], reynolds=c["reynolds"],
                         ref_length=c["ref_length"], bc=c["bc"], theta_inf=c.get("theta_inf", 0.0),
                         use_ac=c.get("use_ac", lbmib.AC_CENTRAL), bulk_ratio=c.get("bulk_ratio", 0.0))
        if k == 0:
            geo = inputs.cylinder((30.3, 32.2), c["ref_length"], 48, tbc=1, t_value=0.0)
            s.set_geometry(geo)
            b.case(k).set_geometry(geo)
        else:
            f, E = s.state()
            rng = np.random.Generator(np.random.PCG64(31))
            f = f * (1.0 + 1e-3 * rng.standard_normal(f.shape))
            s.set_state(f, E)
            b.case(k).set_state(f, E)
        solo.append(s)
    b.step(40)
    for s in solo:
        s.step(40)
    b.sync()
    for k, s in enumerate(solo):
        fa, Ea = b.case(k).state()
        fb, Eb = s.state()
        assert np.isfinite(fa).all() and np.isfinite(Ea).all()
        assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb)
        s.close()
    b.close()


def test_persistent_barrier_timeout_is_reported():
    """A grid barrier that cannot complete (its arrival count set past the
    grid size) ends the persistent launch after its bounded wait; the host
    reads LBM_ETIMEOUT, and the batch steps again afterwards."""
    from paper_2607_07432_b300 import lbmib
    cases, specs = _cases()
    b = lbmib.Batch("D2Q9", "fp32", cases[:2])
    for k, c in enumerate(cases[:2]):
        th = b.case(k).constants()["theta_inf"]
        b.case(k).set_geometry(_geometry(c, specs[k], th))
    b.step(2)
    b.sync()
    b.test_stall_barrier()
    b.step(2)
    with pytest.raises(lbmib.LBMError) as e:
        b.sync()
    assert e.value.status == 6 and "timed out" in str(e.value)     # LBM_ETIMEOUT
    b.sync()          # the barrier was cleared
    b.step(2)
    b.sync()
    b.close()
