"""Two-level static refinement through the C ABI (lbm_refined_*) against
the oracle's refine module: FP64 parity of both levels with a body on
level 1 and far-field boundaries on level 0 (2D and 3D), and the FP32 path
against the FP64 one."""
import numpy as np
import pytest

from paper_2607_07432_b300 import inputs

pytestmark = pytest.mark.gpu


def _maxrel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _case2d():
    # level 0: 40 x 32 with inlet / outlet / far field; level 1: the box
    # [12, 27] x [10, 21] refined by 2, a cylinder of diameter 6 level-0
    # cells (12 level-1 cells) at level-0 (19.3, 15.7)
    G = 4
    ctr1 = (G + 2 * (19.3 - 12), G + 2 * (15.7 - 10))
    return dict(lattice="D2Q9", shape=(40, 32), lo=(12, 10), hi=(27, 21), mach=0.2, reynolds=40.0,
                ref_length=6.0, bc=[1, 2, 3, 3],
                geo=lambda th: inputs.cylinder(ctr1, 12.0, 38, tbc=0, t_value=1.05 * th))


def _case3d():
    G = 4
    ctr1 = (G + 2 * (11.3 - 8), G + 2 * (9.6 - 6), G + 2 * (9.4 - 6))
    return dict(lattice="D3Q19", shape=(24, 20, 20), lo=(8, 6, 6), hi=(15, 13, 13), mach=0.2, reynolds=20.0,
                ref_length=3.0, bc=[1, 2, 3, 3, 3, 3],
                geo=lambda th: inputs.icosphere(ctr1, 6.0, 3, tbc=1, t_value=0.0))


def _oracle(c):
    from oracle import refine
    from oracle import lbm
    r = refine.Refined(c["lattice"], c["shape"], c["lo"], c["hi"], mach=c["mach"], reynolds=c["reynolds"],
                       ref_length=c["ref_length"], bc=c["bc"])
    geo = c["geo"](r.prm0.theta_inf)
    r.s1 = lbm.Sim(r.prm1, geo)
    return r, geo


def _gpu(c, precision, geo):
    from paper_2607_07432_b300 import lbmib
    r = lbmib.Refined(c["lattice"], precision, c["shape"], c["lo"], c["hi"], mach=c["mach"], reynolds=c["reynolds"],
                      ref_length=c["ref_length"], bc=c["bc"])
    r.level1.set_geometry(geo)
    return r


@pytest.mark.parametrize("case_fn,steps", [(_case2d, 20), (_case3d, 4)])
def test_refined_fp64_parity(case_fn, steps):
    """Level 0 and the level-1 nodes inside the ghost layer (populations
    and rho E) equal the oracle's to 1e-12 after `steps` level-0 steps from
    the uniform start with the body (the ghost nodes' own updates are
    scratch, overwritten by the next transfer)."""
    c = case_fn()
    o, geo = _oracle(c)
    g = _gpu(c, "fp64", geo)
    assert abs(g.level0.constants()["theta_inf"] - o.prm0.theta_inf) < 1e-15
    assert abs(g.level1.constants()["mu"] - o.prm1.mu) < 1e-15 * o.prm1.mu
    o.run(steps)
    g.step(steps)
    D = len(c["shape"])
    inner = tuple(slice(g.G, -g.G) for _ in range(D))
    f, E = g.level0.state()
    assert _maxrel(f, o.s0.f) < 1e-12
    assert _maxrel(E, o.s0.E) < 1e-12
    f, E = g.level1.state()
    assert _maxrel(f[(slice(None),) + inner], o.s1.f[(slice(None),) + inner]) < 1e-12
    assert _maxrel(E[inner], o.s1.E[inner]) < 1e-12
    g.check()
    g.close()


def test_refined_fp32_against_fp64():
    """FP32 path: relative L2 of u and T on both levels within 1e-5 of the
    FP64 path after 40 level-0 steps of the 2D case."""
    c = _case2d()
    o, geo = _oracle(c)
    outs = []
    for prec in ("fp64", "fp32"):
        g = _gpu(c, prec, geo)
        g.step(40)
        outs.append([lv.fields() for lv in (g.level0, g.level1)])
        g.close()
    inner = (slice(None),) + (slice(4, -4),) * 2
    for lev in (0, 1):
        _, u64, T64, _ = outs[0][lev]
        _, u32, T32, _ = outs[1][lev]
        if lev == 1:
            u64, u32, T64, T32 = u64[inner], u32[inner], T64[inner[1:]], T32[inner[1:]]
        assert np.linalg.norm(u32 - u64) / np.linalg.norm(u64) < 1e-5
        assert np.linalg.norm(T32 - T64) / np.linalg.norm(T64) < 1e-5


def test_refined_graph_replay_matches_eager(monkeypatch):
    """lbm_refined_step replays pairs of level-0 steps from a captured graph;
    both levels equal eager stepping (LBMIB_NO_GRAPH=1) bit for bit, for
    even and odd step counts."""
    c = _case2d()
    o, geo = _oracle(c)
    out = []
    for off in ("0", "1"):
        monkeypatch.setenv("LBMIB_NO_GRAPH", off)
        g = _gpu(c, "fp32", geo)
        g.step(5)
        g.step(4)
        g.step(1)
        out.append([lv.state() for lv in (g.level0, g.level1)])
        g.close()
    for lev in (0, 1):
        assert np.array_equal(out[0][lev][0], out[1][lev][0])
        assert np.array_equal(out[0][lev][1], out[1][lev][1])
