"""One case split into z slabs (Sec. 2.5 step, partitioned): the host logic
of the decomposition -- the library's slab plan and Lagrangian-point rule
(lbm_slab_plan, lbm_slab_keep; host-only calls, no GPU) and the ghost-plane
exchange after every step -- checked with the FP64 oracle as the per-slab
engine: two gloo ranks, each stepping its slab of a D3Q19 case with an
immersed sphere cut by the slab boundary, exchanging ghost planes through
torch.distributed, give owned planes equal bit for bit to the unsplit
oracle, and wall loads that add up to the unsplit ones."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

SHAPE, HALO, STEPS = (14, 12, 40), 10, 8
SPHERE = dict(center=(6.7, 6.2, 20.3), diameter=6.0, frequency=3)
BC = [1, 2, 3, 3, 3, 3]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _params(**kw):
    from oracle import lbm
    return lbm.Params("D3Q19", kw.pop("shape", SHAPE), mach=0.2, reynolds=20.0, ref_length=6.0, **kw)


def _geometry(theta):
    from paper_2607_07432_b300 import inputs
    return inputs.icosphere(SPHERE["center"], SPHERE["diameter"], SPHERE["frequency"], tbc=0, t_value=1.05 * theta)


def _subset(geo, keep):
    out = dict(geo)
    for k in ("X", "normals", "tbc", "t_value", "u_target"):
        out[k] = np.asarray(geo[k])[keep]
    return out


def _state(sim):
    """The per-step state of an oracle sim as a list of (z, y, x) arrays."""
    D = sim.prm.lat.D
    arrs = [sim.f[i] for i in range(sim.prm.lat.Q)] + [sim.E, sim.P_prev]
    arrs += [sim.devAF_prev[a][b] for a in range(D) for b in range(D)]
    return arrs


def _exchange(sim, info, rank, world):
    """Send the owned planes next to each neighbour, receive its owned planes
    into the ghost planes (the library's lbm_slab_pack / unpack order)."""
    g, own = info["ghost_lo"], info["z1"] - info["z0"]
    arrs = _state(sim)
    reqs, recv = [], []
    if rank > 0:
        send = torch.from_numpy(np.stack([a[g:g + g] for a in arrs]).copy())
        buf = torch.empty_like(send)
        reqs += [dist.isend(send, rank - 1), dist.irecv(buf, rank - 1)]
        recv.append((slice(0, g), buf))
    if rank < world - 1:
        h = info["ghost_hi"]
        send = torch.from_numpy(np.stack([a[g + own - h:g + own] for a in arrs]).copy())
        buf = torch.empty_like(send)
        reqs += [dist.isend(send, rank + 1), dist.irecv(buf, rank + 1)]
        recv.append((slice(g + own, g + own + h), buf))
    for r in reqs:
        r.wait()
    for sl, buf in recv:
        b = buf.numpy()
        for k, a in enumerate(arrs):
            a[sl] = b[k]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import lbm
    from paper_2607_07432_b300 import slab
    info = slab.plan(SHAPE[2], world, HALO)[rank]
    ref = lbm.Sim(_params(bc=BC), _geometry(_params().theta_inf))
    bc = list(BC)
    if info["ghost_lo"]:
        bc[4] = lbm.BC_GHOST
    if info["ghost_hi"]:
        bc[5] = lbm.BC_GHOST
    prm = _params(shape=(SHAPE[0], SHAPE[1], info["nz_local"]), bc=bc, zoff=info["zoff"])
    geo = _geometry(prm.theta_inf)
    keep, own = slab.keep_points(SHAPE, prm.d_n, info["z0"], info["z1"], HALO, geo)
    sim = lbm.Sim(prm, _subset(geo, keep))
    for _ in range(STEPS):
        ref.step()
        sim.step()
        _exchange(sim, info, rank, world)
    z = slice(info["ghost_lo"], info["ghost_lo"] + info["z1"] - info["z0"])
    zg = slice(info["z0"], info["z1"])
    same_f = bool(np.array_equal(sim.f[:, z], ref.f[:, zg]))
    same_E = bool(np.array_equal(sim.E[z], ref.E[zg]))
    L = sim.last_loads
    ok = own[keep]
    force = -(L["F"][ok] * sim.ib.W[ok][:, None]).sum(axis=0)
    heat = (L["Q"][ok] * sim.ib.W[ok]).sum()
    out[rank] = (same_f, same_E, force, heat, ref.last_loads["force"], ref.last_loads["heat"], int(keep.sum()),
                 int(own.sum()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_slabs_equal_the_unsplit_oracle():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    force = sum(out[r][2] for r in range(world))
    heat = sum(out[r][3] for r in range(world))
    for r in range(world):
        same_f, same_E = out[r][0], out[r][1]
        assert same_f and same_E, r
    ref_force, ref_heat = out[0][4], out[0][5]
    assert np.allclose(force, ref_force, rtol=1e-12, atol=1e-14)
    assert abs(heat - ref_heat) <= 1e-12 * abs(ref_heat)
    assert sum(out[r][7] for r in range(world)) == len(_geometry(1.0)["X"])    # each point one owner


def test_slab_plan_and_point_rule():
    """Host-only planning calls: slabs cover the planes once, ghost planes
    only towards neighbours, the first nz % n slabs one plane thicker;
    points whose stencils leave a slab are dropped only far from its owned
    planes, and a halo too narrow for the body is refused."""
    from paper_2607_07432_b300 import inputs, lbmib, slab
    p = slab.plan(50, 4, 10)
    assert [q["z1"] - q["z0"] for q in p] == [13, 13, 12, 12]
    assert p[0]["z0"] == 0 and p[-1]["z1"] == 50
    assert all(p[k]["z1"] == p[k + 1]["z0"] for k in range(3))
    assert p[0]["ghost_lo"] == 0 and p[-1]["ghost_hi"] == 0
    assert all(q["ghost_hi"] == 10 for q in p[:-1]) and all(q["ghost_lo"] == 10 for q in p[1:])
    geo = inputs.icosphere((12.0, 10.0, 25.0), 8.0, 4)
    owners = np.zeros(len(geo["X"]), int)
    for q in p:
        keep, own = slab.keep_points((24, 20, 50), 1.5, q["z0"], q["z1"], 10, geo)
        assert not (own & ~keep).any() or q["z1"] - q["z0"] < 1
        owners += own
    assert (owners == 1).all()
    with pytest.raises(lbmib.LBMError):
        slab.keep_points((24, 20, 50), 1.5, 0, 26, 3, geo)
