"""One case split into z slabs (Sec. 2.5 step, partitioned across devices):
the host side.  The library does the planning (lbm_slab_plan), the point
rule (lbm_slab_keep) and the packing of ghost planes (lbm_slab_pack /
lbm_slab_unpack); this module only marshals them and moves the buffers:
a device copy when the slabs share a GPU, NCCL send / receive through
torch.distributed when they are on different GPUs (one rank per slab).

After every step each slab sends its owned planes next to a neighbour and
receives that neighbour's into its ghost planes; with halo >= MIN_HALO the
owned planes evolve exactly as in the unsplit case."""
import ctypes as ct

import numpy as np

from . import lbmib

MIN_HALO = 10


def plan(nz, n_slabs, halo=MIN_HALO):
    """Per slab: dict(z0, z1, ghost_lo, ghost_hi, zoff, nz_local)."""
    out = (ct.c_int * (4 * n_slabs))()
    st = lbmib.lib().lbm_slab_plan(int(nz), int(n_slabs), int(halo), out)
    if st:
        raise lbmib.LBMError(st, "lbm_slab_plan")
    res = []
    for k in range(n_slabs):
        z0, z1, glo, ghi = out[4 * k:4 * k + 4]
        res.append(dict(z0=z0, z1=z1, ghost_lo=glo, ghost_hi=ghi, zoff=z0 - glo, nz_local=z1 - z0 + glo + ghi))
    return res


def keep_points(shape, d_n, z0, z1, halo, geo):
    """lbm_slab_keep: which Lagrangian points a slab keeps and owns (host
    arrays of 0/1); raises LBMError(LBM_EGEOM) when the halo is too narrow."""
    L = lbmib.lib()
    cfg = lbmib.Config()
    L.lbm_config_default(ct.byref(cfg))
    cfg.lattice = lbmib.D3Q19
    cfg.nx, cfg.ny, cfg.nz = int(shape[0]), int(shape[1]), int(shape[2])
    cfg.d_n = float(d_n)
    X = np.ascontiguousarray(geo["X"], dtype=np.float64).reshape(-1, 3)
    Nn = np.ascontiguousarray(geo["normals"], dtype=np.float64).reshape(-1, 3)
    n = X.shape[0]
    keep = np.zeros(n, dtype=np.int32)
    own = np.zeros(n, dtype=np.int32)
    st = L.lbm_slab_keep(ct.byref(cfg), int(z0), int(z1), int(halo), n, lbmib._ptr(X), lbmib._ptr(Nn),
                         lbmib._ptr(keep), lbmib._ptr(own))
    if st:
        raise lbmib.LBMError(st, "lbm_slab_keep")
    return keep.astype(bool), own.astype(bool)


def owned(arr, info, axis=-3):
    """The owned planes of a local array (z axis `axis`)."""
    sl = [slice(None)] * arr.ndim
    sl[axis] = slice(info["ghost_lo"], info["ghost_lo"] + info["z1"] - info["z0"])
    return arr[tuple(sl)]


class Buffers:
    """Device exchange buffers of one slab handle (torch uint8 tensors)."""

    def __init__(self, solver, device):
        import torch
        self.send = [None, None]
        self.recv = [None, None]
        for side in (0, 1):
            n = solver.exchange_bytes(side)
            if n:
                self.send[side] = torch.empty(n, dtype=torch.uint8, device=device)
                self.recv[side] = torch.empty(n, dtype=torch.uint8, device=device)


def exchange_local(solvers, bufs):
    """Refresh the ghost planes of slabs that share one device (solvers in
    slab order, all on the legacy default stream): pack every facing side,
    then unpack into the neighbours."""
    n = len(solvers)
    for k in range(n - 1):
        solvers[k].slab_pack(1, bufs[k].send[1])
        solvers[k + 1].slab_pack(0, bufs[k + 1].send[0])
    for k in range(n - 1):
        solvers[k + 1].slab_unpack(0, bufs[k].send[1])
        solvers[k].slab_unpack(1, bufs[k + 1].send[0])


def exchange_dist(solver, bufs, rank, world, dist):
    """Refresh the ghost planes of this rank's slab from its neighbours (rank
    - 1 below, rank + 1 above) with point-to-point NCCL transfers; the
    library's copies and torch's transfers run on the same (legacy default)
    stream."""
    ops = []
    if bufs.send[0] is not None:
        solver.slab_pack(0, bufs.send[0])
    if bufs.send[1] is not None:
        solver.slab_pack(1, bufs.send[1])
    if rank > 0 and bufs.send[0] is not None:
        ops.append(dist.P2POp(dist.isend, bufs.send[0], rank - 1))
        ops.append(dist.P2POp(dist.irecv, bufs.recv[0], rank - 1))
    if rank < world - 1 and bufs.send[1] is not None:
        ops.append(dist.P2POp(dist.isend, bufs.send[1], rank + 1))
        ops.append(dist.P2POp(dist.irecv, bufs.recv[1], rank + 1))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    if rank > 0 and bufs.recv[0] is not None:
        solver.slab_unpack(0, bufs.recv[0])
    if rank < world - 1 and bufs.recv[1] is not None:
        solver.slab_unpack(1, bufs.recv[1])


def reduce_loads(parts):
    """Wall loads of the whole body from the slabs' owned shares, added in
    slab order (a fixed order: the same sum on every rank)."""
    force = np.zeros_like(np.asarray(parts[0]["force"], dtype=np.float64))
    heat = work = 0.0
    for p in parts:
        force = force + np.asarray(p["force"])
        heat = heat + p["heat"]
        work = work + p["work"]
    return dict(force=force, heat=heat, work=work)
