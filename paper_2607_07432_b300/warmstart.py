"""Learned warm start for 2D cases: the solver generates its own steady
fields (batched launch), the neural operator is trained on them on the GPU,
and a new case starts from the network's field instead of uniform flow.
The converged plain solve stays the reference: time-to-steady is the number of
steps until the drag stays within a tolerance of the drag that the
uniform-start run converges to.

Orchestration only: the solver steps, the network's forward / backward /
Adam and the hand-off of the predicted field run in the CUDA library; this
module assembles inputs (signed distance, Mach, Re planes), scales the
targets and records drag histories.
"""
import time

import numpy as np

from . import inputs, lbmib
from .nop import NeuralOperator

BC = [lbmib.BC_INLET, lbmib.BC_OUTLET, lbmib.BC_FARFIELD, lbmib.BC_FARFIELD]
# isothermal walls at the free-stream temperature: with walls at 1.1 T_inf,
# bodies of 8-10 cells at Re 30 diverge within a few hundred steps (the
# FP64 oracle shows the same), so the heated wall is left out of this set
WALL_T = 1.0
# high-Mach sets (hm=True below): the Mach-weighted upstream a^C stencil and a
# free-stream lattice speed of at most U_CAP (bluff bodies at Ma 0.75 with the
# built-in theta rule's 0.15 diverge from a uniform start)
U_CAP = 0.1


def case_theta(case, hm):
    """theta_inf of a case: 0 (the library's rule) for the default sets; for
    high-Mach sets the rule's value (u_inf <= 0.15, conduction number <= 0.1)
    lowered until u_inf <= U_CAP."""
    if not hm:
        return 0.0
    g, pr = 1.4, 0.71
    u1 = case["mach"] * np.sqrt(g / 3.0)
    k1 = u1 * case["ref_length"] / case["reynolds"] * g / pr
    th = 1.0
    if u1 > 0.15:
        th = min(th, (0.15 / u1) ** 2)
    if k1 > 0.1:
        th = min(th, (0.1 / k1) ** 2)
    u = u1 * np.sqrt(th)
    return th * (U_CAP / u) ** 2 if u > U_CAP else th


def case_config(case, hm):
    """Keyword arguments of lbmib.Solver / lbmib.Batch for a case."""
    return dict(mach=case["mach"], reynolds=case["reynolds"], ref_length=case["ref_length"], bc=BC,
                theta_inf=case_theta(case, hm), use_ac=lbmib.AC_UPWIND if hm else lbmib.AC_CENTRAL)


def solver_for(case, precision="fp32", hm=False):
    nx, ny = case["shape"]
    s = lbmib.Solver("D2Q9", precision, shape=(nx, ny), **case_config(case, hm))
    th = s.constants()["theta_inf"]
    s.set_geometry(inputs.two_body_geometry(case, WALL_T * th))
    return s


def features(case):
    """Network input [ny][nx][3]: signed distance / reference length, Mach,
    Re / 200."""
    sdf = inputs.signed_distance(case) / case["ref_length"]
    x = np.empty(sdf.shape + (3,), dtype=np.float32)
    x[..., 0] = sdf
    x[..., 1] = case["mach"]
    x[..., 2] = case["reynolds"] / 200.0
    return x


def scales(const, mach):
    """(offset, scale) of the four outputs: rho = rho_inf (1 + Ma^2 y0),
    u_x = u_inf (1 + y1), u_y = u_inf y2, T = T_inf (1 + Ma^2 y3)."""
    r, u, t = const["rho_inf"], const["u_mag"], const["theta_inf"]
    m2 = mach * mach
    return (r, u, 0.0, t), (r * m2, u, u, t * m2)


def normalise(fields, const, mach):
    rho, u, T, _ = fields
    off, sc = scales(const, mach)
    y = np.empty(rho.shape + (4,), dtype=np.float32)
    y[..., 0] = (rho - off[0]) / sc[0]
    y[..., 1] = (u[0] - off[1]) / sc[1]
    y[..., 2] = (u[1] - off[2]) / sc[2]
    y[..., 3] = (T - off[3]) / sc[3]
    return y


def generate(cases, steps, chunk=64, hm=False, failed=None):
    """Steady fields of the cases from uniform starts, `steps` steps each,
    advanced `chunk` cases at a time in one batched launch per step.
    Returns X [n][ny][nx][3] and Y [n][ny][nx][4] (float32).  With a list
    `failed`, a case whose fields fail the health check is left out and its
    index appended there (otherwise the check raises)."""
    X, Y = [], []
    for k0 in range(0, len(cases), chunk):
        part = cases[k0:k0 + chunk]
        b = lbmib.Batch("D2Q9", "fp32", [dict(shape=c["shape"], **case_config(c, hm)) for c in part])
        consts = []
        for k, c in enumerate(part):
            v = b.case(k)
            const = v.constants()
            consts.append(const)
            v.set_geometry(inputs.two_body_geometry(c, WALL_T * const["theta_inf"]))
        b.step(steps + (steps % 2))
        b.sync()
        for k, c in enumerate(part):
            v = b.case(k)
            if failed is None:
                v.check()
            else:
                try:
                    v.check()
                except lbmib.LBMError:
                    failed.append(k0 + k)
                    continue
            X.append(features(c))
            Y.append(normalise(v.fields(), consts[k], c["mach"]))
        b.close()
    return np.stack(X), np.stack(Y)


def train(net, X, Y, steps, batch, lr, seed=0, lr_final=None, log_every=0):
    """Adam on mini-batches drawn (seeded) from the device-resident dataset;
    the learning rate decays linearly to lr_final.  Returns the losses."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    xb = torch.empty((batch,) + tuple(X.shape[1:]), device="cuda", dtype=torch.float32)
    yb = torch.empty((batch,) + tuple(Y.shape[1:]), device="cuda", dtype=torch.float32)
    lr_final = lr if lr_final is None else lr_final
    losses = []
    for s in range(steps):
        idx = torch.from_numpy(rng.integers(0, X.shape[0], size=batch)).cuda()
        torch.index_select(Xd, 0, idx, out=xb)
        torch.index_select(Yd, 0, idx, out=yb)
        torch.cuda.synchronize()
        a = lr + (lr_final - lr) * s / max(1, steps - 1)
        losses.append(net.train_step(xb, yb, a))
        if log_every and s % log_every == 0:
            print("step %d loss %.4e" % (s, losses[-1]), flush=True)
    return np.array(losses)


def drag_history(solver, steps, every):
    """x-force on the bodies every `every` steps."""
    out = []
    for _ in range(steps // every):
        solver.step(every)
        out.append(solver.wall_loads()["force"][0])
    solver.check()
    return np.array(out)


def steps_to_steady(hist, target, every, tol=1e-3):
    """First step count after which every recorded drag stays within
    tol |target| of target; None if the record never settles."""
    ok = np.abs(hist - target) <= tol * abs(target)
    if not ok[-1]:
        return None
    bad = np.nonzero(~ok)[0]
    first = 0 if bad.size == 0 else bad[-1] + 1
    return int((first + 1) * every)


def compare(net, case, steps, every, tol=1e-3, hm=False):
    """Uniform start vs warm start on one case.  The uniform run's final
    drag is the converged answer both are measured against.  A run that
    fails the health check is reported (diverged) instead of measured."""
    import torch
    s = solver_for(case, hm=hm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        h_u = drag_history(s, steps, every)
    except lbmib.LBMError:
        s.close()
        return dict(diverged="uniform", steps_uniform=None, steps_warm=None)
    torch.cuda.synchronize()
    ms_u = (time.perf_counter() - t0) * 1e3
    cd_inf = h_u[-1]
    const = s.constants()
    s.close()
    s = solver_for(case, hm=hm)
    x = torch.from_numpy(features(case)[None]).cuda()
    off, sc = scales(const, case["mach"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.infer_into(s, x, off, sc)
    torch.cuda.synchronize()
    ms_inf = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    try:
        h_w = drag_history(s, steps, every)
    except lbmib.LBMError:
        s.close()
        return dict(diverged="warm", cd_inf=float(cd_inf), steps_uniform=steps_to_steady(h_u, cd_inf, every, tol),
                    steps_warm=None)
    torch.cuda.synchronize()
    ms_w = (time.perf_counter() - t0) * 1e3
    s.close()
    n_u = steps_to_steady(h_u, cd_inf, every, tol)
    n_w = steps_to_steady(h_w, cd_inf, every, tol)
    ms_step_u, ms_step_w = ms_u / steps, ms_w / steps
    return dict(cd_inf=float(cd_inf), warm_final=float(h_w[-1]), steps_uniform=n_u, steps_warm=n_w,
                ms_uniform=None if n_u is None else n_u * ms_step_u,
                ms_warm=None if n_w is None else ms_inf + n_w * ms_step_w, ms_infer=ms_inf)


def new_network(shape, max_batch=8, channels=(32, 64, 96, 128), seed=1):
    nx, ny = shape
    net = NeuralOperator(height=ny, width=nx, max_batch=max_batch, channels=channels)
    net.init_params(seed)
    return net
