"""Benchmark: MLUPS of the full time step (IB on) of the 3D sphere case.

Workload (the 3D case the headline metric is quoted on): D3Q19 hybrid LBM,
grid 256x192x192, sphere D = 48 at (64, 96, 96), 7292 Lagrangian points
(geodesic icosphere, frequency 27), Ma 0.3, Re 300, isothermal wall at
1.1 T_inf, FODIBM-R, inlet / outlet in x, far field elsewhere, FP32.
A step is one pass of the whole hot path (IB interpolation + forcing,
spreading, collision, streaming, energy update, boundaries).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 ranks (one per GPU) the case is
partitioned into z slabs (lbm_create_slab), one per rank, with the ghost
planes exchanged by NCCL after every step: a 256 x 192 x 192N channel with
one sphere per 192 planes (weak scaling, each rank owns a 256 x 192 x 192
slab around its sphere).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS with IBM on (% of HBM roofline); time-to-steady at 0.1% drag vs plain FP32"
UNIT = "MLUPS"
SHAPE = (256, 192, 192)
CASE = dict(lattice="D3Q19", shape=SHAPE, mach=0.3, reynolds=300.0, ref_length=48.0,
            center=(64.0, 96.0, 96.0), diameter=48.0, frequency=27)
# Algorithmic bytes per lattice update: populations read and written once
# (2 Q s_f) plus the state the method carries between steps, read and written
# once: rho E, rho(1-theta) of the previous step (the backward difference of
# Eq. af2) and the deviator of a^F of the previous step (the F_i(t - dt) term
# of Eq. pi2).  With the full a^C reading (off-diagonal advective terms) that
# deviator has all D(D+1)/2 - 1 components (5 in 3D): 208 B for D3Q19 FP32.
# A diagonal-only a^C would need D - 1 slots (184 B for D3Q19 FP32); both
# fractions are reported.
def bytes_per_lu(lattice, precision, ndev=None):
    Q, D = (19, 3) if lattice == "D3Q19" else (9, 2)
    sf = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[precision]
    sa = 8 if precision == "fp64" else 4
    if ndev is None:
        ndev = D * (D + 1) // 2 - 1
    return 2 * Q * sf + 2 * (2 + ndev) * sa


def kernel_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu
    capture, if the kernel sources are unchanged since that capture."""
    import glob
    import hashlib
    p = os.path.join(ROOT, "profiles", "fused_step_sphere256_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    return float(d["dram_bytes_per_launch"]) if fused_sources_sha() == d["src_sha256"] else None


def fused_sources_sha():
    """sha256 over the sources that define the fused step kernel."""
    import hashlib
    h = hashlib.sha256()
    for name in FUSED_SOURCES:
        f = os.path.join(ROOT, "paper_2607_07432_b300", "csrc", name)
        h.update(name.encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


FUSED_SOURCES = ["grid.cuh", "inst_d3q19_fp32.cu", "lattice.cuh", "physics.cuh", "step_fused.cuh"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None
        self.lines = []
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.perf_counter(), line))

    def start(self):
        """Start sampling and wait (at most 5 s) for the first sample, so the
        sampler is running when the timed region begins."""
        import threading
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return
        threading.Thread(target=self._read, daemon=True).start()
        t = time.perf_counter()
        while not self.lines and time.perf_counter() - t < 5.0:
            time.sleep(0.005)

    def begin(self):
        self.t0 = time.perf_counter()

    def end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.05)
        self.p.terminate()
        try:
            self.p.wait(timeout=10)
        except subprocess.TimeoutExpired:
            self.p.kill()
        # samples inside the timed region, plus the last one before it
        t0 = self.t0 if self.t0 is not None else -1e30
        t1 = self.t1 if self.t1 is not None else 1e30
        inside = [ln for (t, ln) in self.lines if t0 <= t <= t1 + 0.025]
        before = [ln for (t, ln) in self.lines if t < t0]
        sel = (before[-1:] + inside) if before else inside
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in sel:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def build_case(lbmib, inputs, precision):
    c = CASE
    s = lbmib.Solver(c["lattice"], precision, c["shape"], mach=c["mach"], reynolds=c["reynolds"],
                     ref_length=c["ref_length"],
                     bc=[lbmib.BC_INLET, lbmib.BC_OUTLET] + [lbmib.BC_FARFIELD] * 4)
    th = s.constants()["theta_inf"]
    geo = inputs.icosphere(c["center"], c["diameter"], c["frequency"], tbc=0, t_value=1.1 * th)
    s.set_geometry(geo)
    return s, geo


def oracle_sample(steps_budget_s=15.0, max_steps=None):
    """The oracle on a 64x48x48 downscale of the same case (D = 12, 492
    points); returns MLUPS, steps and nodes."""
    from oracle import lbm
    from paper_2607_07432_b300 import inputs
    prm = lbm.Params("D3Q19", (64, 48, 48), mach=CASE["mach"], reynolds=CASE["reynolds"], ref_length=12.0,
                     bc=[1, 2, 3, 3, 3, 3])
    geo = inputs.icosphere((16.0, 24.0, 24.0), 12.0, 7, tbc=0, t_value=1.1 * prm.theta_inf)
    sim = lbm.Sim(prm, geo)
    sim.step()  # warm-up
    n = 0
    t0 = time.perf_counter()
    while True:
        sim.step()
        n += 1
        el = time.perf_counter() - t0
        if el > steps_budget_s or (max_steps and n >= max_steps):
            break
    nodes = 64 * 48 * 48
    return nodes * n / el / 1e6, n, nodes, el


def host_cpu():
    """Host cores and CPU model (for the CPU baseline's record)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return os.cpu_count() or 1, model


def _oracle_worker(budget):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    return oracle_sample(budget)


def oracle_all_cores(budget_s, max_procs=32):
    """Independent oracle processes (one per core, at most max_procs), each
    stepping its own copy of the 64x48x48 downscale for budget_s seconds:
    the host's aggregate oracle throughput.  Processes are spawned (never
    forked from a process that has used the GPU)."""
    import multiprocessing as mp
    nproc, _ = host_cpu()
    P = max(1, min(nproc, max_procs))
    ctx = mp.get_context("spawn")
    with ctx.Pool(P) as pool:
        res = pool.map(_oracle_worker, [budget_s] * P)
    return sum(r[0] for r in res), P, sum(r[1] for r in res)


def cpu_baseline_record(budget_s=15.0, all_cores=True):
    """The oracle as it stands on the host: one core, and (optionally) every
    core running independent copies of the same downscale."""
    nproc, model = host_cpu()
    mlups, n, nodes, el = oracle_sample(budget_s)
    rec = {"value": mlups, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d steps of the 64x48x48 downscale of the sphere case (D=12, 492 points), %.1f s, "
                     "one process" % (n, el),
           "host_nproc": nproc, "cpu_model": model}
    if all_cores:
        agg, P, nsteps = oracle_all_cores(budget_s)
        rec["all_cores"] = {"value": agg, "unit": UNIT, "cores": P,
                            "sample": "%d independent oracle processes on the same downscale, %.0f s each, "
                                      "%d steps in total" % (P, budget_s, nsteps)}
    return rec


def run_reference(args, rank):
    if rank != 0:
        return
    nproc, model = host_cpu()
    mlups, n, nodes, el = oracle_sample(steps_budget_s=max(5.0, 10.0 * args.steps / 20.0))
    line = {"metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / n * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "3D sphere D3Q19 256x192x192 (oracle on its 64x48x48 downscale)",
                       "precision": "fp64", "method": "FODIBM-R"},
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d steps of the 64x48x48 downscale (D=12, 492 points), %.1f s" % (n, el),
                             "host_nproc": nproc, "cpu_model": model},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, emit=True):
    """64 uneven 2D cases (seeded circles and ellipses, grids 256x128 ..
    1024x512, Re 20-200, FP32) stepped together (autotuned plan: launch form
    -- one persistent cooperative launch per two steps or one launch per
    phase --, tile rows and schedule; graph replay) against 64 sequential
    per-case launches; both launch forms are timed with the tuned tile and
    schedule.  Mach is
    drawn from [0.1, 0.45]: from an impulsive start, bluff bodies at Ma >= 0.5
    develop transonic pockets that the unlimited MUSCL scheme does not hold."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    specs = inputs.batch_cases(64, seed=20260001, mach_range=(0.1, 0.45))
    bc = [lbmib.BC_INLET, lbmib.BC_OUTLET, lbmib.BC_FARFIELD, lbmib.BC_FARFIELD]
    cases = [dict(shape=(c["nx"], c["ny"]), mach=c["mach"], reynolds=c["reynolds"], ref_length=c["ref_length"],
                  bc=bc) for c in specs]
    b = lbmib.Batch("D2Q9", "fp32", cases)
    nodes = 0
    for k, (c, sp) in enumerate(zip(cases, specs)):
        v = b.case(k)
        th = v.constants()["theta_inf"]
        nx, ny = c["shape"]
        ctr = (nx / 4.0, ny / 2.0)
        if sp["ellipse"]:
            geo = inputs.ellipse(ctr, sp["a"], sp["b"], sp["angle"], sp["n_points"], tbc=0, t_value=1.1 * th)
        else:
            geo = inputs.cylinder(ctr, 2 * sp["a"], sp["n_points"], tbc=0, t_value=1.1 * th)
        v.set_geometry(geo)
        nodes += nx * ny
    plan, tuned_ms = b.autotune(steps=6)
    b.step(args.warmup + (args.warmup % 2))
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = args.steps + (args.steps % 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(K)
    b.sync()
    ms_b = (time.perf_counter() - t0) * 1e3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step_sequential(K)
    b.sync()
    ms_s = (time.perf_counter() - t0) * 1e3
    form = b.launch_form()
    forms = {}
    for fm in (1, 0):
        b.set_launch_form(fm)
        b.set_plan(*plan)
        b.step(2)
        b.sync()
        t0 = time.perf_counter()
        b.step(K)
        b.sync()
        forms["persistent" if fm else "per_phase"] = (time.perf_counter() - t0) * 1e3 / K
    for k in range(len(cases)):
        b.case(k).check()
    line = {"metric": "aggregate MLUPS, 64 uneven 2D cases (batched vs sequential)",
            "value": nodes * K / (ms_b / 1e3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_b / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch of 64 seeded 2D cases (seed 20260001, Ma 0.1-0.45)", "nodes": nodes,
                       "plan": {"tile_rows": plan[0], "schedule": plan[1],
                                "launch_form": "persistent" if form else "per_phase"}},
            "ms_per_step_by_form": forms,
            "sequential": {"value": nodes * K / (ms_s / 1e3) / 1e6, "ms_per_step": ms_s / K},
            "speedup_vs_sequential": ms_s / ms_b}
    b.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


def _sphere(lbmib, inputs, precision, shape, D, freq):
    s = lbmib.Solver("D3Q19", precision, shape, mach=CASE["mach"], reynolds=CASE["reynolds"], ref_length=D,
                     bc=[lbmib.BC_INLET, lbmib.BC_OUTLET] + [lbmib.BC_FARFIELD] * 4)
    th = s.constants()["theta_inf"]
    center = (shape[0] / 4.0, shape[1] / 2.0, shape[2] / 2.0)
    s.set_geometry(inputs.icosphere(center, D, freq, tbc=0, t_value=1.1 * th))
    return s


def coefficient_history(s, steps, every):
    """C_d and Nu of the body sampled every `every` steps."""
    cd, nu = [], []
    for _ in range(steps // every):
        s.step(every)
        d = s.wall_diagnostics(per_point=False)
        cd.append(d["Cd"])
        nu.append(d["Nu"])
    s.check()
    return np.array(cd), np.array(nu)


def steady_summary(cd, nu, every, window):
    """Running means over the last `window` steps and the first step from
    which the trailing-window mean of C_d stays within 0.1% of that final
    value (reading Q28: the criterion is judged on a running mean over at
    least two shedding periods)."""
    w = max(1, window // every)
    cd_f, nu_f = float(cd[-w:].mean()), float(nu[-w:].mean())
    run = np.convolve(cd, np.ones(w) / w, mode="valid")
    ok = np.abs(run - cd_f) <= 1e-3 * abs(cd_f)
    bad = np.nonzero(~ok)[0]
    first = int(bad[-1] + 1) if bad.size else 0
    steady = (first + w) * every if first < run.size else None
    return dict(Cd=cd_f, Nu=nu_f, steps_to_steady=steady)


def run_rotsphere(args):
    """Subsonic flow past a sphere turning about z (Sec. 3.9): Ma 0.3,
    Re 300, adiabatic no-slip wall with targets omega x r, Omega* =
    omega D / (2 u_inf) = 0.3 and 0.6, characteristic far field on the
    outlet and the lateral faces, a uniform 10D x 6D x 6D grid (D = 32
    cells by default).
    Reports time-averaged C_d, C_l (along -y, the side where the surface
    moves with the stream) and the Strouhal number of the lift."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    D = float(args.rot_d)
    shape = (int(10 * D), int(6 * D), int(6 * D))
    freq = int(round(np.sqrt(np.pi * D * D / 10.0)))
    ctr = (2.5 * D, 3.0 * D, 3.0 * D)
    steps, window, every = args.rot_steps, args.rot_window, 20
    paper = {"0.3": {"Cd": 0.750, "Cl": 0.332, "St": 0.202}, "0.6": {"Cd": 0.862, "Cl": 0.512, "St": None}}
    res = {}
    for om in [float(v) for v in args.rot_omegas.split(",")]:
        s = lbmib.Solver("D3Q19", "fp32", shape, mach=0.3, reynolds=300.0, ref_length=D,
                         bc=[lbmib.BC_INLET] + [lbmib.BC_CHAR] * 5)
        u_inf = s.constants()["u_mag"]
        omega = 2.0 * om * u_inf / D
        s.set_geometry(inputs.rotating(inputs.icosphere(ctr, D, freq, tbc=1, t_value=0.0), ctr, (0.0, 0.0, omega)))
        if args.rot_noise > 0:
            # seeded velocity noise on the uniform start, to seed the wake
            # instability without waiting for round-off to grow
            c = s.constants()
            N = s.N
            rng = np.random.default_rng(20260009)
            u0 = args.rot_noise * u_inf * rng.standard_normal(3 * N)
            u0[:N] += u_inf
            s.set_fields(np.ones(N), u0, np.full(N, c["theta_inf"]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cd, cl, cz = [], [], []
        for _ in range(steps // every):
            s.step(every)
            d = s.wall_diagnostics(per_point=False)
            cd.append(d["Cd"])
            cl.append(-d["Cl"])
            cz.append(d["Cl2"])
        s.check()
        wall = time.perf_counter() - t0
        s.close()
        w = window // every
        cd, cl, cz = np.array(cd), np.array(cl), np.array(cz)
        # Strouhal number: the spectral peak of the lift fluctuation (both
        # lateral components) over the averaging window
        best = (0.0, None)
        for sig in (cl[-w:], cz[-w:]):
            x = (sig - sig.mean()) * np.hanning(w)
            p = np.abs(np.fft.rfft(x)) ** 2
            k = int(np.argmax(p[1:]) + 1)
            # peak between bins: vertex of the parabola through the log
            # power of the peak bin and its neighbours
            kf = float(k)
            if 1 <= k < len(p) - 1 and min(p[k - 1], p[k], p[k + 1]) > 0:
                a, b, c = np.log(p[k - 1]), np.log(p[k]), np.log(p[k + 1])
                if a - 2 * b + c < 0:
                    kf = k + 0.5 * (a - c) / (a - 2 * b + c)
            amp = float(np.std(sig))
            if amp > best[0]:
                best = (amp, kf / (w * every) * D / u_inf)
        amp, st = best
        # lift fluctuation per 4000-step block (growth or decay of shedding)
        blk = 4000 // every
        rms_blocks = [float(np.std(cl[i:i + blk])) for i in range(0, len(cl) - blk + 1, blk)]
        res["%.1f" % om] = {"Cd": float(cd[-w:].mean()), "Cl": float(cl[-w:].mean()), "Cl_rms_blocks": rms_blocks,
                            "Cl_rms": amp, "St": st if amp > 1e-3 else None, "omega": omega,
                            "steps": steps, "window": window, "wall_s": wall,
                            "paper_fodibm_r": paper.get("%.1f" % om)}
    line = {"metric": "time-averaged C_d, C_l and lift Strouhal number of a rotating sphere (Ma 0.3, Re 300)",
            "value": next(iter(res.values()))["Cd"], "unit": "C_d at Omega* %s" % next(iter(res)), "n_gpus": 1,
            "higher_is_better": False,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "3D rotating sphere D3Q19 %dx%dx%d, D = %d (%d points), Omega* %s, "
                                   "adiabatic wall, characteristic far field, start noise %g u_inf"
                                   % (shape + (int(D), 10 * freq * freq + 2, args.rot_omegas, args.rot_noise))},
            "results": res}
    print(json.dumps(line), flush=True)


def run_refined(args):
    """Two-level static refinement against uniform grids on the 2D cylinder
    (Ma 0.2, Re 40, isothermal wall 1.1 T_inf): uniform D = 20 (200x100),
    uniform D = 40 (400x200), and level 0 at D = 20 with the box of level-0
    nodes [30, 150] x [20, 80] around the cylinder and its wake (by default)
    refined to D = 40.  All
    three at the theta_inf of the refined case; C_d from running means over
    the last 2000 level-0 steps of `--ref-steps`."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    steps, every, window = args.ref_steps, 50, 2000
    kw = dict(mach=0.2, reynolds=40.0, bc=[lbmib.BC_INLET, lbmib.BC_OUTLET, lbmib.BC_FARFIELD, lbmib.BC_FARFIELD])
    out = {}

    def history(step, diag, n_steps):
        cd = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_steps // every):
            step(every)
            cd.append(diag()["Cd"])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        cd = np.array(cd)
        w = window // every
        return float(cd[-w:].mean()), float(np.abs(cd[-w:] - cd[-w:].mean()).max()), wall

    r = lbmib.Refined("D2Q9", "fp32", (200, 100), tuple(args.ref_lo), tuple(args.ref_hi), ref_length=20.0, **kw)
    th = r.level0.constants()["theta_inf"]
    G = r.G
    lo = r.box_lo
    r.level1.set_geometry(inputs.cylinder((G + 2 * (60.0 - lo[0]), G + 2 * (50.0 - lo[1])), 40.0, 126, tbc=0,
                                          t_value=1.1 * th))
    n1 = int(np.prod(r.level1.shape))
    cd, spread, wall = history(r.step, lambda: r.level1.wall_diagnostics(per_point=False), steps)
    r.check()
    r.close()
    out["refined"] = {"Cd": cd, "Cd_spread": spread, "wall_s": wall, "level0_nodes": 200 * 100,
                      "level1_nodes": n1, "node_updates_per_level0_step": 200 * 100 + 2 * n1}
    for name, shape, D, ctr, n_pts, scale in (("uniform D=20", (200, 100), 20.0, (60.0, 50.0), 63, 1),
                                              ("uniform D=40", (400, 200), 40.0, (120.0, 100.0), 126, 2)):
        s = lbmib.Solver("D2Q9", "fp32", shape, ref_length=D, theta_inf=th, **kw)
        s.set_geometry(inputs.cylinder(ctr, D, n_pts, tbc=0, t_value=1.1 * th))
        cd, spread, wall = history(lambda n: s.step(n * scale), lambda: s.wall_diagnostics(per_point=False), steps)
        s.check()
        s.close()
        out[name] = {"Cd": cd, "Cd_spread": spread, "wall_s": wall,
                     "node_updates_per_level0_step": int(np.prod(shape)) * scale}
    line = {"metric": "C_d of the 2D cylinder on a two-level refined grid against uniform grids",
            "value": out["refined"]["Cd"], "unit": "C_d", "n_gpus": 1, "higher_is_better": False, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "2D cylinder Ma 0.2, Re 40, 200x100 level 0 (D = 20) with [%d,%d]x[%d,%d] "
                                   "refined by 2 (D = 40), against uniform D = 20 and D = 40"
                                   % (args.ref_lo[0], args.ref_hi[0], args.ref_lo[1], args.ref_hi[1]),
                       "theta_inf": th, "level0_steps": steps},
            "results": out}
    print(json.dumps(line), flush=True)


def run_refined_sphere(args):
    """Two-level refinement on the 3D sphere (Ma 0.3, Re 300, isothermal wall
    1.1 T_inf): level 0 192x96x96 at D = 16 with the box of level-0 nodes
    [32, 112] x [24, 72] x [24, 72] around the sphere and its near wake
    refined to D = 32, against the uniform D = 32 grid (384x192x192) and the
    uniform D = 16 grid.  C_d and Nu as running means over the last 3000
    level-0 steps of `--ref-steps`; cost as device time per level-0 step."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    steps, every, window = args.ref_steps, 100, 3000
    kw = dict(mach=0.3, reynolds=300.0, bc=[lbmib.BC_INLET, lbmib.BC_OUTLET] + [lbmib.BC_FARFIELD] * 4)
    lo, hi = (32, 24, 24), (112, 72, 72)
    out = {}

    def history(step, diag, n_steps):
        cd, nu = [], []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(n_steps // every):
            ev0.record()
            step(every)
            ev1.record()
            d = diag()
            ms += ev0.elapsed_time(ev1)
            cd.append(d["Cd"])
            nu.append(d["Nu"])
        w = window // every
        cd, nu = np.array(cd), np.array(nu)
        return dict(Cd=float(cd[-w:].mean()), Nu=float(nu[-w:].mean()),
                    Cd_spread=float(np.abs(cd[-w:] - cd[-w:].mean()).max()), ms_per_level0_step=ms / n_steps)

    r = lbmib.Refined("D3Q19", "fp32", (192, 96, 96), lo, hi, ref_length=16.0, **kw)
    th = r.level0.constants()["theta_inf"]
    G = r.G
    ctr1 = tuple(G + 2.0 * (c - l) for c, l in zip((48.0, 48.0, 48.0), lo))
    r.level1.set_geometry(inputs.icosphere(ctr1, 32.0, 18, tbc=0, t_value=1.1 * th))
    n1 = int(np.prod(r.level1.shape))
    out["refined"] = history(r.step, lambda: r.level1.wall_diagnostics(per_point=False), steps)
    out["refined"].update(level0_nodes=192 * 96 * 96, level1_nodes=n1)
    r.check()
    r.close()
    for name, shape, D, freq, scale in (("uniform D=32", (384, 192, 192), 32.0, 18, 2),
                                        ("uniform D=16", (192, 96, 96), 16.0, 9, 1)):
        s = lbmib.Solver("D3Q19", "fp32", shape, ref_length=D, theta_inf=th, **kw)
        s.set_geometry(inputs.icosphere((3.0 * D, 3.0 * D, 3.0 * D), D, freq, tbc=0, t_value=1.1 * th))
        out[name] = history(lambda n: s.step(n * scale), lambda: s.wall_diagnostics(per_point=False), steps)
        out[name]["nodes"] = int(np.prod(shape))
        s.check()
        s.close()
    ref = out["uniform D=32"]
    line = {"metric": "C_d and Nu of the 3D sphere on a two-level refined grid against uniform grids, and cost",
            "value": out["refined"]["Cd"], "unit": "C_d", "n_gpus": 1, "higher_is_better": False, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "3D sphere Ma 0.3, Re 300, 192x96x96 level 0 (D = 16) with [32,112]x[24,72]x[24,72] "
                                   "refined by 2 (D = 32), against uniform D = 32 and D = 16",
                       "theta_inf": th, "level0_steps": steps},
            "speedup_vs_uniform_fine": ref["ms_per_level0_step"] / out["refined"]["ms_per_level0_step"],
            "results": out}
    print(json.dumps(line), flush=True)


def run_supersonic(args):
    """High-Mach operating points with the Mach-weighted upstream a^C stencil
    (LBM_AC_UPWIND), FP32:
    (1) a seeded uniform Mach 2 stream (theta 0.02, periodic 256x128,
        populations with 1e-3 relative noise): growth of the density deviation
        with the central stencil (20 steps) and with LBM_AC_UPWIND (5000 steps);
    (2) NACA0012 at Mach 0.8, Re 500, 10 degrees (chord 100, 1024x512, inlet
        and characteristic faces, theta 0.1, impulsive start): C_d and C_l,
        running means over the last 10 000 of 30 000 steps;
    (3) the adiabatic sphere at Mach 1.2, Re 300 (D = `--sup-sphere-d`, grid
        12D x 8D x 8D, theta 0.02, bulk viscosity 3 mu): Mach ramp from 0.3 in
        8 restarts of 1500 steps, then 30 000 steps; C_d (mean over the last
        7500) and the shock stand-off on the axis;
    (4) the adiabatic cylinder at Mach 2, Re 300 (D = `--sup-d`, domain
        [-10D, 30D] x [-10D, 10D], theta `--sup-theta`, bulk viscosity
        `--sup-bulk` mu): Mach ramp from 0.5 in 16 restarts of 2000 steps, then
        `--sup-steps` steps with a health check every 2000; C_d and stand-off
        every 10 000 steps and the step at which a check fails, if one does.
    The stand-off is the distance from the stagnation point to where p / p_inf
    first reaches the normal-shock ratio upstream of it."""
    from paper_2607_07432_b300 import inputs, lbmib
    out = {}
    g = 1.4
    CH = lbmib.BC_CHAR
    for name, ac, steps in (("central", lbmib.AC_CENTRAL, 20), ("mach_weighted", lbmib.AC_UPWIND, 5000)):
        s = lbmib.Solver("D2Q9", "fp32", (256, 128), mach=2.0, reynolds=300.0, ref_length=20.0, theta_inf=0.02,
                         bc=[0] * 4, use_ac=ac)
        f0, E0 = s.state()          # the uniform free stream the case starts from
        rng = np.random.Generator(np.random.PCG64(7))
        s.set_state(f0 * (1.0 + 1e-3 * rng.standard_normal(f0.shape)), E0)
        rho = s.fields()[0]
        d0 = float(np.abs(rho - rho.mean()).max())
        s.step(steps)
        rho = s.fields()[0]
        out["stream_" + name] = {"steps": steps, "deviation_ratio": float(np.abs(rho - rho.mean()).max()) / d0}
        s.close()

    def standoff(p_line, x_stag, pinf, mach):
        """Stand-off (cells) from x_stag to where the pressure line (along +x)
        first reaches the normal-shock ratio going upstream."""
        row = p_line / pinf
        ps = 2 * g / (g + 1) * mach * mach - (g - 1) / (g + 1)
        x0 = int(np.floor(x_stag))
        for x in range(x0, 0, -1):
            if row[x - 1] < ps <= row[x]:
                return x_stag - (x - 1 + (ps - row[x - 1]) / (row[x] - row[x - 1]))
        return float("nan")

    def ramp_run(make, mach, stages, per, final, m0, chunk, sample):
        """Restarts at Mach numbers from m0 to mach (fixed theta and mu), then
        `final` steps at mach with a check every `chunk` steps; sample(s, k)
        is called after each chunk of the last stage."""
        state, done, failed = None, 0, None
        machs = [mach] if stages == 1 else list(np.linspace(m0, mach, stages))
        for k, m in enumerate(machs):
            s = make(float(m))
            if state is not None:
                s.set_state(*state)
            n = per if k < len(machs) - 1 else final
            for j in range(n // chunk):
                s.step(chunk)
                done += chunk
                try:
                    s.check()
                except lbmib.LBMError:
                    failed = done
                    break
                if k == len(machs) - 1:
                    sample(s, (j + 1) * chunk)
            if failed is not None or k == len(machs) - 1:
                s.close()
                return done, failed
            state = s.state()
            s.close()

    # (2) NACA0012, Mach 0.8, Re 500, 10 degrees
    t0 = time.perf_counter()
    a = np.deg2rad(10.0)
    hist = []

    def naca(m):
        s = lbmib.Solver("D2Q9", "fp32", (1024, 512), mach=m, reynolds=500.0, ref_length=100.0, theta_inf=0.1,
                         bc=[lbmib.BC_INLET, CH, CH, CH], inflow_dir=(np.cos(a), np.sin(a), 0.0),
                         use_ac=lbmib.AC_UPWIND)
        s.set_geometry(inputs.naca0012((300.0, 256.0), 100.0, 256, tbc=1, t_value=0.0))
        return s

    def naca_sample(s, k):
        if k > 20000:
            d = s.wall_diagnostics(per_point=False)
            hist.append((d["Cd"], d["Cl"]))
    done, failed = ramp_run(naca, 0.8, 1, 0, 30000, 0.8, 100, naca_sample)
    h = np.array(hist) if hist else np.full((1, 2), np.nan)
    out["naca0012_mach0.8"] = {"Cd": float(h[:, 0].mean()), "Cl": float(h[:, 1].mean()), "steps": done,
                               "failed_at_step": failed, "wall_s": time.perf_counter() - t0,
                               "paper_FODIBM_R": {"Cd": 0.2638, "Cl": 0.4196}}

    # (3) sphere, Mach 1.2, Re 300
    t0 = time.perf_counter()
    Ds, ths = args.sup_sphere_d, 0.02
    sh = (12 * Ds, 8 * Ds, 8 * Ds)
    hist, last = [], {}

    def sph(m):
        s = lbmib.Solver("D3Q19", "fp32", sh, mach=m, reynolds=300.0 * m / 1.2, ref_length=float(Ds), theta_inf=ths,
                         bc=[lbmib.BC_INLET] + [CH] * 5, use_ac=lbmib.AC_UPWIND, bulk_ratio=3.0)
        s.set_geometry(inputs.icosphere((3.0 * Ds, 4.0 * Ds, 4.0 * Ds), float(Ds), 16, tbc=1, t_value=0.0))
        return s

    def sph_sample(s, k):
        if k > 22500:
            hist.append(s.wall_diagnostics(per_point=False)["Cd"])
        if k == 30000:
            _, _, _, p = s.fields()
            last["standoff_D"] = standoff(p[4 * Ds, 4 * Ds], 2.5 * Ds, ths / 3.0, 1.2) / Ds
    done, failed = ramp_run(sph, 1.2, 8, 1500, 30000, 0.3, 1500, sph_sample)
    out["sphere_mach1.2"] = {"Cd": float(np.mean(hist)) if hist else float("nan"),
                             "standoff_D": last.get("standoff_D", float("nan")), "D": Ds, "steps": done,
                             "failed_at_step": failed, "wall_s": time.perf_counter() - t0,
                             "paper_FODIBM_R": {"Cd": 1.287, "standoff_D": 0.678}}

    # (4) cylinder, Mach 2, Re 300
    t0 = time.perf_counter()
    D, th, bulk = args.sup_d, args.sup_theta, args.sup_bulk
    nx, ny, xc = 40 * D, 20 * D, 10.0 * D
    yc = ny / 2.0
    hist = []

    def cyl(m):
        s = lbmib.Solver("D2Q9", "fp32", (nx, ny), mach=m, reynolds=300.0 * m / 2.0, ref_length=float(D),
                         theta_inf=th, bc=[lbmib.BC_INLET, CH, CH, CH], use_ac=lbmib.AC_UPWIND, bulk_ratio=bulk)
        s.set_geometry(inputs.cylinder((xc, yc), float(D), int(np.pi * D), tbc=1, t_value=0.0))
        return s

    def cyl_sample(s, k):
        if k % 10000 == 0:
            d = s.wall_diagnostics(per_point=False)
            _, _, _, p = s.fields()
            hist.append({"steps_at_mach2": k, "Cd": float(d["Cd"]),
                         "standoff_D": standoff(p[int(round(yc))], xc - D / 2.0, th / 3.0, 2.0) / D})
    done, failed = ramp_run(cyl, 2.0, 16, 2000, args.sup_steps, 0.5, 2000, cyl_sample)
    out["cylinder_mach2"] = {"history": hist, "failed_at_step": failed, "ramp_steps": 15 * 2000, "D": D,
                             "wall_s": time.perf_counter() - t0, "paper_FODIBM_R": {"Cd": 1.57, "standoff_D": 0.71}}
    line = {"metric": "high-Mach operating points: uniform-stream stability, NACA0012 at Mach 0.8, sphere at "
                      "Mach 1.2, cylinder at Mach 2",
            "value": out["sphere_mach1.2"]["Cd"], "unit": "C_d (sphere, Mach 1.2)", "n_gpus": 1,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Mach 2 uniform stream 256x128; NACA0012 Ma 0.8 Re 500 10 deg chord 100 "
                                   "(1024x512); sphere Ma 1.2 Re 300 D = %d (%dx%dx%d); cylinder Ma 2 Re 300 "
                                   "D = %d (%dx%d), theta_inf %.3f, bulk viscosity %.1f mu"
                                   % (Ds, sh[0], sh[1], sh[2], D, nx, ny, th, bulk)},
            "results": out}
    print(json.dumps(line), flush=True)


def run_airfoil(args):
    """The NACA0012 airfoil case at full size: chord 400 cells, 1024
    Lagrangian points, grid 2048x1024 (leading edge at (512, 512); 5.1 x 2.6
    chords), Re 5000, Mach 0.5 and 0.8 at angles of attack 0-5 degrees in
    steps of 1, adiabatic wall, inlet and characteristic faces, theta_inf from
    the built-in rule at Mach 0.5 (0.193) and 0.05 at Mach 0.8 (the rule's
    0.075 diverges there within 2000 steps), the Mach-weighted upstream a^C
    stencil (LBM_AC_UPWIND), FP32, uniform start.  Per case: C_d and C_l as means over the last 5 of
    `--af-chords` chord flow-through times (spread = largest deviation from
    the mean), the wall C_p extremes and the chordwise position of the upper
    surface's C_p minimum at the end, and the MLUPS of 2000 timed steps."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    chord, nx, ny, le = 400.0, 2048, 1024, (512.0, 512.0)
    geo = inputs.naca0012(le, chord, 1024, tbc=1, t_value=0.0)
    out = {}
    for mach in (0.5, 0.8):
        for aoa in (0.0, 1.0, 2.0, 3.0, 4.0, 5.0):
            a = np.deg2rad(aoa)
            s = lbmib.Solver("D2Q9", "fp32", (nx, ny), mach=mach, reynolds=5000.0, ref_length=chord,
                             theta_inf=0.0 if mach < 0.6 else 0.05,
                             bc=[lbmib.BC_INLET] + [lbmib.BC_CHAR] * 3, inflow_dir=(np.cos(a), np.sin(a), 0.0),
                             use_ac=lbmib.AC_UPWIND)
            s.set_geometry(geo)
            per_chord = int(chord / s.constants()["u_mag"])
            every = 200
            n_total = args.af_chords * per_chord // every * every
            n_avg = 5 * per_chord // every
            s.step(200)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(2000)
            torch.cuda.synchronize()
            mlups = nx * ny * 2000 / (time.perf_counter() - t0) / 1e6
            hist = []
            for _ in range((n_total - 2200) // every):
                s.step(every)
                d = s.wall_diagnostics(per_point=False)
                hist.append((d["Cd"], d["Cl"]))
            s.check()
            d = s.wall_diagnostics(per_point=True)
            h = np.array(hist[-n_avg:])
            cp = d["Cp"]
            out["Ma%.1f_aoa%.1f" % (mach, aoa)] = {
                "Cd": float(h[:, 0].mean()), "Cl": float(h[:, 1].mean()),
                "Cd_spread": float(np.abs(h[:, 0] - h[:, 0].mean()).max()),
                "Cl_spread": float(np.abs(h[:, 1] - h[:, 1].mean()).max()),
                "Cp_min": float(cp.min()), "Cp_max": float(cp.max()),
                "upper_Cp_min_at_x_over_c": _upper_cp_min(geo, cp, le, chord),
                "steps": n_total, "mlups_fp32": mlups}
            s.close()
    line = {"metric": "NACA0012 at full size (chord 400, 2048x1024): C_d, C_l and wall C_p over Mach 0.5 / 0.8 "
                      "and angle of attack 0-5 deg",
            "value": out["Ma0.8_aoa2.0"]["Cl"], "unit": "C_l (Mach 0.8, 2 deg)", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "NACA0012 chord 400, 1024 points, 2048x1024, Re 5000, adiabatic, theta_inf 0.193 "
                                   "(Ma 0.5) / 0.05 (Ma 0.8), LBM_AC_UPWIND, %d chord flow-throughs" % args.af_chords},
            "cases": out}
    print(json.dumps(line), flush=True)


def _upper_cp_min(geo, cp, le, chord):
    """x/c of the smallest C_p among the Lagrangian points above the chord
    line (y > leading-edge y)."""
    X = np.asarray(geo.X if hasattr(geo, "X") else geo["X"], dtype=np.float64).reshape(len(cp), -1)
    up = X[:, 1] > le[1]
    if not up.any():
        return float("nan")
    i = np.argmin(np.where(up, cp, np.inf))
    return float((X[i, 0] - le[0]) / chord)


def run_precision_mach12(args):
    """Reduced-precision storage on the 3D sphere at Mach 1.2 (Re 300,
    isothermal wall 1.1 T_inf, 256x192x192, D = 48 centred at (100, 96, 96),
    inlet and characteristic faces, theta_inf 0.02, the Mach-weighted a^C
    stencil, bulk viscosity 3 mu).  The FP32 path ramps the Mach number from
    0.3 to 1.2 in 8 restarts of 1500 steps and runs `--p12-settle` steps at
    Mach 1.2; from that state FP32, FP16 and BF16 storage each run
    `--p12-steps` steps, and C_d and Nu are averaged over the last half."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    shape, D, center = SHAPE, 48.0, (100.0, 96.0, 96.0)
    CH = lbmib.BC_CHAR
    th = 0.02

    def make(prec, m):
        s = lbmib.Solver("D3Q19", prec, shape, mach=m, reynolds=300.0 * m / 1.2, ref_length=D, theta_inf=th,
                         bc=[lbmib.BC_INLET] + [CH] * 5, use_ac=lbmib.AC_UPWIND, bulk_ratio=3.0)
        s.set_geometry(inputs.icosphere(center, D, 27, tbc=0, t_value=1.1 * th))
        return s

    t0 = time.perf_counter()
    state = None
    for k, m in enumerate(np.linspace(0.3, 1.2, 8)):
        s = make("fp32", float(m))
        if state is not None:
            s.set_state(*state)
        s.step(1500 if k < 7 else args.p12_settle)
        s.check()
        state = s.state()
        s.close()
    ramp_s = time.perf_counter() - t0
    res = {}
    for prec in ("fp32", "fp16", "bf16"):
        s = make(prec, 1.2)
        s.set_state(*state)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        cd, nu = coefficient_history(s, args.p12_steps, 50)
        torch.cuda.synchronize()
        el = time.perf_counter() - t1
        s.check()
        s.close()
        h = len(cd) // 2
        res[prec] = {"Cd": float(np.mean(cd[h:])), "Nu": float(np.mean(nu[h:])), "wall_s": el,
                     "mlups": float(np.prod(shape)) * args.p12_steps / el / 1e6}
    for prec, r in res.items():
        r["Cd_rel_vs_fp32"] = r["Cd"] / res["fp32"]["Cd"] - 1.0
        r["Nu_rel_vs_fp32"] = r["Nu"] / res["fp32"]["Nu"] - 1.0
    line = {"metric": "C_d and Nu by storage form, 3D sphere at Mach 1.2 (Re 300, 256x192x192)",
            "value": res["bf16"]["Cd_rel_vs_fp32"], "unit": "relative C_d vs FP32 (BF16)", "n_gpus": 1,
            "higher_is_better": False, "dtype": "f32 / f16 / bf16 storage, f32 math", "data": "synthetic",
            "config": {"workload": "3D sphere D3Q19 Ma 1.2 Re 300 D = 48, isothermal wall 1.1 T_inf, theta_inf 0.02, "
                                   "LBM_AC_UPWIND, bulk viscosity 3 mu; ramp %.1f s; %d settle + %d steps per form"
                                   % (ramp_s, args.p12_settle, args.p12_steps)},
            "forms": res}
    print(json.dumps(line), flush=True)


def run_nop(args):
    """Speed of the warm-start network (512x256, batch 8, channels
    32-64-96-128, 3 inputs, 4 outputs): forward pass and training step
    (forward, backward, Adam), each timed over `--nop-steps` calls after
    warm-up, with the forward FLOP count of its convolutions."""
    import torch
    from paper_2607_07432_b300.nop import NeuralOperator
    H, W, B, ch = 256, 512, 8, (32, 64, 96, 128)
    n = NeuralOperator(height=H, width=W, max_batch=B, channels=ch)
    n.init_params(1)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((B, H, W, 3), device="cuda", generator=g)
    y = torch.empty((B, H, W, 4), device="cuda")
    t = torch.randn((B, H, W, 4), device="cuda", generator=g)
    K = args.nop_steps
    for _ in range(2):
        n.forward(x, y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        n.forward(x, y)
    torch.cuda.synchronize()
    fw = (time.perf_counter() - t0) / K * 1e3
    for _ in range(2):
        n.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        n.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    tr = (time.perf_counter() - t0) / K * 1e3
    n.close()
    # forward FLOPs: 2 x 9 x c_in x c_out per pixel of each convolution's level
    # (skip connections are added, so a decoder convolution takes the coarser level's channels)
    shapes = [(3, ch[0]), (ch[0], ch[0]), (ch[0], ch[1]), (ch[1], ch[1]), (ch[1], ch[2]), (ch[2], ch[2]),
              (ch[2], ch[3]), (ch[3], ch[3]), (ch[3], ch[2]), (ch[2], ch[2]), (ch[2], ch[1]), (ch[1], ch[1]),
              (ch[1], ch[0]), (ch[0], ch[0]), (ch[0], 4)]
    levels = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0]
    fl = sum(2 * 9 * ci * co * B * (H >> l) * (W >> l) for (ci, co), l in zip(shapes, levels))
    line = {"metric": "warm-start network: forward and training-step time (512x256, batch 8)",
            "value": tr, "unit": "ms per training step", "n_gpus": 1, "higher_is_better": False,
            "dtype": "bf16 x bf16 -> f32", "data": "synthetic",
            "config": {"workload": "4-level U-Net 32-64-96-128 channels, 512x256, batch 8", "calls": K},
            "forward_ms": fw, "forward_tflops": fl / fw / 1e9, "train_tflops_3x_forward": 3 * fl / tr / 1e9}
    print(json.dumps(line), flush=True)


def run_precision(args):
    """Reduced-precision storage on the 3D sphere case (Ma 0.3, Re 300,
    isothermal wall): C_d and Nu as running means, and the steps until the
    running mean of C_d settles within 0.1%, for FP32, FP16 and BF16 on the
    full 256x192x192 grid (D = 48) and, with the FP64 path (which equals the
    oracle to 1e-12), on the 64x48x48 downscale (D = 12)."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    out = {}
    for name, shape, D, freq, steps, window, forms in (
            ("downscale_64x48x48", (64, 48, 48), 12.0, 7, args.prec_steps_small, 2500, ("fp64", "fp32", "fp16", "bf16")),
            ("full_256x192x192", SHAPE, 48.0, 27, args.prec_steps_full, 10000, ("fp32", "fp16", "bf16"))):
        res = {}
        for prec in forms:
            s = _sphere(lbmib, inputs, prec, shape, D, freq)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cd, nu = coefficient_history(s, steps, 50)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            s.close()
            r = steady_summary(cd, nu, 50, window)
            r["wall_s"] = el
            r["mlups"] = float(np.prod(shape)) * steps / el / 1e6
            res[prec] = r
        base = res["fp32"]
        for prec, r in res.items():
            r["Cd_rel_vs_fp32"] = r["Cd"] / base["Cd"] - 1.0
            r["Nu_rel_vs_fp32"] = r["Nu"] / base["Nu"] - 1.0
            if "fp64" in res:
                r["Cd_rel_vs_fp64"] = r["Cd"] / res["fp64"]["Cd"] - 1.0
                r["Nu_rel_vs_fp64"] = r["Nu"] / res["fp64"]["Nu"] - 1.0
        out[name] = dict(steps=steps, window=window, forms=res)
    line = {"metric": "C_d and Nu running means by storage form, 3D sphere (Ma 0.3, Re 300); steps to 0.1% drag",
            "value": out["full_256x192x192"]["forms"]["fp16"]["Cd_rel_vs_fp32"], "unit": "relative C_d vs FP32 (FP16)",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f32 / f16 / bf16 storage, f32 math", "data": "synthetic",
            "config": {"workload": "3D sphere D3Q19, Ma 0.3, Re 300, isothermal wall 1.1 T_inf, uniform start"},
            "cases": out}
    print(json.dumps(line), flush=True)


def run_convergence(args):
    """Grid convergence of the wall pressure coefficient (paper Sec. 3.1: L2
    error of C_p against the finest mesh at identical wall locations), read
    at X_l (Eq. int1, d = 2, nodes on both sides of the wall) and at the
    projection points (d = 1, fluid nodes), and of C_d: the
    2D cylinder case (Ma 0.2, Re 40, isothermal wall 1.1 T_inf, FODIBM-R and
    FODIBM) at D = 20, 40, 80 on 10D x 5D grids, against D = 160; 64 D / 20
    Lagrangian points so that every coarse point is also a fine point; FP32;
    characteristic far field on the outflow and lateral faces; each run to a
    steady C_d (change below 0.01% over two convective times)."""
    import torch
    from paper_2607_07432_b300 import inputs, lbmib
    Ds = (20, 40, 80, 160)
    res = {}
    for method in (lbmib.FODIBM_R, lbmib.FODIBM):
        cps = {}
        for D in Ds:
            nx, ny = 10 * D, 5 * D
            s = lbmib.Solver("D2Q9", "fp32", (nx, ny), mach=0.2, reynolds=40.0, ref_length=float(D),
                             method=method, bc=[lbmib.BC_INLET, lbmib.BC_CHAR, lbmib.BC_CHAR, lbmib.BC_CHAR])
            c = s.constants()
            th = c["theta_inf"]
            s.set_geometry(inputs.cylinder((3.0 * D, 2.5 * D), float(D), 64 * D // 20, tbc=0, t_value=1.1 * th))
            chunk = int(2 * D / c["u_mag"])
            prev, steps = None, 0
            t0 = time.perf_counter()
            while True:
                s.step(chunk)
                steps += chunk
                cd = s.wall_diagnostics(per_point=False)["Cd"]
                if prev is not None and abs(cd - prev) < 1e-4 * abs(cd) and steps > 20 * chunk:
                    break
                prev = cd
                if steps > 400 * chunk:
                    break
            s.check()
            d = s.wall_diagnostics()
            cps[D] = dict(Cp=d["Cp"], CpP=d["CpP"], Cd=d["Cd"], steps=steps, theta_inf=th,
                          wall_s=time.perf_counter() - t0)
            s.close()
        out = {}
        for key in ("Cp", "CpP"):
            ref = cps[Ds[-1]][key]
            err = {}
            for D in Ds[:-1]:
                r = ref[::Ds[-1] // D]
                err[D] = float(np.sqrt(((cps[D][key] - r) ** 2).sum() / (r ** 2).sum()))
            orders = [float(np.log(err[Ds[k]] / err[Ds[k + 1]]) / np.log(2.0)) for k in range(len(Ds) - 2)]
            out[key] = dict(L2_error=err, observed_order=orders)
        cds = [cps[D]["Cd"] for D in Ds]
        out["Cd_order"] = [float(np.log(abs(cds[k] - cds[k + 1]) / abs(cds[k + 1] - cds[k + 2])) / np.log(2.0))
                           for k in range(len(Ds) - 2)]
        out["runs"] = {D: dict(Cd=v["Cd"], steps=v["steps"], theta_inf=v["theta_inf"], wall_s=v["wall_s"])
                       for D, v in cps.items()}
        res["FODIBM-R" if method == lbmib.FODIBM_R else "FODIBM"] = out
    line = {"metric": "L2 error of C_p against D = 160 and observed order (2D cylinder, Ma 0.2, Re 40)",
            "value": res["FODIBM-R"]["CpP"]["observed_order"][-1], "unit": "order", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic", "config": {"workload": "2D cylinder, 10D x 5D, D = 20/40/80/160"},
            "results": res}
    print(json.dumps(line), flush=True)


def run_warmstart(args):
    """Learned warm start on 512x256 two-body cases (a circle and an
    ellipse, diameters 10-40 cells, Ma 0.1 to --ws-mach-max (0.45 at most
    with the default stencil, whose bluff bodies above it diverge; up to 0.8
    with --ws-high-mach, which steps every case with the Mach-weighted
    upstream a^C stencil at u_inf <= 0.1 and counts the cases that still
    fail), Re 20-45 so that every case has a steady state): generate the training fields with the batched
    solver, train the network on the GPU, then report steps and wall-clock
    to the 0.1% drag band of the uniform-start answer, warm vs uniform, on
    held-out cases.  Not a per-step throughput line: the metric is
    time-to-steady."""
    import torch
    from paper_2607_07432_b300 import inputs, warmstart as ws
    shape = (512, 256)
    kw = dict(shape=shape, d_range=(10.0, 40.0), mach_range=(0.1, args.ws_mach_max), re_range=(20.0, 45.0))
    n_train, gen_steps, train_steps, n_test, run_steps = (args.ws_cases, args.ws_gen_steps, args.ws_train_steps,
                                                          args.ws_test, 40000)
    train_cases = inputs.warmstart_cases(n_train, 20260002, **kw)
    test_cases = inputs.warmstart_cases(n_test, 20260003, **kw)
    t0 = time.perf_counter()
    hm = args.ws_high_mach
    gen_failed = []
    X, Y = ws.generate(train_cases, gen_steps, hm=hm, failed=gen_failed if hm else None)
    t_gen = time.perf_counter() - t0
    net = ws.new_network(shape, max_batch=8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = ws.train(net, X, Y, train_steps, 8, 1e-3, lr_final=1e-4)
    t_train = time.perf_counter() - t0
    res = [ws.compare(net, c, run_steps, 100, hm=hm) for c in test_cases]
    net.close()
    # the uniform run's drag at the end of the run is the reference answer;
    # it is trusted only where that run has stayed in the band for the last
    # 10000 steps ("settled"); the other cases are counted, not averaged
    settled = [r for r in res if "diverged" not in r and r["steps_uniform"] and
               r["steps_uniform"] <= run_steps - 10000]
    ok = [r for r in settled if r["steps_warm"]]
    su = float(np.mean([r["steps_uniform"] for r in ok])) if ok else None
    sw = float(np.mean([r["steps_warm"] for r in ok])) if ok else None
    mu = float(np.mean([r["ms_uniform"] for r in ok])) if ok else None
    mw = float(np.mean([r["ms_warm"] for r in ok])) if ok else None
    line = {"metric": "steps to the 0.1% drag band, warm start vs uniform start (mean over settled held-out cases)",
            "value": sw, "unit": "steps", "n_gpus": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 solver, bf16 x bf16 -> f32 network", "data": "synthetic",
            "config": {"workload": "2D two-body cases 512x256 (circle + ellipse, D 10-40, Ma 0.1-%.2f, Re 20-45)%s"
                                   % (args.ws_mach_max, ", Mach-weighted a^C stencil, u_inf <= 0.1" if hm else ""),
                       "train_cases": n_train, "gen_steps": gen_steps, "train_steps": train_steps, "batch": 8,
                       "held_out": n_test},
            "uniform_steps": su, "warm_ms": mw, "uniform_ms": mu, "step_ratio": (sw / su) if ok else None,
            "settled_cases": len(settled), "warm_missed_band": len(settled) - len(ok),
            "warm_faster": sum(r["steps_warm"] < r["steps_uniform"] for r in ok),
            "unsettled_reference": len(res) - len(settled) - sum("diverged" in r for r in res),
            "diverged_uniform": sum(r.get("diverged") == "uniform" for r in res),
            "diverged_warm": sum(r.get("diverged") == "warm" for r in res),
            "training_cases_failed": len(gen_failed),
            "gen_s": t_gen, "train_s": t_train, "final_loss": float(losses[-50:].mean()),
            "cases": res}
    print(json.dumps(line), flush=True)


def time_form(lbmib, inputs, precision, steps, warmup, N, peak):
    """One storage form of the sphere case: device-timed MLUPS of the whole
    step and the fused kernel's time from a profiled pass of the same steps."""
    import torch
    s, _ = build_case(lbmib, inputs, precision)
    s.step(warmup)
    s.check()
    s.profile(True, True)
    torch.cuda.synchronize()
    s.step(steps)
    torch.cuda.synchronize()
    prof = s.get_profile()
    s.profile(False, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    s.step(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.check()
    s.close()
    kern_ms = prof["step"][0] / steps
    bpl = bytes_per_lu("D3Q19", precision)
    return {"value": N * steps / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms / steps,
            "kernel_ms_per_step": kern_ms, "bytes_per_lu": bpl,
            "roofline_frac": bpl * N / (kern_ms / 1e3) / 1e9 / peak}


def other_forms(args, lbmib, inputs, N, peak):
    """The reduced-precision storage forms of the same case and the 64-case
    batch, measured on the same box as the headline (compact sub-records)."""
    out = {}
    for prec in ("fp16", "bf16"):
        out[prec] = time_form(lbmib, inputs, prec, args.steps, args.warmup, N, peak)
    b = run_batch(argparse.Namespace(steps=max(20, args.steps // 2), warmup=args.warmup), emit=False)
    out["batch64"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "sequential", "speedup_vs_sequential",
                                        "ms_per_step_by_form")}
    out["batch64"]["plan"] = b["config"]["plan"]
    out["batch64"]["workload"] = b["config"]["workload"]
    out["batch64"]["nodes"] = b["config"]["nodes"]
    return out


def run_slabs(args, rank, world, local, dist, lbmib, inputs):
    """The partitioned case on N ranks: rank r owns planes [192 r, 192 r +
    192) of a 256 x 192 x 192N channel whose sphere r (D = 48, 7292 points)
    sits at z = 192 r + 96; ghost planes (10 per cut) are exchanged with NCCL
    point-to-point transfers after every step; the wall loads are added over
    ranks in rank order."""
    import torch
    from paper_2607_07432_b300 import slab
    c = CASE
    nz = SHAPE[2] * world
    gshape = (SHAPE[0], SHAPE[1], nz)
    halo = slab.MIN_HALO
    p = slab.plan(nz, world, halo)[rank]
    s = lbmib.Solver(c["lattice"], args.precision, gshape, mach=c["mach"], reynolds=c["reynolds"],
                     ref_length=c["ref_length"], bc=[lbmib.BC_INLET, lbmib.BC_OUTLET] + [lbmib.BC_FARFIELD] * 4,
                     slab=(p["z0"], p["z1"], halo))
    th = s.constants()["theta_inf"]
    center = (c["center"][0], c["center"][1], float(p["z0"]) + c["center"][2])
    s.set_geometry(inputs.icosphere(center, c["diameter"], c["frequency"], tbc=0, t_value=1.1 * th))
    bufs = slab.Buffers(s, "cuda")

    def step(n):
        for _ in range(n):
            s.step(1)
            slab.exchange_dist(s, bufs, rank, world, dist)

    def barrier():
        dist.barrier()
        torch.cuda.synchronize()

    step(args.warmup)
    s.check()
    own = SHAPE[0] * SHAPE[1] * (p["z1"] - p["z0"])
    total = int(np.prod(gshape))
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    l0 = s.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.begin()
    e0.record()
    step(args.steps)
    e1.record()
    barrier()
    clocks.end()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    launches = s.launch_count() - l0
    s.check()
    # end to end: initial fields from pinned host memory, steps with the
    # exchange, the body's loads gathered from every rank each step
    Nloc = s.N
    rho0 = torch.full((Nloc,), 1.0, dtype=torch.float64).pin_memory()
    u0 = torch.zeros((3 * Nloc,), dtype=torch.float64)
    u0[:Nloc] = s.constants()["u_mag"]
    u0 = u0.pin_memory()
    T0 = torch.full((Nloc,), th, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    s.set_fields(rho0.numpy(), u0.numpy(), T0.numpy())
    for _ in range(args.steps):
        step(1)
        wl = s.wall_loads()
        part = torch.tensor(list(wl["force"]) + [wl["heat"], wl["work"]], dtype=torch.float64, device="cuda")
        gathered = [torch.empty_like(part) for _ in range(world)]
        dist.all_gather(gathered, part)
        slab.reduce_loads([dict(force=g[:3].cpu().numpy(), heat=float(g[3]), work=float(g[4])) for g in gathered])
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    if rank != 0:
        s.close()
        return
    peak, _ = peaks()
    line = {"metric": METRIC, "value": total * args.steps / (ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
            "data": "synthetic",
            "config": {"workload": "3D spheres D3Q19 256x192x(192 N), one D=48 sphere (7292 points) per 192 planes, "
                                   "Ma 0.3, Re 300, isothermal walls, FODIBM-R",
                       "precision": args.precision, "parallelism": "z slabs, %d ranks, halo %d" % (world, halo),
                       "l2": "inputs larger than L2, no flush"},
            "roofline": None, "cpu_baseline": None,
            "e2e": {"value": total * args.steps / e2e_s / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": int(Nloc * 5 * 8 / args.steps), "d2h_bytes_per_step": 5 * 8 * world},
            "gpu_launches": launches, "clocks": clk,
            "exchange_bytes_per_step_per_rank": sum(bufs.send[k].numel() for k in (0, 1)
                                                    if bufs.send[k] is not None)}
    print(json.dumps(line), flush=True)
    s.close()


def max_over_ranks(x, dist, device):
    """The slowest rank's time (every rank gets it); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, nodes, steps, seconds):
    """Whole-job throughput: every rank advances its own replica of `nodes`
    nodes by `steps` steps in `seconds` (the slowest rank's time)."""
    return world * nodes * steps / seconds / 1e6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-forms", action="store_true",
                    help="skip the FP16 / BF16 storage and 64-case batch sub-records")
    ap.add_argument("--workload", default="sphere", choices=["sphere", "batch64", "warmstart", "precision",
                                                                    "convergence", "rotsphere", "refined",
                                                                    "refined_sphere", "supersonic", "airfoil",
                                                                    "precision_mach12", "nop"])
    ap.add_argument("--ref-steps", type=int, default=40000)
    ap.add_argument("--ref-lo", type=int, nargs=2, default=[30, 20])
    ap.add_argument("--ref-hi", type=int, nargs=2, default=[150, 80])
    ap.add_argument("--rot-steps", type=int, default=36000)
    ap.add_argument("--rot-window", type=int, default=16000)
    ap.add_argument("--rot-d", type=int, default=48, help="sphere diameter in cells (grid 10D x 6D x 6D)")
    ap.add_argument("--rot-noise", type=float, default=0.01)
    ap.add_argument("--rot-omegas", default="0.3,0.6")
    ap.add_argument("--nop-steps", type=int, default=10)
    ap.add_argument("--p12-settle", type=int, default=12000)
    ap.add_argument("--p12-steps", type=int, default=16000)
    ap.add_argument("--af-chords", type=int, default=15, help="chord flow-through times per airfoil case")
    ap.add_argument("--sup-d", type=int, default=60, help="cylinder diameter in cells (Mach 2 workload)")
    ap.add_argument("--sup-theta", type=float, default=0.02)
    ap.add_argument("--sup-bulk", type=float, default=3.0, help="artificial bulk viscosity over mu")
    ap.add_argument("--sup-steps", type=int, default=40000, help="steps at Mach 2 after the ramp")
    ap.add_argument("--sup-sphere-d", type=int, default=32, help="sphere diameter in cells (Mach 1.2)")
    ap.add_argument("--prec-steps-small", type=int, default=20000)
    ap.add_argument("--prec-steps-full", type=int, default=40000)
    ap.add_argument("--ws-cases", type=int, default=256)
    ap.add_argument("--ws-gen-steps", type=int, default=24000)
    ap.add_argument("--ws-train-steps", type=int, default=2000)
    ap.add_argument("--ws-test", type=int, default=8, help="held-out cases")
    ap.add_argument("--ws-mach-max", type=float, default=0.3)
    ap.add_argument("--ws-high-mach", action="store_true",
                    help="Mach-weighted upstream a^C stencil and u_inf <= 0.1 for every case (for Ma up to 0.8)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "convergence":
        return run_convergence(args)
    if args.workload == "supersonic":
        return run_supersonic(args)
    if args.workload == "airfoil":
        return run_airfoil(args)
    if args.workload == "precision_mach12":
        return run_precision_mach12(args)
    if args.workload == "nop":
        return run_nop(args)
    if args.workload == "rotsphere":
        return run_rotsphere(args)
    if args.workload == "refined":
        return run_refined(args)
    if args.workload == "refined_sphere":
        return run_refined_sphere(args)
    args.warmup = max(args.warmup, 3)
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2607_07432_b300 import inputs, lbmib
    if world > 1:
        return run_slabs(args, rank, world, local, dist, lbmib, inputs)
    s, geo = build_case(lbmib, inputs, args.precision)
    N = int(np.prod(SHAPE))
    s.step(args.warmup)
    s.check()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # device-timed region: K steps, inputs resident in HBM (each step reads
    # about 1 GB of state, far more than L2, so no flush is needed)
    # per-kernel breakdown (roofline of the fused kernel): one pass of the
    # same K steps with CUDA events recorded around every launch
    s.profile(True, True)
    barrier()
    s.step(args.steps)
    barrier()
    prof = s.get_profile()
    s.profile(False, True)
    # timed region: the plain step path, no profiling events
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    l0 = s.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.begin()
    e0.record()
    s.step(args.steps)
    e1.record()
    barrier()
    clocks.end()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = s.launch_count() - l0
    ms = max_over_ranks(ms, dist, "cuda")
    ms_step = ms / args.steps
    value = job_mlups(world, N, args.steps, ms / 1e3)
    s.check()

    # end-to-end through the public API with host buffers: the job uploads
    # its initial fields from pinned host memory, steps, and copies the wall
    # loads of every step into its own row of a pinned host array (queued
    # behind the step, no per-step wait); after the last step it waits once
    # and reads them all.  Every copy is inside the timed region.
    c = s.constants()
    rho0 = torch.full((N,), 1.0, dtype=torch.float64).pin_memory()
    u0 = torch.zeros((3 * N,), dtype=torch.float64)
    u0[:N] = c["u_mag"]
    u0 = u0.pin_memory()
    T0 = torch.full((N,), c["theta_inf"], dtype=torch.float64).pin_memory()
    loads_h = torch.zeros((args.steps, 5), dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    s.set_fields(rho0.numpy(), u0.numpy(), T0.numpy())
    for k in range(args.steps):
        s.step(1)
        s.wall_loads_async(loads_h[k])
    s.sync()
    drag_hist = loads_h[:, 0].numpy().copy()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    if not np.all(np.isfinite(drag_hist)):
        raise RuntimeError("non-finite wall loads in the end-to-end run")
    e2e = {"value": job_mlups(world, N, args.steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(N * 5 * 8 / args.steps), "d2h_bytes_per_step": 5 * 8}

    if rank != 0:
        return
    peak, peak_kind = peaks()
    bpl = bytes_per_lu(CASE["lattice"], args.precision)
    bpl_diag = bytes_per_lu(CASE["lattice"], args.precision, ndev=2)
    step_ms, step_n = prof["step"]
    other_ms, other_n = prof["other"]
    # dominant kernel: the fused collide-stream-energy step kernel
    kern_ms = (step_ms + other_ms) / args.steps
    achieved = bpl * N / (kern_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": kernel_traffic() if args.precision == "fp32" else None, "peak_kind": peak_kind,
            "bytes_per_lu": bpl,
            "frac_at_diagonal_aC_bytes": bpl_diag * N / (kern_ms / 1e3) / 1e9 / peak,
            "bytes_per_lu_diagonal_aC": bpl_diag,
            "kernel_ms_per_step": kern_ms,
            "breakdown_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}
    s.close()
    others = None
    if not args.no_other_forms and world == 1 and args.precision == "fp32":
        others = other_forms(args, lbmib, inputs, N, peak)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_record(15.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
            "data": "synthetic",
            "config": {"workload": "3D sphere D3Q19 256x192x192, D=48, 7292 points, Ma 0.3, Re 300, "
                                   "isothermal wall, FODIBM-R",
                       "precision": args.precision, "parallelism": "single",
                       "l2": "inputs larger than L2: each step reads %.2f GB of state (126 MB L2), no flush"
                             % (bpl * N / 2 / 1e9)},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    if others is not None:
        line["other_forms"] = others
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
