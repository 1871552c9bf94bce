"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds no arithmetic of the method: it only produces geometry
(Lagrangian points, outward normals, a shape description for the
inside/outside test) and case parameters.  Both the CUDA path and the CPU
oracle consume what it returns.

Workload recipes (shapes of the paper's cases, Sec. 3):
  * cylinder: circle of diameter D, N_L points uniform in angle (dx/ds ~ 1)
  * ellipse: aspect ratio a/b, N_L points uniform in arc length
  * NACA0012: closed-trailing-edge 4-digit thickness polynomial, points
    uniform in arc length on each side, leading edge at the given position
  * sphere: class-I geodesic icosphere of frequency nu (10 nu^2 + 2 points)
"""
import math

import numpy as np


def _as_geometry(X, N, shape, tbc, t_value, u_target=None):
    X = np.ascontiguousarray(X, dtype=np.float64)
    N = np.ascontiguousarray(N, dtype=np.float64)
    NL, D = X.shape
    if u_target is None:
        u_target = np.zeros((NL, D))
    return dict(X=X, normals=N, shape=shape,
                tbc=np.full(NL, int(tbc), dtype=np.int64) if np.isscalar(tbc) else np.asarray(tbc, dtype=np.int64),
                t_value=np.full(NL, float(t_value)) if np.isscalar(t_value) else np.asarray(t_value, dtype=np.float64),
                u_target=np.ascontiguousarray(u_target, dtype=np.float64))


def cylinder(center, diameter, n_points, tbc=0, t_value=1.0, phase=0.0):
    """Circle of the given diameter; point l at angle 2 pi l / n + phase."""
    r = 0.5 * diameter
    th = 2.0 * np.pi * np.arange(n_points) / n_points + phase
    N = np.stack([np.cos(th), np.sin(th)], axis=1)
    X = np.array(center[:2], dtype=np.float64)[None, :] + r * N
    shape = dict(kind="circle", center=np.array(center[:2], dtype=np.float64), radius=r)
    return _as_geometry(X, N, shape, tbc, t_value)


def ellipse(center, a, b, angle, n_points, tbc=0, t_value=1.0):
    """Ellipse with semi-axes a (along the rotated x) and b, rotated by
    `angle`; points uniform in arc length, outward normals."""
    t = np.linspace(0.0, 2.0 * np.pi, 20001)
    px, py = a * np.cos(t), b * np.sin(t)
    seg = np.hypot(np.diff(px), np.diff(py))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    tl = np.interp(np.arange(n_points) * s[-1] / n_points, s, t)
    ex, ey = a * np.cos(tl), b * np.sin(tl)
    nx, ny = ex / (a * a), ey / (b * b)
    nn = np.hypot(nx, ny)
    nx, ny = nx / nn, ny / nn
    cs, sn = math.cos(angle), math.sin(angle)
    X = np.stack([center[0] + cs * ex - sn * ey, center[1] + sn * ex + cs * ey], axis=1)
    N = np.stack([cs * nx - sn * ny, sn * nx + cs * ny], axis=1)
    shape = dict(kind="ellipse", center=np.array(center[:2], dtype=np.float64),
                 radii=(float(a), float(b)), cos=cs, sin=sn)
    return _as_geometry(X, N, shape, tbc, t_value)


def naca0012(leading_edge, chord, n_points, tbc=1, t_value=0.0):
    """NACA 0012 (t = 0.12) with the closed trailing edge (last coefficient
    -0.1036), n_points/2 points per side uniform in arc length, ordered
    counter-clockwise starting at the trailing edge."""
    t = 0.12
    xs = np.linspace(0.0, 1.0, 40001)
    yt = 5.0 * t * (0.2969 * np.sqrt(xs) - 0.1260 * xs - 0.3516 * xs ** 2 + 0.2843 * xs ** 3 - 0.1036 * xs ** 4)
    # upper surface from TE to LE, then lower from LE to TE
    ux, uy = xs[::-1], yt[::-1]
    lx, ly = xs[1:], -yt[1:]
    cx = np.concatenate([ux, lx])
    cy = np.concatenate([uy, ly])
    seg = np.hypot(np.diff(cx), np.diff(cy))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    sl = np.arange(n_points) * s[-1] / n_points
    px = np.interp(sl, s, cx)
    py = np.interp(sl, s, cy)
    # outward normal: perpendicular of the central chord through the neighbours
    dx = np.roll(px, -1) - np.roll(px, 1)
    dy = np.roll(py, -1) - np.roll(py, 1)
    nn = np.hypot(dx, dy)
    N = np.stack([dy / nn, -dx / nn], axis=1)
    X = np.stack([leading_edge[0] + chord * px, leading_edge[1] + chord * py], axis=1)
    # the curve runs counter-clockwise (upper surface first, TE -> LE), so
    # (dy, -dx) points outward
    shape = dict(kind="polygon", poly=X.copy())
    return _as_geometry(X, N, shape, tbc, t_value)


def icosphere(center, diameter, frequency, tbc=0, t_value=1.0):
    """Class-I geodesic subdivision of the icosahedron projected on the
    sphere: 10 nu^2 + 2 points, radial normals."""
    p = (1.0 + 5 ** 0.5) / 2.0
    V = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    nu = int(frequency)
    pts = {}
    for (a, b, c) in F:
        A, B, C = V[a], V[b], V[c]
        for i in range(nu + 1):
            for j in range(nu + 1 - i):
                k = nu - i - j
                q = (i * A + j * B + k * C) / nu
                q = q / np.linalg.norm(q)
                key = tuple(np.round(q, 9))
                pts[key] = q
    U = np.array(sorted(pts.values(), key=lambda v: (round(v[2], 9), round(v[1], 9), round(v[0], 9))))
    r = 0.5 * diameter
    X = np.array(center, dtype=np.float64)[None, :] + r * U
    shape = dict(kind="sphere", center=np.array(center, dtype=np.float64), radius=r)
    return _as_geometry(X, U, shape, tbc, t_value)


def rotating(geometry, center, omega):
    """Velocity targets of a body turning rigidly about `center`:
    u_target = omega x (X - center) (3D, omega a vector; 2D, omega the
    scalar rate about z).  Returns the geometry with its targets replaced."""
    X = geometry["X"]
    r = X - np.asarray(center, dtype=np.float64)[None, : X.shape[1]]
    if X.shape[1] == 2:
        w = float(omega)
        u = np.stack([-w * r[:, 1], w * r[:, 0]], axis=1)
    else:
        u = np.cross(np.broadcast_to(np.asarray(omega, dtype=np.float64), r.shape), r)
    out = dict(geometry)
    out["u_target"] = np.ascontiguousarray(u, dtype=np.float64)
    return out


def batch_cases(n_cases, seed, mach_range=(0.1, 0.8)):
    """Seeded uneven 2D case set (circles and ellipses, aspect 1-3, diameters
    10-60, 32-512 points, grids 256x128 .. 1024x512, Ma uniform in
    mach_range, Re in [20, 200])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cases = []
    for _ in range(n_cases):
        nx = int(rng.integers(4, 17)) * 64
        ny = nx // 2
        ellipse_ = rng.random() < 0.5
        aspect = rng.uniform(1.0, 3.0) if ellipse_ else 1.0
        dmaj = rng.uniform(10.0, 60.0)
        a, b = 0.5 * dmaj, 0.5 * dmaj / aspect
        ang = rng.uniform(0.0, np.pi)
        per = np.pi * (3 * (a + b) - np.sqrt((3 * a + b) * (a + 3 * b)))
        nl = int(min(512, max(32, round(per))))
        ma = rng.uniform(mach_range[0], mach_range[1])
        re = rng.uniform(20.0, 200.0)
        cases.append(dict(nx=nx, ny=ny, a=a, b=b, angle=ang, n_points=nl, mach=ma, reynolds=re,
                          ellipse=ellipse_, ref_length=dmaj))
    return cases


def random_state(lattice_q, shape_zyx, seed, amp=1e-3):
    """Small seeded perturbation field (for parity of a single step)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return amp * rng.standard_normal((lattice_q,) + tuple(shape_zyx))


def warmstart_cases(n_cases, seed, shape=(512, 256), d_range=(10.0, 60.0), mach_range=(0.1, 0.45),
                    re_range=(20.0, 200.0)):
    """Seeded two-body 2D cases for the warm-start network: one circle and
    one ellipse (aspect 1-3, random orientation), diameters (major axis for
    the ellipse) uniform in d_range, both centres in the upstream half of
    the grid and at least 10 cells apart surface to surface (bounding
    circles), so that the interpolation and spreading stencils of one body
    never reach the other; ellipse minor semi-axis at least 3 cells; Mach
    and Re uniform in their ranges, Re on the larger diameter."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny = shape
    out = []
    while len(out) < n_cases:
        dc = rng.uniform(*d_range)
        de = rng.uniform(*d_range)
        aspect = rng.uniform(1.0, 3.0)
        ang = rng.uniform(0.0, np.pi)
        lo_x, hi_x = 0.15 * nx, 0.5 * nx
        pc = np.array([rng.uniform(lo_x, hi_x), rng.uniform(0.25 * ny, 0.75 * ny)])
        pe = np.array([rng.uniform(lo_x, hi_x), rng.uniform(0.25 * ny, 0.75 * ny)])
        if np.hypot(*(pc - pe)) < 0.5 * (dc + de) + 10.0 or 0.5 * de / aspect < 3.0:
            continue
        if min(pc[1], pe[1]) - 0.5 * max(dc, de) < 6 or max(pc[1], pe[1]) + 0.5 * max(dc, de) > ny - 6:
            continue
        out.append(dict(shape=(nx, ny), circle=dict(center=(float(pc[0]), float(pc[1])), diameter=dc),
                        ellipse=dict(center=(float(pe[0]), float(pe[1])), a=0.5 * de, b=0.5 * de / aspect,
                                     angle=ang),
                        mach=rng.uniform(*mach_range), reynolds=rng.uniform(*re_range),
                        ref_length=max(dc, de)))
    return out


def two_body_geometry(case, t_value, spacing=1.0):
    """Lagrangian points of both bodies (about one point per cell of
    perimeter), their outward normals, and the inside mask of the union
    (strict interiors) in the solver layout [ny][nx]."""
    nx, ny = case["shape"]
    c, e = case["circle"], case["ellipse"]
    nc = max(16, int(round(np.pi * c["diameter"] / spacing)))
    a, b = e["a"], e["b"]
    per = np.pi * (3 * (a + b) - np.sqrt((3 * a + b) * (a + 3 * b)))
    ne = max(16, int(round(per / spacing)))
    g1 = cylinder(c["center"], c["diameter"], nc, tbc=0, t_value=t_value)
    g2 = ellipse(e["center"], a, b, e["angle"], ne, tbc=0, t_value=t_value)
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = 0.5 * c["diameter"]
    inside = (xx - c["center"][0]) ** 2 + (yy - c["center"][1]) ** 2 < r * r
    cs, sn = math.cos(e["angle"]), math.sin(e["angle"])
    dx, dy = xx - e["center"][0], yy - e["center"][1]
    xr, yr = cs * dx + sn * dy, -sn * dx + cs * dy
    inside |= (xr / a) ** 2 + (yr / b) ** 2 < 1.0
    geo = dict(X=np.concatenate([g1["X"], g2["X"]]), normals=np.concatenate([g1["normals"], g2["normals"]]),
               shape=dict(kind="mask", mask=inside.astype(np.uint8)),
               tbc=np.concatenate([g1["tbc"], g2["tbc"]]), t_value=np.concatenate([g1["t_value"], g2["t_value"]]),
               u_target=np.zeros((nc + ne, 2)))
    return geo


def signed_distance(case):
    """Signed distance to the nearer body surface, negative inside, in cells
    ([ny][nx]); exact for the circle, for the ellipse the distance to its
    surface measured along the ray from its centre (an approximation that is
    exact on the axes)."""
    nx, ny = case["shape"]
    c, e = case["circle"], case["ellipse"]
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d1 = np.hypot(xx - c["center"][0], yy - c["center"][1]) - 0.5 * c["diameter"]
    cs, sn = math.cos(e["angle"]), math.sin(e["angle"])
    dx, dy = xx - e["center"][0], yy - e["center"][1]
    xr, yr = cs * dx + sn * dy, -sn * dx + cs * dy
    rho = np.hypot(xr, yr)
    k = np.hypot(xr / e["a"], yr / e["b"])
    with np.errstate(invalid="ignore", divide="ignore"):
        d2 = np.where(k > 0, rho * (1.0 - 1.0 / k), -min(e["a"], e["b"]))
    return np.minimum(d1, d2)
