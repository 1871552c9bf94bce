"""Thin ctypes binding of the C ABI in include/lbmib.h (argument marshalling
only: every step of the method runs in the CUDA library).

Host arrays are numpy; device arrays may be torch CUDA tensors (their
data_ptr is passed through).  The library must be built first
(``python -m paper_2607_07432_b300.build``); importing this module without
it raises ImportError rather than falling back to anything else.
"""
import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "liblbmib.so")

D2Q9, D3Q19 = 0, 1
FP64, FP32, FP16DEV, BF16DEV = 0, 1, 2, 3
DIBM, FODIBM, FODIBM_R = 0, 1, 2
BC_PERIODIC, BC_INLET, BC_OUTLET, BC_FARFIELD, BC_CHAR = 0, 1, 2, 3, 5
TAU_THETA, TAU_LITERAL = 0, 1
AC_OFF, AC_CUBIC, AC_CENTRAL, AC_UPWIND = 0, 1, 2, 3
SHAPE_SPHERE, SHAPE_ELLIPSE, SHAPE_POLYGON, SHAPE_MASK = 0, 1, 2, 3
STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_EGEOM",
          5: "LBM_ENAN", 6: "LBM_ETIMEOUT", 7: "LBM_ESTATE", 8: "LBM_EUNSUPPORTED"}
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp16": FP16DEV, "bf16": BF16DEV}

EXPORTS = ["lbm_config_default", "lbm_create", "lbm_destroy", "lbm_last_error", "ib_set_geometry",
           "lbm_step", "lbm_check", "lbm_get_fields", "lbm_get_state", "lbm_set_state", "lbm_set_fields",
           "lbm_get_wall_loads", "lbm_get_wall_diagnostics", "lbm_get_constants", "ib_get_sizes", "ib_get_setup", "lbm_profile",
           "lbm_get_profile", "lbm_launch_count", "lbm_get_wall_loads_noalloc", "lbm_get_wall_loads_async", "lbm_sync", "lbm_batch_create",
           "lbm_batch_destroy", "lbm_batch_last_error", "lbm_batch_case", "lbm_batch_step",
           "lbm_batch_step_sequential", "lbm_batch_sync", "lbm_batch_set_plan", "lbm_batch_get_plan",
           "lbm_batch_set_launch_form", "lbm_batch_get_launch_form", "lbm_batch_test_stall_barrier",
           "lbm_batch_autotune", "lbm_save_state", "lbm_load_state", "lbm_create_slab", "lbm_slab_info",
           "lbm_slab_exchange_bytes", "lbm_slab_pack", "lbm_slab_unpack", "lbm_slab_points",
           "lbm_slab_plan", "lbm_slab_keep", "lbm_refined_create", "lbm_refined_destroy",
           "lbm_refined_last_error", "lbm_refined_level", "lbm_refined_info", "lbm_refined_step"]


class Config(ct.Structure):
    _fields_ = [("struct_size", ct.c_size_t), ("lattice", ct.c_int), ("precision", ct.c_int),
                ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("mach", ct.c_double),
                ("reynolds", ct.c_double), ("ref_length", ct.c_double), ("prandtl", ct.c_double),
                ("gamma", ct.c_double), ("theta_inf", ct.c_double), ("inflow_dir", ct.c_double * 3),
                ("sigma_hrr", ct.c_double), ("d_n", ct.c_double), ("method", ct.c_int),
                ("bc", ct.c_int * 6), ("tau_mode", ct.c_int), ("use_ac", ct.c_int), ("device", ct.c_int),
                ("stream", ct.c_void_p), ("bulk_ratio", ct.c_double)]


class Geometry(ct.Structure):
    _fields_ = [("struct_size", ct.c_size_t), ("n_points", ct.c_int), ("X", ct.c_void_p),
                ("normals", ct.c_void_p), ("tbc", ct.c_void_p), ("u_target", ct.c_void_p),
                ("t_value", ct.c_void_p), ("shape", ct.c_int), ("center", ct.c_double * 3),
                ("radius", ct.c_double), ("radii", ct.c_double * 2), ("cos_a", ct.c_double),
                ("sin_a", ct.c_double), ("n_poly", ct.c_int), ("poly", ct.c_void_p), ("mask", ct.c_void_p)]


def load():
    if not os.path.exists(LIBPATH):
        raise ImportError("liblbmib.so is not built; run python -m paper_2607_07432_b300.build")
    lib = ct.CDLL(LIBPATH)
    lib.lbm_last_error.restype = ct.c_char_p
    lib.lbm_launch_count.restype = ct.c_longlong
    lib.lbm_create.argtypes = [ct.POINTER(Config), ct.POINTER(ct.c_void_p)]
    lib.lbm_create_slab.argtypes = [ct.POINTER(Config), ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_void_p)]
    lib.lbm_slab_pack.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.lbm_slab_unpack.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.lbm_slab_exchange_bytes.argtypes = [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_size_t)]
    lib.lbm_save_state.argtypes = [ct.c_void_p, ct.c_char_p]
    lib.lbm_load_state.argtypes = [ct.c_void_p, ct.c_char_p]
    lib.lbm_refined_last_error.restype = ct.c_char_p
    lib.lbm_refined_last_error.argtypes = [ct.c_void_p]
    lib.lbm_refined_destroy.argtypes = [ct.c_void_p]
    lib.lbm_refined_step.argtypes = [ct.c_void_p, ct.c_int]
    lib.lbm_refined_create.argtypes = [ct.POINTER(Config), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                       ct.POINTER(ct.c_void_p)]
    lib.lbm_batch_last_error.restype = ct.c_char_p
    lib.lbm_batch_last_error.argtypes = [ct.c_void_p]
    lib.lbm_batch_destroy.argtypes = [ct.c_void_p]
    lib.lbm_batch_step.argtypes = [ct.c_void_p, ct.c_int]
    lib.lbm_batch_step_sequential.argtypes = [ct.c_void_p, ct.c_int]
    lib.lbm_batch_sync.argtypes = [ct.c_void_p]
    lib.lbm_batch_set_plan.argtypes = [ct.c_void_p, ct.c_int, ct.c_int]
    lib.lbm_batch_set_launch_form.argtypes = [ct.c_void_p, ct.c_int]
    for name in ("lbm_step",):
        getattr(lib, name).argtypes = [ct.c_void_p, ct.c_int]
    for name in ("lbm_destroy", "lbm_check", "lbm_last_error", "lbm_launch_count"):
        getattr(lib, name).argtypes = [ct.c_void_p]
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ct.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ct.c_void_p)


def _config(lattice, precision, shape, mach, reynolds, ref_length, prandtl, gamma, theta_inf, inflow_dir, sigma,
            d_n, method, bc, tau_mode, use_ac, device, stream, bulk_ratio=0.0):
    cfg = Config()
    lib().lbm_config_default(ct.byref(cfg))
    D = 2 if lattice in ("D2Q9", D2Q9) else 3
    cfg.lattice = D2Q9 if D == 2 else D3Q19
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.nx, cfg.ny = int(shape[0]), int(shape[1])
    cfg.nz = int(shape[2]) if D == 3 else 1
    cfg.mach, cfg.reynolds, cfg.ref_length = mach, reynolds, ref_length
    cfg.prandtl, cfg.gamma, cfg.theta_inf = prandtl, gamma, theta_inf
    for a in range(3):
        cfg.inflow_dir[a] = float(inflow_dir[a]) if a < len(inflow_dir) else 0.0
    cfg.sigma_hrr, cfg.d_n, cfg.method = sigma, d_n, int(method)
    bc = list(bc) if bc is not None else [BC_PERIODIC] * (2 * D)
    for k in range(6):
        cfg.bc[k] = int(bc[k]) if k < len(bc) else BC_PERIODIC
    cfg.tau_mode, cfg.use_ac, cfg.device = int(tau_mode), int(use_ac), int(device)
    cfg.stream = ct.c_void_p(stream) if stream else None
    cfg.bulk_ratio = float(bulk_ratio)
    return cfg


class Solver:
    """One case on one GPU (lbm_create ... lbm_destroy)."""

    def __init__(self, lattice="D2Q9", precision="fp32", shape=(64, 64), mach=0.1, reynolds=100.0,
                 ref_length=10.0, prandtl=0.71, gamma=1.4, theta_inf=0.0, inflow_dir=(1.0, 0.0, 0.0),
                 sigma=0.98, d_n=1.5, method=FODIBM_R, bc=None, tau_mode=TAU_LITERAL, use_ac=2,
                 device=0, stream=None, slab=None, bulk_ratio=0.0):
        """slab = (z0, z1, halo): a z slab of the case (lbm_create_slab); shape
        is then the global grid."""
        L = lib()
        cfg = _config(lattice, precision, shape, mach, reynolds, ref_length, prandtl, gamma, theta_inf,
                      inflow_dir, sigma, d_n, method, bc, tau_mode, use_ac, device, stream, bulk_ratio)
        self.D = 2 if lattice in ("D2Q9", D2Q9) else 3
        self.Q = 9 if self.D == 2 else 19
        self.cfg = cfg
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.zyx = tuple(reversed(self.shape))
        h = ct.c_void_p()
        if slab is None:
            st = L.lbm_create(ct.byref(cfg), ct.byref(h))
        else:
            st = L.lbm_create_slab(ct.byref(cfg), int(slab[0]), int(slab[1]), int(slab[2]), ct.byref(h))
        if st:
            raise LBMError(st, "lbm_create failed")
        self.h = h
        self.NL = 0
        self.slab = None
        if slab is not None:
            info = (ct.c_int * 6)()
            self._check(L.lbm_slab_info(h, info))
            self.slab = dict(z0=info[0], z1=info[1], ghost_lo=info[2], ghost_hi=info[3], zoff=info[4],
                             nz_global=info[5])
            nloc = info[1] - info[0] + info[2] + info[3]
            self.shape = (self.shape[0], self.shape[1], nloc)
            self.N = int(np.prod(self.shape))
            self.zyx = tuple(reversed(self.shape))

    def _check(self, st):
        if st:
            raise LBMError(st, lib().lbm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- geometry ----------------------------------------------------------
    def set_geometry(self, geo):
        D = self.D
        X = np.ascontiguousarray(geo["X"], dtype=np.float64).reshape(-1, D)
        N = np.ascontiguousarray(geo["normals"], dtype=np.float64).reshape(-1, D)
        NL = X.shape[0]
        tbc = np.ascontiguousarray(geo.get("tbc", np.zeros(NL)), dtype=np.int32)
        ut = np.ascontiguousarray(geo.get("u_target", np.zeros((NL, D))), dtype=np.float64).reshape(NL, D)
        tv = np.ascontiguousarray(geo["t_value"], dtype=np.float64).reshape(NL)
        g = Geometry()
        g.struct_size = ct.sizeof(Geometry)
        g.n_points = NL
        g.X, g.normals, g.tbc, g.u_target, g.t_value = _ptr(X), _ptr(N), _ptr(tbc), _ptr(ut), _ptr(tv)
        sh = geo["shape"]
        keep = [X, N, tbc, ut, tv]
        kind = sh["kind"]
        if kind in ("circle", "sphere"):
            g.shape = SHAPE_SPHERE
            for a in range(D):
                g.center[a] = float(sh["center"][a])
            g.radius = float(sh["radius"])
        elif kind == "ellipse":
            g.shape = SHAPE_ELLIPSE
            g.center[0], g.center[1] = float(sh["center"][0]), float(sh["center"][1])
            g.radii[0], g.radii[1] = float(sh["radii"][0]), float(sh["radii"][1])
            g.cos_a, g.sin_a = float(sh["cos"]), float(sh["sin"])
        elif kind == "polygon":
            g.shape = SHAPE_POLYGON
            P = np.ascontiguousarray(sh["poly"], dtype=np.float64)
            keep.append(P)
            g.n_poly, g.poly = P.shape[0], _ptr(P)
        elif kind == "mask":
            g.shape = SHAPE_MASK
            M = np.ascontiguousarray(sh["mask"], dtype=np.uint8)
            keep.append(M)
            g.mask = _ptr(M)
        else:
            raise ValueError(kind)
        self._check(lib().ib_set_geometry(self.h, ct.byref(g)))
        self.NL = NL
        if getattr(self, "slab", None) is not None:
            n = ct.c_int()
            self._check(lib().lbm_slab_points(self.h, ct.byref(n), None))
            idx = np.empty(n.value, dtype=np.int32)
            self._check(lib().lbm_slab_points(self.h, ct.byref(n), _ptr(idx)))
            self.NL = n.value
            self.slab_points = idx

    # -- time stepping -----------------------------------------------------
    def step(self, n=1):
        self._check(lib().lbm_step(self.h, int(n)))

    def check(self):
        self._check(lib().lbm_check(self.h))

    # -- data --------------------------------------------------------------
    def fields(self):
        N, D = self.N, self.D
        rho, u, T, p = np.empty(N), np.empty(D * N), np.empty(N), np.empty(N)
        self._check(lib().lbm_get_fields(self.h, 0, _ptr(rho), _ptr(u), _ptr(T), _ptr(p)))
        z = self.zyx
        return rho.reshape(z), u.reshape((D,) + z), T.reshape(z), p.reshape(z)

    def fields_device(self, rho, u, T, p):
        self._check(lib().lbm_get_fields(self.h, 1, _ptr(rho), _ptr(u), _ptr(T), _ptr(p)))

    def state(self):
        f = np.empty(self.Q * self.N)
        E = np.empty(self.N)
        self._check(lib().lbm_get_state(self.h, 0, _ptr(f), _ptr(E)))
        return f.reshape((self.Q,) + self.zyx), E.reshape(self.zyx)

    def set_state(self, f, E):
        f = np.ascontiguousarray(f, dtype=np.float64)
        E = np.ascontiguousarray(E, dtype=np.float64)
        self._check(lib().lbm_set_state(self.h, 0, _ptr(f), _ptr(E)))

    def set_fields(self, rho, u, T, device=False):
        if device:
            self._check(lib().lbm_set_fields(self.h, 1, _ptr(rho), _ptr(u), _ptr(T)))
            return
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        self._check(lib().lbm_set_fields(self.h, 0, _ptr(rho), _ptr(u), _ptr(T)))

    def save_state(self, path):
        self._check(lib().lbm_save_state(self.h, str(path).encode()))

    def load_state(self, path):
        self._check(lib().lbm_load_state(self.h, str(path).encode()))

    def wall_loads(self, per_point=False):
        force = (ct.c_double * 3)()
        heat, work = ct.c_double(), ct.c_double()
        pp = np.empty(self.NL * (self.D + 2)) if per_point else None
        self._check(lib().lbm_get_wall_loads(self.h, force, ct.byref(heat), ct.byref(work), _ptr(pp)))
        out = dict(force=np.array(force[:self.D]), heat=heat.value, work=work.value)
        if per_point:
            pp = pp.reshape(self.NL, self.D + 2)
            out.update(F=pp[:, :self.D].copy(), W=pp[:, self.D].copy(), Q=pp[:, self.D + 1].copy())
        return out

    # -- z slabs ------------------------------------------------------------
    def exchange_bytes(self, side):
        n = ct.c_size_t()
        self._check(lib().lbm_slab_exchange_bytes(self.h, int(side), ct.byref(n)))
        return n.value

    def slab_pack(self, side, dst):
        """Pack the owned planes next to `side` into dst (a torch CUDA uint8
        tensor of exchange_bytes(side) bytes)."""
        self._check(lib().lbm_slab_pack(self.h, int(side), _ptr(dst)))

    def slab_unpack(self, side, src):
        self._check(lib().lbm_slab_unpack(self.h, int(side), _ptr(src)))

    def wall_diagnostics(self, per_point=True):
        """lbm_get_wall_diagnostics: C_d, C_l (C_l2 in 3D), Nu and, per
        Lagrangian point, C_p, tau_w, u^s, T^s, (dT/dn)^s and C_p at the
        projection point of the current field."""
        D = self.D
        co = (ct.c_double * 4)()
        pp = np.empty(self.NL * (2 * D + 4)) if per_point else None
        self._check(lib().lbm_get_wall_diagnostics(self.h, co, _ptr(pp)))
        out = dict(Cd=co[0], Cl=co[1], Cl2=co[2], Nu=co[3])
        if per_point:
            pp = pp.reshape(self.NL, 2 * D + 4)
            out.update(Cp=pp[:, 0].copy(), tau_w=pp[:, 1:1 + D].copy(), u_s=pp[:, 1 + D:1 + 2 * D].copy(),
                       T_s=pp[:, 1 + 2 * D].copy(), dTdn=pp[:, 2 + 2 * D].copy(), CpP=pp[:, 3 + 2 * D].copy())
        return out

    def wall_loads_noalloc(self):
        """lbm_get_wall_loads_noalloc: the same loads with no device allocation
        (static scratch, at most 65536 points)."""
        force = (ct.c_double * 3)()
        heat, work = ct.c_double(), ct.c_double()
        self._check(lib().lbm_get_wall_loads_noalloc(self.h, force, ct.byref(heat), ct.byref(work)))
        return dict(force=np.array(force[:self.D]), heat=heat.value, work=work.value)

    def wall_loads_async(self, out):
        """lbm_get_wall_loads_async: queue the last step's loads (force[3],
        heat, work) into `out`, 5 float64 of host memory (page-locked keeps
        the copy asynchronous), valid after sync()."""
        n = out.numel() if hasattr(out, "numel") else out.size
        if str(out.dtype).rsplit(".", 1)[-1] != "float64" or n < 5 or getattr(out, "is_cuda", False):
            raise ValueError("wall_loads_async needs 5 contiguous float64 host values")
        self._check(lib().lbm_get_wall_loads_async(self.h, _ptr(out)))

    def sync(self):
        """lbm_sync: wait for the work queued on the handle's stream."""
        self._check(lib().lbm_sync(self.h))

    def constants(self):
        out = (ct.c_double * 8)()
        self._check(lib().lbm_get_constants(self.h, out))
        keys = ["u_mag", "mu", "lam", "theta_inf", "Cv", "Cp", "rho_inf", "gamma"]
        return dict(zip(keys, list(out)))

    def ib_setup(self):
        nr, nnz, nl = ct.c_int(), ct.c_int(), ct.c_int()
        self._check(lib().ib_get_sizes(self.h, ct.byref(nr), ct.byref(nnz), ct.byref(nl)))
        nr, nnz, nl = nr.value, nnz.value, nl.value
        D = self.D
        out = dict(phi=np.empty(nl), W=np.empty(nl), Xstar=np.empty(nl * D), dBV=np.empty(nl),
                   inside=np.empty(self.N, dtype=np.uint8), row_ptr=np.empty(nr + 1, dtype=np.int32),
                   cell_id=np.empty(nr, dtype=np.int32), col=np.empty(nnz, dtype=np.int32), wt=np.empty(nnz))
        self._check(lib().ib_get_setup(self.h, *[_ptr(out[k]) for k in
                                                 ("phi", "W", "Xstar", "dBV", "inside", "row_ptr", "cell_id",
                                                  "col", "wt")]))
        out["Xstar"] = out["Xstar"].reshape(nl, D)
        out["inside"] = out["inside"].reshape(self.zyx).astype(bool)
        return out

    def profile(self, enable=True, reset=True):
        self._check(lib().lbm_profile(self.h, int(enable), int(reset)))

    def get_profile(self):
        ms = (ct.c_double * 5)()
        n = (ct.c_longlong * 5)()
        self._check(lib().lbm_get_profile(self.h, ms, n))
        names = ["step", "ib_force", "ib_spread", "bc", "other"]
        return {k: (ms[i], n[i]) for i, k in enumerate(names)}

    def launch_count(self):
        return int(lib().lbm_launch_count(self.h))


class CaseView(Solver):
    """A case owned by a Batch (borrowed handle; not destroyed on close)."""

    def __init__(self, handle, lattice, shape):
        self.h = handle
        self.D = 2 if lattice == "D2Q9" else 3
        self.Q = 9 if self.D == 2 else 19
        self.shape = tuple(int(v) for v in shape)
        self.N = int(np.prod(self.shape))
        self.zyx = tuple(reversed(self.shape))
        self.NL = 0
        self.slab = None

    def close(self):
        self.h = None


class Refined:
    """Two-level static refinement (lbm_refined_*): level 0 over `shape`
    (Reynolds number on ref_length level-0 cells) and level 1, the box of
    level-0 nodes [box_lo, box_hi] refined by 2 with G ghost nodes.  The
    levels are CaseView objects (`level0`, `level1`); a body goes on level 1
    in its node coordinates (`to_level1`)."""

    def __init__(self, lattice, precision, shape, box_lo, box_hi, mach=0.1, reynolds=100.0, ref_length=10.0,
                 prandtl=0.71, gamma=1.4, theta_inf=0.0, inflow_dir=(1.0, 0.0, 0.0), sigma=0.98, d_n=1.5,
                 method=FODIBM_R, bc=None, tau_mode=TAU_LITERAL, use_ac=2, device=0, stream=None, bulk_ratio=0.0):
        L = lib()
        self.cfg = _config(lattice, precision, shape, mach, reynolds, ref_length, prandtl, gamma, theta_inf,
                           inflow_dir, sigma, d_n, method, bc, tau_mode, use_ac, device, stream, bulk_ratio)
        D = 2 if lattice in ("D2Q9", D2Q9) else 3
        lo = (ct.c_int * 3)(*[int(v) for v in (list(box_lo) + [0, 0])[:3]])
        hi = (ct.c_int * 3)(*[int(v) for v in (list(box_hi) + [0, 0])[:3]])
        r = ct.c_void_p()
        st = L.lbm_refined_create(ct.byref(self.cfg), lo, hi, ct.byref(r))
        if st:
            raise LBMError(st, "lbm_refined_create failed")
        self.r = r
        info = (ct.c_int * 8)()
        self._check(L.lbm_refined_info(r, info))
        self.G, self.R = info[0], info[1]
        self.box_lo = tuple(info[5:5 + D])
        shape1 = tuple(info[2:2 + D])
        hs = []
        for lev in (0, 1):
            h = ct.c_void_p()
            self._check(L.lbm_refined_level(r, lev, ct.byref(h)))
            hs.append(h)
        self.level0 = CaseView(hs[0], lattice, tuple(int(v) for v in shape[:D]))
        self.level1 = CaseView(hs[1], lattice, shape1)

    def _check(self, st):
        if st:
            raise LBMError(st, lib().lbm_refined_last_error(self.r).decode() if self.r else "")

    def to_level1(self, X):
        """Level-0 coordinates (N x D) to level-1 node coordinates."""
        X = np.asarray(X, dtype=np.float64)
        lo = np.asarray(self.box_lo, dtype=np.float64)
        return self.G + 2.0 * (X - lo[None, :X.shape[1]])

    def step(self, n=1):
        self._check(lib().lbm_refined_step(self.r, int(n)))

    def check(self):
        self.level0.check()
        self.level1.check()

    def close(self):
        if self.r:
            lib().lbm_refined_destroy(self.r)
            self.r = None
            self.level0.close()
            self.level1.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several cases advanced together (lbm_batch_*)."""

    def __init__(self, lattice, precision, cases, device=0):
        """cases: list of dicts with shape, mach, reynolds, ref_length and
        optional bc, method, inflow_dir, theta_inf, use_ac, bulk_ratio."""
        L = lib()
        n = len(cases)
        cfgs = (Config * n)()
        self.lattice = lattice
        D = 2 if lattice == "D2Q9" else 3
        for k, c in enumerate(cases):
            cfg = cfgs[k]
            L.lbm_config_default(ct.byref(cfg))
            cfg.lattice = D2Q9 if D == 2 else D3Q19
            cfg.precision = PRECISIONS[precision]
            cfg.nx, cfg.ny = int(c["shape"][0]), int(c["shape"][1])
            cfg.nz = int(c["shape"][2]) if D == 3 else 1
            cfg.mach, cfg.reynolds, cfg.ref_length = c["mach"], c["reynolds"], c["ref_length"]
            cfg.theta_inf = c.get("theta_inf", 0.0)
            cfg.method = int(c.get("method", FODIBM_R))
            cfg.use_ac = int(c.get("use_ac", cfg.use_ac))
            cfg.bulk_ratio = float(c.get("bulk_ratio", 0.0))
            d = c.get("inflow_dir", (1.0, 0.0, 0.0))
            for a in range(3):
                cfg.inflow_dir[a] = float(d[a]) if a < len(d) else 0.0
            bc = c.get("bc", [BC_PERIODIC] * (2 * D))
            for f in range(6):
                cfg.bc[f] = int(bc[f]) if f < len(bc) else BC_PERIODIC
            cfg.device = device
        h = ct.c_void_p()
        st = L.lbm_batch_create(n, cfgs, ct.byref(h))
        if st:
            raise LBMError(st, "lbm_batch_create failed")
        self.b = h
        self.views = []
        for k, c in enumerate(cases):
            hk = ct.c_void_p()
            self._check(L.lbm_batch_case(self.b, k, ct.byref(hk)))
            self.views.append(CaseView(hk, lattice, c["shape"]))

    def _check(self, st):
        if st:
            raise LBMError(st, lib().lbm_batch_last_error(self.b).decode())

    def case(self, k):
        return self.views[k]

    def step(self, n=1):
        self._check(lib().lbm_batch_step(self.b, int(n)))

    def step_sequential(self, n=1):
        self._check(lib().lbm_batch_step_sequential(self.b, int(n)))

    def sync(self):
        self._check(lib().lbm_batch_sync(self.b))

    def set_plan(self, tile_rows, schedule):
        self._check(lib().lbm_batch_set_plan(self.b, int(tile_rows), int(schedule)))

    def plan(self):
        tr, sc = ct.c_int(), ct.c_int()
        self._check(lib().lbm_batch_get_plan(self.b, ct.byref(tr), ct.byref(sc)))
        return tr.value, sc.value

    def set_launch_form(self, form):
        """1: one persistent cooperative launch per two steps (2D); 0: one
        launch per phase."""
        self._check(lib().lbm_batch_set_launch_form(self.b, int(form)))

    def test_stall_barrier(self):
        """Failure-path test aid (see lbm_batch_test_stall_barrier)."""
        self._check(lib().lbm_batch_test_stall_barrier(self.b))

    def launch_form(self):
        f = ct.c_int()
        self._check(lib().lbm_batch_get_launch_form(self.b, ct.byref(f)))
        return f.value

    def autotune(self, steps=10, cache_path=None):
        best = ct.c_double()
        p = cache_path.encode() if cache_path else None
        self._check(lib().lbm_batch_autotune(self.b, int(steps), p, ct.byref(best)))
        return self.plan(), best.value

    def close(self):
        if getattr(self, "b", None):
            for v in self.views:
                v.close()
            lib().lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
