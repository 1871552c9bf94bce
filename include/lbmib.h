/*
 * lbmib.h -- C ABI of the B300 hybrid compressible lattice Boltzmann solver
 * with the fully one-sided diffuse-interface immersed boundary method and
 * target-value reconstruction (FODIBM-R), arXiv 2607.07432.
 *
 * One handle = one simulation case on one GPU.  The library owns every
 * device buffer it allocates; buffers passed in by the caller stay owned by
 * the caller and are only read or written during the call.  Every entry
 * point returns an lbm_status; no exception or C++ type crosses the ABI.
 * A handle must be used by one host thread at a time.  Work is issued on
 * the CUDA stream given in lbm_config.stream (NULL = legacy default stream);
 * calls that return data to the caller synchronize that stream.
 *
 * Units are lattice units: dx = dt = 1, c_s^2 = 1/3, T_ref = 1.  Node (i,j,k)
 * sits at coordinates (i,j,k); arrays over nodes are x-fastest
 * (index = i + nx*(j + ny*k)).  Geometry is given in the same units.
 *
 * Errors: LBM_EINVAL bad argument, LBM_ENOMEM allocation failure, LBM_ECUDA a
 * CUDA runtime error (text in lbm_last_error), LBM_EGEOM an immersed-boundary
 * stencil that leaves the domain or a point with no interior node,
 * LBM_ENAN a non-finite or non-positive density/temperature found by the
 * health check (sticky until lbm_set_state / lbm_set_fields),
 * LBM_ESTATE a call out of order (e.g. a step before geometry when a body
 * was declared), LBM_EUNSUPPORTED a precision/lattice combination not built.
 */
#ifndef LBMIB_H
#define LBMIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_handle lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,
  LBM_ENOMEM = 2,
  LBM_ECUDA = 3,
  LBM_EGEOM = 4,
  LBM_ENAN = 5,
  LBM_ETIMEOUT = 6,
  LBM_ESTATE = 7,
  LBM_EUNSUPPORTED = 8
} lbm_status;

/* lattice (Sec. 2.2 and App. A; D2Q9 is the standard 2D set) */
enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 };
/* population storage / arithmetic: FP64 everywhere; FP32 everywhere;
 * FP16 or BF16 storage of f_i - w_i with FP32 arithmetic.  The immersed
 * boundary sums and wall loads are FP64 in every mode. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16DEV = 2, LBM_BF16DEV = 3 };
/* immersed boundary method (Sec. 2.3, 2.4, Table 1) */
enum { IB_DIBM = 0, IB_FODIBM = 1, IB_FODIBM_R = 2 };
/* per-face domain boundary: periodic; free-stream equilibrium (inlet or far
 * field); zero-gradient outlet; characteristic far field (the equilibrium of
 * the state whose linearized one-dimensional Riemann invariants normal to the
 * face, p +- rho c u_n, rho - p/c^2 and u_t, come from the interior neighbour
 * when they leave the domain and from the free stream when they enter; an
 * edge between two characteristic faces takes the free stream; not combined
 * with an outlet face, LBM_EINVAL).  Faces: x-, x+, y-, y+, z-, z+. */
enum { LBM_BC_PERIODIC = 0, LBM_BC_INLET = 1, LBM_BC_OUTLET = 2, LBM_BC_FARFIELD = 3,
       LBM_BC_CHARACTERISTIC = 5 };
/* relaxation time: tau_LB = mu/(rho c_s^2 theta), or tau_LB = nu/c_s^2 = mu/(rho c_s^2)
 * as written in Eq. LB (the default; the theta-scaled variant is not stable for
 * theta < 1 and gives a shear viscosity mu/theta) */
enum { LBM_TAU_THETA = 0, LBM_TAU_LITERAL = 1 };
/* a^C stencils (use_ac) */
enum { LBM_AC_OFF = 0, LBM_AC_CUBIC = 1, LBM_AC_CENTRAL = 2, LBM_AC_UPWIND = 3 };
/* temperature condition at a Lagrangian point (velocity is always Dirichlet) */
enum { IB_T_DIRICHLET = 0, IB_T_NEUMANN = 1 };
/* body shape used to classify Eulerian nodes as inside (Omega') or not */
enum { IB_SHAPE_SPHERE = 0, IB_SHAPE_ELLIPSE = 1, IB_SHAPE_POLYGON = 2, IB_SHAPE_MASK = 3 };

typedef struct {
  size_t struct_size;      /* = sizeof(lbm_config) */
  int lattice;             /* LBM_D2Q9 or LBM_D3Q19 */
  int precision;           /* LBM_FP64 .. LBM_BF16DEV */
  int nx, ny, nz;          /* nz = 1 for D2Q9 */
  double mach;             /* free-stream Mach number u_inf / sqrt(gamma R T_inf) */
  double reynolds;         /* rho_inf u_inf L / mu */
  double ref_length;       /* L in cells */
  double prandtl;          /* lambda = mu C_p / Pr (default 0.71) */
  double gamma;            /* ratio of specific heats (default 1.4) */
  double theta_inf;        /* T_inf / T_ref; <= 0 selects the built-in rule */
  double inflow_dir[3];    /* direction of u_inf (normalized by the library) */
  double sigma_hrr;        /* HRR weight of Eq. pi2 (default 0.98) */
  double d_n;              /* projection distance d_PB in cells (default 1.5) */
  int method;              /* IB_DIBM / IB_FODIBM / IB_FODIBM_R */
  int bc[6];               /* LBM_BC_* per face */
  int tau_mode;            /* LBM_TAU_LITERAL (default) or LBM_TAU_THETA */
  int use_ac;              /* a^C of Eq. af2: 2 = c_s^2 (u_a d_b P + u_b d_a P) - d_ab d_a(rho u_a^3),
                              P = rho(1-theta), central differences (default); 3 = the same terms with
                              first-order differences on the upstream side of each node (needed for
                              streams faster than the sound speed, which central differences leave
                              unstable); 1 = the cubic part only; 0 = none */
  int device;              /* CUDA device ordinal */
  void* stream;            /* cudaStream_t, or NULL */
  double bulk_ratio;       /* artificial bulk viscosity mu_b = bulk_ratio * mu (default 0: the zero bulk
                              viscosity of the trace terms of Eq. af2), added to the trace of a^F as
                              -2 mu_b div u; >= 0 */
} lbm_config;

typedef struct {
  size_t struct_size;      /* = sizeof(ib_geometry) */
  int n_points;            /* number of Lagrangian points N_L */
  const double* X;         /* host, N_L*D, point coordinates (cells) */
  const double* normals;   /* host, N_L*D, outward unit normals */
  const int* tbc;          /* host, N_L, IB_T_*; NULL = all Dirichlet */
  const double* u_target;  /* host, N_L*D, wall velocity u^Bt; NULL = 0 */
  const double* t_value;   /* host, N_L, T^Bt (Dirichlet) or dT/dn (Neumann) */
  int shape;               /* IB_SHAPE_* */
  double center[3];        /* sphere / circle / ellipse centre */
  double radius;           /* sphere / circle radius */
  double radii[2];         /* ellipse semi-axes */
  double cos_a, sin_a;     /* ellipse rotation */
  int n_poly;              /* polygon vertex count (2D) */
  const double* poly;      /* host, n_poly*2, closed polygon vertices */
  const uint8_t* mask;     /* host, nodes, 1 = inside (IB_SHAPE_MASK) */
} ib_geometry;

/* Fill *cfg with defaults (D2Q9, FP32, Pr 0.71, gamma 1.4, sigma 0.98,
 * d_n 1.5, FODIBM-R, periodic faces, tau_LB = nu/c_s^2, full a^C). */
lbm_status lbm_config_default(lbm_config* cfg);

/* Create a case (Sec. 2.2): validates *cfg, derives u_inf, mu, lambda,
 * theta_inf, allocates the device state and initializes every node to the
 * free-stream equilibrium.  *out receives a handle owned by the caller until
 * lbm_destroy. */
lbm_status lbm_create(const lbm_config* cfg, lbm_handle** out);

/* Free every device buffer of the handle.  NULL is accepted. */
void lbm_destroy(lbm_handle* h);

/* Text of the last error on this handle (valid until the next call). */
const char* lbm_last_error(const lbm_handle* h);

/* Immersed-boundary geometry (Sec. 2.3, 2.4): classifies nodes (Omega' =
 * strict interior), builds on the device the one-sided stencils, phi_l
 * (Eq. phi), the Lagrangian weights W_l (Eq. weight), the effective
 * boundary X*_l (Eq. xeffect), d_BV, the projection points P_l and their
 * d = 1 stencils, and the Eulerian-side spreading CSR (Eq. spr2).  Host
 * arrays are copied; the call may be repeated to replace the body. */
lbm_status ib_set_geometry(lbm_handle* h, const ib_geometry* g);

/* Advance n_steps time steps (Sec. 2.5 steps 1-5), asynchronously on the
 * configured stream.  Returns a sticky error found by a previous step. */
lbm_status lbm_step(lbm_handle* h, int n_steps);

/* Synchronize the stream and run the health check (Eq. feq needs rho > 0,
 * theta > 0); LBM_ENAN if any node is non-finite or non-positive. */
lbm_status lbm_check(lbm_handle* h);

/* Macroscopic fields of the current state: rho = sum f, u = sum c f / rho,
 * T = (rho E / rho - |u|^2/2) / C_v, p = rho R T (Sec. 2.2).  Each output
 * is N doubles (u is D planes of N); any pointer may be NULL.  dst_is_device
 * selects device or host destination pointers. */
lbm_status lbm_get_fields(lbm_handle* h, int dst_is_device, double* rho, double* u,
                          double* T, double* p);

/* Raw state as FP64: populations f-bar (Q planes of N) and rho E (N). */
lbm_status lbm_get_state(lbm_handle* h, int dst_is_device, double* f, double* rhoE);

/* Replace the state: populations (Q*N) and rho E (N).  The stored
 * previous-step auxiliaries are reset as for a fresh start.  Host arrays in
 * page-locked memory that the device can address (cudaHostAlloc /
 * cudaMallocHost under unified addressing, cudaHostRegister with mapping)
 * are read by the upload kernel in place; other host memory goes through a
 * device buffer allocated for the call.  Returns after the upload. */
lbm_status lbm_set_state(lbm_handle* h, int src_is_device, const double* f, const double* rhoE);

/* Checkpoint: write the complete time-stepping state of the handle to a
 * file (populations in their storage format, the carried moments or rho E,
 * and the previous-step auxiliaries rho(1-theta) and the a^F deviator), so
 * that lbm_load_state on a handle of the same lattice, precision, grid and
 * step form resumes bit for bit.  The immersed-body geometry is not part of
 * the file: set it again with ib_set_geometry before loading.  LBM_EINVAL
 * for a NULL path, LBM_ECUDA / LBM_ESTATE when the file cannot be written.
 * (The paper has no counterpart: a service of the library.) */
lbm_status lbm_save_state(lbm_handle* h, const char* path);

/* Read a file written by lbm_save_state into the handle.  LBM_ESTATE when
 * the file is missing, truncated or written by a handle of another lattice,
 * precision, grid or step form; the handle is unchanged then.  Clears a
 * sticky LBM_ENAN. */
lbm_status lbm_load_state(lbm_handle* h, const char* path);

/* Set the state to the equilibrium of given fields (warm start): rho (N),
 * u (D*N), T (N).  Host arrays are read as by lbm_set_state (in place when
 * page-locked and device-addressable). */
lbm_status lbm_set_fields(lbm_handle* h, int src_is_device, const double* rho,
                          const double* u, const double* T);

/* Wall loads of the last step, FP64, deterministic fixed-order sums:
 * force on the body = -sum_l F_l W_l (D components, rest 0),
 * heat = sum_l Q_l W_l and work = sum_l W^IB_l W_l injected into the fluid.
 * per_point (optional, host) receives N_L rows of (F_l[D], W^IB_l, Q_l). */
lbm_status lbm_get_wall_loads(lbm_handle* h, double force[3], double* heat, double* work,
                              double* per_point);

/* Wall loads as lbm_get_wall_loads, for callers that cannot allocate device
 * memory when they ask for them (a process whose device memory is fully
 * reserved by another framework's caching pool, or an embedding that forbids
 * cudaMalloc / cudaFree after start-up).  The paper has no counterpart: this
 * is a service of the library.  It allocates nothing: the reduction scratch
 * is a fixed static device array of 257 x 8 doubles, present on every device
 * that loads the library until the process exits, which limits the body to
 * at most 65536 Lagrangian points (LBM_EINVAL beyond).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * must come before any stream capture.  Every call reuses the same array
 * and overwrites every entry it reads, so nothing needs clearing; calls
 * that overlap on the GPU (two handles on different streams of one device)
 * race on it.  The sums are FP64 in a fixed order (per-block trees, then
 * blocks in order), deterministic, equal to lbm_get_wall_loads up to
 * rounding. */
lbm_status lbm_get_wall_loads_noalloc(lbm_handle* h, double force[3], double* heat, double* work);

/* Wall loads of the last step (the sums of lbm_get_wall_loads) queued for
 * the host without waiting: the reduction and a device-to-host copy of
 * out[5] = (force[3], heat, work) are issued on the handle's stream and the
 * call returns at once.  out is host memory that the caller keeps alive and
 * does not read until lbm_sync (or another synchronizing call) returns;
 * page-locked memory (cudaHostAlloc) keeps the copy asynchronous, pageable
 * memory makes the copy wait for the stream.  Each call may name its own
 * out (one per step, read after the run).  On a slab the body does not
 * reach, out is zeroed at once.  LBM_ESTATE without a body. */
lbm_status lbm_get_wall_loads_async(lbm_handle* h, double out[5]);

/* Wait for the work queued on the handle's stream; returns a sticky error
 * found by a previous step, else LBM_ECUDA on a device error. */
lbm_status lbm_sync(lbm_handle* h);

/* Wall diagnostics of the current (updated) flow field (Sec. 3.1-3.2; the
 * paper defines C_p and reads wall values with Eq. int1 at d = 2; the wall
 * shear stress and heat-flux forms are this library's reading).
 * coeffs (optional, host, 4 doubles), from the last step's FP64 loads:
 *   [0] C_d = F . e_d / (q_inf A), e_d the inflow direction,
 *   [1] C_l along e_d rotated by +90 degrees (2D) or the y axis made
 *       orthogonal to e_d (3D), [2] C_l along e_d x e_l1 (3D; 0 in 2D),
 *   [3] Nu = heat L / (lambda (T_w - T_inf) S), T_w the mean Dirichlet
 *       temperature target (0 when every point is Neumann),
 *   with q_inf = rho_inf u_inf^2 / 2, L = ref_length, A = L (2D, per unit
 *   depth) or pi L^2 / 4 (3D), S = pi L (2D) or pi L^2 (3D): the frontal
 *   area and surface of a circle or sphere of diameter L.
 * per_point (optional, host, N_L rows of 2D + 4 doubles):
 *   C_p = (p^s - p_inf) / q_inf with p^s by Eq. int1 (d = 2, nodes on both
 *   sides of the wall) at X_l; tau_w[D] = mu ((u^P - u^B) - its normal
 *   part) / d_n with u^P by Eq. int1 (d = 1) at the projection point;
 *   u^s[D] and T^s by Eq. int1 (d = 2) at X_l; (dT/dn)^s = (T^P - T^s) / d_n;
 *   C_p^P, the pressure coefficient at the projection point (d = 1: fluid
 *   nodes only, d_n cells off the wall).
 * The boundary errors of Sec. 3.2 follow: eps_Dir = |u^s - u^Bt| / u_inf,
 * eps_iso = |T^s - T^Bt| / T_inf, eps_Neu = |(dT/dn)^s - g| D / T_inf.
 * LBM_ESTATE without a body, LBM_EGEOM if a diagnostic stencil leaves a
 * non-periodic domain.  Allocates a device buffer of N_L (2D + 4) doubles
 * for the call when per_point is given. */
lbm_status lbm_get_wall_diagnostics(lbm_handle* h, double coeffs[4], double* per_point);

/* Derived constants: out[0..7] = u_inf magnitude, mu, lambda, theta_inf,
 * C_v, C_p, rho_inf, gamma. */
lbm_status lbm_get_constants(const lbm_handle* h, double out[8]);

/* Sizes of the immersed-boundary setup: rows and nonzeros of the spreading
 * CSR, number of points. */
lbm_status ib_get_sizes(const lbm_handle* h, int* n_rows, int* nnz, int* n_points);

/* Copy the immersed-boundary setup to host arrays (any may be NULL):
 * phi (N_L), W (N_L), Xstar (N_L*D), dBV (N_L), inside (N nodes, 0/1),
 * row_ptr (n_rows+1), cell_id (n_rows), col (nnz), wt (nnz). */
lbm_status ib_get_setup(lbm_handle* h, double* phi, double* W, double* Xstar, double* dBV,
                        uint8_t* inside, int* row_ptr, int* cell_id, int* col, double* wt);

/* Per-kernel timing with CUDA events recorded on the launching stream:
 * enable (1) or disable (0); reset clears the counters. */
lbm_status lbm_profile(lbm_handle* h, int enable, int reset);

/* Accumulated profile: for kernel class k (0 = fused LBM step, 1 = IB
 * interpolation/forcing, 2 = IB spreading, 3 = boundaries, 4 = other),
 * ms[k] total milliseconds and launches[k] count since the last reset. */
lbm_status lbm_get_profile(lbm_handle* h, double ms[5], long long launches[5]);

/* Number of kernels this handle has launched since creation. */
long long lbm_launch_count(const lbm_handle* h);

/* ---- one case split into z slabs (Sec. 2.5 step, partitioned) -----------
 * A slab handle owns the planes [z0, z1) of the D3Q19 case *cfg describes
 * (cfg->nz = the global nz; its z axis must not be periodic:
 * LBM_EUNSUPPORTED), plus `halo` ghost planes on each side that borders
 * another slab (none at a domain face).  It is created, initialised,
 * stepped and read like any handle, on local arrays of nx x ny x
 * (z1 - z0 + ghosts) nodes whose plane k is global plane k + zoff.  No
 * boundary condition is applied on a ghost face.  After every step the
 * ghost planes must be refreshed from the neighbours' owned planes: pack
 * side 1 (high z) of slab s and unpack it into side 0 of slab s + 1, and
 * pack side 0 of slab s + 1 into side 1 of slab s, before the next step
 * (the caller moves the buffers: a device copy on one GPU, NCCL send and
 * receive across GPUs).  With the exchange after every step and halo >= 10
 * the owned planes evolve as the same planes of the unsplit case, bit for
 * bit in FP64 (FP32 to rounding: the fused step's z chunks start at other
 * planes).  ib_set_geometry on a slab takes the whole body in global
 * coordinates and keeps the points whose stencils lie in its local planes
 * (LBM_EGEOM if a point whose stencils leave the slab has its d = 2 stencil
 * within 5 planes of the owned planes; 9 ghost planes always suffice);
 * wall loads, diagnostics coefficients
 * and their per-point arrays cover the points it keeps, the loads and
 * coefficients only those it owns (z0 <= X_z < z1), so the case's loads
 * are the sum over slabs (add them in slab order for a reproducible sum). */
lbm_status lbm_create_slab(const lbm_config* cfg, int z0, int z1, int halo, lbm_handle** out);
/* info[0..5] = z0, z1, ghost planes below, ghost planes above, zoff (global
 * z of local plane 0), global nz.  LBM_ESTATE for a handle that is not a slab. */
lbm_status lbm_slab_info(const lbm_handle* h, int info[6]);
/* Bytes of the exchange buffer of one side (0 = low z, 1 = high z; 0 bytes
 * at a domain face): the side's ghost-plane count x nx x ny x (Q storage
 * elements + D + 3 + NDEV compute elements) -- populations, carried moments
 * rho, rho u, rho E, rho(1-theta) and the a^F deviator of the previous
 * step, component after component, planes in z order. */
lbm_status lbm_slab_exchange_bytes(const lbm_handle* h, int side, size_t* bytes);
/* Copy the owned planes next to `side` into dst (device, caller-owned,
 * lbm_slab_exchange_bytes of that side), asynchronously on the handle's
 * stream. */
lbm_status lbm_slab_pack(lbm_handle* h, int side, void* dst);
/* Copy src (device; the neighbour's pack of its facing side) into the
 * ghost planes of `side`, asynchronously on the handle's stream. */
lbm_status lbm_slab_unpack(lbm_handle* h, int side, const void* src);
/* Number of Lagrangian points the slab keeps and (optional) their indices
 * in the geometry given to ib_set_geometry. */
lbm_status lbm_slab_points(const lbm_handle* h, int* n_points, int* global_index);
/* Host-only planning (no device work, callable without a GPU):
 * lbm_slab_plan writes, for each of n_slabs slabs of nz planes, out[4k..4k+3]
 * = z0, z1, ghost planes below, ghost planes above (the first nz % n_slabs
 * slabs get one plane more).  lbm_slab_keep applies the point rule of
 * ib_set_geometry on a slab: keep[l] (the slab keeps point l) and owned[l]
 * (z0 <= X_z < z1) for n_points points X, normals (host, n_points x 3);
 * LBM_EGEOM when the halo is too narrow for the body. */
lbm_status lbm_slab_plan(int nz, int n_slabs, int halo, int* out);
lbm_status lbm_slab_keep(const lbm_config* cfg, int z0, int z1, int halo, int n_points, const double* X,
                         const double* normals, int* keep, int* owned);

/* ---- two-level static refinement (the locally refined meshes of Secs.
 * 3.2-3.9; the paper gives no refinement algorithm, so what follows is this
 * library's reading) ---------------------------------------------------
 * Level 0 covers the domain described by cfg (its grid, boundary
 * conditions, Reynolds number on ref_length level-0 cells).  Level 1
 * refines the box of level-0 nodes [box_lo, box_hi] (inclusive) by 2: its
 * node k along an axis sits at level-0 coordinate box_lo + (k - G)/2 with G
 * = 4 ghost nodes beyond the box on every side (no boundary condition
 * there).  Acoustic scaling: level 1 steps twice per level-0 step with the
 * same lattice velocities and theta and twice the lattice viscosity and
 * conductivity (Reynolds number on 2 ref_length cells); theta_inf <= 0
 * applies the theta rule to level 1, and level 0 takes the same value.
 * Per level-0 step: the ghost nodes take the nested mean (x, then y, then
 * z) of the level-0 nodes around them of the predicted moments and of
 * f-bar_i - f^eq_i, rebuilt as f^eq + s01 (f-bar - f^eq), s01 = tau-bar_1 /
 * (2 tau-bar_0), tau-bar = mu / (rho c_s^2) + 1/2; the first level-1 step
 * sees level 0 at n, the second the mean of n and n+1; the previous-step
 * rho(1-theta) comes from level 0 (mean of n-1 and n, then n) and the a^F
 * deviator halved.  Level-0 nodes R = 2 or more nodes inside the box then
 * take the coinciding level-1 node's state (f^eq + s10 (f-bar - f^eq), s10
 * = 2 tau-bar_0 / tau-bar_1, rho E, its previous-step values, the deviator
 * doubled).  The energy equation couples through the same values (no
 * refluxing).  A body goes on level 1 (ib_set_geometry on its handle, in
 * level-1 node coordinates) and must stay clear of its ghost nodes. */
typedef struct lbm_refined lbm_refined;
/* LBM_EINVAL unless every box face lies at least 3 level-0 nodes inside
 * level 0 and the box spans more than 2 R nodes per axis. */
lbm_status lbm_refined_create(const lbm_config* cfg, const int box_lo[3], const int box_hi[3],
                              lbm_refined** out);
void lbm_refined_destroy(lbm_refined* r);
const char* lbm_refined_last_error(const lbm_refined* r);
/* The handle of level 0 or 1 (owned by r: fields, state, geometry,
 * diagnostics; step the pair with lbm_refined_step only).  Level 1's ghost
 * nodes hold scratch values between steps (each transfer overwrites them);
 * level-0 nodes inside the box hold the restricted level-1 solution. */
lbm_status lbm_refined_level(lbm_refined* r, int level, lbm_handle** h);
/* info[0] = G, [1] = R, [2..4] level-1 grid, [5..7] box_lo. */
lbm_status lbm_refined_info(const lbm_refined* r, int info[8]);
/* Advance n_steps level-0 steps (2 n_steps level-1 steps), asynchronously
 * on the configured stream. */
lbm_status lbm_refined_step(lbm_refined* r, int n_steps);

/* ---- several cases advanced together ------------------------------------
 * A batch owns n cases (same lattice, precision and device; grids, bodies
 * and flow parameters may differ) on one stream of its own.  A batched step
 * runs the immersed-boundary force, spreading, fused and boundary work of
 * every case (Sec. 2.5 steps 1-5) from work tables in a schedule order,
 * either as one persistent cooperative launch whose CTAs pass grid-wide
 * barriers between the phases (launch form 1, 2D lattices, default there)
 * or as one launch per phase (form 0); two steps are captured once as a CUDA
 * graph and replayed.  Results are bit-identical to stepping each case on
 * its own, in either form. */
typedef struct lbm_batch lbm_batch;

/* Create n cases from cfgs[0..n-1] (their stream fields are ignored). */
lbm_status lbm_batch_create(int n, const lbm_config* cfgs, lbm_batch** out);
void lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);
/* Borrow case i's handle (geometry, fields, loads); owned by the batch. */
lbm_status lbm_batch_case(lbm_batch* b, int i, lbm_handle** h);
/* Advance every case n_steps steps with batched launches (graph replay). */
lbm_status lbm_batch_step(lbm_batch* b, int n_steps);
/* Advance every case n_steps steps one case after another with per-case
 * launches (the unbatched form, for comparison). */
lbm_status lbm_batch_step_sequential(lbm_batch* b, int n_steps);
/* Wait for the batch stream.  LBM_ETIMEOUT when a persistent launch ended
 * early because a grid barrier waited past its limit (about a second; the
 * cases are then not at a whole step). */
lbm_status lbm_batch_sync(lbm_batch* b);
/* Launch form of a batched step: 1 = one persistent cooperative launch per
 * two steps (2D lattices only; the grid is as many CTAs as are resident at
 * once), 0 = one launch per phase.  LBM_EINVAL for form 1 on D3Q19. */
lbm_status lbm_batch_set_launch_form(lbm_batch* b, int form);
lbm_status lbm_batch_get_launch_form(const lbm_batch* b, int* form);
/* Test aid for the failure path of form 1: sets the barrier's arrival count
 * so that the next persistent launch cannot pass its first grid barrier;
 * every CTA then waits out its limit and leaves, and the following
 * lbm_batch_sync returns LBM_ETIMEOUT (and clears the barrier).  The cases
 * are left part-way through a step.  LBM_EINVAL unless the form is 1.  No
 * counterpart in the paper. */
lbm_status lbm_batch_test_stall_barrier(lbm_batch* b);
/* Fused-launch plan: tile_rows 0 (default tile), 16 or 32 (2D FP32 only), and
 * schedule 0 = case-major, 1 = round-robin over cases, 2 = largest first. */
lbm_status lbm_batch_set_plan(lbm_batch* b, int tile_rows, int schedule);
lbm_status lbm_batch_get_plan(const lbm_batch* b, int* tile_rows, int* schedule);
/* Autotuner: times each plan (launch form, tile rows, schedule) over `steps`
 * batched steps on the batch itself
 * (state saved before and restored after) and keeps the fastest; with
 * cache_path, results are read from / appended to that text file keyed by
 * the case set.  *best_ms (optional) receives the best time per step. */
lbm_status lbm_batch_autotune(lbm_batch* b, int steps, const char* cache_path, double* best_ms);

#ifdef __cplusplus
}
#endif
#endif /* LBMIB_H */
