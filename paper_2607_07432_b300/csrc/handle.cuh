// Handle of one simulation case and the host-side helpers shared by the
// C ABI (api.cu) and the per-configuration kernel instantiations.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/lbmib.h"
#include "devguard.cuh"
#include "grid.cuh"

namespace lbmib_host {
using namespace lbmib;
constexpr int kProfClasses = 5;
enum { kProfStep = 0, kProfIBForce = 1, kProfIBSpread = 2, kProfBC = 3, kProfOther = 4 };

struct Ops;

struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  void* f = nullptr;         // population buffer the captured steps start from
  int cur = 0;               // auxiliary-buffer parity they start from
  int geom = -1;             // geometry version they were captured with
  long long launches = 0;    // kernels per replay
};
}  // namespace lbmib_host

struct lbm_handle {
  lbm_config cfg;
  int D = 2, Q = 9, NDEV = 2;
  lbmib::Grid g{};
  cudaStream_t st = nullptr;
  // derived constants (Sec. 2.1, readings Q10-Q11)
  double R = 1.0 / 3.0, gamma = 1.4, Cv = 0, Cp = 0, theta_inf = 1, rho_inf = 1, u_mag = 0, mu = 0, lam = 0;
  double u_inf[3] = {0, 0, 0};
  double E_inf = 0;
  size_t csize = 8, ssize = 8;  // compute / storage element sizes
  // device state
  void* f = nullptr;
  void* M = nullptr;
  void* E = nullptr;
  void* P[2] = {nullptr, nullptr};
  void* A[2] = {nullptr, nullptr};
  void* feq_inf = nullptr;
  int cur = 0;
  int zchunk = 16;           // planes per CTA along z in the fused step
  int zchunk_fixed = 0;      // set by the environment: keep it
  int bc_in_kernel = 1;  // far-field boundaries inside the fused kernel when the faces allow it
  void* f2 = nullptr;        // second population buffer (the fused step reads one, writes the other)
  void* M2 = nullptr;        // second predicted-moment buffer
  unsigned long long* d_bad = nullptr;
  // immersed boundary
  bool has_ib = false;
  int NL = 0, n_rows = 0, nnz = 0;
  unsigned char* inside = nullptr;
  double *X = nullptr, *nrm = nullptr, *uB = nullptr, *tB = nullptr;
  int* tbc = nullptr;
  int *sten_node = nullptr, *psten_node = nullptr;
  double *sten_w = nullptr, *sten_x = nullptr, *psten_w = nullptr;
  double *phi = nullptr, *W = nullptr, *Xstar = nullptr, *dBV = nullptr;
  int *row_ptr = nullptr, *cell_id = nullptr, *col = nullptr, *slot_of_entry = nullptr;
  double* wt = nullptr;
  int* row_of_node = nullptr;
  unsigned char* forced = nullptr;
  double *G = nullptr, *FU = nullptr, *WQ = nullptr, *loads = nullptr;
  double T_wall = 0.0;       // mean Dirichlet temperature target (Nusselt number)
  bool has_dirichlet = false;
  // z slab of a larger case (lbm_create_slab): global owned planes
  // [z0, z1), ghost planes below / above, global nz; the Lagrangian points
  // kept by the slab (global indices) and which of them it owns
  bool slab = false;
  int slab_z0 = 0, slab_z1 = 0, ghost_lo = 0, ghost_hi = 0, nz_global = 0;
  std::vector<int> slab_points;
  unsigned char* owned = nullptr;
  // bookkeeping
  std::string err;
  long long launches = 0;
  int sticky = LBM_OK;
  int geom_version = 0;
  bool prof = false;
  // steps captured as CUDA graphs for lbm_step: [0] two steps (both buffer
  // parities), [1 + cur] one step from buffer parity cur; each is valid
  // while the buffers are at its captured parity and the geometry is
  // unchanged
  lbmib_host::StepGraph graphs[3];
  int use_graph = 1;
  bool stepped = false;      // a first eager step has set the kernels' launch attributes
  cudaStream_t cap_st = nullptr;  // capture stream when the handle runs on the legacy default stream
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  double prof_ms[lbmib_host::kProfClasses] = {0, 0, 0, 0, 0};
  long long prof_n[lbmib_host::kProfClasses] = {0, 0, 0, 0, 0};
  const lbmib_host::Ops* ops = nullptr;
};

namespace lbmib_host {

inline lbm_status fail(lbm_handle* h, lbm_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(h, LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

inline cudaEvent_t ev_get(lbm_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// launch wrapper: counts launches and records profiling events
template <class F>
inline lbm_status launch(lbm_handle* h, int cls, F&& fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->prof) {
    a = ev_get(h);
    b = ev_get(h);
    cudaEventRecord(a, h->st);
  }
  fn();
  h->launches++;
  if (h->prof) {
    cudaEventRecord(b, h->st);
    h->ev_used.push_back({cls, {a, b}});
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return LBM_OK;
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

struct BatchPlan;
struct Ops {
  lbm_status (*init)(lbm_handle*);
  lbm_status (*step)(lbm_handle*);
  lbm_status (*fields)(lbm_handle*, double*, double*, double*, double*);
  lbm_status (*get_state)(lbm_handle*, double*, double*);
  lbm_status (*set_state)(lbm_handle*, const double*, const double*);
  lbm_status (*set_fields)(lbm_handle*, const double*, const double*, const double*);
  lbm_status (*health)(lbm_handle*, unsigned long long*);
  // batched step support: build the case descriptors and the work schedule
  // of a plan, and launch one batched fused step of the given parity
  lbm_status (*batch_build)(BatchPlan*);
  lbm_status (*batch_fused)(BatchPlan*, int parity);
  // the IB part (part 0: interpolation, forcing, spreading) or the boundary
  // part (part 1) of every case of a plan, one launch per kernel
  lbm_status (*batch_aux)(BatchPlan*, int parity, int part);
  // nsteps whole steps of every case from the given parity in one
  // persistent launch (launch_form 1; LBM_EINVAL where not available)
  lbm_status (*batch_persistent)(BatchPlan*, int parity, int nsteps);
  // per-case parts of a step around the fused kernel
  lbm_status (*ib_part)(lbm_handle*);
  lbm_status (*bc_part)(lbm_handle*);
  // wall diagnostics of the current state into a device array (NL rows)
  lbm_status (*wall_diag)(lbm_handle*, double* out, int* err);
  // two-level refinement transfers (level-0 handle, level-1 handle):
  // ghost state of level 1 from level 0 into a device array, its write into
  // level 1 (Gb null: the first level-1 step), restriction into level 0
  lbm_status (*refine_ghost_state)(lbm_handle* h0, const lbmib::RefineDev&, void* out);
  lbm_status (*refine_fill)(lbm_handle* h0, lbm_handle* h1, const lbmib::RefineDev&, const void* Ga,
                            const void* Gb);
  lbm_status (*refine_restrict)(lbm_handle* h0, lbm_handle* h1, const lbmib::RefineDev&);
};

// a handle whose every face is a ghost face (no boundary condition, edge
// reads clamped): the level-1 box of a refined case
lbm_status create_patch_handle(const lbm_config* cfg, lbm_handle** out);

// A set of cases advanced together (lbm_batch_*): one fused launch covers
// every case; the per-case IB and boundary kernels surround it.
struct BatchPlan {
  std::vector<lbm_handle*> cases;
  cudaStream_t st = nullptr;
  int tile_rows = 0;   // 0: the default tile of the lattice / precision
  int schedule = 0;    // 0 case-major, 1 round-robin over cases, 2 largest case first
  void* descs[2] = {nullptr, nullptr};   // device CaseDesc arrays, parity 0 / 1
  void* work = nullptr;                  // device int4 work items
  int n_work = 0;
  // IB force, spread + apply and boundary launches over all cases:
  // per-parity case descriptors and work items (case, block [, face])
  void* ib_descs[2] = {nullptr, nullptr};
  void* ib_work = nullptr;
  int n_ib_work = 0;
  void* sp_descs[2] = {nullptr, nullptr};
  void* sp_work = nullptr;
  int n_sp_work = 0;
  void* bc_descs[2] = {nullptr, nullptr};
  void* bc_work = nullptr;
  int n_bc_work = 0;
  // launch form of a step: 0 = the four batched kernels, 1 = one persistent
  // cooperative launch for all phases (2D lattices), with its grid barrier
  // state and grid size (CTAs resident at once)
  int launch_form = 0;
  void* bar = nullptr;
  int persist_grid = 0;
  std::vector<void*> built_f;            // per case h->f at build time (parity 0)
  std::vector<int> built_geom;           // per case geometry version at build time
  bool built = false;
  std::string err;
};


const Ops* ops_d2q9_fp64();
const Ops* ops_d2q9_fp32();
const Ops* ops_d2q9_fp16();
const Ops* ops_d2q9_bf16();
const Ops* ops_d3q19_fp64();
const Ops* ops_d3q19_fp32();
const Ops* ops_d3q19_fp16();
const Ops* ops_d3q19_bf16();
}  // namespace lbmib_host
