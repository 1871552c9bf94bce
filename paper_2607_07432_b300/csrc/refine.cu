// Two-level static refinement (lbm_refined_*): a level-0 case over the
// whole domain and the level-1 case of a box of it refined by 2, stepped
// together (the transfers are in refine.cuh; the reading is stated there
// and in include/lbmib.h).
#include <cuda_runtime.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

using namespace lbmib_host;

namespace {
constexpr int kRefineG = 4;  // level-1 ghost nodes beyond the box
constexpr int kRefineR = 2;  // restriction margin in level-0 nodes
}  // namespace

struct lbm_refined {
  lbm_handle* h0 = nullptr;
  lbm_handle* h1 = nullptr;
  int D = 2;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  lbmib::RefineDev dev{};
  int4* ghost = nullptr;
  long long* shell = nullptr;
  int* corners = nullptr;
  void* Ga = nullptr;
  void* Gb = nullptr;
  std::string err;
  // two level-0 steps captured as one CUDA graph (both parities of both
  // levels return to the captured ones), valid while the buffers and the
  // geometry versions match
  cudaGraphExec_t gexec = nullptr;
  void* g_f0 = nullptr;
  void* g_f1 = nullptr;
  int g_cur0 = 0, g_cur1 = 0, g_geom0 = -1, g_geom1 = -1;
  long long g_launch0 = 0, g_launch1 = 0;
  cudaStream_t cap_st = nullptr;
  bool stepped = false;
};

namespace {

lbm_status rfail(lbm_refined* r, lbm_status s, const std::string& msg) {
  if (r) r->err = msg;
  return s;
}

void refined_free(lbm_refined* r) {
  if (!r) return;
  if (r->h0) {
    DeviceGuard dg(r->h0->cfg.device);
    if (r->h0->st) cudaStreamSynchronize(r->h0->st);
    if (r->ghost) cudaFree(r->ghost);
    if (r->shell) cudaFree(r->shell);
    if (r->corners) cudaFree(r->corners);
    if (r->Ga) cudaFree(r->Ga);
    if (r->Gb) cudaFree(r->Gb);
    if (r->gexec) cudaGraphExecDestroy(r->gexec);
    if (r->cap_st) cudaStreamDestroy(r->cap_st);
  }
  lbm_destroy(r->h1);
  lbm_destroy(r->h0);
  delete r;
}

}  // namespace

extern "C" {

lbm_status lbm_refined_create(const lbm_config* cfg, const int box_lo[3], const int box_hi[3], lbm_refined** out) {
  if (!cfg || !box_lo || !box_hi || !out || cfg->struct_size != sizeof(lbm_config)) return LBM_EINVAL;
  *out = nullptr;
  const int D = cfg->lattice == LBM_D3Q19 ? 3 : 2;
  const int n[3] = {cfg->nx, cfg->ny, D == 3 ? cfg->nz : 1};
  for (int a = 0; a < D; ++a) {
    // the box, its ghost nodes and the level-0 nodes they read lie inside
    // level 0, and the box holds restricted nodes
    if (box_lo[a] - kRefineG / 2 - 1 < 0 || box_hi[a] + kRefineG / 2 + 1 > n[a] - 1 ||
        box_hi[a] - box_lo[a] <= 2 * kRefineR)
      return LBM_EINVAL;
  }
  lbm_refined* r = new lbm_refined();
  r->D = D;
  // level 1: the box refined by 2 with ghost faces, Reynolds number on
  // 2 L cells; the theta rule (when asked for) applies to it, and level 0
  // takes the same theta
  lbm_config c1 = *cfg;
  c1.nx = 2 * (box_hi[0] - box_lo[0]) + 1 + 2 * kRefineG;
  c1.ny = 2 * (box_hi[1] - box_lo[1]) + 1 + 2 * kRefineG;
  c1.nz = D == 3 ? 2 * (box_hi[2] - box_lo[2]) + 1 + 2 * kRefineG : 1;
  c1.ref_length = 2.0 * cfg->ref_length;
  for (int f = 0; f < 6; ++f) c1.bc[f] = f < 2 * D ? lbmib::kBCGhostFace : LBM_BC_PERIODIC;
  lbm_status s = create_patch_handle(&c1, &r->h1);
  if (s) {
    refined_free(r);
    return s;
  }
  lbm_config c0 = *cfg;
  c0.theta_inf = r->h1->theta_inf;
  s = lbm_create(&c0, &r->h0);
  if (s) {
    refined_free(r);
    return s;
  }
  DeviceGuard dg(cfg->device);
  for (int a = 0; a < 3; ++a) {
    r->lo[a] = a < D ? box_lo[a] : 0;
    r->hi[a] = a < D ? box_hi[a] : 0;
  }
  // ghost nodes of level 1
  std::vector<int4> gh;
  const int m[3] = {c1.nx, c1.ny, c1.nz};
  for (int z = 0; z < m[2]; ++z)
    for (int y = 0; y < m[1]; ++y)
      for (int x = 0; x < m[0]; ++x) {
        const int c[3] = {x, y, z};
        bool g = false;
        for (int a = 0; a < D; ++a) g = g || c[a] < kRefineG || c[a] >= m[a] - kRefineG;
        if (g) gh.push_back(make_int4(x, y, z, 0));
      }
  lbmib::RefineDev& d = r->dev;
  d.g0 = r->h0->g;
  d.g1 = r->h1->g;
  d.G = kRefineG;
  d.n_ghost = (int)gh.size();
  for (int a = 0; a < 3; ++a) {
    d.lo[a] = r->lo[a];
    d.rlo[a] = a < D ? r->lo[a] + kRefineR : 0;
    d.rn[a] = a < D ? r->hi[a] - r->lo[a] - 2 * kRefineR + 1 : 1;
  }
  d.mu0 = r->h0->mu;
  d.mu1 = r->h1->mu;
  d.Cv = r->h0->Cv;
  // the level-0 nodes each ghost node's mean reads (corner sx + 2 sy + 4 sz
  // of the cell above its base node, only along axes where its level-1
  // index is odd) and their union, the shell
  const int NC = D == 3 ? 8 : 4;
  std::vector<int> corners(gh.size() * NC, -1);
  std::vector<long long> shell;
  std::unordered_map<long long, int> shell_of;
  for (size_t k = 0; k < gh.size(); ++k) {
    const int kk[3] = {gh[k].x, gh[k].y, gh[k].z};
    int base[3] = {0, 0, 0}, odd[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      const int v = kk[a] - kRefineG;
      odd[a] = v & 1;
      base[a] = r->lo[a] + (v - (v & 1)) / 2;
    }
    for (int c = 0; c < NC; ++c) {
      const int sc[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
      if ((sc[0] && !odd[0]) || (sc[1] && !odd[1]) || (sc[2] && !odd[2])) continue;
      const long long n0 = r->h0->g.lin(base[0] + sc[0], base[1] + sc[1], D == 3 ? base[2] + sc[2] : 0);
      auto it = shell_of.find(n0);
      int si;
      if (it == shell_of.end()) {
        si = (int)shell.size();
        shell_of.emplace(n0, si);
        shell.push_back(n0);
      } else {
        si = it->second;
      }
      corners[k * NC + c] = si;
    }
  }
  d.n_shell = (int)shell.size();
  // each ghost-state buffer holds the ghost state and its shell scratch
  const size_t gbytes = ((size_t)(r->h0->Q + 1) * gh.size() + (size_t)(r->h0->Q + D + 2) * shell.size()) *
                        r->h0->csize;
  if (cudaMalloc(&r->ghost, gh.size() * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&r->shell, shell.size() * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&r->corners, corners.size() * sizeof(int)) != cudaSuccess || cudaMalloc(&r->Ga, gbytes) != cudaSuccess ||
      cudaMalloc(&r->Gb, gbytes) != cudaSuccess) {
    cudaGetLastError();
    refined_free(r);
    return LBM_ENOMEM;
  }
  if (cudaMemcpy(r->ghost, gh.data(), gh.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(r->shell, shell.data(), shell.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(r->corners, corners.data(), corners.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    refined_free(r);
    return LBM_ECUDA;
  }
  d.ghost = r->ghost;
  d.shell = r->shell;
  d.corners = r->corners;
  *out = r;
  return LBM_OK;
}

void lbm_refined_destroy(lbm_refined* r) { refined_free(r); }

const char* lbm_refined_last_error(const lbm_refined* r) { return r ? r->err.c_str() : "null refined case"; }

lbm_status lbm_refined_level(lbm_refined* r, int level, lbm_handle** h) {
  if (!r || !h || level < 0 || level > 1) return LBM_EINVAL;
  *h = level == 0 ? r->h0 : r->h1;
  return LBM_OK;
}

lbm_status lbm_refined_info(const lbm_refined* r, int info[8]) {
  if (!r || !info) return LBM_EINVAL;
  info[0] = kRefineG;
  info[1] = kRefineR;
  for (int a = 0; a < 3; ++a) {
    info[2 + a] = r->h1->g.n[a];
    info[5 + a] = r->lo[a];
  }
  return LBM_OK;
}

}  // extern "C"

namespace {

// one level-0 step with its two level-1 steps and the transfers; the level
// steps run eagerly (while a graph is captured) or through lbm_step
lbm_status refined_once(lbm_refined* r, bool eager) {
  lbm_handle *h0 = r->h0, *h1 = r->h1;
  const Ops* ops = h0->ops;
  lbmib::RefineDev& d = r->dev;
  auto step = [&](lbm_handle* h) { return eager ? h->ops->step(h) : lbm_step(h, 1); };
  lbm_status s = ops->refine_ghost_state(h0, d, r->Ga);  // level 0 at n
  if (!s) s = step(h0);                                   // level 0: n -> n+1
  if (!s) s = ops->refine_fill(h0, h1, d, r->Ga, nullptr);
  if (!s) s = step(h1);                                   // level 1: n -> n+1/2
  if (!s) s = ops->refine_ghost_state(h0, d, r->Gb);     // level 0 at n+1
  if (!s) s = ops->refine_fill(h0, h1, d, r->Ga, r->Gb);
  if (!s) s = step(h1);                                   // level 1: n+1/2 -> n+1
  if (!s) s = ops->refine_restrict(h0, h1, d);
  return s;
}

// capture two level-0 steps as a graph; the host side of the captured steps
// (buffer swaps) returns both levels to the parities they started from
lbm_status refined_capture(lbm_refined* r) {
  lbm_handle *h0 = r->h0, *h1 = r->h1;
  if (r->gexec) cudaGraphExecDestroy(r->gexec);
  r->gexec = nullptr;
  cudaStream_t run_st = h0->st;
  if (!run_st && !r->cap_st && cudaStreamCreateWithFlags(&r->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return rfail(r, LBM_ECUDA, "capture stream");
  }
  cudaStream_t st = run_st ? run_st : r->cap_st;
  const long long l0 = h0->launches, l1 = h1->launches;
  void* f0 = h0->f;
  void* f1 = h1->f;
  const int c0 = h0->cur, c1 = h1->cur;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return rfail(r, LBM_ECUDA, "graph capture begin");
  }
  h0->st = h1->st = st;
  lbm_status s = refined_once(r, true);
  if (!s) s = refined_once(r, true);
  h0->st = h1->st = run_st;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  r->g_launch0 = h0->launches - l0;
  r->g_launch1 = h1->launches - l1;
  h0->launches = l0;
  h1->launches = l1;
  if (s || e != cudaSuccess || h0->f != f0 || h1->f != f1 || h0->cur != c0 || h1->cur != c1) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rfail(r, s ? s : LBM_ECUDA, "refined step graph capture");
  }
  const cudaError_t ei = cudaGraphInstantiate(&r->gexec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    r->gexec = nullptr;
    cudaGetLastError();
    return rfail(r, LBM_ECUDA, "refined step graph instantiate");
  }
  r->g_f0 = f0;
  r->g_f1 = f1;
  r->g_cur0 = c0;
  r->g_cur1 = c1;
  r->g_geom0 = h0->geom_version;
  r->g_geom1 = h1->geom_version;
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_refined_step(lbm_refined* r, int n_steps) {
  if (!r || n_steps < 0) return LBM_EINVAL;
  lbm_handle *h0 = r->h0, *h1 = r->h1;
  DeviceGuard dg(h0->cfg.device);
  if (h0->sticky) return (lbm_status)h0->sticky;
  if (h1->sticky) return (lbm_status)h1->sticky;
  // after a first eager step, pairs of level-0 steps replay a captured
  // graph; profiling runs and odd remainders step through lbm_step
  const bool graphs = h0->use_graph && h1->use_graph && !h0->prof && !h1->prof;
  int k = 0;
  while (k < n_steps) {
    if (graphs && r->stepped && n_steps - k >= 2) {
      if (!r->gexec || r->g_f0 != h0->f || r->g_f1 != h1->f || r->g_cur0 != h0->cur || r->g_cur1 != h1->cur ||
          r->g_geom0 != h0->geom_version || r->g_geom1 != h1->geom_version) {
        lbm_status s = refined_capture(r);
        if (s) return s;
      }
      if (cudaGraphLaunch(r->gexec, h0->st) != cudaSuccess) return rfail(r, LBM_ECUDA, "refined graph launch");
      h0->launches += r->g_launch0;
      h1->launches += r->g_launch1;
      k += 2;
      continue;
    }
    lbm_status s = refined_once(r, false);
    if (s) {
      const lbm_handle* hb = h1->err.empty() ? h0 : h1;
      return rfail(r, s, hb->err);
    }
    r->stepped = h0->stepped && h1->stepped;
    ++k;
  }
  return LBM_OK;
}

}  // extern "C"
