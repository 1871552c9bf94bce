// Batched stepping of several cases (lbm_batch_*), from work tables, in one
// of two launch forms: one persistent cooperative launch that runs every
// phase of the step for all cases with grid-wide barriers between them (2D
// lattices, the default there), or one launch each of the immersed-boundary
// force, spreading, fused and boundary kernels.  Two consecutive steps (both
// buffer parities) are captured once as a CUDA graph and replayed.  The
// autotuner times the tile heights, schedules and launch forms on the batch
// and keeps the fastest; it restores the state it advanced.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace lbmib_host;

struct lbm_batch {
  BatchPlan plan;
  cudaStream_t st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  const Ops* ops = nullptr;
  std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

void drop_graph(lbm_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_ok = false;
}

// the plan matches the handles when every case is at the parity it was
// built for and no geometry changed since
bool plan_current(lbm_batch* b) {
  BatchPlan& p = b->plan;
  if (!p.built) return false;
  for (size_t k = 0; k < p.cases.size(); ++k)
    if (p.cases[k]->f != p.built_f[k] || p.cases[k]->geom_version != p.built_geom[k]) return false;
  return true;
}

lbm_status rebuild(lbm_batch* b) {
  drop_graph(b);
  BatchPlan& p = b->plan;
  lbm_status s = b->ops->batch_build(&p);
  if (s) return bfail(b, s, p.err.empty() ? "batch plan" : p.err);
  if (p.launch_form == 1) {
    // barrier state (zero) and the grid of CTAs resident at once
    if (!p.bar && cudaMalloc(&p.bar, sizeof(lbmib::GridBarrier)) != cudaSuccess)
      return bfail(b, LBM_ENOMEM, "barrier state");
    if (cudaMemsetAsync(p.bar, 0, sizeof(lbmib::GridBarrier), b->st) != cudaSuccess)
      return bfail(b, LBM_ECUDA, "barrier state");
    s = b->ops->batch_persistent(&p, 0, 0);
    if (s) return bfail(b, s, "persistent launch: no resident grid for this plan");
  }
  p.built_f.clear();
  p.built_geom.clear();
  for (lbm_handle* h : p.cases) {
    p.built_f.push_back(h->f);
    p.built_geom.push_back(h->geom_version);
  }
  p.built = true;
  return LBM_OK;
}

// one step of every case, eager (also used while capturing)
lbm_status one_step(lbm_batch* b, int parity) {
  BatchPlan& p = b->plan;
  for (lbm_handle* h : p.cases)
    if (h->sticky) return (lbm_status)h->sticky;
  if (p.launch_form == 1) {
    lbm_status s = b->ops->batch_persistent(&p, parity, 1);
    if (s) return bfail(b, s, p.err);
    for (lbm_handle* h : p.cases) {
      std::swap(h->f, h->f2);
      std::swap(h->M, h->M2);
      h->cur = 1 - h->cur;
    }
    return LBM_OK;
  }
  lbm_status s = b->ops->batch_aux(&p, parity, 0);
  if (!s) s = b->ops->batch_fused(&p, parity);
  if (s) return bfail(b, s, p.err);
  for (lbm_handle* h : p.cases) {
    std::swap(h->f, h->f2);
    std::swap(h->M, h->M2);
    h->cur = 1 - h->cur;
  }
  s = b->ops->batch_aux(&p, parity, 1);
  if (s) return bfail(b, s, p.err);
  return LBM_OK;
}

// two steps from parity 0 (eager, also used while capturing): one
// persistent launch, or the launches of two single steps
lbm_status two_steps(lbm_batch* b) {
  BatchPlan& p = b->plan;
  if (p.launch_form != 1) {
    lbm_status s = one_step(b, 0);
    return s ? s : one_step(b, 1);
  }
  for (lbm_handle* h : p.cases)
    if (h->sticky) return (lbm_status)h->sticky;
  lbm_status s = b->ops->batch_persistent(&p, 0, 2);
  if (s) return bfail(b, s, p.err);
  return LBM_OK;  // two buffer swaps: every handle is back at parity 0
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int n, const lbm_config* cfgs, lbm_batch** out) {
  if (n <= 0 || !cfgs || !out) return LBM_EINVAL;
  *out = nullptr;
  for (int k = 1; k < n; ++k)
    if (cfgs[k].lattice != cfgs[0].lattice || cfgs[k].precision != cfgs[0].precision ||
        cfgs[k].device != cfgs[0].device)
      return LBM_EINVAL;
  DeviceGuard dg(cfgs[0].device);
  lbm_batch* b = new lbm_batch();
  if (dg.status() != cudaSuccess || cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return LBM_ECUDA;
  }
  b->plan.st = b->st;
  b->plan.launch_form = cfgs[0].lattice == LBM_D2Q9 ? 1 : 0;
  for (int k = 0; k < n; ++k) {
    lbm_config c = cfgs[k];
    c.stream = b->st;
    lbm_handle* h = nullptr;
    lbm_status s = lbm_create(&c, &h);
    if (s) {
      lbm_batch_destroy(b);
      return s;
    }
    b->plan.cases.push_back(h);
  }
  b->ops = b->plan.cases[0]->ops;
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->plan.cases.empty() ? 0 : b->plan.cases[0]->cfg.device);
  drop_graph(b);
  for (lbm_handle* h : b->plan.cases) lbm_destroy(h);
  BatchPlan& pl = b->plan;
  for (int p = 0; p < 2; ++p)
    for (void* d : {pl.descs[p], pl.ib_descs[p], pl.sp_descs[p], pl.bc_descs[p]})
      if (d) cudaFree(d);
  for (void* d : {pl.work, pl.ib_work, pl.sp_work, pl.bc_work, pl.bar})
    if (d) cudaFree(d);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : "null batch"; }

lbm_status lbm_batch_case(lbm_batch* b, int i, lbm_handle** h) {
  if (!b || !h || i < 0 || i >= (int)b->plan.cases.size()) return LBM_EINVAL;
  *h = b->plan.cases[i];
  return LBM_OK;
}

lbm_status lbm_batch_set_plan(lbm_batch* b, int tile_rows, int schedule) {
  if (!b || (tile_rows != 0 && tile_rows != 16 && tile_rows != 32) || schedule < 0 || schedule > 2) return LBM_EINVAL;
  b->plan.tile_rows = tile_rows;
  b->plan.schedule = schedule;
  b->plan.built = false;
  drop_graph(b);
  return LBM_OK;
}

lbm_status lbm_batch_set_launch_form(lbm_batch* b, int form) {
  if (!b || form < 0 || form > 1 || (form == 1 && b->plan.cases[0]->D != 2)) return LBM_EINVAL;
  b->plan.launch_form = form;
  b->plan.built = false;
  drop_graph(b);
  return LBM_OK;
}

lbm_status lbm_batch_test_stall_barrier(lbm_batch* b) {
  if (!b || b->plan.launch_form != 1) return LBM_EINVAL;
  DeviceGuard dg(b->plan.cases[0]->cfg.device);
  if (!plan_current(b)) {
    lbm_status s = rebuild(b);
    if (s) return s;
  }
  // an arrival count past any grid size: the next barrier cannot complete
  const unsigned stuck = 0x40000000u;
  if (cudaStreamSynchronize(b->st) != cudaSuccess ||
      cudaMemcpy(b->plan.bar, &stuck, sizeof(stuck), cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, LBM_ECUDA, "barrier state write");
  return LBM_OK;
}

lbm_status lbm_batch_get_launch_form(const lbm_batch* b, int* form) {
  if (!b || !form) return LBM_EINVAL;
  *form = b->plan.launch_form;
  return LBM_OK;
}

lbm_status lbm_batch_get_plan(const lbm_batch* b, int* tile_rows, int* schedule) {
  if (!b) return LBM_EINVAL;
  if (tile_rows) *tile_rows = b->plan.tile_rows;
  if (schedule) *schedule = b->plan.schedule;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n_steps) {
  if (!b || n_steps < 0) return LBM_EINVAL;
  DeviceGuard dg(b->plan.cases[0]->cfg.device);
  int done = 0;
  while (done < n_steps) {
    if (!plan_current(b)) {
      // the cases are at the other parity (odd number of eager steps) or a
      // geometry changed: rebuild the plan for the current state
      lbm_status s = rebuild(b);
      if (s) return s;
    }
    if (n_steps - done >= 2) {
      if (!b->graph_ok) {
        cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
        lbm_status s2 = two_steps(b);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->st, &g);
        if (s2 || e != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          return s2 ? s2 : bfail(b, LBM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        b->graph = g;
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
          drop_graph(b);
          return bfail(b, LBM_ECUDA, "graph instantiate");
        }
        b->graph_ok = true;
      }
      if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) return bfail(b, LBM_ECUDA, "graph launch");
      done += 2;
    } else {
      lbm_status s = one_step(b, 0);
      if (s) return s;
      done += 1;
    }
  }
  return LBM_OK;
}

lbm_status lbm_batch_step_sequential(lbm_batch* b, int n_steps) {
  if (!b || n_steps < 0) return LBM_EINVAL;
  DeviceGuard dg(b->plan.cases[0]->cfg.device);
  for (lbm_handle* h : b->plan.cases) {
    lbm_status s = lbm_step(h, n_steps);
    if (s) return bfail(b, s, h->err);
  }
  return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  DeviceGuard dg(b->plan.cases[0]->cfg.device);
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return bfail(b, LBM_ECUDA, "sync");
  if (b->plan.bar) {
    // a persistent launch whose grid barrier gave up ended early: the state
    // is not a whole step; clear the barrier for the next launch
    lbmib::GridBarrier gb;
    if (cudaMemcpy(&gb, b->plan.bar, sizeof(gb), cudaMemcpyDeviceToHost) != cudaSuccess)
      return bfail(b, LBM_ECUDA, "barrier status read");
    if (gb.err) {
      cudaMemset(b->plan.bar, 0, sizeof(gb));
      return bfail(b, LBM_ETIMEOUT, "persistent batched step: a grid barrier timed out");
    }
  }
  return LBM_OK;
}

// Time every (launch form, tile rows, schedule) candidate over `steps`
// batched steps and keep the fastest.  The state each trial advances is
// saved before and restored after.  With cache_path, a result for the same
// case set is read from / appended to that text file ("key tile_rows
// schedule launch_form" lines; a line without the form means form 0).
lbm_status lbm_batch_autotune(lbm_batch* b, int steps, const char* cache_path, double* best_ms) {
  if (!b || steps <= 0) return LBM_EINVAL;
  DeviceGuard dg(b->plan.cases[0]->cfg.device);
  BatchPlan& p = b->plan;
  std::ostringstream key;
  key << p.cases.size() << ":" << p.cases[0]->cfg.lattice << ":" << p.cases[0]->cfg.precision;
  for (lbm_handle* h : p.cases) key << ":" << h->g.n[0] << "x" << h->g.n[1] << "x" << h->g.n[2] << "/" << h->NL;
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string k;
      int tr = 0, sc = 0, fm = 0;
      if (!(ls >> k >> tr >> sc) || k != key.str()) continue;
      if (!(ls >> fm)) fm = 0;
      lbm_status s = lbm_batch_set_launch_form(b, fm);
      return s ? s : lbm_batch_set_plan(b, tr, sc);
    }
  }
  // save the state
  struct Saved {
    std::vector<std::pair<void*, size_t>> bufs;
    std::vector<void*> copies;
  } sv;
  for (lbm_handle* h : p.cases) {
    const size_t N = (size_t)h->g.N;
    sv.bufs.push_back({h->f, N * h->Q * h->ssize});
    sv.bufs.push_back({h->M, N * (h->D + 2) * h->csize});
    sv.bufs.push_back({h->P[h->cur], N * h->csize});
    sv.bufs.push_back({h->A[h->cur], N * h->NDEV * h->csize});
  }
  for (auto& bf : sv.bufs) {
    void* c = nullptr;
    if (cudaMalloc(&c, bf.second) != cudaSuccess) {
      for (void* q : sv.copies) cudaFree(q);
      return bfail(b, LBM_ENOMEM, "autotune snapshot");
    }
    cudaMemcpyAsync(c, bf.first, bf.second, cudaMemcpyDeviceToDevice, b->st);
    sv.copies.push_back(c);
  }
  std::vector<void*> f0, M0;
  std::vector<int> cur0;
  for (lbm_handle* h : p.cases) {
    f0.push_back(h->f);
    M0.push_back(h->M);
    cur0.push_back(h->cur);
  }
  auto restore = [&]() {
    for (size_t k = 0; k < p.cases.size(); ++k) {
      lbm_handle* h = p.cases[k];
      if (h->f != f0[k]) {
        std::swap(h->f, h->f2);
        std::swap(h->M, h->M2);
      }
      h->cur = cur0[k];
    }
    for (size_t i = 0; i < sv.bufs.size(); ++i)
      cudaMemcpyAsync(sv.bufs[i].first, sv.copies[i], sv.bufs[i].second, cudaMemcpyDeviceToDevice, b->st);
  };
  const int rows[3] = {0, 16, 32};
  const int nrows = (p.cases[0]->D == 2 && p.cases[0]->csize == 4) ? 3 : 1;
  const int nforms = p.cases[0]->D == 2 ? 2 : 1;
  double best = 1e300;
  int best_r = 0, best_s = 0, best_f = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  lbm_status st = LBM_OK;
  for (int fm = 0; fm < nforms && !st; ++fm)
  for (int ri = 0; ri < nrows && !st; ++ri)
    for (int sc = 0; sc < 3 && !st; ++sc) {
      lbm_batch_set_launch_form(b, fm);
      lbm_batch_set_plan(b, rows[ri], sc);
      st = lbm_batch_step(b, 2);  // warm-up and capture
      if (st) break;
      cudaEventRecord(e0, b->st);
      st = lbm_batch_step(b, 2 * ((steps + 1) / 2));
      cudaEventRecord(e1, b->st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_r = rows[ri];
        best_s = sc;
        best_f = fm;
      }
      restore();
    }
  cudaStreamSynchronize(b->st);
  for (void* q : sv.copies) cudaFree(q);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  lbm_batch_set_launch_form(b, best_f);
  lbm_batch_set_plan(b, best_r, best_s);
  if (best_ms) *best_ms = best / (2 * ((steps + 1) / 2));
  if (cache_path) {
    std::ofstream o(cache_path, std::ios::app);
    o << key.str() << " " << best_r << " " << best_s << " " << best_f << "\n";
  }
  return LBM_OK;
}

}  // extern "C"
