// C ABI of the solver (include/lbmib.h): handle management, derived
// constants, immersed-boundary setup orchestration and the time loop.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <cub/cub.cuh>
#include <string>
#include <vector>

#include "handle.cuh"
#include "ib.cuh"

using namespace lbmib;
using namespace lbmib_host;

namespace {

const Ops* pick_ops(int lattice, int precision) {
  if (lattice == LBM_D2Q9) {
    switch (precision) {
      case LBM_FP64: return ops_d2q9_fp64();
      case LBM_FP32: return ops_d2q9_fp32();
      case LBM_FP16DEV: return ops_d2q9_fp16();
      case LBM_BF16DEV: return ops_d2q9_bf16();
    }
  } else if (lattice == LBM_D3Q19) {
    switch (precision) {
      case LBM_FP64: return ops_d3q19_fp64();
      case LBM_FP32: return ops_d3q19_fp32();
      case LBM_FP16DEV: return ops_d3q19_fp16();
      case LBM_BF16DEV: return ops_d3q19_bf16();
    }
  }
  return nullptr;
}

// reading Q11: largest theta_inf <= 1 with u_inf <= 0.15 (lattice units) and
// an explicit conduction number kappa = mu gamma / Pr <= kappa_max
double theta_rule(double mach, double gamma, double re, double L, double pr, int D) {
  const double umax = 0.15;
  const double u1 = mach * std::sqrt(gamma * (1.0 / 3.0));
  const double k1 = (u1 * L / re) * gamma / pr;
  const double kmax = D == 2 ? 0.10 : 0.0667;
  double th = 1.0;
  if (u1 > umax) th = std::fmin(th, (umax / u1) * (umax / u1));
  if (k1 > kmax) th = std::fmin(th, (kmax / k1) * (kmax / k1));
  return th;
}

void free_ib(lbm_handle* h) {
  void* ptrs[] = {h->inside, h->X, h->nrm, h->uB, h->tB, h->tbc, h->sten_node, h->psten_node, h->sten_w,
                  h->sten_x, h->psten_w, h->phi, h->W, h->Xstar, h->dBV, h->row_ptr, h->cell_id, h->col,
                  h->slot_of_entry, h->wt, h->row_of_node, h->forced, h->G, h->FU, h->WQ, h->loads, h->owned};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->inside = nullptr;
  h->X = h->nrm = h->uB = h->tB = nullptr;
  h->tbc = nullptr;
  h->sten_node = h->psten_node = nullptr;
  h->sten_w = h->sten_x = h->psten_w = h->phi = h->W = h->Xstar = h->dBV = nullptr;
  h->row_ptr = h->cell_id = h->col = h->slot_of_entry = nullptr;
  h->wt = nullptr;
  h->row_of_node = nullptr;
  h->forced = nullptr;
  h->G = h->FU = h->WQ = h->loads = nullptr;
  h->owned = nullptr;
  h->has_ib = false;
  h->NL = h->n_rows = h->nnz = 0;
}

}  // namespace

extern "C" {

lbm_status lbm_config_default(lbm_config* c) {
  if (!c) return LBM_EINVAL;
  std::memset(c, 0, sizeof(*c));
  c->struct_size = sizeof(lbm_config);
  c->lattice = LBM_D2Q9;
  c->precision = LBM_FP32;
  c->nx = 64;
  c->ny = 64;
  c->nz = 1;
  c->mach = 0.1;
  c->reynolds = 100;
  c->ref_length = 10;
  c->prandtl = 0.71;
  c->gamma = 1.4;
  c->theta_inf = 0.0;
  c->inflow_dir[0] = 1.0;
  c->sigma_hrr = 0.98;
  c->d_n = 1.5;
  c->method = IB_FODIBM_R;
  c->tau_mode = LBM_TAU_LITERAL;
  c->use_ac = 2;
  c->bulk_ratio = 0.0;
  return LBM_OK;
}

}  // extern "C"

namespace {

// z slab of a larger case: global owned planes [z0, z1), ghost planes
// below / above, global nz
struct SlabSpec {
  int z0, z1, ghost_lo, ghost_hi, nz_global;
};

lbm_status create_impl(const lbm_config* cfg, const SlabSpec* slab, lbm_handle** out, bool ghost_faces = false) {
  if (!cfg || !out || cfg->struct_size != sizeof(lbm_config)) return LBM_EINVAL;
  *out = nullptr;
  const int D = cfg->lattice == LBM_D3Q19 ? 3 : 2;
  if ((cfg->lattice != LBM_D2Q9 && cfg->lattice != LBM_D3Q19) || cfg->nx < 3 || cfg->ny < 3 ||
      (D == 3 && cfg->nz < 3) || (D == 2 && cfg->nz != 1) || cfg->mach <= 0 || cfg->reynolds <= 0 ||
      cfg->ref_length <= 0 || cfg->gamma <= 1.0 || cfg->prandtl <= 0 || cfg->precision < 0 ||
      cfg->precision > LBM_BF16DEV || cfg->method < IB_DIBM || cfg->method > IB_FODIBM_R || cfg->use_ac < 0 ||
      cfg->use_ac > 3 || !(cfg->bulk_ratio >= 0.0) || !std::isfinite(cfg->bulk_ratio))
    return LBM_EINVAL;
  bool has_char = false, has_outlet = false;
  for (int f = 0; f < 2 * D; ++f) {
    const int t = cfg->bc[f];
    if ((t < LBM_BC_PERIODIC || t > LBM_BC_FARFIELD) && t != LBM_BC_CHARACTERISTIC &&
        !((slab || ghost_faces) && t == kBCGhostFace))
      return LBM_EINVAL;
    has_char = has_char || t == LBM_BC_CHARACTERISTIC;
    has_outlet = has_outlet || t == LBM_BC_OUTLET;
  }
  if (has_char && has_outlet) return LBM_EINVAL;  // a characteristic face is the outflow face
  for (int a = 0; a < D; ++a)
    if ((cfg->bc[2 * a] == LBM_BC_PERIODIC) != (cfg->bc[2 * a + 1] == LBM_BC_PERIODIC)) return LBM_EINVAL;
  const Ops* ops = pick_ops(cfg->lattice, cfg->precision);
  if (!ops) return LBM_EUNSUPPORTED;
  lbm_handle* h = new lbm_handle();
  h->cfg = *cfg;
  h->ops = ops;
  if (slab) {
    h->slab = true;
    h->slab_z0 = slab->z0;
    h->slab_z1 = slab->z1;
    h->ghost_lo = slab->ghost_lo;
    h->ghost_hi = slab->ghost_hi;
    h->nz_global = slab->nz_global;
    h->g.zoff = slab->z0 - slab->ghost_lo;
  }
  h->D = D;
  h->Q = D == 3 ? 19 : 9;
  h->NDEV = D == 3 ? 5 : 2;
  h->g.n[0] = cfg->nx;
  h->g.n[1] = cfg->ny;
  h->g.n[2] = D == 3 ? cfg->nz : 1;
  for (int a = 0; a < 3; ++a) h->g.per[a] = a < D ? (cfg->bc[2 * a] == LBM_BC_PERIODIC) : 1;
  h->g.N = (long long)h->g.n[0] * h->g.n[1] * h->g.n[2];
  h->st = (cudaStream_t)cfg->stream;
  h->csize = cfg->precision == LBM_FP64 ? 8 : 4;
  h->ssize = cfg->precision == LBM_FP64 ? 8 : (cfg->precision == LBM_FP32 ? 4 : 2);
  // derived constants (Sec. 2.1; readings Q10, Q11)
  h->gamma = cfg->gamma;
  h->R = 1.0 / 3.0;
  h->Cv = h->R / (h->gamma - 1.0);
  h->Cp = h->gamma * h->R / (h->gamma - 1.0);
  h->theta_inf = cfg->theta_inf > 0 ? cfg->theta_inf
                                    : theta_rule(cfg->mach, cfg->gamma, cfg->reynolds, cfg->ref_length,
                                                 cfg->prandtl, D);
  h->rho_inf = 1.0;
  for (float& o : h->g.off) o = 0.f;  // storage offsets: set by the engine's init
  const double c_inf = std::sqrt(h->gamma * h->R * h->theta_inf);
  h->u_mag = cfg->mach * c_inf;
  double dn = 0.0;
  for (int a = 0; a < D; ++a) dn += cfg->inflow_dir[a] * cfg->inflow_dir[a];
  dn = std::sqrt(dn);
  if (!(dn > 0)) {
    delete h;
    return LBM_EINVAL;
  }
  for (int a = 0; a < D; ++a) h->u_inf[a] = h->u_mag * (cfg->inflow_dir[a] / dn);
  h->mu = h->rho_inf * h->u_mag * cfg->ref_length / cfg->reynolds;
  h->lam = h->mu * h->Cp / cfg->prandtl;
  double k = 0.0;
  for (int a = 0; a < D; ++a) k += h->u_inf[a] * h->u_inf[a];
  h->E_inf = h->rho_inf * (0.5 * k + h->Cv * h->theta_inf);
  DeviceGuard dg(cfg->device);
  if (dg.status() != cudaSuccess) {
    delete h;
    return LBM_ECUDA;
  }
  const long long N = h->g.N;
  lbm_status s = LBM_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (s) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      s = fail(h, LBM_ENOMEM, "device allocation failed");
    }
  };
  {
    const char* zc = std::getenv("LBMIB_ZCHUNK");
    if (zc) {
      h->zchunk = std::max(1, std::atoi(zc));
      h->zchunk_fixed = 1;
    }
    const char* ng = std::getenv("LBMIB_NO_GRAPH");
    if (ng && ng[0] == '1') h->use_graph = 0;
    const char* bk = std::getenv("LBMIB_BC_SEPARATE");
    if (bk && bk[0] == '1') h->bc_in_kernel = 0;
  }
  alloc(&h->f, N * h->Q * h->ssize);
  alloc(&h->f2, N * h->Q * h->ssize);
  alloc(&h->M2, N * (D + 2) * h->csize);
  alloc(&h->M, N * (D + 3) * h->csize);
  alloc(&h->E, N * h->csize);
  for (int k2 = 0; k2 < 2; ++k2) {
    alloc(&h->P[k2], N * h->csize);
    alloc(&h->A[k2], N * h->NDEV * h->csize);
  }
  alloc(&h->feq_inf, 32 * h->csize);
  alloc((void**)&h->d_bad, sizeof(unsigned long long));
  if (!s) s = h->ops->init(h);
  if (!s && cudaStreamSynchronize(h->st) != cudaSuccess) s = fail(h, LBM_ECUDA, "init");
  if (s) {
    lbm_destroy(h);
    return s;
  }
  *out = h;
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_config* cfg, lbm_handle** out) { return create_impl(cfg, nullptr, out); }

}  // extern "C"

lbm_status lbmib_host::create_patch_handle(const lbm_config* cfg, lbm_handle** out) {
  return create_impl(cfg, nullptr, out, true);
}

extern "C" {

lbm_status lbm_create_slab(const lbm_config* cfg, int z0, int z1, int halo, lbm_handle** out) {
  if (!cfg || !out || cfg->struct_size != sizeof(lbm_config)) return LBM_EINVAL;
  *out = nullptr;
  if (cfg->lattice != LBM_D3Q19) return LBM_EINVAL;
  if (cfg->bc[4] == LBM_BC_PERIODIC) return LBM_EUNSUPPORTED;
  const int nz = cfg->nz;
  if (z0 < 0 || z1 > nz || z1 - z0 < 1 || halo < 1) return LBM_EINVAL;
  SlabSpec sp;
  sp.z0 = z0;
  sp.z1 = z1;
  sp.ghost_lo = z0 > 0 ? std::min(halo, z0) : 0;
  sp.ghost_hi = z1 < nz ? std::min(halo, nz - z1) : 0;
  sp.nz_global = nz;
  lbm_config c = *cfg;
  c.nz = (z1 - z0) + sp.ghost_lo + sp.ghost_hi;
  if (c.nz < 3) return LBM_EINVAL;
  if (sp.ghost_lo) c.bc[4] = kBCGhostFace;
  if (sp.ghost_hi) c.bc[5] = kBCGhostFace;
  return create_impl(&c, &sp, out);
}

lbm_status lbm_slab_info(const lbm_handle* h, int info[6]) {
  if (!h || !info) return LBM_EINVAL;
  if (!h->slab) return LBM_ESTATE;
  info[0] = h->slab_z0;
  info[1] = h->slab_z1;
  info[2] = h->ghost_lo;
  info[3] = h->ghost_hi;
  info[4] = h->g.zoff;
  info[5] = h->nz_global;
  return LBM_OK;
}

}  // extern "C"

namespace {

// the stepping state of a slab as (device pointer, plane bytes, planes) per
// component: populations (storage type), carried moments, rho(1-theta) of
// the previous step, deviator of a^F of the previous step
struct StateComp {
  char* base;
  size_t elem;
};
std::vector<StateComp> slab_components(lbm_handle* h) {
  std::vector<StateComp> v;
  const size_t N = (size_t)h->g.N;
  for (int i = 0; i < h->Q; ++i) v.push_back({(char*)h->f + i * N * h->ssize, h->ssize});
  for (int k = 0; k < h->D + 2; ++k) v.push_back({(char*)h->M + k * N * h->csize, h->csize});
  v.push_back({(char*)h->P[h->cur], h->csize});
  for (int k = 0; k < h->NDEV; ++k) v.push_back({(char*)h->A[h->cur] + k * N * h->csize, h->csize});
  return v;
}

// planes of one side: the first plane and the count
void slab_planes(const lbm_handle* h, int side, bool ghost, int* p0, int* cnt) {
  const int nloc = h->g.n[2];
  const int own = h->slab_z1 - h->slab_z0;
  if (side == 0) {
    *cnt = h->ghost_lo;
    *p0 = ghost ? 0 : h->ghost_lo;
  } else {
    *cnt = h->ghost_hi;
    *p0 = ghost ? nloc - h->ghost_hi : h->ghost_lo + own - h->ghost_hi;
  }
}

lbm_status slab_copy(lbm_handle* h, int side, void* buf, bool pack) {
  if (!h->slab) return fail(h, LBM_ESTATE, "not a slab handle");
  if (side != 0 && side != 1) return fail(h, LBM_EINVAL, "side must be 0 (low z) or 1 (high z)");
  int p0 = 0, cnt = 0;
  slab_planes(h, side, !pack, &p0, &cnt);
  if (!cnt) return LBM_OK;
  if (pack && h->slab_z1 - h->slab_z0 < cnt) return fail(h, LBM_EINVAL, "slab thinner than its halo");
  const size_t plane = (size_t)h->g.n[0] * h->g.n[1];
  char* b = static_cast<char*>(buf);
  for (const StateComp& c : slab_components(h)) {
    const size_t bytes = (size_t)cnt * plane * c.elem;
    char* field = c.base + (size_t)p0 * plane * c.elem;
    const cudaError_t e = pack ? cudaMemcpyAsync(b, field, bytes, cudaMemcpyDeviceToDevice, h->st)
                               : cudaMemcpyAsync(field, b, bytes, cudaMemcpyDeviceToDevice, h->st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, LBM_ECUDA, std::string("slab exchange copy: ") + cudaGetErrorString(e));
    }
    b += bytes;
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_slab_exchange_bytes(const lbm_handle* h, int side, size_t* bytes) {
  if (!h || !bytes || (side != 0 && side != 1)) return LBM_EINVAL;
  if (!h->slab) return LBM_ESTATE;
  const int cnt = side == 0 ? h->ghost_lo : h->ghost_hi;
  const size_t plane = (size_t)h->g.n[0] * h->g.n[1];
  *bytes = (size_t)cnt * plane * (h->Q * h->ssize + (h->D + 3 + h->NDEV) * h->csize);
  return LBM_OK;
}

lbm_status lbm_slab_pack(lbm_handle* h, int side, void* dst) {
  if (!h || !dst) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  return slab_copy(h, side, dst, true);
}

lbm_status lbm_slab_unpack(lbm_handle* h, int side, const void* src) {
  if (!h || !src) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  lbm_status s = slab_copy(h, side, const_cast<void*>(src), false);
  // the ghost planes changed: a captured step graph stays valid (same
  // buffers), the stream orders the copies before the next step
  return s;
}

namespace {
void drop_step_graph(lbm_handle* h);
}

void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  DeviceGuard dg(h->cfg.device);
  cudaStreamSynchronize(h->st);
  drop_step_graph(h);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  free_ib(h);
  void* ptrs[] = {h->f, h->f2, h->M, h->M2, h->E, h->P[0], h->P[1], h->A[0], h->A[1], h->feq_inf, h->d_bad};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& e : h->ev_pool) cudaEventDestroy(e);
  for (auto& e : h->ev_used) {
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  delete h;
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err.c_str() : "null handle"; }

// Points of a z slab (host only, no device work): keep[l] = 1 when the
// point's interpolation (d = 2) and projection (d = 1) stencils lie in the
// local planes [zlo, zhi) (global z), owned[l] = 1 when z0 <= X_z < z1 (each
// point has one owner).  The owned planes read the carried moments up to two
// planes beyond them; those take forcing from points whose d = 2 stencils
// reach them (within three more planes), whose Lagrangian weights (Eq.
// weight) need every point sharing one of their nodes (three more).  So a
// point may only be dropped when its d = 2 stencil stays more than four
// planes beyond the owned planes; returns 1 when a dropped point comes
// closer (the halo is too narrow there; 9 ghost planes always suffice).
static int slab_keep_points(int D, double d_n, int zlo, int zhi, int ghost_lo, int ghost_hi, int z0, int z1, int NL,
                            const double* X, const double* nrm, int* keep, int* owned) {
  for (int l = 0; l < NL; ++l) {
    const double xz = X[l * D + 2];
    const double fz = std::floor(xz);
    const int s_lo = int(fz) - 1, s_hi = int(fz) + (xz > fz ? 2 : 1);
    const double pz = xz + d_n * nrm[l * D + 2];
    const double fp = std::floor(pz);
    const int p_lo = int(fp), p_hi = int(fp) + (pz > fp ? 1 : 0);
    const int f_lo = std::min(s_lo, p_lo), f_hi = std::max(s_hi, p_hi);
    const bool out_lo = f_lo < zlo && ghost_lo > 0;
    const bool out_hi = f_hi >= zhi && ghost_hi > 0;
    keep[l] = (!out_lo && !out_hi) ? 1 : 0;
    owned[l] = (xz >= double(z0) && xz < double(z1)) ? 1 : 0;
    if ((out_lo && s_hi >= zlo + ghost_lo - 5) || (out_hi && s_lo < zhi - ghost_hi + 5)) return 1;
  }
  return 0;
}

// z ranges of n slabs of nz planes: owned [z0, z1), ghost planes below and
// above (halo, none at the domain faces)
static void slab_ranges(int nz, int n, int halo, int k, int* z0, int* z1, int* glo, int* ghi) {
  const int base = nz / n, extra = nz % n;
  *z0 = k * base + std::min(k, extra);
  *z1 = *z0 + base + (k < extra ? 1 : 0);
  *glo = *z0 > 0 ? std::min(halo, *z0) : 0;
  *ghi = *z1 < nz ? std::min(halo, nz - *z1) : 0;
}

lbm_status lbm_slab_plan(int nz, int n_slabs, int halo, int* out) {
  if (nz < 1 || n_slabs < 1 || n_slabs > nz || halo < 1 || !out) return LBM_EINVAL;
  for (int k = 0; k < n_slabs; ++k) slab_ranges(nz, n_slabs, halo, k, out + 4 * k, out + 4 * k + 1, out + 4 * k + 2,
                                                 out + 4 * k + 3);
  return LBM_OK;
}

lbm_status lbm_slab_keep(const lbm_config* cfg, int z0, int z1, int halo, int n_points, const double* X,
                         const double* normals, int* keep, int* owned) {
  if (!cfg || cfg->lattice != LBM_D3Q19 || !X || !normals || !keep || !owned || n_points < 0 || z0 < 0 ||
      z1 > cfg->nz || z1 <= z0 || halo < 1)
    return LBM_EINVAL;
  const int glo = z0 > 0 ? std::min(halo, z0) : 0, ghi = z1 < cfg->nz ? std::min(halo, cfg->nz - z1) : 0;
  return slab_keep_points(3, cfg->d_n, z0 - glo, z1 + ghi, glo, ghi, z0, z1, n_points, X, normals, keep, owned)
             ? LBM_EGEOM
             : LBM_OK;
}

static lbm_status set_geometry_impl(lbm_handle* h, const ib_geometry* gm) {
  if (!h || !gm || gm->struct_size != sizeof(ib_geometry) || gm->n_points <= 0 || !gm->X || !gm->normals ||
      !gm->t_value)
    return fail(h, LBM_EINVAL, "invalid geometry arguments");
  if (gm->shape < IB_SHAPE_SPHERE || gm->shape > IB_SHAPE_MASK) return fail(h, LBM_EINVAL, "invalid shape");
  if (gm->shape == IB_SHAPE_POLYGON && (gm->n_poly < 3 || !gm->poly || h->D != 2))
    return fail(h, LBM_EINVAL, "invalid polygon");
  if (gm->shape == IB_SHAPE_ELLIPSE && h->D != 2) return fail(h, LBM_EINVAL, "ellipse is 2D only");
  if (gm->shape == IB_SHAPE_MASK && !gm->mask) return fail(h, LBM_EINVAL, "mask missing");
  DeviceGuard dg(h->cfg.device);
  CK(cudaStreamSynchronize(h->st));
  free_ib(h);
  const int D = h->D, NL = gm->n_points;
  const int KS = D == 2 ? 16 : 64, KP = D == 2 ? 4 : 8;
  const long long N = h->g.N;
  h->NL = NL;
  double* dpoly = nullptr;
  unsigned char* dmask = nullptr;
  int* derr = nullptr;
  unsigned long long *keys = nullptr, *keys_sorted = nullptr;
  int *count = nullptr, *head = nullptr, *head_scan = nullptr;
  double* s_row = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  lbm_status s = LBM_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (s) return;
    if (cudaMalloc(p, bytes ? bytes : 8) != cudaSuccess) {
      cudaGetLastError();
      s = fail(h, LBM_ENOMEM, "device allocation failed");
    }
  };
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (s) return;
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->st) != cudaSuccess)
      s = fail(h, LBM_ECUDA, "upload failed");
  };
  alloc((void**)&h->inside, N);
  alloc((void**)&h->X, NL * D * 8);
  alloc((void**)&h->nrm, NL * D * 8);
  alloc((void**)&h->uB, NL * D * 8);
  alloc((void**)&h->tB, NL * 8);
  alloc((void**)&h->tbc, NL * 4);
  alloc((void**)&h->sten_node, (size_t)NL * KS * 4);
  alloc((void**)&h->sten_w, (size_t)NL * KS * 8);
  alloc((void**)&h->sten_x, (size_t)NL * KS * 3 * 8);
  alloc((void**)&h->psten_node, (size_t)NL * KP * 4);
  alloc((void**)&h->psten_w, (size_t)NL * KP * 8);
  alloc((void**)&h->phi, NL * 8);
  alloc((void**)&h->W, NL * 8);
  alloc((void**)&h->Xstar, NL * D * 8);
  alloc((void**)&h->dBV, NL * 8);
  alloc((void**)&h->G, NL * (D + 2) * 8);
  alloc((void**)&h->loads, 8 * 8);
  alloc((void**)&h->row_of_node, N * 4);
  alloc((void**)&h->forced, N);
  alloc((void**)&derr, 4);
  alloc((void**)&keys, (size_t)NL * KS * 8);
  alloc((void**)&keys_sorted, (size_t)NL * KS * 8);
  alloc((void**)&count, 4);
  if (s) goto done;
  {
// a CUDA error from here on releases the temporaries and the partial setup
#define GCK(call)                                                                                     \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      cudaGetLastError();                                                                             \
      s = fail(h, LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));                     \
      goto done;                                                                                      \
    }                                                                                                 \
  } while (0)
    std::vector<double> zeros((size_t)NL * D, 0.0);
    std::vector<int> tb(NL, 0);
    if (gm->tbc)
      for (int l = 0; l < NL; ++l) tb[l] = gm->tbc[l];
    up(h->X, gm->X, NL * D * 8);
    up(h->nrm, gm->normals, NL * D * 8);
    up(h->uB, gm->u_target ? gm->u_target : zeros.data(), NL * D * 8);
    up(h->tB, gm->t_value, NL * 8);
    up(h->tbc, tb.data(), NL * 4);
    if (s) goto done;
    {
      double tsum = 0.0;
      int nd = 0;
      for (int l = 0; l < NL; ++l)
        if (tb[l] == IB_T_DIRICHLET) {
          tsum += gm->t_value[l];
          ++nd;
        }
      h->has_dirichlet = nd > 0;
      h->T_wall = nd > 0 ? tsum / nd : 0.0;
    }
    ShapeDev sd{};
    sd.kind = gm->shape;
    for (int a = 0; a < 3; ++a) sd.c[a] = gm->center[a];
    sd.r = gm->radius;
    sd.ra = gm->radii[0];
    sd.rb = gm->radii[1];
    sd.cs = gm->cos_a;
    sd.sn = gm->sin_a;
    sd.n_poly = gm->n_poly;
    if (gm->shape == IB_SHAPE_POLYGON) {
      alloc((void**)&dpoly, gm->n_poly * 2 * 8);
      up(dpoly, gm->poly, gm->n_poly * 2 * 8);
      sd.poly = dpoly;
    }
    if (gm->shape == IB_SHAPE_MASK) {
      alloc((void**)&dmask, N);
      up(dmask, gm->mask, N);
      sd.mask = dmask;
    }
    if (s) goto done;
    GCK(cudaMemsetAsync(derr, 0, 4, h->st));
    GCK(cudaMemsetAsync(count, 0, 4, h->st));
    GCK(cudaMemsetAsync(h->row_of_node, 0xff, N * 4, h->st));
    GCK(cudaMemsetAsync(h->forced, 0, N, h->st));
    if ((s = launch(h, kProfOther, [&] { k_classify<<<nblk(N, 256), 256, 0, h->st>>>(h->g, D, sd, h->inside); })))
      goto done;
    IBSetupDev sdv;
    sdv.D = D;
    sdv.NL = NL;
    sdv.one_sided = h->cfg.method != IB_DIBM;
    sdv.d_n = h->cfg.d_n;
    sdv.X = h->X;
    sdv.nrm = h->nrm;
    sdv.inside = h->inside;
    sdv.sten_node = h->sten_node;
    sdv.sten_w = h->sten_w;
    sdv.sten_x = h->sten_x;
    sdv.phi = h->phi;
    sdv.psten_node = h->psten_node;
    sdv.psten_w = h->psten_w;
    sdv.err = derr;
    if ((s = launch(h, kProfOther, [&] { k_stencils<<<nblk(NL, 64), 64, 0, h->st>>>(h->g, sdv); }))) goto done;
    if ((s = launch(h, kProfOther, [&] {
           k_csr_keys<<<nblk((long long)NL * KS, 256), 256, 0, h->st>>>(NL, KS, h->sten_node, keys, count);
         })))
      goto done;
    int herr = 0, hcount = 0;
    GCK(cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, h->st));
    GCK(cudaMemcpyAsync(&hcount, count, 4, cudaMemcpyDeviceToHost, h->st));
    GCK(cudaStreamSynchronize(h->st));
    if (herr) {
      s = fail(h, LBM_EGEOM, herr == 1 ? "an immersed-boundary stencil leaves the domain"
                                       : "a Lagrangian point has no interior node in its support");
      goto done;
    }
    const int nnz = hcount;
    h->nnz = nnz;
    // sort (node, point, slot) keys: rows ascending, entries ascending in l
    const int bits = 64;
    cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, keys, keys_sorted, nnz, 0, bits, h->st);
    alloc(&tmp, tmp_bytes);
    alloc((void**)&head, (size_t)nnz * 4);
    alloc((void**)&head_scan, (size_t)nnz * 4);
    if (s) goto done;
    GCK(cub::DeviceRadixSort::SortKeys(tmp, tmp_bytes, keys, keys_sorted, nnz, 0, bits, h->st));
    const int NLKS = NL * KS;
    if ((s = launch(h, kProfOther, [&] {
           k_csr_heads<<<nblk(nnz, 256), 256, 0, h->st>>>(nnz, NLKS, keys_sorted, head);
         })))
      goto done;
    size_t tmp2 = 0;
    cub::DeviceScan::InclusiveSum(nullptr, tmp2, head, head_scan, nnz, h->st);
    if (tmp2 > tmp_bytes) {
      GCK(cudaStreamSynchronize(h->st));
      cudaFree(tmp);
      tmp = nullptr;
      tmp_bytes = tmp2;
      alloc(&tmp, tmp_bytes);
      if (s) goto done;
    }
    GCK(cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, head, head_scan, nnz, h->st));
    int nrows = 0;
    GCK(cudaMemcpyAsync(&nrows, head_scan + (nnz - 1), 4, cudaMemcpyDeviceToHost, h->st));
    GCK(cudaStreamSynchronize(h->st));
    h->n_rows = nrows;
    alloc((void**)&h->row_ptr, (size_t)(nrows + 1) * 4);
    alloc((void**)&h->cell_id, (size_t)nrows * 4);
    alloc((void**)&h->col, (size_t)nnz * 4);
    alloc((void**)&h->slot_of_entry, (size_t)nnz * 4);
    alloc((void**)&h->wt, (size_t)nnz * 8);
    alloc((void**)&s_row, (size_t)nrows * 8);
    alloc((void**)&h->FU, (size_t)nrows * D * 8);
    alloc((void**)&h->WQ, (size_t)nrows * 8);
    if (s) goto done;
    GCK(cudaMemcpyAsync(h->row_ptr + nrows, &h->nnz, 4, cudaMemcpyHostToDevice, h->st));
    if ((s = launch(h, kProfOther, [&] {
           k_csr_fill<<<nblk(nnz, 256), 256, 0, h->st>>>(nnz, NLKS, KS, keys_sorted, head_scan, h->row_ptr,
                                                          h->cell_id, h->col, h->slot_of_entry);
         })))
      goto done;
    if ((s = launch(h, kProfOther, [&] {
           k_row_density<<<nblk(nrows, 256), 256, 0, h->st>>>(nrows, h->row_ptr, h->slot_of_entry, h->col,
                                                               h->phi, h->sten_w, s_row);
         })))
      goto done;
    if ((s = launch(h, kProfOther, [&] {
           k_weights<<<nblk(NL, 64), 64, 0, h->st>>>(D, NL, KS, nrows, h->cell_id, s_row, h->sten_node,
                                                     h->sten_w, h->sten_x, h->phi, h->X, h->nrm, h->W,
                                                     h->Xstar, h->dBV);
         })))
      goto done;
    if ((s = launch(h, kProfOther, [&] {
           k_csr_weights<<<nblk(nnz, 256), 256, 0, h->st>>>(nnz, h->col, h->slot_of_entry, h->phi, h->W,
                                                            h->sten_w, h->wt);
         })))
      goto done;
    if ((s = launch(h, kProfOther, [&] {
           k_row_map<<<nblk(nrows, 256), 256, 0, h->st>>>(nrows, h->cell_id, h->row_of_node, h->forced);
         })))
      goto done;
    GCK(cudaMemsetAsync(h->G, 0, NL * (D + 2) * 8, h->st));
    GCK(cudaMemsetAsync(h->FU, 0, (size_t)nrows * D * 8, h->st));
    GCK(cudaMemsetAsync(h->WQ, 0, (size_t)nrows * 8, h->st));
    GCK(cudaStreamSynchronize(h->st));
    h->has_ib = true;
    h->geom_version++;
  }
done:
  cudaStreamSynchronize(h->st);
  void* tmps[] = {dpoly, dmask, derr, keys, keys_sorted, count, head, head_scan, s_row, tmp};
  for (void* p : tmps)
    if (p) cudaFree(p);
  if (s) free_ib(h);
  return s;
#undef GCK
}

lbm_status ib_set_geometry(lbm_handle* h, const ib_geometry* gm) {
  if (!h || !gm || gm->struct_size != sizeof(ib_geometry) || gm->n_points <= 0 || !gm->X || !gm->normals ||
      !gm->t_value)
    return fail(h, LBM_EINVAL, "invalid geometry arguments");
  if (!h->slab) return set_geometry_impl(h, gm);
  // A z slab keeps the points whose interpolation (d = 2) and projection
  // (d = 1) stencils lie in its local planes (slab_keep_points); the
  // geometry stays in global coordinates.
  const int D = h->D, NL = gm->n_points;
  std::vector<int> kflag(NL), oflag(NL);
  if (slab_keep_points(D, h->cfg.d_n, h->g.zoff, h->g.zoff + h->g.n[2], h->ghost_lo, h->ghost_hi, h->slab_z0,
                       h->slab_z1, NL, gm->X, gm->normals, kflag.data(), oflag.data()))
    return fail(h, LBM_EGEOM, "slab halo too narrow for the immersed body at a slab boundary");
  std::vector<int> keep;
  for (int l = 0; l < NL; ++l)
    if (kflag[l]) keep.push_back(l);
  DeviceGuard dg(h->cfg.device);
  if (keep.empty()) {
    CK(cudaStreamSynchronize(h->st));
    free_ib(h);
    h->slab_points.clear();
    h->geom_version++;
    return LBM_OK;
  }
  const int n = (int)keep.size();
  std::vector<double> X((size_t)n * D), nrm((size_t)n * D), ut((size_t)n * D), tv(n);
  std::vector<int> tb(n, 0);
  for (int k = 0; k < n; ++k) {
    const int l = keep[k];
    for (int a = 0; a < D; ++a) {
      X[k * D + a] = gm->X[l * D + a];
      nrm[k * D + a] = gm->normals[l * D + a];
      ut[k * D + a] = gm->u_target ? gm->u_target[l * D + a] : 0.0;
    }
    tv[k] = gm->t_value[l];
    if (gm->tbc) tb[k] = gm->tbc[l];
  }
  ib_geometry g2 = *gm;
  g2.n_points = n;
  g2.X = X.data();
  g2.normals = nrm.data();
  g2.u_target = ut.data();
  g2.t_value = tv.data();
  g2.tbc = tb.data();
  if (gm->shape == IB_SHAPE_MASK) g2.mask = gm->mask + (size_t)h->g.zoff * h->g.n[0] * h->g.n[1];
  lbm_status s = set_geometry_impl(h, &g2);
  if (s) return s;
  h->slab_points = keep;
  std::vector<unsigned char> own(n);
  for (int k = 0; k < n; ++k) own[k] = (unsigned char)oflag[keep[k]];
  if (cudaMalloc((void**)&h->owned, n) != cudaSuccess) {
    cudaGetLastError();
    free_ib(h);
    return fail(h, LBM_ENOMEM, "device allocation failed");
  }
  CK(cudaMemcpy(h->owned, own.data(), n, cudaMemcpyHostToDevice));
  return LBM_OK;
}

lbm_status lbm_slab_points(const lbm_handle* h, int* n_points, int* global_index) {
  if (!h || !n_points) return LBM_EINVAL;
  if (!h->slab) return LBM_ESTATE;
  *n_points = (int)h->slab_points.size();
  if (global_index)
    for (size_t k = 0; k < h->slab_points.size(); ++k) global_index[k] = h->slab_points[k];
  return LBM_OK;
}

namespace {

void drop_step_graph(lbm_handle* h) {
  for (StepGraph& g : h->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = StepGraph{};
  }
}

// Capture n_steps (1 or 2) steps from the current buffer parity as a graph.
// Capturing runs the host side of the steps (the buffer swaps) but no
// kernel: the handle is left at the parity after them, where a launch of
// the graph brings the device as well.
lbm_status capture_steps(lbm_handle* h, int n_steps, StepGraph& out) {
  if (out.exec) cudaGraphExecDestroy(out.exec);
  out = StepGraph{};
  // the legacy default stream cannot be captured: record on a private
  // stream (the graph keeps no stream) and launch on the handle's stream
  cudaStream_t run_st = h->st;
  if (!run_st && !h->cap_st && cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, LBM_ECUDA, "capture stream");
  }
  cudaStream_t st = run_st ? run_st : h->cap_st;
  void* f0 = h->f;
  const int cur0 = h->cur;
  const long long l0 = h->launches;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, LBM_ECUDA, "graph capture begin");
  }
  h->st = st;
  lbm_status s = LBM_OK;
  for (int k = 0; k < n_steps && !s; ++k) s = h->ops->step(h);
  h->st = run_st;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  const long long nl = h->launches - l0;
  h->launches = l0;
  auto rewind = [&] {
    // nothing ran: put the host side back at the starting parity
    if (h->f != f0) {
      std::swap(h->f, h->f2);
      std::swap(h->M, h->M2);
    }
    h->cur = cur0;
  };
  if (s || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    rewind();
    return s ? s : fail(h, LBM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&out.exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    out.exec = nullptr;
    cudaGetLastError();
    rewind();
    return fail(h, LBM_ECUDA, "graph instantiate");
  }
  out.f = f0;
  out.cur = cur0;
  out.geom = h->geom_version;
  out.launches = nl;
  rewind();
  return LBM_OK;
}

}  // namespace

lbm_status lbm_step(lbm_handle* h, int n_steps) {
  if (!h || n_steps < 0) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  if (h->sticky) return (lbm_status)h->sticky;
  // after a first eager step (which sets the kernels' launch attributes)
  // steps replay captured graphs, two at a time and one for an odd
  // remainder (fewer host launches for small grids); profiling runs step
  // eagerly
  const bool graphs = h->use_graph && !h->prof;
  int k = 0;
  while (k < n_steps) {
    if (graphs && h->stepped) {
      const int n = n_steps - k >= 2 ? 2 : 1;
      StepGraph& g = h->graphs[n == 2 ? 0 : 1 + h->cur];
      if (!g.exec || g.f != h->f || g.cur != h->cur || g.geom != h->geom_version) {
        lbm_status s = capture_steps(h, n, g);
        if (s) return s;
      }
      if (cudaGraphLaunch(g.exec, h->st) != cudaSuccess) return fail(h, LBM_ECUDA, "graph launch");
      h->launches += g.launches;
      // the host side of the replayed steps: one buffer swap per step
      if (n == 1) {
        std::swap(h->f, h->f2);
        std::swap(h->M, h->M2);
        h->cur = 1 - h->cur;
      }
      k += n;
      continue;
    }
    lbm_status s = h->ops->step(h);
    if (s) return s;
    h->stepped = true;
    ++k;
  }
  return LBM_OK;
}

lbm_status lbm_check(lbm_handle* h) {
  if (!h) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  CK(cudaMemsetAsync(h->d_bad, 0, sizeof(unsigned long long), h->st));
  lbm_status s = h->ops->health(h, h->d_bad);
  if (s) return s;
  unsigned long long bad = 0;
  CK(cudaMemcpyAsync(&bad, h->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (bad) {
    h->sticky = LBM_ENAN;
    return fail(h, LBM_ENAN, std::to_string(bad) + " nodes with non-finite or non-positive rho / T");
  }
  return LBM_OK;
}

lbm_status lbm_get_fields(lbm_handle* h, int dst_is_device, double* rho, double* u, double* T, double* p) {
  if (!h) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  const long long N = h->g.N;
  if (dst_is_device) {
    lbm_status s = h->ops->fields(h, rho, u, T, p);
    if (s) return s;
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
  }
  double* buf = nullptr;
  CK(cudaMalloc(&buf, N * 8 * (h->D + 3)));
  double *dr = buf, *du = buf + N, *dT = buf + N * (1 + h->D), *dp = buf + N * (2 + h->D);
  lbm_status s = h->ops->fields(h, rho ? dr : nullptr, u ? du : nullptr, T ? dT : nullptr, p ? dp : nullptr);
  if (!s) {
    if (rho) cudaMemcpyAsync(rho, dr, N * 8, cudaMemcpyDeviceToHost, h->st);
    if (u) cudaMemcpyAsync(u, du, N * 8 * h->D, cudaMemcpyDeviceToHost, h->st);
    if (T) cudaMemcpyAsync(T, dT, N * 8, cudaMemcpyDeviceToHost, h->st);
    if (p) cudaMemcpyAsync(p, dp, N * 8, cudaMemcpyDeviceToHost, h->st);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) s = fail(h, LBM_ECUDA, "get_fields copy");
  }
  cudaFree(buf);
  return s;
}

lbm_status lbm_get_state(lbm_handle* h, int dst_is_device, double* f, double* E) {
  if (!h || !f || !E) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  const long long N = h->g.N;
  if (dst_is_device) {
    lbm_status s = h->ops->get_state(h, f, E);
    if (s) return s;
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
  }
  double* buf = nullptr;
  CK(cudaMalloc(&buf, N * 8 * (h->Q + 1)));
  lbm_status s = h->ops->get_state(h, buf, buf + N * h->Q);
  if (!s) {
    cudaMemcpyAsync(f, buf, N * 8 * h->Q, cudaMemcpyDeviceToHost, h->st);
    cudaMemcpyAsync(E, buf + N * h->Q, N * 8, cudaMemcpyDeviceToHost, h->st);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) s = fail(h, LBM_ECUDA, "get_state copy");
  }
  cudaFree(buf);
  return s;
}

}  // extern "C"

namespace {
// the device address of page-locked host memory the device can read in
// place (null for pageable memory): the upload kernels then read it over
// the bus directly, with no device staging buffer and no separate copy
const double* mapped_host(const double* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? (const double*)a.devicePointer : nullptr;
}
}  // namespace

extern "C" {

lbm_status lbm_set_state(lbm_handle* h, int src_is_device, const double* f, const double* E) {
  if (!h || !f || !E) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  const long long N = h->g.N;
  if (src_is_device) {
    lbm_status s = h->ops->set_state(h, f, E);
    if (s) return s;
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
  }
  const double *mf = mapped_host(f), *mE = mapped_host(E);
  if (mf && mE) {
    lbm_status s = h->ops->set_state(h, mf, mE);
    if (s) return s;
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
  }
  double* buf = nullptr;
  CK(cudaMalloc(&buf, N * 8 * (h->Q + 1)));
  lbm_status s = LBM_OK;
  if (cudaMemcpyAsync(buf, f, N * 8 * h->Q, cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
      cudaMemcpyAsync(buf + N * h->Q, E, N * 8, cudaMemcpyHostToDevice, h->st) != cudaSuccess)
    s = fail(h, LBM_ECUDA, "set_state copy");
  if (!s) s = h->ops->set_state(h, buf, buf + N * h->Q);
  cudaStreamSynchronize(h->st);
  cudaFree(buf);
  return s;
}

namespace {

struct StateHeader {
  char magic[8];
  int version, lattice, precision, nx, ny, nz, fused, pad;
  long long N;
};

// device arrays of the stepping state and their byte sizes
int state_arrays(lbm_handle* h, void** ptr, size_t* bytes) {
  const size_t N = (size_t)h->g.N;
  int k = 0;
  ptr[k] = h->f;
  bytes[k++] = N * h->Q * h->ssize;
  ptr[k] = h->M;
  bytes[k++] = N * (h->D + 2) * h->csize;
  ptr[k] = h->P[h->cur];
  bytes[k++] = N * h->csize;
  ptr[k] = h->A[h->cur];
  bytes[k++] = N * h->NDEV * h->csize;
  return k;
}

StateHeader state_header(lbm_handle* h) {
  StateHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "LBMIBST1", 8);
  hd.version = 1;
  hd.lattice = h->cfg.lattice;
  hd.precision = h->cfg.precision;
  hd.nx = h->g.n[0];
  hd.ny = h->g.n[1];
  hd.nz = h->g.n[2];
  hd.fused = 1;
  hd.N = h->g.N;
  return hd;
}

}  // namespace

lbm_status lbm_save_state(lbm_handle* h, const char* path) {
  if (!h || !path) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  void* ptr[4];
  size_t bytes[4];
  const int n = state_arrays(h, ptr, bytes);
  const StateHeader hd = state_header(h);
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(h, LBM_ESTATE, std::string("cannot open ") + path);
  bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1;
  std::vector<unsigned char> host;
  CK(cudaStreamSynchronize(h->st));
  for (int k = 0; k < n && ok; ++k) {
    host.resize(bytes[k]);
    if (cudaMemcpy(host.data(), ptr[k], bytes[k], cudaMemcpyDeviceToHost) != cudaSuccess) {
      std::fclose(fp);
      return fail(h, LBM_ECUDA, "state copy to host");
    }
    ok = std::fwrite(host.data(), 1, bytes[k], fp) == bytes[k];
  }
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) return fail(h, LBM_ESTATE, std::string("cannot write ") + path);
  return LBM_OK;
}

lbm_status lbm_load_state(lbm_handle* h, const char* path) {
  if (!h || !path) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  void* ptr[4];
  size_t bytes[4];
  const int n = state_arrays(h, ptr, bytes);
  const StateHeader want = state_header(h);
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(h, LBM_ESTATE, std::string("cannot open ") + path);
  StateHeader hd;
  if (std::fread(&hd, sizeof(hd), 1, fp) != 1 || std::memcmp(&hd, &want, sizeof(hd)) != 0) {
    std::fclose(fp);
    return fail(h, LBM_ESTATE, "state file of another lattice, precision, grid or step form");
  }
  std::vector<std::vector<unsigned char>> host(n);
  for (int k = 0; k < n; ++k) {
    host[k].resize(bytes[k]);
    if (std::fread(host[k].data(), 1, bytes[k], fp) != bytes[k]) {
      std::fclose(fp);
      return fail(h, LBM_ESTATE, "state file truncated");
    }
  }
  std::fclose(fp);
  CK(cudaStreamSynchronize(h->st));
  for (int k = 0; k < n; ++k)
    if (cudaMemcpy(ptr[k], host[k].data(), bytes[k], cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(h, LBM_ECUDA, "state copy to device");
  h->sticky = LBM_OK;
  return LBM_OK;
}

lbm_status lbm_set_fields(lbm_handle* h, int src_is_device, const double* rho, const double* u,
                          const double* T) {
  if (!h || !rho || !u || !T) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  const long long N = h->g.N;
  if (src_is_device) {
    lbm_status s = h->ops->set_fields(h, rho, u, T);
    if (s) return s;
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
  }
  const double *mr = mapped_host(rho), *mu = mapped_host(u), *mT = mapped_host(T);
  if (mr && mu && mT) {
    lbm_status s = h->ops->set_fields(h, mr, mu, mT);
    if (s) return s;
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
  }
  double* buf = nullptr;
  CK(cudaMalloc(&buf, N * 8 * (h->D + 2)));
  lbm_status s = LBM_OK;
  if (cudaMemcpyAsync(buf, rho, N * 8, cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
      cudaMemcpyAsync(buf + N, u, N * 8 * h->D, cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
      cudaMemcpyAsync(buf + N * (1 + h->D), T, N * 8, cudaMemcpyHostToDevice, h->st) != cudaSuccess)
    s = fail(h, LBM_ECUDA, "set_fields copy");
  if (!s) s = h->ops->set_fields(h, buf, buf + N, buf + N * (1 + h->D));
  cudaStreamSynchronize(h->st);
  cudaFree(buf);
  return s;
}

lbm_status lbm_get_wall_loads(lbm_handle* h, double force[3], double* heat, double* work, double* per_point) {
  if (!h) return LBM_EINVAL;
  if (h->slab && !h->has_ib) {
    // a slab the body does not reach contributes nothing
    if (force)
      for (int a = 0; a < 3; ++a) force[a] = 0.0;
    if (heat) *heat = 0.0;
    if (work) *work = 0.0;
    return LBM_OK;
  }
  DeviceGuard dg(h->cfg.device);
  if (!h->has_ib) return fail(h, LBM_ESTATE, "no immersed body");
  lbm_status s = launch(h, kProfOther, [&] { k_wall_loads<<<1, 256, 0, h->st>>>(h->D, h->NL, h->G, h->W, h->owned, h->loads); });
  if (s) return s;
  double out[5];
  CK(cudaMemcpyAsync(out, h->loads, 5 * 8, cudaMemcpyDeviceToHost, h->st));
  if (per_point) CK(cudaMemcpyAsync(per_point, h->G, (size_t)h->NL * (h->D + 2) * 8, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (force)
    for (int a = 0; a < 3; ++a) force[a] = out[a];
  if (heat) *heat = out[3];
  if (work) *work = out[4];
  return LBM_OK;
}

lbm_status lbm_get_wall_loads_async(lbm_handle* h, double out[5]) {
  if (!h || !out) return LBM_EINVAL;
  if (h->slab && !h->has_ib) {
    for (int a = 0; a < 5; ++a) out[a] = 0.0;
    return LBM_OK;
  }
  DeviceGuard dg(h->cfg.device);
  if (!h->has_ib) return fail(h, LBM_ESTATE, "no immersed body");
  lbm_status s = launch(h, kProfOther, [&] { k_wall_loads<<<1, 256, 0, h->st>>>(h->D, h->NL, h->G, h->W, h->owned, h->loads); });
  if (s) return s;
  // stream order keeps the next call's reduction behind this copy, so one
  // device slot serves every call
  CK(cudaMemcpyAsync(out, h->loads, 5 * 8, cudaMemcpyDeviceToHost, h->st));
  return LBM_OK;
}

lbm_status lbm_sync(lbm_handle* h) {
  if (!h) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  CK(cudaStreamSynchronize(h->st));
  return (lbm_status)h->sticky;
}

lbm_status lbm_get_wall_diagnostics(lbm_handle* h, double coeffs[4], double* per_point) {
  if (!h) return LBM_EINVAL;
  if (!h->has_ib) return fail(h, LBM_ESTATE, "no immersed body");
  DeviceGuard dg(h->cfg.device);
  const int D = h->D;
  if (coeffs) {
    double force[3], heat = 0.0;
    lbm_status s = lbm_get_wall_loads(h, force, &heat, nullptr, nullptr);
    if (s) return s;
    // drag along the inflow direction, lift along the perpendicular axes
    double ed[3] = {0, 0, 0}, e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0}, nd = 0.0;
    for (int a = 0; a < D; ++a) nd += h->cfg.inflow_dir[a] * h->cfg.inflow_dir[a];
    nd = std::sqrt(nd);
    for (int a = 0; a < D; ++a) ed[a] = h->cfg.inflow_dir[a] / nd;
    if (D == 2) {
      e1[0] = -ed[1];
      e1[1] = ed[0];
    } else {
      e1[0] = -ed[1] * ed[0];
      e1[1] = 1.0 - ed[1] * ed[1];
      e1[2] = -ed[1] * ed[2];
      const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
      for (int a = 0; a < 3; ++a) e1[a] /= n1;
      e2[0] = ed[1] * e1[2] - ed[2] * e1[1];
      e2[1] = ed[2] * e1[0] - ed[0] * e1[2];
      e2[2] = ed[0] * e1[1] - ed[1] * e1[0];
    }
    const double Lr = h->cfg.ref_length;
    const double q = 0.5 * h->rho_inf * h->u_mag * h->u_mag;
    const double A = D == 2 ? Lr : M_PI * Lr * Lr / 4.0;
    const double S = D == 2 ? M_PI * Lr : M_PI * Lr * Lr;
    double fd = 0.0, f1 = 0.0, f2 = 0.0;
    for (int a = 0; a < D; ++a) {
      fd += force[a] * ed[a];
      f1 += force[a] * e1[a];
      f2 += force[a] * e2[a];
    }
    coeffs[0] = fd / (q * A);
    coeffs[1] = f1 / (q * A);
    coeffs[2] = D == 3 ? f2 / (q * A) : 0.0;
    coeffs[3] = (h->has_dirichlet && h->T_wall != h->theta_inf)
                    ? heat * Lr / (h->lam * (h->T_wall - h->theta_inf) * S)
                    : 0.0;
  }
  if (per_point) {
    const size_t bytes = (size_t)h->NL * (2 * D + 4) * 8;
    double* buf = nullptr;
    int* derr = nullptr;
    CK(cudaMalloc(&buf, bytes + 16));
    derr = reinterpret_cast<int*>(reinterpret_cast<char*>(buf) + bytes);
    lbm_status s = LBM_OK;
    if (cudaMemsetAsync(derr, 0, 4, h->st) != cudaSuccess) s = fail(h, LBM_ECUDA, "diagnostics memset");
    if (!s) s = h->ops->wall_diag(h, buf, derr);
    int herr = 0;
    if (!s && (cudaMemcpyAsync(per_point, buf, bytes, cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
               cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
               cudaStreamSynchronize(h->st) != cudaSuccess))
      s = fail(h, LBM_ECUDA, "diagnostics copy");
    cudaStreamSynchronize(h->st);
    cudaFree(buf);
    if (!s && herr) s = fail(h, LBM_EGEOM, "a diagnostic stencil leaves the domain");
    if (s) return s;
  }
  return LBM_OK;
}

lbm_status lbm_get_constants(const lbm_handle* h, double out[8]) {
  if (!h || !out) return LBM_EINVAL;
  out[0] = h->u_mag;
  out[1] = h->mu;
  out[2] = h->lam;
  out[3] = h->theta_inf;
  out[4] = h->Cv;
  out[5] = h->Cp;
  out[6] = h->rho_inf;
  out[7] = h->gamma;
  return LBM_OK;
}

lbm_status ib_get_sizes(const lbm_handle* h, int* n_rows, int* nnz, int* n_points) {
  if (!h) return LBM_EINVAL;
  if (n_rows) *n_rows = h->n_rows;
  if (nnz) *nnz = h->nnz;
  if (n_points) *n_points = h->NL;
  return LBM_OK;
}

lbm_status ib_get_setup(lbm_handle* h, double* phi, double* W, double* Xstar, double* dBV, uint8_t* inside,
                        int* row_ptr, int* cell_id, int* col, double* wt) {
  if (!h) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  if (!h->has_ib) return fail(h, LBM_ESTATE, "no immersed body");
  const int NL = h->NL, D = h->D;
  if (phi) CK(cudaMemcpyAsync(phi, h->phi, NL * 8, cudaMemcpyDeviceToHost, h->st));
  if (W) CK(cudaMemcpyAsync(W, h->W, NL * 8, cudaMemcpyDeviceToHost, h->st));
  if (Xstar) CK(cudaMemcpyAsync(Xstar, h->Xstar, NL * D * 8, cudaMemcpyDeviceToHost, h->st));
  if (dBV) CK(cudaMemcpyAsync(dBV, h->dBV, NL * 8, cudaMemcpyDeviceToHost, h->st));
  if (inside) CK(cudaMemcpyAsync(inside, h->inside, h->g.N, cudaMemcpyDeviceToHost, h->st));
  if (row_ptr) CK(cudaMemcpyAsync(row_ptr, h->row_ptr, (size_t)(h->n_rows + 1) * 4, cudaMemcpyDeviceToHost, h->st));
  if (cell_id) CK(cudaMemcpyAsync(cell_id, h->cell_id, (size_t)h->n_rows * 4, cudaMemcpyDeviceToHost, h->st));
  if (col) CK(cudaMemcpyAsync(col, h->col, (size_t)h->nnz * 4, cudaMemcpyDeviceToHost, h->st));
  if (wt) CK(cudaMemcpyAsync(wt, h->wt, (size_t)h->nnz * 8, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return LBM_OK;
}

lbm_status lbm_profile(lbm_handle* h, int enable, int reset) {
  if (!h) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  CK(cudaStreamSynchronize(h->st));
  if (reset) {
    for (auto& e : h->ev_used) {
      h->ev_pool.push_back(e.second.first);
      h->ev_pool.push_back(e.second.second);
    }
    h->ev_used.clear();
    for (int k = 0; k < kProfClasses; ++k) {
      h->prof_ms[k] = 0;
      h->prof_n[k] = 0;
    }
  }
  h->prof = enable != 0;
  return LBM_OK;
}

lbm_status lbm_get_profile(lbm_handle* h, double ms[5], long long launches[5]) {
  if (!h) return LBM_EINVAL;
  DeviceGuard dg(h->cfg.device);
  CK(cudaStreamSynchronize(h->st));
  for (auto& e : h->ev_used) {
    float t = 0.f;
    cudaEventElapsedTime(&t, e.second.first, e.second.second);
    h->prof_ms[e.first] += t;
    h->prof_n[e.first] += 1;
    h->ev_pool.push_back(e.second.first);
    h->ev_pool.push_back(e.second.second);
  }
  h->ev_used.clear();
  for (int k = 0; k < kProfClasses; ++k) {
    if (ms) ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->prof_n[k];
  }
  return LBM_OK;
}

long long lbm_launch_count(const lbm_handle* h) { return h ? h->launches : -1; }

}  // extern "C"
