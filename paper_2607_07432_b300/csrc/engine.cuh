// Per-configuration engine: the time step and state conversions for one
// (lattice, storage, compute) combination.  Included by one instantiation
// file per combination so that they compile in parallel.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "handle.cuh"
#include "ib.cuh"
#include "persist.cuh"
#include "physics.cuh"
#include "refine.cuh"
#include "state.cuh"
#include "step_fused.cuh"

namespace lbmib_host {

template <class L, class S, class C>
struct Engine {
  static Phys<C> phys(const lbm_handle* h) {
    Phys<C> p;
    p.cs2 = C(1.0 / 3.0);
    p.Cv = C(h->Cv);
    p.Cp = C(h->Cp);
    p.mu = C(h->mu);
    p.lam = C(h->lam);
    p.sigma = C(h->cfg.sigma_hrr);
    p.theta_tau = h->cfg.tau_mode == LBM_TAU_THETA ? 1 : 0;
    p.use_ac = h->cfg.use_ac;
    p.gcs2 = C(h->cfg.gamma * kCs2);
    p.mub2 = C(2.0 * (h->cfg.bulk_ratio * h->mu));
    return p;
  }
  static lbm_status reset_aux(lbm_handle* h) {
    lbm_handle* hh = h;
    return launch(hh, kProfOther, [&] {
      k_reset_aux<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, (const S*)h->f, (const C*)h->E, C(h->Cv),
                                                                  (C*)h->P[h->cur], (C*)h->A[h->cur]);
    });
  }
  // Planes per CTA of the 3D fused step: every chunk recomputes two
  // collision planes, and the last wave of CTAs runs partly empty, so take
  // the chunk that minimises (waves of CTAs) x (planes a CTA collides).
  static void choose_zchunk(lbm_handle* h) {
    if (L::D != 3 || h->zchunk_fixed) return;
    using Lay = FusedLayout<L, S, C, 0>;
    int sms = 0, occ = 0;
    // both index widths have the same launch shape and shared memory
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->cfg.device) != cudaSuccess ||
        cudaFuncSetAttribute(k_fused<L, S, C, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Lay::bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused<L, S, C, 0, false>, Lay::NT, Lay::bytes) !=
            cudaSuccess ||
        sms <= 0 || occ <= 0) {
      cudaGetLastError();
      return;
    }
    const long long tiles = (long long)((h->g.n[0] + Lay::TX - 1) / Lay::TX) * ((h->g.n[1] + Lay::TY - 1) / Lay::TY);
    const int nz = h->g.n[2];
    long long best = -1;
    // chunks longer than 24 planes measured slower on the 256x192x192 sphere
    // (24: 0.893, 28: 0.912, 32: 0.959 ms per step) although they need fewer
    // waves, so the search stops there
    constexpr int kMaxZChunk = 24;
    for (int zc = 4; zc <= std::max(4, std::min(nz, kMaxZChunk)); ++zc) {
      const long long ctas = tiles * ((nz + zc - 1) / zc);
      const long long waves = (ctas + (long long)sms * occ - 1) / ((long long)sms * occ);
      const long long cost = waves * (zc + 2);
      if (best < 0 || cost < best) {
        best = cost;
        h->zchunk = zc;
      }
    }
  }
  static lbm_status init(lbm_handle* h) {
    choose_zchunk(h);
    lbm_status s = launch(h, kProfOther, [&] {
      k_feq_inf<L, C><<<1, 32, 0, h->st>>>((C*)h->feq_inf, C(h->rho_inf), C(h->u_inf[0]), C(h->u_inf[1]),
                                           C(h->u_inf[2]), C(h->theta_inf));
    });
    if (s) return s;
    // storage offsets (pop_offset): the free-stream equilibrium for 16-bit
    // storage, read back before any state is stored; w_i otherwise
    if constexpr (sizeof(S) == 2) {
      C fe[L::Q];
      CK(cudaMemcpyAsync(fe, h->feq_inf, sizeof(fe), cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      for (int i = 0; i < L::Q; ++i) h->g.off[i] = float(fe[i]);
    } else {
      for (int i = 0; i < L::Q; ++i) h->g.off[i] = float(L::w(i));
    }
    // uniform free-stream start (reading Q25)
    std::vector<double> rho(h->g.N, h->rho_inf), T(h->g.N, h->theta_inf), u(h->g.N * L::D);
    for (int a = 0; a < L::D; ++a)
      for (long long n = 0; n < h->g.N; ++n) u[a * h->g.N + n] = h->u_inf[a];
    return set_fields(h, rho.data(), u.data(), T.data(), false);
  }
  static lbm_status set_fields(lbm_handle* h, const double* rho, const double* u, const double* T, bool dev) {
    const long long N = h->g.N;
    double *dr = nullptr, *du = nullptr, *dT = nullptr;
    if (!dev) {
      CK(cudaMalloc(&dr, N * 8));
      CK(cudaMalloc(&du, N * 8 * L::D));
      CK(cudaMalloc(&dT, N * 8));
      CK(cudaMemcpyAsync(dr, rho, N * 8, cudaMemcpyHostToDevice, h->st));
      CK(cudaMemcpyAsync(du, u, N * 8 * L::D, cudaMemcpyHostToDevice, h->st));
      CK(cudaMemcpyAsync(dT, T, N * 8, cudaMemcpyHostToDevice, h->st));
    }
    lbm_status s = launch(h, kProfOther, [&] {
      k_set_fields<L, S, C><<<nblk(N, 256), 256, 0, h->st>>>(h->g, (S*)h->f, (C*)h->E, dev ? rho : dr,
                                                             dev ? u : du, dev ? T : dT, C(h->Cv));
    });
    if (!s) s = reset_aux(h);
    if (!s) s = refresh_moments(h);
    if (!dev) {
      cudaStreamSynchronize(h->st);
      cudaFree(dr);
      cudaFree(du);
      cudaFree(dT);
    }
    h->sticky = LBM_OK;
    return s;
  }
  static lbm_status set_fields_api(lbm_handle* h, const double* rho, const double* u, const double* T) {
    return set_fields(h, rho, u, T, true);
  }
  static IBStepDev ib_step_dev(lbm_handle* h) {
    IBStepDev s;
    s.NL = h->NL;
    s.method = h->cfg.method;
    s.D = L::D;
    s.d_n = h->cfg.d_n;
    s.Cv = h->Cv;
    s.sten_node = h->sten_node;
    s.sten_w = h->sten_w;
    s.psten_node = h->psten_node;
    s.psten_w = h->psten_w;
    s.phi = h->phi;
    s.dBV = h->dBV;
    s.tbc = h->tbc;
    s.uB = h->uB;
    s.tB = h->tB;
    s.G = h->G;
    return s;
  }
  static BCFaces bc_faces(lbm_handle* h) {
    BCFaces bf;
    for (int face = 0; face < 6; ++face) bf.type[face] = face < 2 * L::D ? h->cfg.bc[face] : 0;
    bf.rho_inf = h->rho_inf;
    for (int a = 0; a < 3; ++a) bf.u_inf[a] = h->u_inf[a];
    bf.p_inf = h->rho_inf * h->R * h->theta_inf;
    bf.gamma = h->gamma;
    bf.R = h->R;
    bf.Cv = h->Cv;
    return bf;
  }
  static lbm_status ib_force(lbm_handle* h) {
    const IBStepDev s = ib_step_dev(h);
    lbm_status st = launch(h, kProfIBForce, [&] {
      k_ib_force<L, S, C><<<nblk(h->NL, kIBPointsPerWarp * kIBWarps), 32 * kIBWarps, 0, h->st>>>(h->g, s,
                                                                                              (const C*)h->M);
    });
    if (st) return st;
    return launch(h, kProfIBSpread, [&] {
      k_ib_spread_apply<C><<<nblk(h->n_rows, 128), 128, 0, h->st>>>(L::D, h->g.N, h->n_rows, h->row_ptr, h->col,
                                                                    h->wt, h->G, h->cell_id, h->FU, h->WQ,
                                                                    (C*)h->M);
    });
  }
  static lbm_status bc(lbm_handle* h) {
    BCFaces bf = bc_faces(h);
    int maxplane = 0;
    const int skip_x = bc_in_kernel(h) ? 1 : 0;
    for (int face = 0; face < 6; ++face) {
      if (face < 2 * L::D && bf.type[face] && !(skip_x && face < 2)) {
        FacePlane fp{face / 2, face % 2};
        maxplane = std::max(maxplane, fp.count(h->g));
      }
    }
    if (!maxplane) return LBM_OK;
    return launch(h, kProfBC, [&] {
      k_bc_all_m<L, S, C><<<dim3(nblk(maxplane, 128), 2 * L::D), 128, 0, h->st>>>(
          h->g, (S*)h->f, (C*)h->M, bf, (const C*)h->feq_inf, C(h->E_inf), skip_x);
    });
  }
  // predicted moments from the populations and rho E
  static lbm_status refresh_moments(lbm_handle* h) {
    return launch(h, kProfOther, [&] {
      k_moments<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, (const S*)h->f, (const C*)h->E, (C*)h->M);
    });
  }
  // rho E lives in the moment buffer; copy it out for readback
  static lbm_status sync_energy(lbm_handle* h) {
    CK(cudaMemcpyAsync(h->E, (const C*)h->M + (size_t)(L::D + 1) * h->g.N, h->g.N * sizeof(C),
                       cudaMemcpyDeviceToDevice, h->st));
    return LBM_OK;
  }
  static lbm_status ib_part(lbm_handle* h) { return h->has_ib ? ib_force(h) : LBM_OK; }
  static lbm_status wall_diag(lbm_handle* h, double* out, int* err) {
    DiagDev d;
    d.NL = h->NL;
    d.D = L::D;
    d.R = h->R;
    d.Cv = h->Cv;
    d.mu = h->mu;
    d.d_n = h->cfg.d_n;
    d.p_inf = h->rho_inf * h->R * h->theta_inf;
    d.q_inf = 0.5 * h->rho_inf * h->u_mag * h->u_mag;
    d.X = h->X;
    d.nrm = h->nrm;
    d.uB = h->uB;
    d.psten_node = h->psten_node;
    d.psten_w = h->psten_w;
    d.out = out;
    d.err = err;
    return launch(h, kProfOther, [&] {
      k_wall_diag<L, C><<<nblk(h->NL, 128), 128, 0, h->st>>>(h->g, d, (const C*)h->M);
    });
  }
  static lbm_status bc_part(lbm_handle* h) { return bc(h); }
  static FusedArgs<S, C> fused_args(lbm_handle* h, int parity) {
    // parity 0: the handle's current buffers; parity 1: the swapped ones
    FusedArgs<S, C> a;
    const bool sw = parity != 0;
    a.f_in = (const S*)(sw ? h->f2 : h->f);
    a.f_out = (S*)(sw ? h->f : h->f2);
    a.M_in = (const C*)(sw ? h->M2 : h->M);
    a.M_out = (C*)(sw ? h->M : h->M2);
    const int c0 = sw ? 1 - h->cur : h->cur;
    a.Pp = (const C*)h->P[c0];
    a.Pn = (C*)h->P[1 - c0];
    a.Ap = (const C*)h->A[c0];
    a.An = (C*)h->A[1 - c0];
    a.forced = h->has_ib ? h->forced : nullptr;
    a.cell_id = h->cell_id;
    a.row_of_node = h->has_ib ? h->row_of_node : nullptr;
    a.n_rows = h->n_rows;
    a.FU = h->FU;
    a.bc_fused = bc_in_kernel(h) ? 1 : 0;
    a.bct[0] = h->cfg.bc[0];
    a.bct[1] = h->cfg.bc[1];
    a.feq_inf = (const C*)h->feq_inf;
    a.E_inf = C(h->E_inf);
    return a;
  }
  // x faces inside the fused kernel: both x faces non-periodic, at least
  // four nodes along x, an x+ outlet node in the same tile as its inner
  // neighbour, and no outlet face on y or z (whose copies would read x-face
  // nodes before the kernel's equilibrium wins on the edges)
  static bool bc_in_kernel(lbm_handle* h) {
    if (!h->bc_in_kernel || h->g.n[0] < 4) return false;
    for (int f = 0; f < 2 * L::D; ++f)
      if (h->cfg.bc[f] == kBCChar) return false;
    if (h->cfg.bc[0] == LBM_BC_PERIODIC || h->cfg.bc[1] == LBM_BC_PERIODIC) return false;
    if (h->cfg.bc[1] == LBM_BC_OUTLET && (h->g.n[0] - 1) % FusedTile<L, C>::TX == 0) return false;
    for (int f = 2; f < 2 * L::D; ++f)
      if (h->cfg.bc[f] == LBM_BC_OUTLET) return false;
    return true;
  }
  template <int HY>
  static void batch_tiles(lbm_handle* h, int& tx, int& ty, int& tz) {
    using Lay = FusedLayout<L, S, C, HY>;
    tx = (h->g.n[0] + Lay::TX - 1) / Lay::TX;
    ty = (h->g.n[1] + Lay::TY - 1) / Lay::TY;
    tz = L::D == 3 ? (h->g.n[2] + h->zchunk - 1) / h->zchunk : 1;
  }
  static lbm_status batch_build(BatchPlan* b) {
    const int n = (int)b->cases.size();
    std::vector<CaseDesc<S, C>> d0(n), d1(n);
    std::vector<int> tx(n), ty(n), tz(n);
    for (int k = 0; k < n; ++k) {
      lbm_handle* h = b->cases[k];
      for (int p = 0; p < 2; ++p) {
        CaseDesc<S, C>& d = p ? d1[k] : d0[k];
        d.g = h->g;
        d.a = fused_args(h, p);
        d.ph = phys(h);
        d.zchunk = h->zchunk;
      }
      bool done = false;
      if constexpr (L::D == 2 && sizeof(C) == 4) {
        if (b->tile_rows == 16) {
          batch_tiles<16>(h, tx[k], ty[k], tz[k]);
          done = true;
        } else if (b->tile_rows == 32) {
          batch_tiles<32>(h, tx[k], ty[k], tz[k]);
          done = true;
        }
      }
      if (!done) batch_tiles<0>(h, tx[k], ty[k], tz[k]);
    }
    // work items in schedule order
    std::vector<int4> w;
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    if (b->schedule == 2)
      std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return tx[p] * ty[p] * tz[p] > tx[q] * ty[q] * tz[q]; });
    if (b->schedule == 1) {
      std::vector<int> left(n);
      size_t total = 0;
      for (int k = 0; k < n; ++k) total += (size_t)tx[k] * ty[k] * tz[k];
      std::vector<int> pos(n, 0);
      while (w.size() < total)
        for (int k = 0; k < n; ++k) {
          const int cnt = tx[k] * ty[k] * tz[k];
          if (pos[k] < cnt) {
            const int i = pos[k]++;
            w.push_back(make_int4(k, i % tx[k], (i / tx[k]) % ty[k], i / (tx[k] * ty[k])));
          }
        }
    } else {
      for (int k : order)
        for (int bz = 0; bz < tz[k]; ++bz)
          for (int by = 0; by < ty[k]; ++by)
            for (int bx = 0; bx < tx[k]; ++bx) w.push_back(make_int4(k, bx, by, bz));
    }
    if (lbm_status sa = batch_aux_build(b)) return sa;
    for (int p = 0; p < 2; ++p) {
      if (b->descs[p]) cudaFree(b->descs[p]);
      if (cudaMalloc(&b->descs[p], sizeof(CaseDesc<S, C>) * n) != cudaSuccess) return LBM_ENOMEM;
      if (cudaMemcpy(b->descs[p], p ? d1.data() : d0.data(), sizeof(CaseDesc<S, C>) * n, cudaMemcpyHostToDevice) !=
          cudaSuccess)
        return LBM_ECUDA;
    }
    if (b->work) cudaFree(b->work);
    if (cudaMalloc(&b->work, sizeof(int4) * w.size()) != cudaSuccess) return LBM_ENOMEM;
    if (cudaMemcpy(b->work, w.data(), sizeof(int4) * w.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return LBM_ECUDA;
    b->n_work = (int)w.size();
    return LBM_OK;
  }
  template <class T>
  static lbm_status upload(void*& dst, const std::vector<T>& v) {
    if (dst) cudaFree(dst);
    dst = nullptr;
    if (v.empty()) return LBM_OK;
    if (cudaMalloc(&dst, sizeof(T) * v.size()) != cudaSuccess) return LBM_ENOMEM;
    if (cudaMemcpy(dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
  }
  // descriptors and work items of the batched IB and boundary launches; the
  // pointers of parity p are those the per-case kernels would use after p
  // buffer swaps from the build-time state
  static lbm_status batch_aux_build(BatchPlan* b) {
    const int n = (int)b->cases.size();
    std::vector<IBCaseDesc<S, C>> ib[2];
    std::vector<SpreadCaseDesc<C>> sp[2];
    std::vector<BCCaseDesc<S, C>> bcd[2];
    std::vector<int2> ibw, spw;
    std::vector<int4> bcw;
    for (int k = 0; k < n; ++k) {
      lbm_handle* h = b->cases[k];
      for (int p = 0; p < 2; ++p) {
        IBCaseDesc<S, C> d;
        d.g = h->g;
        d.s = ib_step_dev(h);
        d.M = (const C*)(p ? h->M2 : h->M);
        ib[p].push_back(d);
        SpreadCaseDesc<C> q;
        q.D = L::D;
        q.N = h->g.N;
        q.n_rows = h->n_rows;
        q.row_ptr = h->row_ptr;
        q.col = h->col;
        q.wt = h->wt;
        q.G = h->G;
        q.cell_id = h->cell_id;
        q.FU = h->FU;
        q.WQ = h->WQ;
        q.M = (C*)(p ? h->M2 : h->M);
        sp[p].push_back(q);
        BCCaseDesc<S, C> c;
        c.g = h->g;
        c.f = (S*)(p ? h->f : h->f2);
        c.M = (C*)(p ? h->M : h->M2);
        c.bf = bc_faces(h);
        c.feq_inf = (const C*)h->feq_inf;
        c.E_inf = C(h->E_inf);
        c.skip_x = bc_in_kernel(h) ? 1 : 0;
        bcd[p].push_back(c);
      }
      if (h->has_ib) {
        const int nb = (int)nblk(h->NL, kIBPointsPerWarp * kIBWarps);
        for (int q = 0; q < nb; ++q) ibw.push_back(make_int2(k, q));
        const int nr = (int)nblk(h->n_rows, 128);
        for (int q = 0; q < nr; ++q) spw.push_back(make_int2(k, q));
      }
      const BCFaces bf = bc_faces(h);
      const int skip_x = bc_in_kernel(h) ? 1 : 0;
      for (int face = 0; face < 2 * L::D; ++face) {
        if (!bf.type[face] || (skip_x && face < 2)) continue;
        FacePlane fp{face / 2, face % 2};
        const int nb = (int)nblk(fp.count(h->g), 128);
        for (int q = 0; q < nb; ++q) bcw.push_back(make_int4(k, face, q, 0));
      }
    }
    lbm_status s = LBM_OK;
    for (int p = 0; p < 2 && !s; ++p) {
      s = upload(b->ib_descs[p], ib[p]);
      if (!s) s = upload(b->sp_descs[p], sp[p]);
      if (!s) s = upload(b->bc_descs[p], bcd[p]);
    }
    if (!s) s = upload(b->ib_work, ibw);
    if (!s) s = upload(b->sp_work, spw);
    if (!s) s = upload(b->bc_work, bcw);
    b->n_ib_work = (int)ibw.size();
    b->n_sp_work = (int)spw.size();
    b->n_bc_work = (int)bcw.size();
    return s;
  }
  static lbm_status batch_aux(BatchPlan* b, int parity, int part) {
    if (part == 0) {
      if (b->n_ib_work) {
        k_ib_force_batched<L, S, C><<<b->n_ib_work, 32 * kIBWarps, 0, b->st>>>(
            (const IBCaseDesc<S, C>*)b->ib_descs[parity], (const int2*)b->ib_work);
        k_spread_apply_batched<C><<<b->n_sp_work, 128, 0, b->st>>>((const SpreadCaseDesc<C>*)b->sp_descs[parity],
                                                                   (const int2*)b->sp_work);
        for (lbm_handle* h : b->cases)
          if (h->has_ib) h->launches += 2;
      }
    } else if (b->n_bc_work) {
      k_bc_batched<L, S, C><<<b->n_bc_work, 128, 0, b->st>>>((const BCCaseDesc<S, C>*)b->bc_descs[parity],
                                                            (const int4*)b->bc_work);
      for (lbm_handle* h : b->cases) h->launches++;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      b->err = std::string("batched launch: ") + cudaGetErrorString(e);
      return LBM_ECUDA;
    }
    return LBM_OK;
  }
  // the persistent form (2D): one cooperative launch of as many CTAs as are
  // resident at once runs nsteps steps; the grid size is found at plan build
  template <int HY, bool NARROW>
  static lbm_status persist_tile(BatchPlan* b, int parity, int nsteps, bool size_only) {
    if constexpr (L::D != 2) {
      return LBM_EINVAL;
    } else {
      using Lay = FusedLayout<L, S, C, HY>;
      auto kern = k_batch_persistent<L, S, C, HY, NARROW>;
      if (size_only) {
        int dev = 0, sms = 0, occ = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Lay::NT, Lay::bytes) != cudaSuccess) {
          cudaGetLastError();
          return LBM_ECUDA;
        }
        b->persist_grid = occ * sms;
        return occ > 0 ? LBM_OK : LBM_EINVAL;
      }
      PersistDesc<S, C> p;
      for (int q = 0; q < 2; ++q) {
        p.descs[q] = (const CaseDesc<S, C>*)b->descs[q];
        p.ib[q] = (const IBCaseDesc<S, C>*)b->ib_descs[q];
        p.sp[q] = (const SpreadCaseDesc<C>*)b->sp_descs[q];
        p.bc[q] = (const BCCaseDesc<S, C>*)b->bc_descs[q];
      }
      p.work = (const int4*)b->work;
      p.n_work = b->n_work;
      p.ib_work = (const int2*)b->ib_work;
      p.n_ib = b->n_ib_work;
      p.sp_work = (const int2*)b->sp_work;
      p.n_sp = b->n_sp_work;
      p.bc_work = (const int4*)b->bc_work;
      p.n_bc = b->n_bc_work;
      p.bar = (GridBarrier*)b->bar;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)b->persist_grid);
      cfg.blockDim = dim3(Lay::NT);
      cfg.dynamicSmemBytes = Lay::bytes;
      cfg.stream = b->st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, kern, p, parity, nsteps) != cudaSuccess) return LBM_ECUDA;
      return LBM_OK;
    }
  }
  template <bool NARROW>
  static lbm_status persist_rows(BatchPlan* b, int parity, int nsteps, bool size_only) {
    if constexpr (L::D == 2 && sizeof(C) == 4) {
      if (b->tile_rows == 16) return persist_tile<16, NARROW>(b, parity, nsteps, size_only);
      if (b->tile_rows == 32) return persist_tile<32, NARROW>(b, parity, nsteps, size_only);
    }
    return persist_tile<0, NARROW>(b, parity, nsteps, size_only);
  }
  // nsteps >= 1: launch; nsteps == 0: size the grid of the plan's tile
  static lbm_status batch_persistent(BatchPlan* b, int parity, int nsteps) {
    if (L::D != 2 || !b->bar) return LBM_EINVAL;
    bool narrow = true;
    for (lbm_handle* h : b->cases) narrow = narrow && narrow_index<L>(h->g.N);
    const bool size_only = nsteps == 0;
    if (!size_only && b->persist_grid <= 0) return LBM_EINVAL;
    lbm_status s = narrow ? persist_rows<true>(b, parity, nsteps, size_only)
                          : persist_rows<false>(b, parity, nsteps, size_only);
    if (s) {
      cudaError_t e = cudaGetLastError();
      b->err = std::string("persistent batched launch: ") + cudaGetErrorString(e);
      return s;
    }
    if (!size_only)
      for (lbm_handle* h : b->cases) h->launches++;
    return LBM_OK;
  }
  template <int HY>
  static void batch_launch(BatchPlan* b, int parity) {
    using Lay = FusedLayout<L, S, C, HY>;
    bool narrow = true;
    for (lbm_handle* h : b->cases) narrow = narrow && narrow_index<L>(h->g.N);
    if (narrow) {
      smem_attr_once<k_fused_batched<L, S, C, HY, true>>((int)Lay::bytes);
      k_fused_batched<L, S, C, HY, true><<<b->n_work, Lay::NT, Lay::bytes, b->st>>>(
          (const CaseDesc<S, C>*)b->descs[parity], (const int4*)b->work);
    } else {
      smem_attr_once<k_fused_batched<L, S, C, HY, false>>((int)Lay::bytes);
      k_fused_batched<L, S, C, HY, false><<<b->n_work, Lay::NT, Lay::bytes, b->st>>>(
          (const CaseDesc<S, C>*)b->descs[parity], (const int4*)b->work);
    }
  }
  static lbm_status batch_fused(BatchPlan* b, int parity) {
    bool done = false;
    if constexpr (L::D == 2 && sizeof(C) == 4) {
      if (b->tile_rows == 16) {
        batch_launch<16>(b, parity);
        done = true;
      } else if (b->tile_rows == 32) {
        batch_launch<32>(b, parity);
        done = true;
      }
    }
    if (!done) batch_launch<0>(b, parity);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      b->err = std::string("batched launch: ") + cudaGetErrorString(e);
      return LBM_ECUDA;
    }
    for (lbm_handle* h : b->cases) h->launches++;
    return LBM_OK;
  }
  static lbm_status step(lbm_handle* h) {
    lbm_status s;
    if (h->has_ib && (s = ib_force(h))) return s;
    if ((s = fused_step(h, phys(h)))) return s;
    if ((s = bc(h))) return s;
    h->cur = 1 - h->cur;
    return LBM_OK;
  }
  static lbm_status fused_step(lbm_handle* h, const Phys<C>& ph);
  static lbm_status fields(lbm_handle* h, double* rho, double* u, double* T, double* p) {
    if (lbm_status s0 = sync_energy(h)) return s0;
    return launch(h, kProfOther, [&] {
      k_fields<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, (const S*)h->f, (const C*)h->E, C(h->Cv),
                                                              C(h->R), rho, u, T, p);
    });
  }
  static lbm_status get_state(lbm_handle* h, double* f, double* E) {
    if (lbm_status s0 = sync_energy(h)) return s0;
    return launch(h, kProfOther, [&] {
      k_get_state<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, (const S*)h->f, (const C*)h->E, f, E);
    });
  }
  static lbm_status set_state(lbm_handle* h, const double* f, const double* E) {
    lbm_status s = launch(h, kProfOther, [&] {
      k_set_state<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, (S*)h->f, (C*)h->E, f, E);
    });
    if (s) return s;
    h->sticky = LBM_OK;
    s = reset_aux(h);
    if (!s) s = refresh_moments(h);
    return s;
  }
  static lbm_status health(lbm_handle* h, unsigned long long* bad) {
    if (lbm_status s0 = sync_energy(h)) return s0;
    return launch(h, kProfOther, [&] {
      k_health<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, (const S*)h->f, (const C*)h->E, C(h->Cv),
                                                              bad);
    });
  }
  // two-level refinement transfers (kernels in refine.cuh)
  // out: the ghost state (Q + 1 values per ghost node) followed by the
  // shell scratch (Q + D + 2 values per shell node)
  static lbm_status refine_ghost_state(lbm_handle* h0, const RefineDev& r, void* out) {
    C* g = (C*)out;
    C* B = g + (size_t)(L::Q + 1) * r.n_ghost;
    lbm_status s = launch(h0, kProfOther, [&] {
      k_refine_shell<L, S, C><<<nblk(r.n_shell, 128), 128, 0, h0->st>>>(r, (const S*)h0->f, (const C*)h0->M, B);
    });
    if (s) return s;
    return launch(h0, kProfOther, [&] {
      k_refine_ghost_state<L, S, C><<<nblk(r.n_ghost, 128), 128, 0, h0->st>>>(r, B, g);
    });
  }
  // level 0 has stepped to n+1: its P / A [cur] hold time n, [1 - cur] time
  // n-1; level 1's [cur] buffers are the previous-step values its next
  // step reads
  static lbm_status refine_fill(lbm_handle* h0, lbm_handle* h1, const RefineDev& r, const void* Ga,
                                const void* Gb) {
    return launch(h1, kProfOther, [&] {
      k_refine_fill<L, S, C><<<nblk(r.n_ghost, 128), 128, 0, h1->st>>>(
          r, (S*)h1->f, (C*)h1->M, (C*)h1->P[h1->cur], (C*)h1->A[h1->cur], (const C*)Ga, (const C*)Gb,
          (const C*)h0->P[1 - h0->cur], (const C*)h0->P[h0->cur], (const C*)h0->A[1 - h0->cur],
          (const C*)h0->A[h0->cur]);
    });
  }
  // after level 1's second step its [1 - cur] buffers hold level-1 time n
  static lbm_status refine_restrict(lbm_handle* h0, lbm_handle* h1, const RefineDev& r) {
    const long long nr = (long long)r.rn[0] * r.rn[1] * (L::D == 3 ? r.rn[2] : 1);
    return launch(h0, kProfOther, [&] {
      k_refine_restrict<L, S, C><<<nblk(nr, 128), 128, 0, h0->st>>>(
          r, (S*)h0->f, (C*)h0->M, (C*)h0->P[h0->cur], (C*)h0->A[h0->cur], (const S*)h1->f, (const C*)h1->M,
          (const C*)h1->P[1 - h1->cur], (const C*)h1->A[1 - h1->cur]);
    });
  }
  static const Ops* ops() {
    static const Ops o = {&init,        &step,        &fields,    &get_state, &set_state,
                          &set_fields_api, &health, &batch_build, &batch_fused, &batch_aux,
                          &batch_persistent, &ib_part,     &bc_part,     &wall_diag, &refine_ghost_state, &refine_fill,
                          &refine_restrict};
    return &o;
  }
};

template <class L, class S, class C>
inline lbm_status Engine<L, S, C>::fused_step(lbm_handle* h, const Phys<C>& ph) {
  const FusedArgs<S, C> a = fused_args(h, 0);
  lbm_status s = launch(h, kProfStep, [&] { launch_fused<L, S, C>(h->g, a, ph, h->st, h->zchunk, 0); });
  if (s) return s;
  std::swap(h->f, h->f2);
  std::swap(h->M, h->M2);
  return LBM_OK;
}

}  // namespace lbmib_host
