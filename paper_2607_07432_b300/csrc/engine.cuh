// Per-configuration engine: the time step and state conversions for one
// (lattice, storage, compute) combination.  Included by one instantiation
// file per combination so that they compile in parallel.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "handle.cuh"
#include "ib.cuh"
#include "physics.cuh"
#include "step_fused.cuh"
#include "step_v1.cuh"

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
    return p;
  }
  static StepBufs<S, C> bufs(lbm_handle* h) {
    StepBufs<S, C> b;
    b.f = (S*)h->f;
    b.fcol = (C*)h->fcol;
    b.M = (C*)h->M;
    b.E = (C*)h->E;
    b.Pp = (const C*)h->P[h->cur];
    b.Pn = (C*)h->P[1 - h->cur];
    b.Ap = (const C*)h->A[h->cur];
    b.An = (C*)h->A[1 - h->cur];
    b.row_of_node = h->has_ib ? h->row_of_node : nullptr;
    b.FU = h->FU;
    b.WQ = h->WQ;
    return b;
  }
  static lbm_status reset_aux(lbm_handle* h) {
    lbm_handle* hh = h;
    return launch(hh, kProfOther, [&] {
      k_reset_aux<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, (const S*)h->f, (const C*)h->E, C(h->Cv),
                                                                  (C*)h->P[h->cur], (C*)h->A[h->cur]);
    });
  }
  static lbm_status init(lbm_handle* h) {
    lbm_status s = launch(h, kProfOther, [&] {
      k_feq_inf<L, C><<<1, 32, 0, h->st>>>((C*)h->feq_inf, C(h->rho_inf), C(h->u_inf[0]), C(h->u_inf[1]),
                                           C(h->u_inf[2]), C(h->theta_inf));
    });
    if (s) return s;
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
  static lbm_status ib_force(lbm_handle* h) {
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
    lbm_status st = launch(h, kProfIBForce, [&] {
      k_ib_force<L, S, C><<<nblk((long long)h->NL * 32, 128), 128, 0, h->st>>>(
          h->g, s, (const S*)h->f, (const C*)h->E, h->use_fused ? (const C*)h->M : nullptr);
    });
    if (st) return st;
    st = launch(h, kProfIBSpread, [&] {
      k_ib_spread<<<nblk(h->n_rows, 128), 128, 0, h->st>>>(L::D, h->n_rows, h->row_ptr, h->col, h->wt, h->G,
                                                          h->FU, h->WQ);
    });
    if (st || !h->use_fused) return st;
    return launch(h, kProfIBSpread, [&] {
      k_apply_forcing<C><<<nblk(h->n_rows, 128), 128, 0, h->st>>>(L::D, h->g.N, h->n_rows, h->cell_id, h->FU,
                                                                  h->WQ, (C*)h->M);
    });
  }
  static lbm_status bc(lbm_handle* h) {
    if (h->use_fused) return bc_fused(h);
    for (int face = 0; face < 2 * L::D; ++face) {
      if (h->cfg.bc[face] != LBM_BC_OUTLET) continue;
      FacePlane fp{face / 2, face % 2};
      lbm_status s = launch(h, kProfBC, [&] {
        k_bc_outlet<L, S, C><<<nblk(fp.count(h->g), 128), 128, 0, h->st>>>(h->g, (S*)h->f, (C*)h->E, fp);
      });
      if (s) return s;
    }
    for (int face = 0; face < 2 * L::D; ++face) {
      const int t = h->cfg.bc[face];
      if (t != LBM_BC_INLET && t != LBM_BC_FARFIELD) continue;
      FacePlane fp{face / 2, face % 2};
      lbm_status s = launch(h, kProfBC, [&] {
        k_bc_equilibrium<L, S, C><<<nblk(fp.count(h->g), 128), 128, 0, h->st>>>(
            h->g, (S*)h->f, (C*)h->E, fp, (const C*)h->feq_inf, C(h->E_inf));
      });
      if (s) return s;
    }
    return LBM_OK;
  }
  static lbm_status bc_fused(lbm_handle* h) {
    BCFaces bf;
    int maxplane = 0;
    for (int face = 0; face < 6; ++face) {
      bf.type[face] = face < 2 * L::D ? h->cfg.bc[face] : 0;
      if (face < 2 * L::D && bf.type[face]) {
        FacePlane fp{face / 2, face % 2};
        maxplane = std::max(maxplane, fp.count(h->g));
      }
    }
    if (!maxplane) return LBM_OK;
    return launch(h, kProfBC, [&] {
      k_bc_all_m<L, S, C><<<dim3(nblk(maxplane, 128), 2 * L::D), 128, 0, h->st>>>(
          h->g, (S*)h->f, (C*)h->M, bf, (const C*)h->feq_inf, C(h->E_inf));
    });
  }
  // fused form: predicted moments from the populations and rho E
  static lbm_status refresh_moments(lbm_handle* h) {
    if (!h->use_fused) return LBM_OK;
    return launch(h, kProfOther, [&] {
      k_moments<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, (const S*)h->f, (const C*)h->E, (C*)h->M);
    });
  }
  // fused form: rho E lives in the moment buffer; copy it out for readback
  static lbm_status sync_energy(lbm_handle* h) {
    if (!h->use_fused) return LBM_OK;
    CK(cudaMemcpyAsync(h->E, (const C*)h->M + (size_t)(L::D + 1) * h->g.N, h->g.N * sizeof(C),
                       cudaMemcpyDeviceToDevice, h->st));
    return LBM_OK;
  }
  static lbm_status step(lbm_handle* h) {
    lbm_status s;
    if (h->has_ib && (s = ib_force(h))) return s;
    const Phys<C> ph = phys(h);
    if (h->use_fused) {
      s = fused_step(h, ph);
    } else {
      StepBufs<S, C> b = bufs(h);
      if ((s = launch(h, kProfOther, [&] { k_macro<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, b, ph); })))
        return s;
      if ((s = launch(h, kProfStep, [&] { k_collide<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, b, ph); })))
        return s;
      s = launch(h, kProfStep,
                 [&] { k_stream_energy<L, S, C><<<nblk(h->g.N, 256), 256, 0, h->st>>>(h->g, b, ph); });
    }
    if (s) return s;
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
  static const Ops* ops() {
    static const Ops o = {&init, &step, &fields, &get_state, &set_state, &set_fields_api, &health};
    return &o;
  }
};

template <class L, class S, class C>
inline lbm_status Engine<L, S, C>::fused_step(lbm_handle* h, const Phys<C>& ph) {
  FusedArgs<S, C> a;
  a.f_in = (const S*)h->f;
  a.f_out = (S*)h->f2;
  a.M_in = (const C*)h->M;
  a.M_out = (C*)h->M2;
  a.Pp = (const C*)h->P[h->cur];
  a.Pn = (C*)h->P[1 - h->cur];
  a.Ap = (const C*)h->A[h->cur];
  a.An = (C*)h->A[1 - h->cur];
  a.forced = h->has_ib ? h->forced : nullptr;
  a.cell_id = h->cell_id;
  a.n_rows = h->n_rows;
  a.FU = h->FU;
  lbm_status s = launch(h, kProfStep, [&] { launch_fused<L, S, C>(h->g, a, ph, h->st, h->zchunk, h->tile_rows); });
  if (s) return s;
  std::swap(h->f, h->f2);
  std::swap(h->M, h->M2);
  return LBM_OK;
}

}  // namespace lbmib_host
