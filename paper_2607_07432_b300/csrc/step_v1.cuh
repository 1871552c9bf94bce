// Unfused global-memory form of the time step: one kernel each for the
// corrected macroscopic fields, the collision and the pull-stream + energy
// update, then the domain boundaries.  It is the reference form of the
// CUDA path (every intermediate lives in HBM) and the one used for FP64.
#pragma once
#include "grid.cuh"
#include "physics.cuh"

namespace lbmib {

template <class S, class C>
struct StepBufs {
  S* f;          // Q*N post-stream populations (storage format)
  C* fcol;       // Q*N post-collision populations
  C* M;          // (D+3)*N corrected macros: rho, u_0..u_{D-1}, theta, rhoE'
  C* E;          // N: rho E (state, before this step's IB energy forcing)
  const C* Pp;   // N: rho(1-theta) of the previous step
  C* Pn;         // N: rho(1-theta) of this step
  const C* Ap;   // NDEV*N: deviator of a^F of the previous step
  C* An;         // NDEV*N: deviator of a^F of this step
  const int* row_of_node;  // N: CSR row of a forced node, -1 otherwise
  const double* FU;        // n_rows*D: spread momentum forcing f_u
  const double* WQ;        // n_rows: spread energy forcing w + q
};

template <class C, int D>
__device__ __forceinline__ Macro<C> load_macro(const C* M, long long N, long long n) {
  Macro<C> m;
  m.rho = M[n];
#pragma unroll
  for (int a = 0; a < 3; ++a) m.u[a] = a < D ? M[(1 + a) * N + n] : C(0);
  m.th = M[(1 + D) * N + n];
  m.E = M[(2 + D) * N + n];
  return m;
}

// Sec. 2.2: rho = sum f-bar, rho u = sum c f-bar + f_u/2; rho E' = rho E +
// w + q (Q15); T = (E'/rho - |u|^2/2)/C_v, theta = T / T_ref.
template <class L, class S, class C>
__global__ void __launch_bounds__(256) k_macro(Grid g, StepBufs<S, C> b, Phys<C> ph) {
  constexpr int D = L::D;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  C rho = C(0), j[3] = {C(0), C(0), C(0)};
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const C v = load_pop<L, S, C>(b.f, i, g.N, n);
    rho += v;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (L::c(i, a) != 0) j[a] += C(L::c(i, a)) * v;
  }
  C fu[3] = {C(0), C(0), C(0)};
  C wq = C(0);
  const int r = b.row_of_node ? b.row_of_node[n] : -1;
  if (r >= 0) {
#pragma unroll
    for (int a = 0; a < D; ++a) fu[a] = C(b.FU[(long long)r * D + a]);
    wq = C(b.WQ[r]);
  }
  C u[3];
  C uu = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    u[a] = (j[a] + C(0.5) * fu[a]) / rho;
    uu += u[a] * u[a];
  }
  const C E = b.E[n] + wq;
  const C th = (E / rho - C(0.5) * uu) / ph.Cv;
  b.M[n] = rho;
#pragma unroll
  for (int a = 0; a < D; ++a) b.M[(1 + a) * g.N + n] = u[a];
  b.M[(1 + D) * g.N + n] = th;
  b.M[(2 + D) * g.N + n] = E;
}

template <class L, class S, class C>
__global__ void __launch_bounds__(256) k_collide(Grid g, StepBufs<S, C> b, Phys<C> ph) {
  constexpr int D = L::D;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const int x = int(n % g.n[0]);
  const int y = int((n / g.n[0]) % g.n[1]);
  const int z = int(n / ((long long)g.n[0] * g.n[1]));
  auto MA = [&](int dx, int dy, int dz) { return load_macro<C, D>(b.M, g.N, g.nb(x, y, z, dx, dy, dz)); };
  C du[3][3], aC[3][3];
  gradients<L, C>(MA, du, aC, ph.use_ac);
  const Macro<C> m = load_macro<C, D>(b.M, g.N, n);
  C fbar[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) fbar[i] = load_pop<L, S, C>(b.f, i, g.N, n);
  C fu[3] = {C(0), C(0), C(0)};
  const int r = b.row_of_node ? b.row_of_node[n] : -1;
  if (r >= 0) {
#pragma unroll
    for (int a = 0; a < D; ++a) fu[a] = C(b.FU[(long long)r * D + a]);
  }
  C dAFp[L::NDEV];
#pragma unroll
  for (int k = 0; k < L::NDEV; ++k) dAFp[k] = b.Ap[k * g.N + n];
  C fcol[L::Q], Pn, dAFn[L::NDEV];
  collide<L, C>(fbar, m, du, aC, b.Pp[n], dAFp, fu, ph, fcol, Pn, dAFn);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) b.fcol[(long long)i * g.N + n] = fcol[i];
  b.Pn[n] = Pn;
#pragma unroll
  for (int k = 0; k < L::NDEV; ++k) b.An[k * g.N + n] = dAFn[k];
}

template <class L, class C, int AX>
__device__ __forceinline__ C face_flux_global(const Grid& g, const C* M, const C* fcol, int x, int y, int z,
                                              const Phys<C>& ph) {
  constexpr int D = L::D;
  auto MA = [&](int k) {
    return load_macro<C, D>(M, g.N, g.nb(x, y, z, AX == 0 ? k : 0, AX == 1 ? k : 0, AX == 2 ? k : 0));
  };
  auto FC = [&](int i, int dx, int dy, int dz) { return fcol[(long long)i * g.N + g.nb(x, y, z, dx, dy, dz)]; };
  return energy_face_flux<L, C, AX>(MA, FC, ph);
}

// Eq. LB pull streaming and Eq. energy update of rho E.
template <class L, class S, class C>
__global__ void __launch_bounds__(256) k_stream_energy(Grid g, StepBufs<S, C> b, Phys<C> ph) {
  constexpr int D = L::D;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const int x = int(n % g.n[0]);
  const int y = int((n / g.n[0]) % g.n[1]);
  const int z = int(n / ((long long)g.n[0] * g.n[1]));
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const C v = b.fcol[(long long)i * g.N + g.nb(x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2))];
    store_pop<L, S, C>(b.f, i, g.N, n, v);
  }
  C E = b.M[(2 + D) * g.N + n];
  {
    const C Fp = face_flux_global<L, C, 0>(g, b.M, b.fcol, x, y, z, ph);
    const C Fm = face_flux_global<L, C, 0>(g, b.M, b.fcol, g.wrap(0, x - 1), y, z, ph);
    E = E - (Fp - Fm);
  }
  {
    const C Fp = face_flux_global<L, C, 1>(g, b.M, b.fcol, x, y, z, ph);
    const C Fm = face_flux_global<L, C, 1>(g, b.M, b.fcol, x, g.wrap(1, y - 1), z, ph);
    E = E - (Fp - Fm);
  }
  if (D == 3) {
    const C Fp = face_flux_global<L, C, 2>(g, b.M, b.fcol, x, y, z, ph);
    const C Fm = face_flux_global<L, C, 2>(g, b.M, b.fcol, x, y, g.wrap(2, z - 1), ph);
    E = E - (Fp - Fm);
  }
  b.E[n] = E;
}

// ---------------------------------------------------------------------------
// domain boundaries (reading Q24): outlet faces copy the inner neighbour
// plane, then inlet / far-field faces take the free-stream equilibrium.
// ---------------------------------------------------------------------------
struct FacePlane {
  int axis, side;
  __host__ __device__ int count(const Grid& g) const {
    const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
    return g.n[a1] * g.n[a2];
  }
};

template <class L, class S, class C>
__global__ void k_bc_outlet(Grid g, S* f, C* E, FacePlane fp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int a1 = fp.axis == 0 ? 1 : 0, a2 = fp.axis == 2 ? 1 : 2;
  if (t >= g.n[a1] * g.n[a2]) return;
  int c[3];
  c[a1] = t % g.n[a1];
  c[a2] = t / g.n[a1];
  const int nax = g.n[fp.axis];
  c[fp.axis] = fp.side ? nax - 1 : 0;
  const long long dst = g.lin(c[0], c[1], c[2]);
  c[fp.axis] = fp.side ? nax - 2 : 1;
  const long long src = g.lin(c[0], c[1], c[2]);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) f[(long long)i * g.N + dst] = f[(long long)i * g.N + src];
  E[dst] = E[src];
}

template <class L, class S, class C>
__global__ void k_bc_equilibrium(Grid g, S* f, C* E, FacePlane fp, const C* feq_inf, C E_inf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int a1 = fp.axis == 0 ? 1 : 0, a2 = fp.axis == 2 ? 1 : 2;
  if (t >= g.n[a1] * g.n[a2]) return;
  int c[3];
  c[a1] = t % g.n[a1];
  c[a2] = t / g.n[a1];
  c[fp.axis] = fp.side ? g.n[fp.axis] - 1 : 0;
  const long long dst = g.lin(c[0], c[1], c[2]);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) store_pop<L, S, C>(f, i, g.N, dst, feq_inf[i]);
  E[dst] = E_inf;
}

// free-stream equilibrium populations (Eq. feq at rho_inf, u_inf, theta_inf)
template <class L, class C>
__global__ void k_feq_inf(C* out, C rho, C ux, C uy, C uz, C th) {
  const int i = threadIdx.x;
  if (i >= L::Q) return;
  const C u[3] = {ux, uy, uz};
  sfor<0, L::Q>([&](auto K) {
    constexpr int k = decltype(K)::value;
    if (k == i) out[k] = feq_i<L, C, k>(rho, u, th);
  });
}

// set every node to the equilibrium of (rho, u, T) fields given in FP64
template <class L, class S, class C>
__global__ void k_set_fields(Grid g, S* f, C* E, const double* rho, const double* u, const double* T, C Cv) {
  constexpr int D = L::D;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const C r = C(rho[n]);
  C uu[3] = {C(0), C(0), C(0)};
  C k = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    uu[a] = C(u[a * g.N + n]);
    k += uu[a] * uu[a];
  }
  const C th = C(T[n]);
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    store_pop<L, S, C>(f, i, g.N, n, feq_i<L, C, i>(r, uu, th));
  });
  E[n] = r * (C(0.5) * k + Cv * th);
}

template <class L, class S, class C>
__global__ void k_fields(Grid g, const S* f, const C* E, C Cv, C R, double* rho, double* u, double* T,
                         double* p) {
  constexpr int D = L::D;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  C r = C(0), j[3] = {C(0), C(0), C(0)};
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const C v = load_pop<L, S, C>(f, i, g.N, n);
    r += v;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (L::c(i, a) != 0) j[a] += C(L::c(i, a)) * v;
  }
  C uu = C(0), uv[3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    uv[a] = j[a] / r;
    uu += uv[a] * uv[a];
  }
  const C Tn = (E[n] / r - C(0.5) * uu) / Cv;
  if (rho) rho[n] = double(r);
  if (u)
#pragma unroll
    for (int a = 0; a < D; ++a) u[a * g.N + n] = double(uv[a]);
  if (T) T[n] = double(Tn);
  if (p) p[n] = double(r * R * Tn);
}

template <class L, class S, class C>
__global__ void k_get_state(Grid g, const S* f, const C* E, double* fo, double* Eo) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) fo[(long long)i * g.N + n] = double(load_pop<L, S, C>(f, i, g.N, n));
  Eo[n] = double(E[n]);
}

template <class L, class S, class C>
__global__ void k_set_state(Grid g, S* f, C* E, const double* fi, const double* Ei) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) store_pop<L, S, C>(f, i, g.N, n, C(fi[(long long)i * g.N + n]));
  E[n] = C(Ei[n]);
}

// previous-step auxiliaries for a fresh start: rho(1-theta) of the state,
// zero deviator of a^F
template <class L, class S, class C>
__global__ void k_reset_aux(Grid g, const S* f, const C* E, C Cv, C* Pp, C* Ap) {
  constexpr int D = L::D;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  C r = C(0), j[3] = {C(0), C(0), C(0)};
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const C v = load_pop<L, S, C>(f, i, g.N, n);
    r += v;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (L::c(i, a) != 0) j[a] += C(L::c(i, a)) * v;
  }
  C uu = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) uu += (j[a] / r) * (j[a] / r);
  const C th = (E[n] / r - C(0.5) * uu) / Cv;
  Pp[n] = r * (C(1) - th);
#pragma unroll
  for (int k = 0; k < L::NDEV; ++k) Ap[k * g.N + n] = C(0);
}

// health check: count nodes whose density or temperature is not finite
// and positive
template <class L, class S, class C>
__global__ void k_health(Grid g, const S* f, const C* E, C Cv, unsigned long long* bad) {
  constexpr int D = L::D;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  C r = C(0), j[3] = {C(0), C(0), C(0)};
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const C v = load_pop<L, S, C>(f, i, g.N, n);
    r += v;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (L::c(i, a) != 0) j[a] += C(L::c(i, a)) * v;
  }
  C uu = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) uu += (j[a] / r) * (j[a] / r);
  const C th = (E[n] / r - C(0.5) * uu) / Cv;
  const bool ok = (r > C(0)) && (th > C(0)) && isfinite(double(r)) && isfinite(double(th));
  if (!ok) atomicAdd(bad, 1ull);
}

}  // namespace lbmib
