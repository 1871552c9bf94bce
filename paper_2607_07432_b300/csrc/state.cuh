// State conversions of one case: free-stream equilibrium (Eq. feq at the
// far-field state), equilibrium initialisation from given fields (uniform
// start, reading Q25, and warm starts), macroscopic fields and raw state for
// readback, previous-step auxiliaries of a fresh start, and the health check.
#pragma once
#include "grid.cuh"
#include "physics.cuh"

namespace lbmib {

// one face plane of the domain (axis, side) and its node count
struct FacePlane {
  int axis, side;
  __host__ __device__ int count(const Grid& g) const {
    const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
    return g.n[a1] * g.n[a2];
  }
};

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
    store_pop<L, S, C>(f, i, g.N, n, feq_i<L, C, i>(r, uu, th), g.off);
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
    const C v = load_pop<L, S, C>(f, i, g.N, n, g.off);
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
  for (int i = 0; i < L::Q; ++i) fo[(long long)i * g.N + n] = double(load_pop<L, S, C>(f, i, g.N, n, g.off));
  Eo[n] = double(E[n]);
}

template <class L, class S, class C>
__global__ void k_set_state(Grid g, S* f, C* E, const double* fi, const double* Ei) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) store_pop<L, S, C>(f, i, g.N, n, C(fi[(long long)i * g.N + n]), g.off);
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
    const C v = load_pop<L, S, C>(f, i, g.N, n, g.off);
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
    const C v = load_pop<L, S, C>(f, i, g.N, n, g.off);
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
