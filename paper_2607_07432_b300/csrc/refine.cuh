// Two-level static refinement: the transfers between a level-0 case and the
// level-1 case of a box refined by 2 (the locally refined meshes of the
// paper's Secs. 3.2-3.9, which give no algorithm; the reading taken here):
//
//   * level-1 node k along an axis sits at level-0 coordinate lo + (k - G)/2;
//     level 1 has G ghost nodes beyond the box on every side and steps twice
//     per level-0 step (acoustic scaling: same lattice velocities and
//     theta, twice the lattice viscosity and conductivity);
//   * ghost nodes take the nested mean (along x, then y, then z) of the
//     level-0 nodes around them of the predicted moments and of
//     f-bar_i - f^eq_i, and are rebuilt as f^eq + s01 (f-bar - f^eq),
//     s01 = tau-bar_1 / (2 tau-bar_0); the first level-1 step takes level 0
//     at n, the second the mean of level 0 at n and n+1; the previous-step
//     rho(1-theta) and a^F deviator (halved) come from level 0's;
//   * level-0 nodes R nodes or more inside the box take the coinciding
//     level-1 node's state: f^eq + s10 (f-bar - f^eq), s10 = 2 tau-bar_0 /
//     tau-bar_1, rho E, and its previous-step values (deviator doubled).
#pragma once
#include "grid.cuh"
#include "physics.cuh"

namespace lbmib {

__device__ __forceinline__ int floor_half(int v) { return (v - (v & 1)) / 2; }

// nested mean over the level-0 nodes around a ghost node: val(sx, sy, sz)
// is the level-0 value at base + (sx, sy, sz)
template <int D, class C, class F>
__device__ __forceinline__ C refine_mean(const int odd[3], const F& val) {
  auto ax = [&](int sy, int sz) {
    const C v0 = val(0, sy, sz);
    return odd[0] ? C(0.5) * (v0 + val(1, sy, sz)) : v0;
  };
  auto ay = [&](int sz) {
    const C v0 = ax(0, sz);
    return odd[1] ? C(0.5) * (v0 + ax(1, sz)) : v0;
  };
  if constexpr (D == 2) {
    return ay(0);
  } else {
    const C v0 = ay(0);
    return odd[2] ? C(0.5) * (v0 + ay(1)) : v0;
  }
}

// rho, u, theta of the predicted moments at a node (as the oracle's
// predicted(): u = j / rho, theta = (E / rho - |u|^2 / 2) / C_v)
template <int D, class C>
__device__ __forceinline__ void refine_macros(const C* M, long long N, long long n, C Cv, C& rho, C* u, C& th) {
  rho = M[n];
  C uu = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    u[a] = M[(1 + a) * N + n] / rho;
    uu = uu + u[a] * u[a];
  }
  th = (M[(1 + D) * N + n] / rho - C(0.5) * uu) / Cv;
}

template <class C>
__device__ __forceinline__ C refine_tau_bar(double mu, C rho) {
  return C(mu) / (rho * C(kCs2) * C(1)) + C(0.5);
}

// per level-0 node the ghost nodes read: out[i * n_shell + s] = f-bar_i -
// f^eq_i (i < Q), then rho, rho u, rho E (the predicted moments)
template <class L, class S, class C>
__global__ void k_refine_shell(RefineDev r, const S* f0, const C* M0, C* out) {
  constexpr int D = L::D, Q = L::Q;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= r.n_shell) return;
  const long long N0 = r.g0.N, n = r.shell[s], ns = r.n_shell;
  C rho, u[3] = {C(0), C(0), C(0)}, th;
  refine_macros<D, C>(M0, N0, n, C(r.Cv), rho, u, th);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    out[i * ns + s] = load_pop<L, S, C>(f0, i, N0, n, r.g0.off) - feq_i<L, C, i>(rho, u, th);
  });
#pragma unroll
  for (int q = 0; q < D + 2; ++q) out[(Q + q) * ns + s] = M0[q * N0 + n];
}

// ghost state from the shell values: out[i * n_ghost + k] = f-bar_i
// (i < Q), out[Q * n_ghost + k] = rho E
template <class L, class S, class C>
__global__ void k_refine_ghost_state(RefineDev r, const C* B, C* out) {
  constexpr int D = L::D, Q = L::Q;
  constexpr int NC = D == 3 ? 8 : 4;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= r.n_ghost) return;
  const int4 q = r.ghost[k];
  const int kk[3] = {q.x, q.y, q.z};
  int odd[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a) odd[a] = (kk[a] - r.G) & 1;
  int cs[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) cs[c] = r.corners[(long long)k * NC + c];
  const long long ns = r.n_shell;
  auto mean_of = [&](int comp) {
    return refine_mean<D, C>(odd, [&](int sx, int sy, int sz) { return B[comp * ns + cs[sx + 2 * sy + 4 * sz]]; });
  };
  const C rho = mean_of(Q);
  C j[3] = {C(0), C(0), C(0)};
#pragma unroll
  for (int a = 0; a < D; ++a) j[a] = mean_of(Q + 1 + a);
  const C E = mean_of(Q + 1 + D);
  C u[3] = {C(0), C(0), C(0)}, uu = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    u[a] = j[a] / rho;
    uu = uu + u[a] * u[a];
  }
  const C th = (E / rho - C(0.5) * uu) / C(r.Cv);
  const C s01 = refine_tau_bar<C>(r.mu1, rho) / (C(2) * refine_tau_bar<C>(r.mu0, rho));
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    out[(long long)i * r.n_ghost + k] = feq_i<L, C, i>(rho, u, th) + s01 * mean_of(i);
  });
  out[(long long)Q * r.n_ghost + k] = E;
}

// write a ghost state into level 1: Ga alone (mode 1, the first level-1
// step) or the mean of Ga and Gb (mode 2); the previous-step rho(1-theta)
// and a^F deviator from level 0's buffers (old: level-0 time n-1, new: n)
template <class L, class S, class C>
__global__ void k_refine_fill(RefineDev r, S* f1, C* M1, C* P1, C* A1, const C* Ga, const C* Gb,
                              const C* P0_old, const C* P0_new, const C* A0_old, const C* A0_new) {
  constexpr int D = L::D, Q = L::Q;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= r.n_ghost) return;
  const int4 q = r.ghost[k];
  const int kk[3] = {q.x, q.y, q.z};
  int base[3] = {0, 0, 0}, odd[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int v = kk[a] - r.G;
    odd[a] = v & 1;
    base[a] = r.lo[a] + floor_half(v);
  }
  const long long N0 = r.g0.N, N1 = r.g1.N;
  const long long n1 = r.g1.lin(kk[0], kk[1], D == 3 ? kk[2] : 0);
  auto node = [&](int sx, int sy, int sz) {
    return r.g0.lin(base[0] + sx, base[1] + sy, D == 3 ? base[2] + sz : 0);
  };
  const bool second = Gb != nullptr;
  C rho = C(0), j[3] = {C(0), C(0), C(0)};
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const long long e = (long long)i * r.n_ghost + k;
    const C fv = second ? C(0.5) * (Ga[e] + Gb[e]) : Ga[e];
    store_pop<L, S, C>(f1, i, N1, n1, fv, r.g1.off);
    const C v = roundtrip_pop<L, S, C>(i, fv, r.g1.off);
    rho += v;
    sfor<0, D>([&](auto A) {
      constexpr int d = decltype(A)::value;
      if constexpr (L::c(i, d) != 0) j[d] += C(L::c(i, d)) * v;
    });
  });
  const long long eE = (long long)Q * r.n_ghost + k;
  M1[n1] = rho;
#pragma unroll
  for (int a = 0; a < D; ++a) M1[(1 + a) * N1 + n1] = j[a];
  M1[(1 + D) * N1 + n1] = second ? C(0.5) * (Ga[eE] + Gb[eE]) : Ga[eE];
  auto mean_of = [&](const C* src) {
    return refine_mean<D, C>(odd, [&](int sx, int sy, int sz) { return src[node(sx, sy, sz)]; });
  };
  P1[n1] = second ? mean_of(P0_new) : C(0.5) * (mean_of(P0_old) + mean_of(P0_new));
#pragma unroll
  for (int s = 0; s < L::NDEV; ++s) {
    const C an = refine_mean<D, C>(odd, [&](int sx, int sy, int sz) { return A0_new[s * N0 + node(sx, sy, sz)]; });
    if (second) {
      A1[s * N1 + n1] = C(0.5) * an;
    } else {
      const C ao =
          refine_mean<D, C>(odd, [&](int sx, int sy, int sz) { return A0_old[s * N0 + node(sx, sy, sz)]; });
      A1[s * N1 + n1] = C(0.25) * (ao + an);
    }
  }
}

// restriction of level 1 into the level-0 nodes R or more nodes inside the
// box (P1_n, A1_n: level 1's previous-step buffers after its second step,
// i.e. its values at level-1 time n)
template <class L, class S, class C>
__global__ void k_refine_restrict(RefineDev r, S* f0, C* M0, C* P0, C* A0, const S* f1, const C* M1,
                                  const C* P1_n, const C* A1_n) {
  constexpr int D = L::D, Q = L::Q;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nr = (long long)r.rn[0] * r.rn[1] * (D == 3 ? r.rn[2] : 1);
  if (t >= nr) return;
  int c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
  c0[0] = r.rlo[0] + (int)(t % r.rn[0]);
  c0[1] = r.rlo[1] + (int)((t / r.rn[0]) % r.rn[1]);
  if (D == 3) c0[2] = r.rlo[2] + (int)(t / ((long long)r.rn[0] * r.rn[1]));
#pragma unroll
  for (int a = 0; a < D; ++a) c1[a] = r.G + 2 * (c0[a] - r.lo[a]);
  const long long N0 = r.g0.N, N1 = r.g1.N;
  const long long n0 = r.g0.lin(c0[0], c0[1], c0[2]);
  const long long n1 = r.g1.lin(c1[0], c1[1], c1[2]);
  C rho1, u[3] = {C(0), C(0), C(0)}, th;
  refine_macros<D, C>(M1, N1, n1, C(r.Cv), rho1, u, th);
  const C s10 = C(2) * refine_tau_bar<C>(r.mu0, rho1) / refine_tau_bar<C>(r.mu1, rho1);
  C rho = C(0), j[3] = {C(0), C(0), C(0)};
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const C fe = feq_i<L, C, i>(rho1, u, th);
    const C fv = fe + s10 * (load_pop<L, S, C>(f1, i, N1, n1, r.g1.off) - fe);
    store_pop<L, S, C>(f0, i, N0, n0, fv, r.g0.off);
    const C v = roundtrip_pop<L, S, C>(i, fv, r.g0.off);
    rho += v;
    sfor<0, D>([&](auto A) {
      constexpr int d = decltype(A)::value;
      if constexpr (L::c(i, d) != 0) j[d] += C(L::c(i, d)) * v;
    });
  });
  M0[n0] = rho;
#pragma unroll
  for (int a = 0; a < D; ++a) M0[(1 + a) * N0 + n0] = j[a];
  M0[(1 + D) * N0 + n0] = M1[(1 + D) * N1 + n1];
  P0[n0] = P1_n[n1];
#pragma unroll
  for (int s = 0; s < L::NDEV; ++s) A0[s * N0 + n0] = C(2) * A1_n[s * N1 + n1];
}

}  // namespace lbmib
