// Lattice constants for the device kernels: D2Q9 and D3Q19 (App. A of
// arXiv 2607.07432).  Every table is a constexpr function so that fully
// unrolled loops fold the velocities, weights and Hermite coefficients into
// immediates.  D3Q19 uses the paper's ordering (Eq. cid3q19; opposite of i
// is i + 9); its weights follow |c_i|^2 (1/3, 1/18, 1/36) because the
// printed list (Eq. wi) is garbled.  D2Q9: 0 rest, 1..4 = +x,+y,-x,-y,
// 5..8 = (1,1),(-1,1),(-1,-1),(1,-1).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace lbmib {

// compile-time loop: f(std::integral_constant<int, i>) for i in [B, E)
template <int B, int E, class F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(f);
  }
}

constexpr double kCs2 = 1.0 / 3.0;

struct D2Q9 {
  static constexpr int D = 2;
  static constexpr int Q = 9;
  static constexpr int N3 = 2;     // H_xxy, H_xyy
  static constexpr int NDEV = 2;   // symmetric traceless tensor: xx, xy
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return a == 0 ? cx[i] : (a == 1 ? cy[i] : 0);
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  // third-order combination k = sum_t sign * H3_{a b g}
  __host__ __device__ static constexpr int h3terms(int) { return 1; }
  __host__ __device__ static constexpr int h3sign(int, int) { return 1; }
  __host__ __device__ static constexpr int h3idx(int k, int, int which) {
    // k = 0: (x,x,y); k = 1: (x,y,y)
    return k == 0 ? (which == 2 ? 1 : 0) : (which == 0 ? 0 : 1);
  }
};

struct D3Q19 {
  static constexpr int D = 3;
  static constexpr int Q = 19;
  static constexpr int N3 = 6;
  static constexpr int NDEV = 5;   // xx, yy, xy, xz, yz (zz = -xx-yy)
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int cx[19] = {0, 1, 1, 0, -1, 0, 0, 0, 1, -1, -1, -1, 0, 1, 0, 0, 0, -1, 1};
    constexpr int cy[19] = {0, 0, 0, 0, 0, 1, 1, -1, 1, 1, 0, 0, 0, 0, -1, -1, 1, -1, -1};
    constexpr int cz[19] = {0, 0, 1, 1, 1, 0, 1, 1, 0, 0, 0, -1, -1, -1, 0, -1, -1, 0, 0};
    return a == 0 ? cx[i] : (a == 1 ? cy[i] : cz[i]);
  }
  __host__ __device__ static constexpr double w(int i) {
    return (c(i, 0) * c(i, 0) + c(i, 1) * c(i, 1) + c(i, 2) * c(i, 2)) == 0
               ? 1.0 / 3.0
               : ((c(i, 0) * c(i, 0) + c(i, 1) * c(i, 1) + c(i, 2) * c(i, 2)) == 1 ? 1.0 / 18.0
                                                                                  : 1.0 / 36.0);
  }
  // Eq. hi3: k=0 xxy+yzz, 1 xzz+xyy, 2 yyz+xxz, 3 xxy-yzz, 4 xzz-xyy, 5 yyz-xxz
  __host__ __device__ static constexpr int h3terms(int) { return 2; }
  __host__ __device__ static constexpr int h3sign(int k, int t) { return (t == 1 && k >= 3) ? -1 : 1; }
  __host__ __device__ static constexpr int h3idx(int k, int t, int which) {
    constexpr int tab[3][2][3] = {{{0, 0, 1}, {1, 2, 2}},   // xxy, yzz
                                  {{0, 2, 2}, {0, 1, 1}},   // xzz, xyy
                                  {{1, 1, 2}, {0, 0, 2}}};  // yyz, xxz
    return tab[k % 3][t][which];
  }
};

// opposite direction: c_opp(i) = -c_i
template <class L>
__host__ __device__ constexpr int opposite(int i) {
  for (int j = 0; j < L::Q; ++j)
    if (L::c(j, 0) == -L::c(i, 0) && L::c(j, 1) == -L::c(i, 1) && L::c(j, 2) == -L::c(i, 2)) return j;
  return -1;
}

// ---------------------------------------------------------------------------
// Hermite polynomials (Eq. hi), evaluated at compile time
// ---------------------------------------------------------------------------
template <class L>
__host__ __device__ constexpr double H2(int i, int a, int b) {
  return double(L::c(i, a) * L::c(i, b)) - (a == b ? kCs2 : 0.0);
}
template <class L>
__host__ __device__ constexpr double H3(int i, int a, int b, int g) {
  return double(L::c(i, a) * L::c(i, b) * L::c(i, g)) -
         kCs2 * ((a == b ? L::c(i, g) : 0) + (b == g ? L::c(i, a) : 0) + (a == g ? L::c(i, b) : 0));
}
template <class L>
__host__ __device__ constexpr double H3r(int k, int i) {
  double v = 0.0;
  for (int t = 0; t < L::h3terms(k); ++t)
    v += L::h3sign(k, t) * H3<L>(i, L::h3idx(k, t, 0), L::h3idx(k, t, 1), L::h3idx(k, t, 2));
  return v;
}
template <class L>
__host__ __device__ constexpr int c2(int i) {
  int s = 0;
  for (int a = 0; a < L::D; ++a) s += L::c(i, a) * L::c(i, a);
  return s;
}
// lattice norm N_k = sum_i w_i H3r_k,i^2 (orthogonal projection, 1/N_k),
// evaluated exactly and rounded once: 36 w_i and 3 H3r_k,i are integers,
// so N_k = (sum_i 36 w_i (3 H3r_k,i)^2) / 324
template <class L>
__host__ __device__ constexpr int w36(int i) {
  return c2<L>(i) == 0 ? (L::D == 3 ? 12 : 16) : (c2<L>(i) == 1 ? (L::D == 3 ? 2 : 4) : 1);
}
template <class L>
__host__ __device__ constexpr int H3x3(int i, int a, int b, int g) {
  return 3 * L::c(i, a) * L::c(i, b) * L::c(i, g) -
         ((a == b ? L::c(i, g) : 0) + (b == g ? L::c(i, a) : 0) + (a == g ? L::c(i, b) : 0));
}
template <class L>
__host__ __device__ constexpr double N3r(int k) {
  long long s = 0;
  for (int i = 0; i < L::Q; ++i) {
    long long h = 0;
    for (int t = 0; t < L::h3terms(k); ++t)
      h += L::h3sign(k, t) * H3x3<L>(i, L::h3idx(k, t, 0), L::h3idx(k, t, 1), L::h3idx(k, t, 2));
    s += w36<L>(i) * h * h;
  }
  return double(s) / 324.0;
}
// number of nonzero transverse components of c_i with respect to axis a
template <class L>
__host__ __device__ constexpr int transverse_axis(int i, int a) {
  for (int t = 0; t < L::D; ++t)
    if (t != a && L::c(i, t) != 0) return t;
  return -1;
}

// index of the symmetric traceless tensor component (a,b) in NDEV storage;
// returns -1 for the dependent last diagonal entry
template <class L>
__host__ __device__ constexpr int dev_slot(int a, int b) {
  if (L::D == 2) {
    if (a == 0 && b == 0) return 0;
    if (a != b) return 1;
    return -1;  // yy = -xx
  } else {
    if (a == b) return a < 2 ? a : -1;  // zz = -xx-yy
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? (hi == 1 ? 2 : 3) : 4;
  }
}

}  // namespace lbmib
