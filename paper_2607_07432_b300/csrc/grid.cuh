// Grid geometry and storage conversions shared by the device kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbmib {

// A face of a z slab that borders a neighbour slab (boundary type next to
// the LBM_BC_* values): no boundary condition there; its ghost planes are
// refreshed by the slab exchange.
constexpr int kBCGhostFace = 4;
// characteristic far field (LBM_BC_CHARACTERISTIC)
constexpr int kBCChar = 5;

// Domain extent and per-axis periodicity.  Non-periodic axes clamp
// out-of-range stencil reads to the edge node (zero-gradient).
struct Grid {
  int n[3];
  int per[3];
  long long N;
  int zoff;  // global z of local plane 0 (a z slab of a larger case; 0 otherwise)
  float off[19];  // values 16-bit storage subtracts from the populations (see pop_offset)
  __host__ __device__ __forceinline__ int wrap(int a, int v) const {
    if (per[a]) {
      v = v % n[a];
      return v < 0 ? v + n[a] : v;
    }
    return v < 0 ? 0 : (v >= n[a] ? n[a] - 1 : v);
  }
  __host__ __device__ __forceinline__ long long lin(int x, int y, int z) const {
    return (long long)x + (long long)n[0] * ((long long)y + (long long)n[1] * z);
  }
  __host__ __device__ __forceinline__ long long nb(int x, int y, int z, int dx, int dy, int dz) const {
    return lin(wrap(0, x + dx), wrap(1, y + dy), wrap(2, z + dz));
  }
};

// Grid-wide barrier state (device memory, zero at plan build).  count: CTAs
// arrived at the current barrier; gen: barriers completed; err: set when a
// CTA waited past the spin limit (the launch then ends early and the host
// reports LBM_ETIMEOUT); next: the next work item of a dynamically shared
// phase.
struct GridBarrier {
  unsigned count;
  unsigned gen;
  int err;
  unsigned next;  // work counter of the phase that follows the barrier
};

// Transfers between the two levels of a refined case (lbm_refined_*):
// level-1 node k along an axis sits at level-0 coordinate lo + (k - G)/2
struct RefineDev {
  Grid g0, g1;            // level-0 and level-1 grids
  int lo[3];              // level-0 node of level-1 node G (per axis)
  int G;                  // ghost width (level-1 nodes)
  int n_ghost;
  const int4* ghost;      // level-1 coordinates of the ghost nodes
  int n_shell;            // level-0 nodes the ghost nodes read
  const long long* shell; // their level-0 indices
  const int* corners;     // per ghost node 2^D shell indices (corner sx + 2 sy + 4 sz; -1: not read)
  int rlo[3], rn[3];      // restricted level-0 nodes: first node and count per axis
  double mu0, mu1, Cv;
};

// Population storage.  FP64 stores f-bar as is; the other formats store
// the deviation f-bar_i - w_i (reference density 1), converted to the
// compute type on load.
template <class S>
struct Store;
template <>
struct Store<double> {
  static constexpr bool dev = false;
  __device__ __forceinline__ static double load(double v) { return v; }
  __device__ __forceinline__ static double save(double v) { return v; }
};
template <>
struct Store<float> {
  static constexpr bool dev = true;
  __device__ __forceinline__ static float load(float v) { return v; }
  __device__ __forceinline__ static float save(float v) { return v; }
};
template <>
struct Store<__half> {
  static constexpr bool dev = true;
  __device__ __forceinline__ static float load(__half v) { return __half2float(v); }
  __device__ __forceinline__ static __half save(float v) { return __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
  static constexpr bool dev = true;
  __device__ __forceinline__ static float load(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static __nv_bfloat16 save(float v) { return __float2bfloat16_rn(v); }
};

// Reference value subtracted from population i before it is stored: w_i for
// FP32 storage; for FP16 / BF16 storage the free-stream equilibrium of the
// case, f^eq_i(rho_inf, u_inf, theta_inf) (Eq. feq; off[i], set when the
// case is created), so that the stored deviations stay small wherever the
// flow is near the free stream and lose little to the 16-bit rounding
template <class L, class S, class C>
__device__ __forceinline__ C pop_offset(int i, const float* off) {
  if constexpr (sizeof(S) == 2) {
    return C(off[i]);
  } else {
    return C(L::w(i));
  }
}
template <class L, class S, class C, class I = long long>
__device__ __forceinline__ C load_pop(const S* f, int i, I N, I n, const float* off) {
  const C v = C(Store<S>::load(f[(I)i * N + n]));
  return Store<S>::dev ? v + pop_offset<L, S, C>(i, off) : v;
}
// the value a population takes after a store and a reload
template <class L, class S, class C>
__device__ __forceinline__ C roundtrip_pop(int i, C v, const float* off) {
  if (Store<S>::dev) {
    const C o = pop_offset<L, S, C>(i, off);
    return C(Store<S>::load(Store<S>::save(v - o))) + o;
  }
  return C(Store<S>::load(Store<S>::save(v)));
}
template <class L, class S, class C, class I = long long>
__device__ __forceinline__ void store_pop(S* f, int i, I N, I n, C v, const float* off) {
  f[(I)i * N + n] = Store<S>::save(Store<S>::dev ? v - pop_offset<L, S, C>(i, off) : v);
}

}  // namespace lbmib
