// Grid geometry and storage conversions shared by the device kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbmib {

// Domain extent and per-axis periodicity.  Non-periodic axes clamp
// out-of-range stencil reads to the edge node (zero-gradient).
struct Grid {
  int n[3];
  int per[3];
  long long N;
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

template <class L, class S, class C>
__device__ __forceinline__ C load_pop(const S* f, int i, long long N, long long n) {
  const C v = C(Store<S>::load(f[(long long)i * N + n]));
  return Store<S>::dev ? v + C(L::w(i)) : v;
}
// the value a population takes after a store and a reload
template <class L, class S, class C>
__device__ __forceinline__ C roundtrip_pop(int i, C v) {
  if (Store<S>::dev) return C(Store<S>::load(Store<S>::save(v - C(L::w(i))))) + C(L::w(i));
  return C(Store<S>::load(Store<S>::save(v)));
}
template <class L, class S, class C>
__device__ __forceinline__ void store_pop(S* f, int i, long long N, long long n, C v) {
  f[(long long)i * N + n] = Store<S>::save(Store<S>::dev ? v - C(L::w(i)) : v);
}

}  // namespace lbmib
