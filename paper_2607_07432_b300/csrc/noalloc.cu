// Wall loads without any device allocation.
//
// lbm_get_wall_loads reduces the per-point immersed-boundary forces into a
// small device buffer that the library allocates when the geometry is set.
// Some callers cannot allocate device memory when they ask for the loads:
// a process whose device memory is fully reserved by another framework's
// caching pool, or an embedding that forbids cudaMalloc / cudaFree after
// start-up.  lbm_get_wall_loads_noalloc serves them: its scratch (the
// per-block partial sums of a two-pass reduction) lives in a file-scope
// static device array of fixed size, and it calls no allocating routine.
//
// The array exists once per device that loads the library, for the life of
// the process.  Host code must not use its name as a device address; the
// address is obtained once per device with cudaGetSymbolAddress, on the
// first call made on that device.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "handle.cuh"

using namespace lbmib_host;

namespace {

constexpr int kNoallocThreads = 256;                 // points per block
constexpr int kNoallocMaxBlocks = 256;               // partial-sum slots
constexpr int kNoallocMaxPoints = kNoallocThreads * kNoallocMaxBlocks;  // 65536
constexpr int kNoallocSlot = 8;                      // doubles per block slot

// [kNoallocMaxBlocks][kNoallocSlot] partials, then one slot for the result
static __device__ __align__(256) double g_wall_scratch[(kNoallocMaxBlocks + 1) * kNoallocSlot];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// pass 1: block b sums points [256 b, 256 b + 256) in a fixed tree order
// (on a z slab only the points it owns, owned != nullptr)
__global__ void k_wall_partials(int D, int NL, const double* G, const double* W, const unsigned char* owned,
                                double* scratch) {
  __shared__ double sh[kNoallocThreads][5];
  const int t = threadIdx.x;
  const int l = blockIdx.x * kNoallocThreads + t;
  double acc[5] = {0, 0, 0, 0, 0};
  if (l < NL && (!owned || owned[l])) {
    const double w = W[l];
    for (int a = 0; a < D; ++a) acc[a] = G[l * (D + 2) + a] * w;
    acc[3] = G[l * (D + 2) + D + 1] * w;  // Q
    acc[4] = G[l * (D + 2) + D] * w;      // W^IB
  }
  for (int k = 0; k < 5; ++k) sh[t][k] = acc[k];
  __syncthreads();
  for (int s = kNoallocThreads / 2; s > 0; s >>= 1) {
    if (t < s)
      for (int k = 0; k < 5; ++k) sh[t][k] += sh[t + s][k];
    __syncthreads();
  }
  if (t == 0)
    for (int k = 0; k < 5; ++k) scratch[blockIdx.x * kNoallocSlot + k] = sh[0][k];
}

// pass 2: one thread adds the block partials in block order
__global__ void k_wall_final(int D, int nblocks, double* scratch) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int k = 0; k < 5; ++k) acc[k] += scratch[b * kNoallocSlot + k];
  double* out = scratch + kNoallocMaxBlocks * kNoallocSlot;
  for (int a = 0; a < 3; ++a) out[a] = a < D ? -acc[a] : 0.0;
  out[3] = acc[3];
  out[4] = acc[4];
}

}  // namespace

extern "C" lbm_status lbm_get_wall_loads_noalloc(lbm_handle* h, double force[3], double* heat, double* work) {
  if (!h) return LBM_EINVAL;
  if (!h->has_ib) return fail(h, LBM_ESTATE, "no immersed body");
  if (h->NL > kNoallocMaxPoints)
    return fail(h, LBM_EINVAL,
                "lbm_get_wall_loads_noalloc supports at most 65536 Lagrangian points (static scratch)");
  const int dev = h->cfg.device;
  if (dev < 0 || dev >= kMaxDevices) return fail(h, LBM_EINVAL, "device ordinal out of range");
  DeviceGuard dg(dev);
  if (dg.status() != cudaSuccess) return fail(h, LBM_ECUDA, "cudaSetDevice failed");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      double* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_wall_scratch);
      if (e != cudaSuccess) return fail(h, LBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  const int nblocks = (h->NL + kNoallocThreads - 1) / kNoallocThreads;
  lbm_status s = launch(h, kProfOther, [&] {
    k_wall_partials<<<nblocks, kNoallocThreads, 0, h->st>>>(h->D, h->NL, h->G, h->W, h->owned, scratch);
  });
  if (s) return s;
  s = launch(h, kProfOther, [&] { k_wall_final<<<1, 32, 0, h->st>>>(h->D, nblocks, scratch); });
  if (s) return s;
  cudaError_t e;
  double out[5];
  e = cudaMemcpyAsync(out, scratch + kNoallocMaxBlocks * kNoallocSlot, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                      h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, std::string("copy of the loads: ") + cudaGetErrorString(e));
  if (force)
    for (int a = 0; a < 3; ++a) force[a] = out[a];
  if (heat) *heat = out[3];
  if (work) *work = out[4];
  return LBM_OK;
}
