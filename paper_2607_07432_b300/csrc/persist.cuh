// Batched step of several 2D cases as one persistent cooperative launch:
// every CTA of the grid (all resident at once, as the cooperative launch
// guarantees) takes the work items of the four phases of a step in turn --
// immersed-boundary force (Sec. 2.3-2.4), spreading and its application to
// the moments (Eq. spr2), the fused collide-stream-energy step (Eq. LB,
// Eq. energy) and the boundary faces -- with a grid-wide barrier between
// phases, for one or more steps.  The operations per work item are those
// of the separate batched kernels, so both forms give the same state bit for
// bit.
#pragma once
#include "ib.cuh"
#include "step_fused.cuh"

namespace lbmib {

// about a second of waiting (64 ns sleeps) before a CTA gives up
constexpr unsigned long long kBarrierSpins = 1ull << 24;

// All CTAs of the launch arrive; the last releases the others.  Returns
// false (in every thread of the CTA) when the barrier failed: the caller
// then returns without further work.
__device__ __forceinline__ bool grid_barrier(GridBarrier* b) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    volatile int* verr = &b->err;
    const unsigned g0 = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&b->count, 0u);
      atomicExch(&b->next, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == g0 && *verr == 0) {
        if (++spins > kBarrierSpins) {
          atomicExch(&b->err, 1);
          break;
        }
        if (spins > 4096) __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = *verr == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class S, class C>
struct PersistDesc {
  const CaseDesc<S, C>* descs[2];
  const int4* work;
  int n_work;
  const IBCaseDesc<S, C>* ib[2];
  const int2* ib_work;
  int n_ib;
  const SpreadCaseDesc<C>* sp[2];
  const int2* sp_work;
  int n_sp;
  const BCCaseDesc<S, C>* bc[2];
  const int4* bc_work;
  int n_bc;
  GridBarrier* bar;
};

// work items of 128 threads (spreading rows, boundary nodes) and IB blocks
// (kIBWarps warps) run NT / 128 and up to 256 / (32 kIBWarps) to a CTA; 64
// registers per thread, as the separate fused kernel takes, so that as many
// CTAs are resident for the fused phase
template <class L, class S, class C, int HY, bool NARROW>
__global__ void __launch_bounds__(FusedLayout<L, S, C, HY>::NT, 1024 / FusedLayout<L, S, C, HY>::NT)
    k_batch_persistent(PersistDesc<S, C> p, int parity0, int nsteps) {
  constexpr int NT = FusedLayout<L, S, C, HY>::NT;
  static_assert(L::D == 2, "2D cases");
  static_assert(NT % 128 == 0, "whole 128-thread items");
  // IB blocks on at most eight warps of the CTA (their staging is static
  // shared memory per warp)
  constexpr int IBW = 32 * kIBWarps, SUB = NT / 128, IBSUB = (NT < 256 ? NT : 256) / IBW;
  const int tid = threadIdx.x;
  for (int k = 0; k < nsteps; ++k) {
    const int par = (parity0 + k) & 1;
    if (k > 0 && !grid_barrier(p.bar)) return;
    if (p.n_ib) {
      if (tid < IBSUB * IBW) {
        for (int it = blockIdx.x * IBSUB + tid / IBW; it < p.n_ib; it += gridDim.x * IBSUB) {
          const int2 w = p.ib_work[it];
          const IBCaseDesc<S, C>& c = p.ib[par][w.x];
          ib_force_body<L, S, C, IBSUB * kIBWarps>(c.g, c.s, c.M, w.y);
        }
      }
      if (!grid_barrier(p.bar)) return;
      for (int it = blockIdx.x * SUB + tid / 128; it < p.n_sp; it += gridDim.x * SUB) {
        const int2 w = p.sp_work[it];
        spread_apply_row<C>(p.sp[par][w.x], w.y * 128 + tid % 128);
      }
      if (!grid_barrier(p.bar)) return;
    }
    {
      // tiles taken in schedule order from a shared counter (reset by the
      // host before the launch and by the barrier that opens the phase);
      // the next index is fetched while the current tile runs
      __shared__ int s_next;
      if (tid == 0) s_next = (int)atomicAdd(&p.bar->next, 1u);
      __syncthreads();
      int it = s_next;
      __syncthreads();
      while (it < p.n_work) {
        int nxt = 0;
        if (tid == 0) nxt = (int)atomicAdd(&p.bar->next, 1u);
        const int4 w = p.work[it];
        const CaseDesc<S, C>& d = p.descs[par][w.x];
        fused_body<L, S, C, HY, NARROW>(d.g, d.a, d.ph, d.zchunk, w.y, w.z, w.w);
        if (tid == 0) s_next = nxt;
        __syncthreads();
        it = s_next;
        __syncthreads();
      }
    }
    if (!grid_barrier(p.bar)) return;
    for (int it = blockIdx.x * SUB + tid / 128; it < p.n_bc; it += gridDim.x * SUB) {
      const int4 w = p.bc_work[it];
      const BCCaseDesc<S, C>& c = p.bc[par][w.x];
      bc_node<L, S, C>(c.g, c.f, c.M, c.bf, c.feq_inf, c.E_inf, c.skip_x, w.y, w.z * 128 + tid % 128);
    }
  }
}

}  // namespace lbmib
