// Kernels of the warm-start neural operator: 3x3 convolution as an implicit
// GEMM on the tensor cores (BF16 operands, FP32 accumulation), its weight
// gradient with deterministic split-K partials, and the elementwise pieces
// (pooling, up-sampling, skip sums, ReLU masks, loss, Adam).
//
// Layout: activations and gradients NHWC FP32, pixel index
// p = (b H + y) W + x, channels fastest.  Weights of a layer are BF16
// Wt[c_out][tap][c_in] with tap = 3 ky + kx multiplying pixel
// (y + ky - 1, x + kx - 1), channel counts padded to multiples of 16.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmib {
namespace nop {

constexpr int kTN = 32;    // output channels per CTA tile
constexpr int kWChunk = 1024;  // pixels per weight-gradient partial

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// D = A B + D for one m16n8k16 tile: A row-major 16x16, B column-major 16x8,
// BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Y[p][co] (+)= sum_{tap, ci} X[p + tap][ci] Wt[co][tap][ci] (+ bias[co]),
// optionally followed by ReLU, zero padding outside the image.  GEMM view:
// M = pixels, N = c_out, K = 9 c_in.  A CTA computes 64 consecutive
// pixels of one image row for 32 output channels: per chunk of 32 input
// channels it stages the three input rows (66 columns, BF16) and the
// chunk's weights of all nine taps once, and every tap's A fragments are
// read from that tile at a column offset.  accumulate adds the previous
// content of Y (gradient sums; every element is written by one thread, so
// the sum is deterministic).  Cin and Cout are multiples of 16; the input
// gradient of a convolution is this kernel applied to the output gradient
// with the flipped, transposed weights Wf[ci][8 - tap][co] = Wt[co][tap][ci].
constexpr int kRowPx = 64;            // pixels per CTA tile (one image row)
constexpr int kRowCols = kRowPx + 2;  // staged input columns
constexpr int kChunk = 32;            // input channels per staged chunk
constexpr int kChLd = 40;             // padded channel stride of a staged pixel (bank-conflict free)

__global__ void __launch_bounds__(128) k_conv3x3(const float* __restrict__ X,
                                                 const __nv_bfloat16* __restrict__ Wt,
                                                 const float* __restrict__ bias, float* __restrict__ Y, int B,
                                                 int H, int W, int Cin, int Cout, int relu, int accumulate) {
  __shared__ __align__(16) __nv_bfloat16 In[3][kRowCols][kChLd];
  __shared__ __align__(16) __nv_bfloat16 Ws[9][kTN][kChLd];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  const int tiles_x = (W + kRowPx - 1) / kRowPx;
  int bid = blockIdx.x;
  const int xt = bid % tiles_x;
  bid /= tiles_x;
  const int y = bid % H;
  const int b = bid / H;
  const int x0 = xt * kRowPx;
  const int n0 = blockIdx.y * kTN;
  const int m0 = warp * 16;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  for (int c0 = 0; c0 < Cin; c0 += kChunk) {
    // input rows y-1..y+1, columns x0-1..x0+64, channels c0..c0+31, in units of 8 channels
    for (int u = tid; u < 3 * kRowCols * 4; u += 128) {
      const int r = u / (kRowCols * 4), rem = u - r * (kRowCols * 4);
      const int col = rem >> 2, q = rem & 3;
      const int yy = y + r - 1, xx = x0 + col - 1, c = c0 + q * 8;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = 0.f;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W && c < Cin) {
        const float4* src = reinterpret_cast<const float4*>(X + (((long long)b * H + yy) * W + xx) * Cin + c);
        const float4 u0 = src[0], u1 = src[1];
        v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
        v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
      }
      uint4 pk;
      pk.x = pack_bf16x2(v[0], v[1]);
      pk.y = pack_bf16x2(v[2], v[3]);
      pk.z = pack_bf16x2(v[4], v[5]);
      pk.w = pack_bf16x2(v[6], v[7]);
      *reinterpret_cast<uint4*>(&In[r][col][q * 8]) = pk;
    }
    // weights of the 32 output channels, all taps, the chunk's channels
    for (int u = tid; u < 9 * kTN * 4; u += 128) {
      const int tap = u / (kTN * 4), rem = u - tap * (kTN * 4);
      const int co = rem >> 2, q = rem & 3;
      const int c = c0 + q * 8;
      uint4 w = make_uint4(0u, 0u, 0u, 0u);
      if (n0 + co < Cout && c < Cin) w = *reinterpret_cast<const uint4*>(Wt + ((long long)(n0 + co) * 9 + tap) * Cin + c);
      *reinterpret_cast<uint4*>(&Ws[tap][co][q * 8]) = w;
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap % 3;
#pragma unroll
      for (int kk = 0; kk < kChunk / 16; ++kk) {
        const int kc = kk * 16 + 2 * tq;
        const uint32_t a0 = lds32(&In[ky][m0 + g + kx][kc]);
        const uint32_t a1 = lds32(&In[ky][m0 + g + 8 + kx][kc]);
        const uint32_t a2 = lds32(&In[ky][m0 + g + kx][kc + 8]);
        const uint32_t a3 = lds32(&In[ky][m0 + g + 8 + kx][kc + 8]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const uint32_t b0 = lds32(&Ws[tap][nt * 8 + g][kc]);
          const uint32_t b1 = lds32(&Ws[tap][nt * 8 + g][kc + 8]);
          mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int co = n0 + nt * 8 + 2 * tq;
    if (co >= Cout) continue;
    const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int x = x0 + m0 + g + hr * 8;
      if (x >= W) continue;
      float v0 = acc[nt][2 * hr] + b0, v1 = acc[nt][2 * hr + 1] + b1;
      if (relu) {
        v0 = v0 > 0.f ? v0 : 0.f;
        v1 = v1 > 0.f ? v1 : 0.f;
      }
      float2* dst = reinterpret_cast<float2*>(Y + (((long long)b * H + y) * W + x) * Cout + co);
      if (accumulate) {
        const float2 o = *dst;
        v0 = o.x + v0;
        v1 = o.y + v1;
      }
      *dst = make_float2(v0, v1);
    }
  }
}

// ---------------------------------------------------------------------------
// The same convolution on the 5th-generation tensor cores (tcgen05): one CTA
// of 128 R threads computes R image rows of 128 consecutive pixels each
// (one M = 128 accumulator per row) for all Cout output channels (N = Cout
// <= 128), accumulating in tensor memory (row rr at columns rr Cout ..).
//
// Per chunk of 8 NG input channels (NG = 4 groups of 8, or 2 when Cin is
// not a multiple of 32) the CTA stages, as BF16 in the canonical K-major
// layout without swizzling (8 x 16-byte core matrices), the R + 2 input rows
// its outputs need (130 columns: In[row][group][column][8 channels]) and the
// chunk's weights of all nine taps (Ws[tap][group][c_out][8 channels]), so
// each staged row and weight serves R output rows.  One thread issues the
// chunk's 9 R NG / 2 MMAs of K = 16 (per output row and tap, the A operand
// is the staged row ky below it from column offset kx) and commits them to
// an mbarrier.  With one staging buffer (DB false, the form the network
// uses) the CTA waits for them before staging the next chunk; with two (DB
// true) it stages the next chunk into the other buffer while they run.  On
// the 512x256 network one buffer is faster (at R = 1: 2.46 against 3.58 ms
// per forward pass): the staging loads, not the MMAs, set the pace, and a
// second buffer halves the CTAs resident per SM.  R = 4 (512 threads) is
// the fastest of 1, 2 and 4 there (1.51 ms).  In the epilogue warp w reads
// TMEM lanes 32 (w % 4) .. (its 32 pixels) of row w / 4 with tcgen05.ld,
// adds the bias, applies ReLU and writes (or accumulates into) Y.  Waits are
// bounded: on a timeout the CTA records it in *status and skips its stores.
constexpr int kTcM = 128;               // pixels per CTA
constexpr int kTcCols = kTcM + 2;       // staged input columns
constexpr unsigned long long kTcWaitNs = 200000000ull;  // MMA-completion wait limit (0.2 s)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading-dimension (K direction)
// and stride-dimension (M / N direction) byte offsets, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;               // base offset 0, relative LBO, layout: no swizzle
}

// instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both operands
// K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4)                      // D format FP32
         | (1u << 7)                    // A format BF16
         | (1u << 10)                   // B format BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

template <int NCOL>
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// bytes of one staging buffer (In then Ws) and of the dynamic shared memory:
// one or two buffers (DB), two mbarriers and the TMEM address
__host__ __device__ constexpr size_t conv_tc_stage_bytes(int NG, int N, int R) {
  return (size_t)(R + 2) * NG * kTcCols * 16 + (size_t)9 * NG * N * 16;
}
__host__ __device__ constexpr size_t conv_tc_smem(int NG, int N, bool DB, int R) {
  return (DB ? 2 : 1) * conv_tc_stage_bytes(NG, N, R) + 32;
}

// wait (bounded) for phase `phase` of an mbarrier; true when it completed
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t phase) {
  uint32_t done = 0;
  const unsigned long long t0 = global_ns();
  while (!done) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
    if (!done && global_ns() - t0 > kTcWaitNs) break;
  }
  return done != 0;
}

// stage input channels c0 .. c0 + 8 NG - 1 of rows y-1..y+1, columns
// x0-1..x0+128 (zero outside the image) and the weights of all taps for
// those channels, as BF16; consecutive threads read consecutive 32-byte
// pieces of one pixel's channels
template <int NG, int R, int NT>
__device__ __forceinline__ void tc_stage(unsigned char* In, unsigned char* Ws, const float* __restrict__ X,
                                         const __nv_bfloat16* __restrict__ Wt, int b, int y, int x0, int c0, int H,
                                         int W, int Cin, int Cout, int tid) {
  // four items per thread per pass: all eight loads are issued before the
  // first conversion, so each thread keeps several loads in flight
  constexpr int kBatch = 4;
  constexpr int total = (R + 2) * kTcCols * NG;
  for (int u0 = tid; u0 < total; u0 += kBatch * NT) {
    float4 lo[kBatch], hi[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const int u = u0 + k * NT;
      lo[k] = hi[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (u < total) {
        const int g = u % NG, rc = u / NG;
        const int col = rc % kTcCols, r = rc / kTcCols;
        const int yy = y + r - 1, xx = x0 + col - 1;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
          const float4* src =
              reinterpret_cast<const float4*>(X + (((long long)b * H + yy) * W + xx) * Cin + c0 + g * 8);
          lo[k] = src[0];
          hi[k] = src[1];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const int u = u0 + k * NT;
      if (u >= total) break;
      const int g = u % NG, rc = u / NG;
      const int col = rc % kTcCols, r = rc / kTcCols;
      uint4 pk;
      pk.x = pack_bf16x2(lo[k].x, lo[k].y);
      pk.y = pack_bf16x2(lo[k].z, lo[k].w);
      pk.z = pack_bf16x2(hi[k].x, hi[k].y);
      pk.w = pack_bf16x2(hi[k].z, hi[k].w);
      *reinterpret_cast<uint4*>(In + ((size_t)(r * NG + g) * kTcCols + col) * 16) = pk;
    }
  }
  const int wtotal = 9 * NG * Cout;
  for (int u0 = tid; u0 < wtotal; u0 += kBatch * NT) {
    uint4 w[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const int u = u0 + k * NT;
      w[k] = make_uint4(0u, 0u, 0u, 0u);
      if (u < wtotal) {
        const int g = u % NG, rc = u / NG;
        const int tap = rc % 9, co = rc / 9;
        w[k] = *reinterpret_cast<const uint4*>(Wt + ((long long)co * 9 + tap) * Cin + c0 + g * 8);
      }
    }
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const int u = u0 + k * NT;
      if (u >= wtotal) break;
      const int g = u % NG, rc = u / NG;
      const int tap = rc % 9, co = rc / 9;
      *reinterpret_cast<uint4*>(Ws + ((size_t)(tap * NG + g) * Cout + co) * 16) = w[k];
    }
  }
}

template <int NG, bool DB, int R>
__global__ void __launch_bounds__(128 * R) k_conv3x3_tc(const float* __restrict__ X, const __nv_bfloat16* __restrict__ Wt,
                                                    const float* __restrict__ bias, float* __restrict__ Y, int B,
                                                    int H, int W, int Cin, int Cout, int relu, int accumulate,
                                                    int* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  const size_t stage = conv_tc_stage_bytes(NG, Cout, R);
  const size_t in_bytes = (size_t)(R + 2) * NG * kTcCols * 16;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + (DB ? 2 : 1) * stage);   // two barriers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // after a timed-out wait anywhere in the launch, the remaining CTAs do
  // nothing (the caller reports the status); one read decides for the CTA
  __shared__ int skip;
  if (tid == 0) skip = *reinterpret_cast<volatile int*>(status);
  __syncthreads();
  if (skip) return;
  const int tiles_x = W / kTcM;
  int bid = blockIdx.x;
  const int xt = bid % tiles_x;
  bid /= tiles_x;
  const int y = (bid % (H / R)) * R;  // first of the CTA's R output rows
  const int b = bid / (H / R);
  const int x0 = xt * kTcM;
  // TMEM columns: a power of two >= 32 holding R x Cout FP32 accumulators
  // (row rr's at columns rr Cout ..)
  uint32_t ncols = 32u;
  while (ncols < (uint32_t)(R * Cout)) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const int nch = Cin / (8 * NG);
  tc_stage<NG, R, 128 * R>(sm, sm + in_bytes, X, Wt, b, y, x0, 0, H, W, Cin, Cout, tid);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = umma_idesc_bf16(kTcM, Cout);
  bool ok = true;
  uint32_t phases = 0u;  // bit b: the phase awaited next on buffer b's barrier
  for (int ch = 0; ch < nch; ++ch) {
    const int bb = DB ? (ch & 1) : 0;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned char* In = sm + bb * stage;
      const unsigned char* Ws = In + in_bytes;
#pragma unroll
      for (int rr = 0; rr < R; ++rr)
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int ky = tap / 3, kx = tap % 3;
#pragma unroll
          for (int sl = 0; sl < NG / 2; ++sl) {
            const uint64_t ad = umma_desc(smem_u32(In + ((size_t)((rr + ky) * NG + 2 * sl) * kTcCols + kx) * 16),
                                          kTcCols * 16, 128);
            const uint64_t bd = umma_desc(smem_u32(Ws + (size_t)(tap * NG + 2 * sl) * Cout * 16), Cout * 16, 128);
            const uint32_t acc = (ch > 0 || tap > 0 || sl > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(rr * Cout)),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(mbar + bb))
                   : "memory");
    }
    if (!DB) {
      // one buffer: the next chunk is staged once this chunk's MMAs are done
      const bool done = tc_wait(mbar, phases & 1u);
      if (!__syncthreads_and((int)done)) {
        ok = false;
        break;
      }
      phases ^= 1u;
      if (ch + 1 < nch) {
        tc_stage<NG, R, 128 * R>(sm, sm + in_bytes, X, Wt, b, y, x0, (ch + 1) * 8 * NG, H, W, Cin, Cout, tid);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
      }
    } else if (ch + 1 < nch) {
      // the other buffer is free once the MMAs of chunk ch-1 completed
      if (ch >= 1) {
        const bool done = tc_wait(mbar + (bb ^ 1), (phases >> (bb ^ 1)) & 1u);
        if (!__syncthreads_and((int)done)) {
          ok = false;
          break;
        }
        phases ^= 1u << (bb ^ 1);
      }
      unsigned char* nb = sm + (bb ^ 1) * stage;
      tc_stage<NG, R, 128 * R>(nb, nb + in_bytes, X, Wt, b, y, x0, (ch + 1) * 8 * NG, H, W, Cin, Cout, tid);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
    }
  }
  if (DB && ok) {
    // the last commit covers every MMA of the CTA
    const int last = (nch - 1) & 1;
    const bool done = tc_wait(mbar + last, (phases >> last) & 1u);
    ok = __syncthreads_and((int)done) != 0;
  }
  if (!ok && tid == 0) atomicExch(status, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. (pixels x0 + 32 (w % 4) + lane)
    // of row y + w / 4, 32 columns at a time
    const int rr = warp >> 2;
    const int x = x0 + (warp & 3) * 32 + lane;
    float* dst = Y + (((long long)b * H + y + rr) * W + x) * Cout;
    for (int n0 = 0; n0 < Cout; n0 += 32) {
      float v[32];
      tmem_ld32<32>(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(rr * Cout + n0), v);
      const int nv = Cout - n0 < 32 ? Cout - n0 : 32;
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        if (j >= nv) break;
        float4 o = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        if (bias) {
          o.x += bias[n0 + j];
          o.y += bias[n0 + j + 1];
          o.z += bias[n0 + j + 2];
          o.w += bias[n0 + j + 3];
        }
        if (relu) {
          o.x = o.x > 0.f ? o.x : 0.f;
          o.y = o.y > 0.f ? o.y : 0.f;
          o.z = o.z > 0.f ? o.z : 0.f;
          o.w = o.w > 0.f ? o.w : 0.f;
        }
        float4* d4 = reinterpret_cast<float4*>(dst + n0 + j);
        if (accumulate) {
          const float4 p = *d4;
          o.x = p.x + o.x;
          o.y = p.y + o.y;
          o.z = p.z + o.z;
          o.w = p.w + o.w;
        }
        *d4 = o;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
  }
}


// Weight-gradient partials:
// part[chunk][co][tap][ci] = sum_{p in chunk} G[p][co] X[p + tap][ci].
// GEMM view per tap: M = c_out (tile 32), N = c_in (tile 32), K = pixels.
// A chunk is kWUnits consecutive row segments of 64 pixels (segment u =
// (b H + y) tiles_x + xt).  For each segment the CTA stages G^T (32 c_out x
// 64 pixels) and the three input rows it meets, transposed (32 c_in x 66
// columns) in two copies, the second shifted by one column so that every
// tap's operand pairs start on an even column, and accumulates all nine taps.
// The chunk partials are added in chunk order by k_sum_chunks.
constexpr int kWUnits = 16;
constexpr int kWLd = 72;  // padded row (bf16) of the transposed tiles

__global__ void __launch_bounds__(128) k_conv3x3_wgrad(const float* __restrict__ G,
                                                       const float* __restrict__ X,
                                                       float* __restrict__ part, int B, int H, int W, int Cin,
                                                       int Cout) {
  __shared__ __align__(16) __nv_bfloat16 Gs[32][kWLd];        // [co][pixel]
  __shared__ __align__(16) __nv_bfloat16 Xs[2][3][32][kWLd];  // [shift][row][ci][column]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  const int chunk = blockIdx.x;
  const int m0 = blockIdx.y * 32;   // c_out tile
  const int c00 = blockIdx.z * 32;  // c_in tile
  const int wm = warp & 1, wn = warp >> 1;
  const int tiles_x = (W + kRowPx - 1) / kRowPx;
  const long long n_units = (long long)B * H * tiles_x;
  float acc[9][2][4];
#pragma unroll
  for (int tp = 0; tp < 9; ++tp)
#pragma unroll
    for (int i = 0; i < 2; ++i) acc[tp][i][0] = acc[tp][i][1] = acc[tp][i][2] = acc[tp][i][3] = 0.f;
  for (int uu = 0; uu < kWUnits; ++uu) {
    const long long unit = (long long)chunk * kWUnits + uu;
    if (unit >= n_units) break;
    const int xt = (int)(unit % tiles_x);
    const long long r0 = unit / tiles_x;
    const int y = (int)(r0 % H);
    const long long b = r0 / H;
    const int x0 = xt * kRowPx;
    // G^T of the segment: 64 pixels x 32 c_out, in units of 4 channels
    for (int e = tid; e < kRowPx * 8; e += 128) {
      const int px = e >> 3, q = e & 7;
      const int x = x0 + px, co = m0 + q * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (x < W && co < Cout) v = *reinterpret_cast<const float4*>(G + ((b * H + y) * W + x) * Cout + co);
      Gs[q * 4 + 0][px] = __float2bfloat16_rn(v.x);
      Gs[q * 4 + 1][px] = __float2bfloat16_rn(v.y);
      Gs[q * 4 + 2][px] = __float2bfloat16_rn(v.z);
      Gs[q * 4 + 3][px] = __float2bfloat16_rn(v.w);
    }
    // input rows y-1..y+1, columns x0-1..x0+64 (column c at index c), 32 c_in
    for (int e = tid; e < 3 * kRowCols * 8; e += 128) {
      const int r = e / (kRowCols * 8), rem = e - r * (kRowCols * 8);
      const int col = rem >> 3, q = rem & 7;
      const int yy = y + r - 1, xx = x0 + col - 1, ci = c00 + q * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (yy >= 0 && yy < H && xx >= 0 && xx < W && ci < Cin)
        v = *reinterpret_cast<const float4*>(X + ((b * H + yy) * W + xx) * Cin + ci);
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y);
      const __nv_bfloat16 h2 = __float2bfloat16_rn(v.z), h3 = __float2bfloat16_rn(v.w);
      Xs[0][r][q * 4 + 0][col] = h0;
      Xs[0][r][q * 4 + 1][col] = h1;
      Xs[0][r][q * 4 + 2][col] = h2;
      Xs[0][r][q * 4 + 3][col] = h3;
      if (col >= 1) {
        Xs[1][r][q * 4 + 0][col - 1] = h0;
        Xs[1][r][q * 4 + 1][col - 1] = h1;
        Xs[1][r][q * 4 + 2][col - 1] = h2;
        Xs[1][r][q * 4 + 3][col - 1] = h3;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kRowPx / 16; ++kk) {
      const int kc = kk * 16 + 2 * tq;  // pixel of the operand pair
      const uint32_t a0 = lds32(&Gs[wm * 16 + g][kc]);
      const uint32_t a1 = lds32(&Gs[wm * 16 + g + 8][kc]);
      const uint32_t a2 = lds32(&Gs[wm * 16 + g][kc + 8]);
      const uint32_t a3 = lds32(&Gs[wm * 16 + g + 8][kc + 8]);
#pragma unroll
      for (int tp = 0; tp < 9; ++tp) {
        const int ky = tp / 3, kx = tp % 3;
        // pixel p meets input column p + kx: even offsets from copy 0, odd from copy 1
        const int sh = kx & 1, off = kx - sh;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int n = wn * 16 + nt * 8 + g;
          const uint32_t b0 = lds32(&Xs[sh][ky][n][kc + off]);
          const uint32_t b1 = lds32(&Xs[sh][ky][n][kc + off + 8]);
          mma_bf16(acc[tp][nt], a0, a1, a2, a3, b0, b1);
        }
      }
    }
    __syncthreads();
  }
  float* out = part + (long long)chunk * Cout * 9 * Cin;
#pragma unroll
  for (int tp = 0; tp < 9; ++tp)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int ci = c00 + wn * 16 + nt * 8 + 2 * tq;
      if (ci >= Cin) continue;
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const int co = m0 + wm * 16 + g + hr * 8;
        if (co >= Cout) continue;
        *reinterpret_cast<float2*>(out + ((long long)co * 9 + tp) * Cin + ci) =
            make_float2(acc[tp][nt][2 * hr], acc[tp][nt][2 * hr + 1]);
      }
    }
}

// Weight-gradient partials on the tensor cores (tcgen05, accumulators in
// TMEM), same partial layout and chunking as k_conv3x3_wgrad:
// part[chunk][co][tap][ci] = sum_{p in chunk} G[p][co] X[p + tap][ci].
// GEMM per tap: M = c_out (128 rows, zero beyond Cout), N = 32 c_in of the
// CTA's tile, K = pixels.  Both operands are staged MN-major as BF16: for
// each group of 8 channels the pixels of the segment follow one another at
// 16 bytes, so the operand of input column shift dx starts 16 dx bytes
// later in the same staged row and every shift reads one copy.  A CTA takes
// one row shift dy and the three column shifts, 3 x 32 TMEM
// columns; per 64-pixel segment it issues 4 (K steps of 16) x 3 MMAs.  The
// MMA wait is bounded as in k_conv3x3_tc.  grid = chunks x c_in tiles x 3.
constexpr int kWtM = 128;                 // c_out rows of the MMA
constexpr int kWtN = 32;                  // c_in per CTA
constexpr int kWtCols = kRowPx + 2;       // staged input columns x0-1 .. x0+64
constexpr int kWtABytes = (kWtM / 8) * kRowPx * 16;
constexpr int kWtBBytes = (kWtN / 8) * kWtCols * 16;
constexpr int kWtSmem = kWtABytes + kWtBBytes + 32;

__global__ void __launch_bounds__(128) k_conv3x3_wgrad_tc(const float* __restrict__ G, const float* __restrict__ X,
                                                          float* __restrict__ part, int B, int H, int W, int Cin,
                                                          int Cout, int* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* As = sm;
  unsigned char* Bs = sm + kWtABytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bs + kWtBBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ int skip;
  if (tid == 0) skip = *reinterpret_cast<volatile int*>(status);
  __syncthreads();
  if (skip) return;
  // the CTAs of a chunk (3 row shifts x input-channel tiles) are
  // neighbours, so they run together and re-reads of its operand rows hit L2
  const int n_ct = (Cin + kWtN - 1) / kWtN;
  const int dy = blockIdx.x % 3;
  const int c00 = (blockIdx.x / 3 % n_ct) * kWtN;
  const int chunk = blockIdx.x / (3 * n_ct);
  const int tiles_x = W / kRowPx;
  const long long n_units = (long long)B * H * tiles_x;
  constexpr uint32_t ncols = 128u;  // 3 x 32 accumulator columns
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // kind::f16, BF16 x BF16 -> FP32, M = 128, N = 32, A and B MN-major
  const uint32_t idesc = umma_idesc_bf16(kWtM, kWtN) | (1u << 15) | (1u << 16);
  bool ok = true;
  int done_units = 0;
  uint32_t phase = 0u;
  // the operands of the next segment are loaded into registers while the
  // MMAs of the current one run: A items u = tid + 128 k (k < 8), B items
  // u = tid + 128 k (k < 3, u < 264)
  constexpr int kAI = kRowPx * (kWtM / 8) / 128, kBI = (kWtCols * (kWtN / 8) + 127) / 128;
  float4 ra[kAI][2], rb[kBI][2];
  auto load_unit = [&](long long unit) {
    const int xt = (int)(unit % tiles_x);
    const long long r0 = unit / tiles_x;
    const int y = (int)(r0 % H);
    const long long b = r0 / H;
    const int x0 = xt * kRowPx, yy = y + dy - 1;
#pragma unroll
    for (int k = 0; k < kAI; ++k) {
      const int u = tid + 128 * k;
      const int g = u % (kWtM / 8), px = u / (kWtM / 8);
      ra[k][0] = ra[k][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (g * 8 < Cout) {
        const float4* src = reinterpret_cast<const float4*>(G + ((b * H + y) * W + x0 + px) * Cout + g * 8);
        ra[k][0] = src[0];
        ra[k][1] = src[1];
      }
    }
#pragma unroll
    for (int k = 0; k < kBI; ++k) {
      const int u = tid + 128 * k;
      const int g = u % (kWtN / 8), col = u / (kWtN / 8);
      const int xx = x0 + col - 1, ci = c00 + g * 8;
      rb[k][0] = rb[k][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (u < kWtCols * (kWtN / 8) && yy >= 0 && yy < H && xx >= 0 && xx < W && ci < Cin) {
        const float4* src = reinterpret_cast<const float4*>(X + ((b * H + yy) * W + xx) * Cin + ci);
        rb[k][0] = src[0];
        rb[k][1] = src[1];
      }
    }
  };
  auto pack = [](const float4& lo, const float4& hi) {
    uint4 pk;
    pk.x = pack_bf16x2(lo.x, lo.y);
    pk.y = pack_bf16x2(lo.z, lo.w);
    pk.z = pack_bf16x2(hi.x, hi.y);
    pk.w = pack_bf16x2(hi.z, hi.w);
    return pk;
  };
  const long long first = (long long)chunk * kWUnits;
  if (first < n_units) load_unit(first);
  for (int uu = 0; uu < kWUnits; ++uu) {
    const long long unit = first + uu;
    if (unit >= n_units) break;
    // A: [c_out group of 8][pixel][8 c_out]; B: input row y + dy - 1, columns
    // x0 - 1 .. x0 + 64, [c_in group][column][8 c_in]
#pragma unroll
    for (int k = 0; k < kAI; ++k) {
      const int u = tid + 128 * k;
      const int g = u % (kWtM / 8), px = u / (kWtM / 8);
      *reinterpret_cast<uint4*>(As + ((size_t)g * kRowPx + px) * 16) = pack(ra[k][0], ra[k][1]);
    }
#pragma unroll
    for (int k = 0; k < kBI; ++k) {
      const int u = tid + 128 * k;
      if (u < kWtCols * (kWtN / 8)) {
        const int g = u % (kWtN / 8), col = u / (kWtN / 8);
        *reinterpret_cast<uint4*>(Bs + ((size_t)g * kWtCols + col) * 16) = pack(rb[k][0], rb[k][1]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < kRowPx / 16; ++ks)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          // MN-major: leading offset between groups of 8 pixels along K
          // (contiguous, 128 bytes), stride offset between groups of 8
          // channels along M / N
          const uint64_t ad = umma_desc(smem_u32(As + (size_t)(ks * 16) * 16), 128, kRowPx * 16);
          const uint64_t bd = umma_desc(smem_u32(Bs + (size_t)(ks * 16 + dx) * 16), 128, kWtCols * 16);
          const uint32_t acc = (uu > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(dx * kWtN)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    if (uu + 1 < kWUnits && unit + 1 < n_units) load_unit(unit + 1);
    // the staged operands are rewritten only after this segment's MMAs
    const bool fin = tc_wait(mbar, phase);
    if (!__syncthreads_and((int)fin)) {
      ok = false;
      break;
    }
    phase ^= 1u;
    ++done_units;
  }
  if (!ok && tid == 0) atomicExch(status, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok && done_units > 0) {
    // warp w reads TMEM lanes 32 w .. 32 w + 31 (c_out = lane row)
    const int co = warp * 32 + lane;
    float* out = part + (long long)chunk * Cout * 9 * Cin;
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      float v[32];
      tmem_ld32<32>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dx * kWtN), v);
      if (co < Cout) {
        float* dst = out + ((long long)co * 9 + dy * 3 + dx) * Cin + c00;
        const int nv = Cin - c00 < kWtN ? Cin - c00 : kWtN;
#pragma unroll
        for (int j = 0; j < kWtN; j += 4) {
          if (j >= nv) break;
          *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
  }
}

// Bias-gradient partials: part[chunk][co] = sum_{p in chunk} G[p][co], pixels
// in order.  grid = chunks, block = Cout threads.
__global__ void k_bias_partial(const float* __restrict__ G, float* __restrict__ part, long long P, int Cout) {
  // threadIdx.x = c_out, threadIdx.y = stripe: stripe k sums the chunk's
  // pixels p = k, k + 4, ... in order; the four stripes are added in order
  __shared__ float red[4][256];  // Cout <= 256
  const int co = threadIdx.x, k = threadIdx.y;
  const long long pbeg = (long long)blockIdx.x * kWChunk;
  const long long pend = pbeg + kWChunk < P ? pbeg + kWChunk : P;
  float s = 0.f;
  for (long long p = pbeg + k; p < pend; p += 4) s += G[p * Cout + co];
  red[k][co] = s;
  __syncthreads();
  if (k == 0) part[(long long)blockIdx.x * Cout + co] = ((red[0][co] + red[1][co]) + red[2][co]) + red[3][co];
}

// out[j] = sum_{c = 0..n-1} part[c][j], deterministic: 32 j per block
// (threadIdx.x), eight stripes of chunks c = y, y + 8, ... summed in order
// (threadIdx.y = y), the stripes added in order.
__global__ void k_sum_chunks(const float* __restrict__ part, int n, long long len, float* __restrict__ out) {
  __shared__ float red[8][32];
  const long long j = (long long)blockIdx.x * 32 + threadIdx.x;
  const int y = threadIdx.y;
  float s = 0.f;
  if (j < len)
    for (int c = y; c < n; c += 8) s += part[(long long)c * len + j];
  red[y][threadIdx.x] = s;
  __syncthreads();
  if (y == 0 && j < len) {
    float t = red[0][threadIdx.x];
#pragma unroll
    for (int k = 1; k < 8; ++k) t += red[k][threadIdx.x];
    out[j] = t;
  }
}

}  // namespace nop
}  // namespace lbmib

namespace lbmib {
namespace nop {

// The resampling and elementwise kernels work on float4 groups of channels
// (C is a multiple of 16).  The resampling ones take one image row per
// blockIdx.y (grid-stride over rows = b H + y of the tensor they iterate)
// and (x, channel group) along blockIdx.x, with 32-bit index arithmetic.

// 2x2 average pooling: out (H/2 x W/2) = mean of the four children, summed
// in the order (2y,2x), (2y,2x+1), (2y+1,2x), (2y+1,2x+1).
__global__ void k_pool2(const float* __restrict__ in, float* __restrict__ out, int rows, int Ho, int Wo, int C) {
  const int C4 = C >> 2, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Wo * C4) return;
  const int x = j / C4, c4 = j - x * C4;
  const int Wi = 2 * Wo;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int y = r % Ho;
    const long long b = r / Ho;
    const float4* p0 = reinterpret_cast<const float4*>(in + ((b * 2 * Ho + 2 * y) * Wi + 2 * x) * C) + c4;
    const float4 a = p0[0], bq = p0[C4], c = p0[(long long)Wi * C4], d = p0[(long long)Wi * C4 + C4];
    float4 o;
    o.x = 0.25f * (((a.x + bq.x) + c.x) + d.x);
    o.y = 0.25f * (((a.y + bq.y) + c.y) + d.y);
    o.z = 0.25f * (((a.z + bq.z) + c.z) + d.z);
    o.w = 0.25f * (((a.w + bq.w) + c.w) + d.w);
    reinterpret_cast<float4*>(out + ((long long)r * Wo + x) * C)[c4] = o;
  }
}

// adjoint of k_pool2, accumulated: din(y, x) += dout(y/2, x/2) / 4
__global__ void k_pool2_bwd(const float* __restrict__ dout, float* __restrict__ din, int rows, int Hi, int Wi,
                            int C) {
  const int C4 = C >> 2, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Wi * C4) return;
  const int x = j / C4, c4 = j - x * C4;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int y = r % Hi;
    const long long b = r / Hi;
    const float4 g = reinterpret_cast<const float4*>(dout + ((b * (Hi / 2) + y / 2) * (Wi / 2) + x / 2) * C)[c4];
    float4* d = reinterpret_cast<float4*>(din + ((long long)r * Wi + x) * C) + c4;
    float4 o = *d;
    o.x += 0.25f * g.x;
    o.y += 0.25f * g.y;
    o.z += 0.25f * g.z;
    o.w += 0.25f * g.w;
    *d = o;
  }
}

// nearest-neighbour x2 up-sampling: out(y, x) = in(y/2, x/2)
__global__ void k_up2(const float* __restrict__ in, float* __restrict__ out, int rows, int Ho, int Wo, int C) {
  const int C4 = C >> 2, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Wo * C4) return;
  const int x = j / C4, c4 = j - x * C4;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int y = r % Ho;
    const long long b = r / Ho;
    reinterpret_cast<float4*>(out + ((long long)r * Wo + x) * C)[c4] =
        reinterpret_cast<const float4*>(in + ((b * (Ho / 2) + y / 2) * (Wo / 2) + x / 2) * C)[c4];
  }
}

// adjoint of k_up2, accumulated: din(y, x) += sum of the four children
__global__ void k_up2_bwd(const float* __restrict__ dout, float* __restrict__ din, int rows, int Hi, int Wi,
                          int C) {
  const int C4 = C >> 2, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Wi * C4) return;
  const int x = j / C4, c4 = j - x * C4;
  const int Wo = 2 * Wi;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int y = r % Hi;
    const long long b = r / Hi;
    const float4* p0 = reinterpret_cast<const float4*>(dout + ((b * 2 * Hi + 2 * y) * Wo + 2 * x) * C) + c4;
    const float4 a = p0[0], bq = p0[C4], c = p0[(long long)Wo * C4], d = p0[(long long)Wo * C4 + C4];
    float4* q = reinterpret_cast<float4*>(din + ((long long)r * Wi + x) * C) + c4;
    float4 o = *q;
    o.x += ((a.x + bq.x) + c.x) + d.x;
    o.y += ((a.y + bq.y) + c.y) + d.y;
    o.z += ((a.z + bq.z) + c.z) + d.z;
    o.w += ((a.w + bq.w) + c.w) + d.w;
    *q = o;
  }
}

// out = a + b (n4 float4 groups)
__global__ void k_add(const float4* __restrict__ a, const float4* __restrict__ b, float4* __restrict__ out,
                      long long n4) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 u = a[i], v = b[i];
  out[i] = make_float4(u.x + v.x, u.y + v.y, u.z + v.z, u.w + v.w);
}

// dst += src (n4 float4 groups)
__global__ void k_acc(const float4* __restrict__ src, float4* __restrict__ dst, long long n4) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 u = src[i];
  float4 v = dst[i];
  v.x += u.x;
  v.y += u.y;
  v.z += u.z;
  v.w += u.w;
  dst[i] = v;
}

// ReLU backward in place: g = g if y > 0 else 0 (y is the activation output)
__global__ void k_relu_mask(const float4* __restrict__ y, float4* __restrict__ g, long long n4) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 a = y[i];
  float4 v = g[i];
  if (!(a.x > 0.f)) v.x = 0.f;
  if (!(a.y > 0.f)) v.y = 0.f;
  if (!(a.z > 0.f)) v.z = 0.f;
  if (!(a.w > 0.f)) v.w = 0.f;
  g[i] = v;
}

// channel padding: dst[p][c] = c < Cs ? src[p][c] : 0 (Cd >= Cs)
__global__ void k_pad_channels(const float* __restrict__ src, float* __restrict__ dst, long long P, int Cs,
                               int Cd) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * Cd) return;
  const int c = (int)(i % Cd);
  const long long p = i / Cd;
  dst[i] = c < Cs ? src[p * Cs + c] : 0.f;
}

// channel cropping: dst[p][c] = src[p][c] for c < Cd (Cs >= Cd)
__global__ void k_crop_channels(const float* __restrict__ src, float* __restrict__ dst, long long P, int Cs,
                                int Cd) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * Cd) return;
  const int c = (int)(i % Cd);
  const long long p = i / Cd;
  dst[i] = src[p * Cs + c];
}

// Mean-squared error over the first Cr of Cp channels: per-block partial
// sums of (y - t)^2 (fixed tree order) and the output gradient
// dy = 2 (y - t) / count (zero in the padding channels).
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                      double* __restrict__ part, long long P, int Cp, int Cr, double inv_count) {
  __shared__ double red[256];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (i < P * Cp) {
    const int c = (int)(i % Cp);
    const long long p = i / Cp;
    float d = 0.f;
    if (c < Cr) {
      d = y[i] - t[p * Cr + c];
      e2 = (double)d * (double)d;
    }
    dy[i] = (float)(2.0 * inv_count) * d;
  }
  red[threadIdx.x] = e2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// loss = inv_count * sum_b part[b], blocks in order (one thread)
// one block of 1024 threads: thread t sums the partials of blocks t, t +
// 1024, ... in order, then a fixed-order tree (deterministic)
__global__ void k_mse_total(const double* __restrict__ part, int n, double inv_count, double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += 1024) s += part[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * inv_count;
}

// Adam with bias correction on the FP32 master weights.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Master FP32 layer (W[co][tap][ci] real sizes, then b[co]) -> padded BF16
// forward weights Wt[co][tap][ci], flipped transposed weights
// Wf[ci][8 - tap][co] for the input gradient, and the padded FP32 bias.
__global__ void k_prep_layer(const float* __restrict__ master, int cin, int cout, int cinp, int coutp,
                             __nv_bfloat16* __restrict__ Wt, __nv_bfloat16* __restrict__ Wf,
                             float* __restrict__ bias) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)coutp * 9 * cinp;
  if (i < coutp) bias[i] = i < cout ? master[(long long)cout * 9 * cin + i] : 0.f;
  if (i >= n) return;
  const int ci = (int)(i % cinp);
  const long long q = i / cinp;
  const int tap = (int)(q % 9);
  const int co = (int)(q / 9);
  const float w = (co < cout && ci < cin) ? master[((long long)co * 9 + tap) * cin + ci] : 0.f;
  const __nv_bfloat16 wb = __float2bfloat16_rn(w);
  Wt[i] = wb;
  Wf[((long long)ci * 9 + (8 - tap)) * coutp + co] = wb;
}

// FP32 operand form of the convolutions (the gradient-check mode of the
// network: no BF16 rounding of weights or activations, FP32 products and
// sums in a fixed order, CUDA cores).  Weights in the padded layouts of
// k_prep_layer: Wt32[co][tap][ci] and the flipped, transposed
// Wf32[ci][8 - tap][co].
__global__ void k_prep_layer_f32(const float* __restrict__ master, int cin, int cout, int cinp, int coutp,
                                 float* __restrict__ Wt32, float* __restrict__ Wf32) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)coutp * 9 * cinp;
  if (i >= n) return;
  const int ci = (int)(i % cinp);
  const long long q = i / cinp;
  const int tap = (int)(q % 9);
  const int co = (int)(q / 9);
  const float w = (co < cout && ci < cin) ? master[((long long)co * 9 + tap) * cin + ci] : 0.f;
  Wt32[i] = w;
  Wf32[((long long)ci * 9 + (8 - tap)) * coutp + co] = w;
}

// Y[p][co] (+)= sum over taps (row-major 3x3, offsets -1..1) and c_in of
// X[p + tap][ci] W32[co][tap][ci] (+ bias[co]), then ReLU if relu; zero
// padding outside the image; one thread per output value, sums in tap then
// channel order.
__global__ void k_conv3x3_f32(const float* __restrict__ X, const float* __restrict__ W32,
                              const float* __restrict__ bias, float* __restrict__ Y, int B, int H, int W, int Cin,
                              int Cout, int relu, int accumulate) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)B * H * W * Cout;
  if (i >= n) return;
  const int co = (int)(i % Cout);
  const long long p = i / Cout;
  const int x = (int)(p % W);
  const int y = (int)((p / W) % H);
  const long long b = p / ((long long)W * H);
  float acc = 0.f;
  for (int tap = 0; tap < 9; ++tap) {
    const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
    const float* xr = X + ((b * H + yy) * W + xx) * Cin;
    const float* wr = W32 + ((long long)co * 9 + tap) * Cin;
    for (int ci = 0; ci < Cin; ++ci) acc = fmaf(xr[ci], wr[ci], acc);
  }
  if (bias) acc += bias[co];
  if (relu) acc = fmaxf(acc, 0.f);
  Y[i] = accumulate ? Y[i] + acc : acc;
}

// Weight-gradient partials of the FP32 form: part[c][(co tap) ci] = sum over
// the pixels p of chunk c (pixels [c P_c, (c + 1) P_c), in order) of
// G[p][co] X[p + tap][ci]; the chunks are added in order by k_sum_chunks.
__global__ void k_conv3x3_wgrad_f32(const float* __restrict__ G, const float* __restrict__ X,
                                    float* __restrict__ part, int B, int H, int W, int Cin, int Cout,
                                    long long chunk_px) {
  const long long len = (long long)Cout * 9 * Cin;
  const long long j = (long long)blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= len) return;
  const int ci = (int)(j % Cin);
  const long long q = j / Cin;
  const int tap = (int)(q % 9);
  const int co = (int)(q / 9);
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const long long P = (long long)B * H * W;
  const long long p0 = (long long)blockIdx.x * chunk_px;
  const long long p1 = p0 + chunk_px < P ? p0 + chunk_px : P;
  float acc = 0.f;
  for (long long p = p0; p < p1; ++p) {
    const int x = (int)(p % W);
    const int y = (int)((p / W) % H);
    const int yy = y + dy, xx = x + dx;
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
    const long long pp = p + (long long)dy * W + dx;
    acc = fmaf(G[p * Cout + co], X[pp * Cin + ci], acc);
  }
  part[(long long)blockIdx.x * len + j] = acc;
}

// Padded weight / bias gradients -> the master layout of the layer.
__global__ void k_unpad_grad(const float* __restrict__ dW, const float* __restrict__ db, int cin, int cout,
                             int cinp, float* __restrict__ grad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)cout * 9 * cin;
  if (i < cout) grad[n + i] = db[i];
  if (i >= n) return;
  const int ci = (int)(i % cin);
  const long long q = i / cin;
  const int tap = (int)(q % 9);
  const int co = (int)(q / 9);
  grad[i] = dW[((long long)co * 9 + tap) * cinp + ci];
}

// He-uniform initialisation from splitmix64(seed, index): weights uniform in
// [-a, a] with a = sqrt(6 / (9 cin)), biases zero.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_init_layer(float* __restrict__ master, int cin, int cout, unsigned long long seed,
                             long long offset) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nw = (long long)cout * 9 * cin;
  if (i >= nw + cout) return;
  if (i >= nw) {
    master[i] = 0.f;
    return;
  }
  const unsigned long long r = splitmix64(seed ^ splitmix64((unsigned long long)(offset + i)));
  const float u = (float)(r >> 40) * (1.0f / 16777216.0f);
  const float a = sqrtf(6.0f / (9.0f * (float)cin));
  master[i] = (2.f * u - 1.f) * a;
}

// Network output (NHWC, Cp channels, first four used) -> solver fields in
// the solver's layout (x fastest): rho, u (two planes), T as doubles.
__global__ void k_to_fields(const float* __restrict__ y, int Cp, long long N, double o0, double o1, double o2,
                            double o3, double s0, double s1, double s2, double s3, double* __restrict__ rho,
                            double* __restrict__ u, double* __restrict__ T) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const float* q = y + p * Cp;
  rho[p] = o0 + s0 * (double)q[0];
  u[p] = o1 + s1 * (double)q[1];
  u[N + p] = o2 + s2 * (double)q[2];
  T[p] = o3 + s3 * (double)q[3];
}

}  // namespace nop
}  // namespace lbmib
