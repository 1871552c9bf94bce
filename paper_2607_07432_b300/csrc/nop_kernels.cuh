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

// Bias-gradient partials: part[chunk][co] = sum_{p in chunk} G[p][co], pixels
// in order.  grid = chunks, block = Cout threads.
__global__ void k_bias_partial(const float* __restrict__ G, float* __restrict__ part, long long P, int Cout) {
  const int co = threadIdx.x;
  const long long pbeg = (long long)blockIdx.x * kWChunk;
  const long long pend = pbeg + kWChunk < P ? pbeg + kWChunk : P;
  float s = 0.f;
  for (long long p = pbeg; p < pend; ++p) s += G[p * Cout + co];
  part[(long long)blockIdx.x * Cout + co] = s;
}

// out[j] = sum_{c = 0..n-1} part[c][j] in chunk order (deterministic).
__global__ void k_sum_chunks(const float* __restrict__ part, int n, long long len, float* __restrict__ out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= len) return;
  float s = 0.f;
  for (int c = 0; c < n; ++c) s += part[(long long)c * len + j];
  out[j] = s;
}

}  // namespace nop
}  // namespace lbmib

namespace lbmib {
namespace nop {

// 2x2 average pooling: out (H/2 x W/2) = mean of the four children, summed
// in the order (2y,2x), (2y,2x+1), (2y+1,2x), (2y+1,2x+1).
__global__ void k_pool2(const float* __restrict__ in, float* __restrict__ out, long long n_out, int Ho, int Wo,
                        int C) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out) return;
  const int c = (int)(i % C);
  const long long q = i / C;
  const int x = (int)(q % Wo);
  const long long r = q / Wo;
  const int y = (int)(r % Ho);
  const long long b = r / Ho;
  const int Wi = 2 * Wo;
  const long long base = ((b * 2 * Ho + 2 * y) * Wi + 2 * x) * C + c;
  const float s = ((in[base] + in[base + C]) + in[base + (long long)Wi * C]) + in[base + (long long)Wi * C + C];
  out[i] = 0.25f * s;
}

// adjoint of k_pool2, accumulated: din(y, x) += dout(y/2, x/2) / 4
__global__ void k_pool2_bwd(const float* __restrict__ dout, float* __restrict__ din, long long n_in, int Hi,
                            int Wi, int C) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_in) return;
  const int c = (int)(i % C);
  const long long q = i / C;
  const int x = (int)(q % Wi);
  const long long r = q / Wi;
  const int y = (int)(r % Hi);
  const long long b = r / Hi;
  din[i] += 0.25f * dout[((b * (Hi / 2) + y / 2) * (Wi / 2) + x / 2) * C + c];
}

// nearest-neighbour x2 up-sampling: out(y, x) = in(y/2, x/2)
__global__ void k_up2(const float* __restrict__ in, float* __restrict__ out, long long n_out, int Ho, int Wo,
                      int C) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out) return;
  const int c = (int)(i % C);
  const long long q = i / C;
  const int x = (int)(q % Wo);
  const long long r = q / Wo;
  const int y = (int)(r % Ho);
  const long long b = r / Ho;
  out[i] = in[((b * (Ho / 2) + y / 2) * (Wo / 2) + x / 2) * C + c];
}

// adjoint of k_up2, accumulated: din(y, x) += sum of the four children
__global__ void k_up2_bwd(const float* __restrict__ dout, float* __restrict__ din, long long n_in, int Hi,
                          int Wi, int C) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_in) return;
  const int c = (int)(i % C);
  const long long q = i / C;
  const int x = (int)(q % Wi);
  const long long r = q / Wi;
  const int y = (int)(r % Hi);
  const long long b = r / Hi;
  const int Wo = 2 * Wi;
  const long long base = ((b * 2 * Hi + 2 * y) * Wo + 2 * x) * C + c;
  const float s = ((dout[base] + dout[base + C]) + dout[base + (long long)Wo * C]) + dout[base + (long long)Wo * C + C];
  din[i] += s;
}

// out = a + b
__global__ void k_add(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out,
                      long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + b[i];
}

// dst += src
__global__ void k_acc(const float* __restrict__ src, float* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] += src[i];
}

// ReLU backward in place: g = g if y > 0 else 0 (y is the activation output)
__global__ void k_relu_mask(const float* __restrict__ y, float* __restrict__ g, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(y[i] > 0.f)) g[i] = 0.f;
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
__global__ void k_mse_total(const double* __restrict__ part, int n, double inv_count, double* __restrict__ out) {
  double s = 0.0;
  for (int b = 0; b < n; ++b) s += part[b];
  *out = s * inv_count;
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
