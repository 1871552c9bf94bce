// Immersed-boundary kernels (arXiv 2607.07432, Sec. 2.3-2.5), FP64.
//
// Setup (geometry only): node classification (Omega' = strict interior of
// the shape), one-sided d = 2 stencils and phi_l (Eq. phi), the spreading
// CSR (Eulerian side, rows = forced nodes ascending, entries = points
// ascending), the Lagrangian weights W_l (Eq. weight), the effective
// boundary X*_l (Eq. xeffect), d_BV and the d = 1 projection stencils.
//
// Per step: one warp per Lagrangian point interpolates the predicted
// density, momentum, velocity and temperature (Eq. int2) and u, T at the
// projection point (Eq. int1, d = 1) with shuffle reductions, reconstructs
// the target (Eqs. virtualdir, virtualneu) and forms F, W, Q (Eqs. fib2,
// wib2, qib2); one thread per CSR row then gathers the spread forcing
// (Eq. spr2) in a fixed order, so the step is deterministic without atomics.
#pragma once
#include <math_constants.h>

#include "grid.cuh"
#include "lattice.cuh"

namespace lbmib {

enum { kShapeSphere = 0, kShapeEllipse = 1, kShapePolygon = 2, kShapeMask = 3 };

struct ShapeDev {
  int kind;
  double c[3];
  double r;
  double ra, rb, cs, sn;
  int n_poly;
  const double* poly;
  const unsigned char* mask;
};

// Q18: strict interior, evaluated in FP64 with explicitly rounded
// operations (no fused multiply-add) so that the classification is
// bit-identical to a plain IEEE evaluation in the same order.
static __global__ void k_classify(Grid g, int D, ShapeDev s, unsigned char* inside) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const int x = int(n % g.n[0]);
  const int y = int((n / g.n[0]) % g.n[1]);
  const int z = int(n / ((long long)g.n[0] * g.n[1]));
  const double p[3] = {double(x), double(y), double(z + g.zoff)};
  bool in = false;
  if (s.kind == kShapeMask) {
    in = s.mask[n] != 0;
  } else if (s.kind == kShapeSphere) {
    double d2 = 0.0;
    for (int a = 0; a < D; ++a) {
      const double da = __dsub_rn(p[a], s.c[a]);
      d2 = a == 0 ? __dmul_rn(da, da) : __dadd_rn(d2, __dmul_rn(da, da));
    }
    in = d2 < __dmul_rn(s.r, s.r);
  } else if (s.kind == kShapeEllipse) {
    const double dx = __dsub_rn(p[0], s.c[0]);
    const double dy = __dsub_rn(p[1], s.c[1]);
    const double xr = __dadd_rn(__dmul_rn(dx, s.cs), __dmul_rn(dy, s.sn));
    const double yr = __dsub_rn(__dmul_rn(dy, s.cs), __dmul_rn(dx, s.sn));
    const double q1 = __ddiv_rn(xr, s.ra);
    const double q2 = __ddiv_rn(yr, s.rb);
    in = __dadd_rn(__dmul_rn(q1, q1), __dmul_rn(q2, q2)) < 1.0;
  } else if (s.kind == kShapePolygon) {
    const double px = p[0], py = p[1];
    for (int k = 0; k < s.n_poly; ++k) {
      const int k2 = (k + 1) % s.n_poly;
      const double ax = s.poly[2 * k], ay = s.poly[2 * k + 1];
      const double bx = s.poly[2 * k2], by = s.poly[2 * k2 + 1];
      const bool crosses = (ay > py) != (by > py);
      double xint = CUDART_INF;
      if (by != ay) {
        const double t = __ddiv_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(py, ay)), __dsub_rn(by, ay));
        xint = __dadd_rn(t, ax);
      }
      if (crosses && (px < xint)) in = !in;
    }
  }
  inside[n] = in ? 1 : 0;
}

// Correctly rounded cosine for |x| <= pi, so that the kernel weights are
// the unique IEEE doubles nearest to the exact values (any correctly
// rounded evaluation agrees bit for bit).  Double-double arithmetic
// (Dekker / Knuth error-free transforms), reduction by k pi/2 with a
// two-term pi/2, Taylor series of sin / cos on |y| <= pi/4 to 1/29!.
struct dd {
  double hi, lo;
};
static __device__ __forceinline__ dd dd_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
static __device__ __forceinline__ dd dd_quick(double a, double b) {
  const double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
static __device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  return dd_quick(s.hi, __dadd_rn(s.lo, __dadd_rn(a.lo, b.lo)));
}
static __device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const double p = __dmul_rn(a.hi, b.hi);
  const double e = __fma_rn(a.hi, b.hi, -p);
  return dd_quick(p, __dadd_rn(e, __dadd_rn(__dmul_rn(a.hi, b.lo), __dmul_rn(a.lo, b.hi))));
}
static __device__ double cos_rn(double x) {
  // 1/n! as double-double, n = 0..29 (computed to 300 bits, split hi + lo)
  const double IF[30][2] = {
      {0x1.0p+0, 0.0}, {0x1.0p+0, 0.0}, {0x1.0p-1, 0.0},
      {0x1.5555555555555p-3, 0x1.5555555555555p-57}, {0x1.5555555555555p-5, 0x1.5555555555555p-59},
      {0x1.1111111111111p-7, 0x1.1111111111111p-63}, {0x1.6c16c16c16c17p-10, -0x1.f49f49f49f49fp-65},
      {0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-73}, {0x1.a01a01a01a01ap-16, 0x1.a01a01a01a01ap-76},
      {0x1.71de3a556c734p-19, -0x1.c154f8ddc6c00p-73}, {0x1.27e4fb7789f5cp-22, 0x1.cbbc05b4fa99ap-76},
      {0x1.ae64567f544e4p-26, -0x1.c062e06d1f209p-80}, {0x1.1eed8eff8d898p-29, -0x1.2aec959e14c06p-83},
      {0x1.6124613a86d09p-33, 0x1.f28e0cc748ebep-87}, {0x1.93974a8c07c9dp-37, 0x1.05d6f8a2efd1fp-92},
      {0x1.ae7f3e733b81fp-41, 0x1.1d8656b0ee8cbp-97}, {0x1.ae7f3e733b81fp-45, 0x1.1d8656b0ee8cbp-101},
      {0x1.952c77030ad4ap-49, 0x1.ac981465ddc6cp-103}, {0x1.6827863b97d97p-53, 0x1.eec01221a8b0bp-107},
      {0x1.2f49b46814157p-57, 0x1.2650f61dbdcb4p-112}, {0x1.e542ba4020225p-62, 0x1.ea72b4afe3c2fp-120},
      {0x1.71b8ef6dcf572p-66, -0x1.d043ae40c4647p-120}, {0x1.0ce396db7f853p-70, -0x1.aebcdbd20331cp-124},
      {0x1.761b41316381ap-75, -0x1.3423c7d91404fp-130}, {0x1.f2cf01972f578p-80, -0x1.9ada5fcc1ab14p-135},
      {0x1.3f3ccdd165fa9p-84, -0x1.58ddadf344487p-139}, {0x1.88e85fc6a4e5ap-89, -0x1.71c37ebd16540p-143},
      {0x1.d1ab1c2dccea3p-94, 0x1.054d0c78aea14p-149}, {0x1.0a18a2635085dp-98, 0x1.b9e2e28e1aa54p-153},
      {0x1.259f98b4358adp-103, 0x1.eaf8c39dd9bc5p-157}};
  const double PIO2_HI = 0x1.921fb54442d18p+0, PIO2_LO = 0x1.1a62633145c07p-54;
  const double k = rint(x / PIO2_HI);
  dd y = dd_two_sum(x, -k * PIO2_HI);  // k in [-2, 2]: k * PIO2_HI is exact
  y = dd_add(y, {-k * PIO2_LO, 0.0});
  const dd y2 = dd_mul(y, y);
  const int q = (((int)k) % 4 + 4) % 4;
  const int first = (q & 1) ? 29 : 28;  // odd terms for sin, even for cos
  dd p = {IF[first][0], IF[first][1]};
  for (int n = first - 2; n >= 0; n -= 2) {
    p = dd_mul(p, y2);
    p = {-p.hi, -p.lo};
    p = dd_add(p, {IF[n][0], IF[n][1]});
  }
  if (q & 1) p = dd_mul(p, y);
  double r = p.hi + p.lo;
  if (q == 1 || q == 2) r = -r;
  return r;
}

static __device__ __forceinline__ double delta_tilde(double r, double d) {
  return (1.0 / (2.0 * d)) * (1.0 + cos_rn((CUDART_PI * r) / d));
}

struct IBSetupDev {
  int D, NL, one_sided;
  double d_n;
  const double* X;
  const double* nrm;
  const unsigned char* inside;
  int* sten_node;   // NL*KS, -1 = empty slot
  double* sten_w;   // NL*KS, delta_il
  double* sten_x;   // NL*KS*3, unwrapped node coordinates
  double* phi;      // NL
  int* psten_node;  // NL*KP
  double* psten_w;  // NL*KP
  int* err;         // geometry error flag
};

// one thread per point: d = 2 one-sided stencil and phi_l; projection
// point and its d = 1 stencil over Omega.
static __global__ void k_stencils(Grid g, IBSetupDev s) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= s.NL) return;
  const int D = s.D;
  const int KS = D == 2 ? 16 : 64;
  const int KP = D == 2 ? 4 : 8;
  double X[3] = {0, 0, 0};
  int base[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    X[a] = s.X[l * D + a];
    base[a] = int(floor(X[a])) - 1;
  }
  double wsum = 0.0;
  int slot = 0;
  for (int oz = 0; oz < (D == 3 ? 4 : 1); ++oz)
    for (int oy = 0; oy < 4; ++oy)
      for (int ox = 0; ox < 4; ++ox, ++slot) {
        const int node[3] = {base[0] + ox, base[1] + oy, D == 3 ? base[2] + oz : 0};
        s.sten_node[l * KS + slot] = -1;
        s.sten_w[l * KS + slot] = 0.0;
        double r[3];
        bool inbox = true;
        for (int a = 0; a < D; ++a) {
          r[a] = double(node[a]) - X[a];
          if (fabs(r[a]) >= 2.0) inbox = false;
        }
        if (!inbox) continue;
        int idx[3] = {0, 0, 0};
        bool ok = true;
        for (int a = 0; a < D; ++a) {
          int v = node[a] - (a == 2 ? g.zoff : 0);
          if (g.per[a]) {
            v = v % g.n[a];
            if (v < 0) v += g.n[a];
          } else if (v < 0 || v >= g.n[a]) {
            ok = false;
          }
          idx[a] = v;
        }
        if (!ok) {
          atomicExch(s.err, 1);
          continue;
        }
        const long long lin = g.lin(idx[0], idx[1], idx[2]);
        if (s.one_sided && !s.inside[lin]) continue;
        double wt = 1.0;
        for (int a = 0; a < D; ++a) wt = wt * delta_tilde(r[a], 2.0);
        s.sten_node[l * KS + slot] = int(lin);
        s.sten_w[l * KS + slot] = wt;
        for (int a = 0; a < 3; ++a) s.sten_x[(l * KS + slot) * 3 + a] = double(node[a]);
        wsum += wt;
      }
  if (wsum == 0.0) atomicExch(s.err, 2);
  s.phi[l] = s.one_sided ? 1.0 / wsum : 1.0;
  // projection point (d = 1 over Omega)
  double P[3] = {0, 0, 0};
  int pb[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    P[a] = __dadd_rn(X[a], __dmul_rn(s.d_n, s.nrm[l * D + a]));
    pb[a] = int(floor(P[a]));
  }
  slot = 0;
  for (int oz = 0; oz < (D == 3 ? 2 : 1); ++oz)
    for (int oy = 0; oy < 2; ++oy)
      for (int ox = 0; ox < 2; ++ox, ++slot) {
        const int node[3] = {pb[0] + ox, pb[1] + oy, D == 3 ? pb[2] + oz : 0};
        s.psten_node[l * KP + slot] = -1;
        s.psten_w[l * KP + slot] = 0.0;
        double r[3];
        bool inbox = true;
        for (int a = 0; a < D; ++a) {
          r[a] = double(node[a]) - P[a];
          if (fabs(r[a]) >= 1.0) inbox = false;
        }
        if (!inbox) continue;
        int idx[3] = {0, 0, 0};
        bool ok = true;
        for (int a = 0; a < D; ++a) {
          int v = node[a] - (a == 2 ? g.zoff : 0);
          if (g.per[a]) {
            v = v % g.n[a];
            if (v < 0) v += g.n[a];
          } else if (v < 0 || v >= g.n[a]) {
            ok = false;
          }
          idx[a] = v;
        }
        if (!ok) {
          atomicExch(s.err, 1);
          continue;
        }
        double wt = 1.0;
        for (int a = 0; a < D; ++a) wt = wt * delta_tilde(r[a], 1.0);
        s.psten_node[l * KP + slot] = int(g.lin(idx[0], idx[1], idx[2]));
        s.psten_w[l * KP + slot] = wt;
      }
}

// CSR keys: node * (NL*KS) + l*KS + slot for every occupied slot
static __global__ void k_csr_keys(int NL, int KS, const int* sten_node, unsigned long long* keys, int* count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NL * KS) return;
  const int n = sten_node[t];
  if (n < 0) return;
  const int pos = atomicAdd(count, 1);
  keys[pos] = (unsigned long long)n * (unsigned long long)(NL * KS) + (unsigned long long)t;
}

// rows from the sorted keys: row starts where the node changes
static __global__ void k_csr_heads(int nnz, int NLKS, const unsigned long long* keys, int* head) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  head[e] = (e == 0 || keys[e] / NLKS != keys[e - 1] / NLKS) ? 1 : 0;
}

static __global__ void k_csr_fill(int nnz, int NLKS, int KS, const unsigned long long* keys, const int* head_scan,
                           int* row_ptr, int* cell_id, int* col, int* slot_of_entry) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const unsigned long long k = keys[e];
  const int n = int(k / NLKS);
  const int t = int(k % NLKS);
  const int r = head_scan[e] - 1;  // inclusive scan of the row-head flags
  if (e == 0 || keys[e - 1] / NLKS != (unsigned long long)n) {
    row_ptr[r] = e;
    cell_id[r] = n;
  }
  col[e] = t / KS;
  slot_of_entry[e] = t;
}

// s_i = sum_k phi_k delta_ik (inner sum of Eq. weight), per row in l order
static __global__ void k_row_density(int n_rows, const int* row_ptr, const int* slot_of_entry, const int* col,
                              const double* phi, const double* sten_w, double* s) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  double acc = 0.0;
  for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
    const double v = phi[col[e]] * sten_w[slot_of_entry[e]];
    acc = e == row_ptr[r] ? v : acc + v;
  }
  s[r] = acc;
}

static __device__ __forceinline__ int find_row(const int* cell_id, int n_rows, int node) {
  int lo = 0, hi = n_rows - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = cell_id[mid];
    if (v == node) return mid;
    if (v < node) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// Eq. weight, Eq. xeffect, d_BV (Q20)
static __global__ void k_weights(int D, int NL, int KS, int n_rows, const int* cell_id, const double* s_row,
                          const int* sten_node, const double* sten_w, const double* sten_x, const double* phi,
                          const double* X, const double* nrm, double* W, double* Xstar, double* dBV) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= NL) return;
  double acc = 0.0;
  double xs[3] = {0.0, 0.0, 0.0};
  bool first = true;
  for (int k = 0; k < KS; ++k) {
    const int n = sten_node[l * KS + k];
    if (n < 0) continue;
    const double w = sten_w[l * KS + k];
    const int r = find_row(cell_id, n_rows, n);
    const double v = (phi[l] * w) * s_row[r];
    acc = first ? v : acc + v;
    for (int a = 0; a < D; ++a) {
      const double t = sten_x[(l * KS + k) * 3 + a] * w;
      xs[a] = first ? t : xs[a] + t;
    }
    first = false;
  }
  W[l] = 1.0 / acc;
  double d = 0.0;
  for (int a = 0; a < D; ++a) {
    const double xa = phi[l] * xs[a];
    Xstar[l * D + a] = xa;
    const double t = (X[l * D + a] - xa) * nrm[l * D + a];
    d = a == 0 ? t : d + t;
  }
  dBV[l] = d > 0.0 ? d : 0.0;
}

static __global__ void k_csr_weights(int nnz, const int* col, const int* slot_of_entry, const double* phi,
                              const double* W, const double* sten_w, double* wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int l = col[e];
  wt[e] = phi[l] * W[l] * sten_w[slot_of_entry[e]];
}

static __global__ void k_row_map(int n_rows, const int* cell_id, int* row_of_node, unsigned char* forced) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  row_of_node[cell_id[r]] = r;
  forced[cell_id[r]] = 1;
}

// ---------------------------------------------------------------------------
// per step
// ---------------------------------------------------------------------------
struct IBStepDev {
  int NL, method, D;
  double d_n, Cv;
  const int* sten_node;
  const double* sten_w;
  const int* psten_node;
  const double* psten_w;
  const double* phi;
  const double* dBV;
  const int* tbc;
  const double* uB;
  const double* tB;
  double* G;       // NL*(D+2): F_l (D), W^IB_l, Q_l
};

static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// predicted moments of one node (Sec. 2.2) from the carried moments rho,
// rho u, rho E, evaluated in the compute type C (the precision of the
// stored state) and widened to FP64 for the Lagrangian sums.
template <class L, class C>
__device__ __forceinline__ void node_pred_c(const C* M, long long N, long long n, C& rho_o, C* j_o, C* u_o,
                                            C& T_o, C Cv) {
  constexpr int D = L::D;
  C rho, j[3], En;
  rho = M[n];
#pragma unroll
  for (int a = 0; a < D; ++a) j[a] = M[(1 + a) * N + n];
  En = M[(1 + D) * N + n];
  C uu = C(0), u[3], T;
  if constexpr (sizeof(C) == 8) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u[a] = j[a] / rho;
      uu += u[a] * u[a];
    }
    T = (En / rho - C(0.5) * uu) / Cv;
  } else {
    const C ir = C(1) / rho;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u[a] = j[a] * ir;
      uu += u[a] * u[a];
    }
    T = (En * ir - C(0.5) * uu) * (C(1) / Cv);
  }
  rho_o = rho;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    j_o[a] = j[a];
    u_o[a] = u[a];
  }
  T_o = T;
}

template <class L, class C>
__device__ __forceinline__ void node_pred(const C* M, long long N, long long n, double& rho_o, double* j_o,
                                          double* u_o, double& T_o, C Cv) {
  C rho, j[3], u[3], T;
  node_pred_c<L, C>(M, N, n, rho, j, u, T, Cv);
  rho_o = double(rho);
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    j_o[a] = double(j[a]);
    u_o[a] = double(u[a]);
  }
  T_o = double(T);
}



// Points per warp of k_ib_force and warps per block.
constexpr int kIBPointsPerWarp = 4;
constexpr int kIBWarps = 2;

// Body of the IB force step for block blk (kIBWarps warps of
// kIBPointsPerWarp Lagrangian points each) of one case.  Warp w of the CTA
// stages in shared-memory slot w (NSLOT slots) and takes the points of warp
// w % kIBWarps of the block; a CTA of NSLOT warps runs NSLOT / kIBWarps
// such blocks at once (each caller passes its own blk).
template <class L, class S, class C, int NSLOT = kIBWarps>
__device__ __forceinline__ void ib_force_body(const Grid& g, const IBStepDev& s, const C* M, int blk) {
  constexpr int D = L::D;
  constexpr int KS = D == 2 ? 16 : 64;
  constexpr int KP = D == 2 ? 4 : 8;
  constexpr int NV = 2 + 2 * D;
  constexpr int NP = kIBPointsPerWarp;
  static_assert(NP * 8 == 32 && NV <= 8, "one lane per (point, quantity)");
  // slot values staged per (point, quantity) row, slots contiguous; rows
  // padded by one so that a lane per row reads distinct banks
  static_assert(NSLOT % kIBWarps == 0, "whole blocks per CTA");
  __shared__ double stage[NSLOT][NP * NV][KS + 1];
  __shared__ double pstage[NSLOT][NP * (D + 1)][KP + 1];
  const int wsl = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int l0 = (blk * kIBWarps + wsl % kIBWarps) * NP;
  if (l0 >= s.NL) return;
  // Eq. int2: every lane evaluates stencil slots of each of the warp's points
#pragma unroll 1
  for (int p = 0; p < NP; ++p) {
    const int l = l0 + p;
    if (l >= s.NL) break;
#pragma unroll
    for (int rep = 0; rep < (KS + 31) / 32; ++rep) {
      const int k = lane + 32 * rep;
      if (k < KS) {
        double v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = 0.0;
        const int n = s.sten_node[l * KS + k];
        if (n >= 0) {
          if constexpr (sizeof(C) == 8) {
            const double w = s.sten_w[l * KS + k];
            double rho, j[3], u[3], T;
            node_pred<L, C>(M, g.N, n, rho, j, u, T, C(s.Cv));
            v[0] = rho * w;
#pragma unroll
            for (int a = 0; a < D; ++a) {
              v[1 + a] = j[a] * w;
              v[1 + D + a] = u[a] * w;
            }
            v[1 + 2 * D] = T * w;
          } else {
            // FP32 state: the slot products in FP32, their sums in FP64
            const C w = C(s.sten_w[l * KS + k]);
            C rho, j[3], u[3], T;
            node_pred_c<L, C>(M, g.N, n, rho, j, u, T, C(s.Cv));
            v[0] = double(rho * w);
#pragma unroll
            for (int a = 0; a < D; ++a) {
              v[1 + a] = double(j[a] * w);
              v[1 + D + a] = double(u[a] * w);
            }
            v[1 + 2 * D] = double(T * w);
          }
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) stage[wsl][p * NV + q][k] = v[q];
      }
    }
  }
  // Eq. int1 at the projection points: lane (p, k) evaluates slot k of
  // point p, all of the warp's points in one pass
  {
    const int p = lane >> 3, k = lane & 7;
    const int l = l0 + p;
    if (k < KP && l < s.NL) {
      double pv[D + 1];
#pragma unroll
      for (int q = 0; q < D + 1; ++q) pv[q] = 0.0;
      const int n = s.psten_node[l * KP + k];
      if (n >= 0) {
        const double w = s.psten_w[l * KP + k];
        double rho, j[3], u[3], T;
        node_pred<L, C>(M, g.N, n, rho, j, u, T, C(s.Cv));
#pragma unroll
        for (int a = 0; a < D; ++a) pv[a] = u[a] * w;
        pv[D] = T * w;
      }
#pragma unroll
      for (int q = 0; q < D + 1; ++q) pstage[wsl][p * (D + 1) + q][k] = pv[q];
    }
  }
  __syncwarp();
  // lane (p, q) adds quantity q of point p over the slots in slot order
  // (z, y, x), the order of a plain sequential sum, so FP64 results are
  // reproducible bit for bit
  {
    const int p = lane >> 3, q = lane & 7;
    if (l0 + p < s.NL) {
      if (q < NV) {
        double a_ = 0.0;
        for (int k = 0; k < KS; ++k) a_ = a_ + stage[wsl][p * NV + q][k];
        stage[wsl][p * NV + q][0] = a_;
      }
      if (q < D + 1) {
        double a_ = 0.0;
        for (int k = 0; k < KP; ++k) a_ = a_ + pstage[wsl][p * (D + 1) + q][k];
        pstage[wsl][p * (D + 1) + q][0] = a_;
      }
    }
  }
  __syncwarp();
  if ((lane & 7) != 0) return;
  const int pp = lane >> 3;
  const int l = l0 + pp;
  if (l >= s.NL) return;
  double acc[NV], pacc[D + 1];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = stage[wsl][pp * NV + q][0];
#pragma unroll
  for (int q = 0; q < D + 1; ++q) pacc[q] = pstage[wsl][pp * (D + 1) + q][0];
  const double ph = s.phi[l];
  const double rho_s = ph * acc[0];
  double j_s[3], u_s[3], uP[3], uV[3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    j_s[a] = ph * acc[1 + a];
    u_s[a] = ph * acc[1 + D + a];
    uP[a] = pacc[a];
  }
  const double T_s = ph * acc[1 + 2 * D];
  const double TP = pacc[D];
  const double dn = s.d_n;
  const double dbv = s.dBV[l];
  double TV;
  const int neu = s.tbc ? s.tbc[l] : 0;
  const double tb = s.tB[l];
  if (s.method == 2) {
    // Eq. virtualdir (velocity) and Eq. virtualdir / virtualneu (temperature)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double ub = s.uB ? s.uB[l * D + a] : 0.0;
      uV[a] = ub - (dbv / dn) * (uP[a] - ub);
    }
    TV = neu ? TP - tb * (dn + dbv) : tb - (dbv / dn) * (TP - tb);
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) uV[a] = s.uB ? s.uB[l * D + a] : 0.0;
    TV = neu ? TP - tb * dn : tb;
  }
  // Eqs. fib2, wib2, qib2 (dt = 1)
  double uv2 = 0.0, us2 = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    s.G[l * (D + 2) + a] = 2.0 * (rho_s * uV[a] - j_s[a]);
    uv2 += uV[a] * uV[a];
    us2 += u_s[a] * u_s[a];
  }
  s.G[l * (D + 2) + D] = rho_s * (uv2 - us2) / 2.0;
  s.G[l * (D + 2) + D + 1] = s.Cv * rho_s * (TV - T_s);
}

template <class L, class S, class C>
static __global__ void __launch_bounds__(32 * kIBWarps) k_ib_force(Grid g, IBStepDev s, const C* M) {
  ib_force_body<L, S, C>(g, s, M, blockIdx.x);
}

// Several cases in one launch: work item = (case, block of the case).
template <class S, class C>
struct IBCaseDesc {
  Grid g;
  IBStepDev s;
  const C* M;
};

template <class L, class S, class C>
static __global__ void __launch_bounds__(32 * kIBWarps) k_ib_force_batched(const IBCaseDesc<S, C>* d,
                                                                           const int2* work) {
  const int2 w = work[blockIdx.x];
  const IBCaseDesc<S, C>& c = d[w.x];
  ib_force_body<L, S, C>(c.g, c.s, c.M, w.y);
}

// Eq. spr2 as an Eulerian-side gather: f_u, w + q of each forced node.
// Entries are fetched eight at a time (independent loads in flight) and
// added in CSR order.  acc receives f_u (D components) and w + q (slot 3).
__device__ __forceinline__ void spread_row(int D, int r, const int* row_ptr, const int* col, const double* wt,
                                           const double* G, double (&acc)[4]) {
  acc[0] = acc[1] = acc[2] = acc[3] = 0.0;
  const int e0 = row_ptr[r], e1 = row_ptr[r + 1];
  for (int eb = e0; eb < e1; eb += 8) {
    int lc[8];
    double wc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      lc[k] = eb + k < e1 ? col[eb + k] : -1;
      wc[k] = eb + k < e1 ? wt[eb + k] : 0.0;
    }
    double gv[8][4];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
      for (int a = 0; a < 4; ++a) gv[k][a] = 0.0;
      if (lc[k] >= 0) {
        const double* gl = G + (long long)lc[k] * (D + 2);
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (a < D) gv[k][a] = gl[a];
        gv[k][3] = gl[D] + gl[D + 1];
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (lc[k] < 0) break;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < D) acc[a] = acc[a] + wc[k] * gv[k][a];
      acc[3] = acc[3] + wc[k] * gv[k][3];
    }
  }
}

// Spreading and its application to the moments, several cases in one
// launch: the same sums and updates as k_ib_spread_apply, one row per
// thread.
template <class C>
struct SpreadCaseDesc {
  int D;
  long long N;
  int n_rows;
  const int* row_ptr;
  const int* col;
  const double* wt;
  const double* G;
  const int* cell_id;
  double* FU;
  double* WQ;
  C* M;
};

template <class C>
__device__ __forceinline__ void spread_apply_row(const SpreadCaseDesc<C>& c, int r) {
  if (r >= c.n_rows) return;
  const int D = c.D;
  double acc[4];
  spread_row(D, r, c.row_ptr, c.col, c.wt, c.G, acc);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < D) c.FU[(long long)r * D + a] = acc[a];
  c.WQ[r] = acc[3];
  const long long n = c.cell_id[r];
  const long long N = c.N;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < D) c.M[(1 + a) * N + n] = c.M[(1 + a) * N + n] + C(0.5) * C(acc[a]);
  c.M[(1 + D) * N + n] = c.M[(1 + D) * N + n] + C(acc[3]);
}

template <class C>
static __global__ void k_spread_apply_batched(const SpreadCaseDesc<C>* d, const int2* work) {
  const int2 w = work[blockIdx.x];
  spread_apply_row<C>(d[w.x], w.y * blockDim.x + threadIdx.x);
}

// One case: spreading (Eq. spr2, the sums of spread_row) and its application to the
// predicted moments in place, rho u += f_u / 2 and rho E += w + q on the
// row's node (Sec. 2.2, reading Q15), one thread per row.
template <class C>
static __global__ void k_ib_spread_apply(int D, long long N, int n_rows, const int* row_ptr, const int* col,
                                         const double* wt, const double* G, const int* cell_id, double* FU,
                                         double* WQ, C* M) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  double acc[4];
  spread_row(D, r, row_ptr, col, wt, G, acc);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < D) FU[(long long)r * D + a] = acc[a];
  WQ[r] = acc[3];
  const long long n = cell_id[r];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < D) M[(1 + a) * N + n] = M[(1 + a) * N + n] + C(0.5) * C(acc[a]);
  M[(1 + D) * N + n] = M[(1 + D) * N + n] + C(acc[3]);
}

// Wall diagnostics of the updated field (Sec. 3.1-3.2, reading Q26), one
// thread per Lagrangian point: p, u, T at X_l by Eq. int1 with d = 2 over
// Omega (nodes on both sides of the wall), u and T at the projection point
// P_l by Eq. int1 with d = 1 (the per-step stencils), then per point
//   C_p = (p^s - p_inf) / q_inf, tau_w = mu [(u^P - u^B) - normal part] / d_n,
//   u^s, T^s, (dT/dn)^s = (T^P - T^s) / d_n, and C_p at P_l (d = 1, fluid
//   nodes only)
// in out[l * (2D + 4) + ...] (C_p, tau_w[D], u^s[D], T^s, (dT/dn)^s, C_p^P).
struct DiagDev {
  int NL, D;
  double R, Cv, mu, d_n, p_inf, q_inf;
  const double* X;
  const double* nrm;
  const double* uB;
  const int* psten_node;
  const double* psten_w;
  double* out;
  int* err;
};

template <class L, class C>
static __global__ void k_wall_diag(Grid g, DiagDev d, const C* M) {
  constexpr int D = L::D;
  constexpr int KP = D == 2 ? 4 : 8;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= d.NL) return;
  double X[3] = {0, 0, 0};
  int base[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    X[a] = d.X[l * D + a];
    base[a] = int(floor(X[a])) - 1;
  }
  double ps = 0.0, us[3] = {0, 0, 0}, Ts = 0.0;
  for (int oz = 0; oz < (D == 3 ? 4 : 1); ++oz)
    for (int oy = 0; oy < 4; ++oy)
      for (int ox = 0; ox < 4; ++ox) {
        const int node[3] = {base[0] + ox, base[1] + oy, D == 3 ? base[2] + oz : 0};
        double r[3];
        bool inbox = true;
        for (int a = 0; a < D; ++a) {
          r[a] = double(node[a]) - X[a];
          if (fabs(r[a]) >= 2.0) inbox = false;
        }
        if (!inbox) continue;
        int idx[3] = {0, 0, 0};
        bool ok = true;
        for (int a = 0; a < D; ++a) {
          int v = node[a] - (a == 2 ? g.zoff : 0);
          if (g.per[a]) {
            v = v % g.n[a];
            if (v < 0) v += g.n[a];
          } else if (v < 0 || v >= g.n[a]) {
            ok = false;
          }
          idx[a] = v;
        }
        if (!ok) {
          atomicExch(d.err, 1);
          continue;
        }
        double wt = 1.0;
        for (int a = 0; a < D; ++a) wt = wt * delta_tilde(r[a], 2.0);
        double rho, j[3], u[3], T;
        node_pred<L, C>(M, g.N, g.lin(idx[0], idx[1], idx[2]), rho, j, u, T, C(d.Cv));
        ps = ps + ((rho * d.R) * T) * wt;
        for (int a = 0; a < D; ++a) us[a] = us[a] + u[a] * wt;
        Ts = Ts + T * wt;
      }
  double uP[3] = {0, 0, 0}, TP = 0.0, pP = 0.0;
  for (int k = 0; k < KP; ++k) {
    const int n = d.psten_node[l * KP + k];
    if (n < 0) continue;
    const double w = d.psten_w[l * KP + k];
    double rho, j[3], u[3], T;
    node_pred<L, C>(M, g.N, n, rho, j, u, T, C(d.Cv));
    for (int a = 0; a < D; ++a) uP[a] = uP[a] + u[a] * w;
    TP = TP + T * w;
    pP = pP + ((rho * d.R) * T) * w;
  }
  double du[3], dn = 0.0;
  for (int a = 0; a < D; ++a) {
    du[a] = uP[a] - (d.uB ? d.uB[l * D + a] : 0.0);
    dn = dn + du[a] * d.nrm[l * D + a];
  }
  double* o = d.out + (long long)l * (2 * D + 4);
  o[0] = (ps - d.p_inf) / d.q_inf;
  for (int a = 0; a < D; ++a) {
    o[1 + a] = d.mu * (du[a] - dn * d.nrm[l * D + a]) / d.d_n;
    o[1 + D + a] = us[a];
  }
  o[1 + 2 * D] = Ts;
  o[2 + 2 * D] = (TP - Ts) / d.d_n;
  o[3 + 2 * D] = (pP - d.p_inf) / d.q_inf;
}

// wall loads: fixed-order block reduction (deterministic)
// owned (optional, slabs): only points with owned[l] != 0 are summed
static __global__ void k_wall_loads(int D, int NL, const double* G, const double* W, const unsigned char* owned,
                                    double* out) {
  __shared__ double sh[256][5];
  const int t = threadIdx.x;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int l = t; l < NL; l += 256) {
    if (owned && !owned[l]) continue;
    const double w = W[l];
    for (int a = 0; a < D; ++a) acc[a] += G[l * (D + 2) + a] * w;
    acc[3] += G[l * (D + 2) + D + 1] * w;  // Q
    acc[4] += G[l * (D + 2) + D] * w;      // W^IB
  }
  for (int k = 0; k < 5; ++k) sh[t][k] = acc[k];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s)
      for (int k = 0; k < 5; ++k) sh[t][k] += sh[t + s][k];
    __syncthreads();
  }
  if (t == 0) {
    for (int a = 0; a < 3; ++a) out[a] = a < D ? -sh[0][a] : 0.0;
    out[3] = sh[0][3];
    out[4] = sh[0][4];
  }
}

}  // namespace lbmib
