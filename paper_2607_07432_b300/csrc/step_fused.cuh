// Fused time step: collision, pull streaming and the total-energy update in
// one pass over HBM (arXiv 2607.07432, Eq. LB, Eq. energy, Sec. 2.5 step 5).
//
// Each CTA owns a TX x TY column of the (x, y) plane and marches along z
// (2.5D blocking).  Shared memory holds two rings of planes:
//   * corrected macroscopic fields (rho, u, theta, rho E') of five planes
//     z-1..z+3 with a halo of two nodes in x and y (MUSCL stencils and the
//     velocity gradients of halo nodes), and
//   * post-collision populations of three planes z-1..z+1 with a halo of one
//     node (pull streaming and the face-crossing flux tables).
// Per plane: load the macros of plane z+3, collide plane z+1 (halo included),
// then stream, form the energy face fluxes and update rho E of plane z.
//
// Between steps the state carries, besides the populations, the predicted
// moments rho, rho u (sums of the streamed populations) and rho E of every
// node, so halo nodes cost D+2 values instead of Q populations.  The IB
// spreading kernel adds f_u/2 and w + q to those moments in place before
// this kernel runs; forced nodes then look up f_u for the force populations.
// In 2D the same kernel runs with a single plane.
#pragma once
#include "grid.cuh"
#include "physics.cuh"

namespace lbmib {

template <class S, class C>
struct FusedArgs {
  const S* f_in;       // Q*N populations of step n
  S* f_out;            // Q*N populations of step n+1
  const C* M_in;       // (D+2)*N: rho, rho u (+ f_u/2 on forced nodes), rho E (+ w + q)
  C* M_out;            // (D+2)*N: predicted moments of step n+1
  const C* Pp;         // N
  C* Pn;               // N
  const C* Ap;         // NDEV*N
  C* An;               // NDEV*N
  const unsigned char* forced;  // N flags (nullptr: no body)
  const int* cell_id;  // n_rows, ascending
  const int* row_of_node;  // N: CSR row of a forced node, -1 otherwise (nullptr: search cell_id)
  int n_rows;
  const double* FU;    // n_rows*D
  // The two x faces applied in the kernel (bc_fused != 0; their nodes are
  // one per grid row, so a separate kernel would touch a 32-byte sector per
  // value): a node on an inlet / far-field x face stores the free-stream
  // equilibrium and E_inf; a node on an outlet x face stores what its inner
  // neighbour stores (zero gradient), computed by the same operations from
  // the neighbour's data in shared memory.  The y and z faces, and
  // equilibrium on shared edges, follow in the boundary kernel.
  int bc_fused;
  int bct[2];          // LBM_BC_* of the x- and x+ faces
  const C* feq_inf;    // Q free-stream equilibrium populations
  C E_inf;
};

// Tile: one thread per node of the halo-1 region HX1 x HY1 (the collision
// region), interior TX x TY = (HX1-2) x (HY1-2).  The D3Q19 FP32 tile uses
// 512 threads and about 180 KB of shared memory.
template <class L, class C, int HY = 0>
struct FusedTile {
  static constexpr int HX1 = sizeof(C) == 8 ? 16 : 32;
  static constexpr int HY1 = HY ? HY : (sizeof(C) == 8 ? 8 : (L::D == 3 ? 16 : 8));
  static constexpr int TX = HX1 - 2, TY = HY1 - 2;
};

template <class L, class S, class C, int HY = 0>
struct FusedLayout {
  static constexpr int D = L::D;
  static constexpr int TX = FusedTile<L, C, HY>::TX, TY = FusedTile<L, C, HY>::TY;
  static constexpr int HX1 = TX + 2, HY1 = TY + 2, NH1 = HX1 * HY1;
  static constexpr int HX2 = TX + 4, HY2 = TY + 4, NH2 = HX2 * HY2;
  static constexpr int NT = NH1;
  // macro planes: iteration z reads planes z-1..z+2 and fills plane z+3;
  // plane z-2 was last read (z face of plane z-1) before the barrier that
  // opens iteration z, so its slot takes plane z+3
  static constexpr int RM = D == 3 ? 5 : 1;
  static constexpr int RF = D == 3 ? 3 : 1;   // f^col planes
  // corrected macros of a plane: rho, u (3 slots), theta, E' per node, kept
  // as vectors so that one shared-memory load reads several fields
  // (FP32: a float4 (rho, u) and a float2 (theta, E') array; FP64: three
  // double2 arrays (rho, u_x), (u_y, u_z), (theta, E')), 6 values per node
  static constexpr int NMF = 6;
  static constexpr int min_blocks = 1;
  static constexpr size_t bytes =
      sizeof(C) * ((size_t)RM * NMF * NH2 + (size_t)RF * L::Q * NH1 + 4 * (size_t)NH1);
};

__device__ __forceinline__ int find_row_dev(const int* cell_id, int n_rows, int node) {
  int lo = 0, hi = n_rows - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = __ldg(cell_id + mid);
    if (v == node) return mid;
    if (v < node) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// body of the fused step for the tile (bx, by) and z-chunk bz of one case
// NARROW: element offsets in 32 bits (the host takes it when Q N < 2^32)
template <class L, class S, class C, int HY, bool NARROW>
__device__ __forceinline__ void fused_body(const Grid& g, const FusedArgs<S, C>& a, const Phys<C>& ph, int zchunk,
                                           int bx, int by, int bz) {
  using Lay = FusedLayout<L, S, C, HY>;
  constexpr int D = L::D, Q = L::Q;
  constexpr int TX = Lay::TX, TY = Lay::TY, NT = Lay::NT;
  constexpr int HX2 = Lay::HX2, NH2 = Lay::NH2, HX1 = Lay::HX1, NH1 = Lay::NH1;
  constexpr int RM = Lay::RM, RF = Lay::RF, NMF = Lay::NMF;
  constexpr bool exact = std::is_same<C, double>::value;  // FP64: operations as in the oracle
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* mr = reinterpret_cast<C*>(smem_raw);        // [RM][6 NH2] vector arrays (see FusedLayout)
  C* fr = mr + (size_t)RM * NMF * NH2;           // [RF][Q][NH1]
  C* Fx = fr + (size_t)RF * Q * NH1;             // [2][NH1] +x face fluxes (plane parity)
  C* Fy = Fx + 2 * NH1;                          // [2][NH1] +y face fluxes
  const int t = threadIdx.x;
  const int cx = t % HX1, cy = t / HX1;          // halo-1 coordinates of this thread's node
  const int hx = cx + 1, hy = cy + 1;            // halo-2 coordinates
  const int x0 = bx * TX, y0 = by * TY;
  const int gx = x0 + cx - 1, gy = y0 + cy - 1;
  const int nz = g.n[2];
  const int z0 = D == 3 ? bz * zchunk : 0;
  const int z1 = D == 3 ? min(nz, z0 + zchunk) : 1;
  using Ix = std::conditional_t<NARROW, unsigned, long long>;
  const Ix N = (Ix)g.N;
  auto lin = [&](int x, int y, int z) { return (Ix)x + (Ix)g.n[0] * ((Ix)y + (Ix)g.n[1] * (Ix)z); };
  const bool interior = cx >= 1 && cx <= TX && cy >= 1 && cy <= TY && gx < g.n[0] && gy < g.n[1];
  const int wx = g.wrap(0, gx), wy = g.wrap(1, gy);

  // ring slots of plane z (z >= z0 - 3 >= -3 here): unsigned remainders
  auto mslot = [&](int z) { return D == 3 ? (int)((unsigned)(z + 4 * RM) % (unsigned)RM) : 0; };
  auto fslot = [&](int z) { return D == 3 ? (int)((unsigned)(z + 4 * RF) % (unsigned)RF) : 0; };
  auto halo2_node = [&](int k, int gz) {
    const int kx = k % HX2, ky = k / HX2;
    return lin(g.wrap(0, x0 + kx - 2), g.wrap(1, y0 + ky - 2), gz);
  };

  // corrected macros (rho, u, theta, rho E') of plane z over the halo-2 region,
  // from the moments rho, rho u, rho E
  constexpr bool RPM = D == 3 && !exact && NH2 <= 2 * NT;
  C rm[RPM ? 2 : 1][RPM ? D + 2 : 1];
  auto prefetch_moments = [&](int z) {
    if constexpr (RPM) {
      const int gz = g.wrap(2, z);
      {
        const Ix n = halo2_node(t, gz);
#pragma unroll
        for (int q = 0; q < D + 2; ++q) rm[0][RPM ? q : 0] = a.M_in[q * N + n];
      }
      if (t + NT < NH2) {
        const Ix n = halo2_node(t + NT, gz);
#pragma unroll
        for (int q = 0; q < D + 2; ++q) rm[RPM ? 1 : 0][RPM ? q : 0] = a.M_in[q * N + n];
      }
    }
  };
  // convert the moments rho, rho u, rho E of halo-2 node k into the corrected
  // macros rho, u, theta, rho E' of the ring slot dst
  auto put_macro = [&](C* dst, int k, C rho, const C* jm, C E) {
    C u[3], uu = C(0);
    C th;
    if constexpr (exact) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        u[d] = jm[d] / rho;
        uu += u[d] * u[d];
      }
      th = (E / rho - C(0.5) * uu) / ph.Cv;
    } else {
      const C ir = fdiv(C(1), rho);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        u[d] = jm[d] * ir;
        uu += u[d] * u[d];
      }
      th = (E * ir - C(0.5) * uu) * (C(1) / ph.Cv);
    }
    const C u2 = D == 3 ? u[D - 1] : C(0);
    if constexpr (sizeof(C) == 4) {
      reinterpret_cast<float4*>(dst)[k] = make_float4(rho, u[0], u[1], u2);
      reinterpret_cast<float2*>(dst + 4 * NH2)[k] = make_float2(th, E);
    } else {
      reinterpret_cast<double2*>(dst)[k] = make_double2(rho, u[0]);
      reinterpret_cast<double2*>(dst + 2 * NH2)[k] = make_double2(u[1], u2);
      reinterpret_cast<double2*>(dst + 4 * NH2)[k] = make_double2(th, E);
    }
  };
  // corrected macros of plane z over the halo-2 region, from the moments in
  // registers (prefetched) or global memory
  auto load_macros = [&](int z, bool regs = false) {
    C* dst = mr + (size_t)mslot(z) * NMF * NH2;
    if constexpr (RPM) {
      if (regs) {
        C jm[3];
#pragma unroll
        for (int d = 0; d < D; ++d) jm[d] = rm[0][RPM ? 1 + d : 0];
        put_macro(dst, t, rm[0][0], jm, rm[0][RPM ? 1 + D : 0]);
        if (t + NT < NH2) {
#pragma unroll
          for (int d = 0; d < D; ++d) jm[d] = rm[1][RPM ? 1 + d : 0];
          put_macro(dst, t + NT, rm[1][0], jm, rm[1][RPM ? 1 + D : 0]);
        }
        return;
      }
    }
    const int gz = g.wrap(2, z);
    for (int k = t; k < NH2; k += NT) {
      C rho, jm[3], E;
      const Ix n = halo2_node(k, gz);
      rho = a.M_in[n];
#pragma unroll
      for (int d = 0; d < D; ++d) jm[d] = a.M_in[(1 + d) * N + n];
      E = a.M_in[(1 + D) * N + n];
      put_macro(dst, k, rho, jm, E);
    }
  };
  auto macro_at = [&](int z, int kx, int ky) {
    const C* src = mr + (size_t)mslot(z) * NMF * NH2;
    const int k = ky * HX2 + kx;
    Macro<C> m;
    if constexpr (sizeof(C) == 4) {
      const float4 a4 = reinterpret_cast<const float4*>(src)[k];
      const float2 a2 = reinterpret_cast<const float2*>(src + 4 * NH2)[k];
      m.rho = a4.x;
      m.u[0] = a4.y;
      m.u[1] = a4.z;
      m.u[2] = a4.w;
      m.th = a2.x;
      m.E = a2.y;
    } else {
      const double2 a = reinterpret_cast<const double2*>(src)[k];
      const double2 b = reinterpret_cast<const double2*>(src + 2 * NH2)[k];
      const double2 c = reinterpret_cast<const double2*>(src + 4 * NH2)[k];
      m.rho = a.x;
      m.u[0] = a.y;
      m.u[1] = b.x;
      m.u[2] = b.y;
      m.th = c.x;
      m.E = c.y;
    }
    return m;
  };
  // 3D FP32 arithmetic (FP32, FP16 or BF16 storage): the populations and
  // auxiliaries of the next collision plane are loaded into registers one
  // plane ahead, so their latency overlaps the streaming and energy stage
  // of the current plane.
  // The loads are issued in three groups (populations [LO, HI), the
  // auxiliaries with the last): a warp whose load queue is full stalls, so
  // one group goes out before the pull stream, one after it and one after
  // the x face flux, where the arithmetic gives the queue time to drain.
  constexpr bool RP = D == 3 && !exact;
  constexpr int QA = (Q + 2) / 3, QB = (2 * Q + 1) / 3;  // population groups [0,QA) [QA,QB) [QB,Q)
  S rf[RP ? Q : 1];
  C rP = C(0);
  C rA[RP ? L::NDEV : 1];
  unsigned char rfl = 0;
  auto prefetch_regs = [&](int z, auto LO, auto HI, bool aux) {
    if constexpr (RP) {
      const Ix n = lin(wx, wy, g.wrap(2, z));
#pragma unroll
      for (int i = decltype(LO)::value; i < decltype(HI)::value; ++i) rf[i] = a.f_in[(Ix)i * N + n];
      if (aux) {
        rP = a.Pp[n];
#pragma unroll
        for (int q = 0; q < L::NDEV; ++q) rA[q] = a.Ap[q * N + n];
        rfl = a.forced ? a.forced[n] : 0;
      }
    }
  };
  // collision of this thread's node of plane z (halo-1 region, one node per thread)
  auto collide_plane = [&](int z, bool regs) {
    C* dst = fr + (size_t)fslot(z) * Q * NH1;
    const Ix n = lin(wx, wy, g.wrap(2, z));
    auto MA = [&](int dx, int dy, int dz) { return macro_at(z + dz, hx + dx, hy + dy); };
    const Macro<C> m = macro_at(z, hx, hy);
    C du[3][3], aC[3][3];
    gradients<L, C>(MA, m, du, aC, ph.use_ac, ph.gcs2);
    C fbar[Q];
    C dAFp[L::NDEV];
    C Pp;
    bool is_forced;
    if (RP && regs) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const C v = C(Store<S>::load(rf[RP ? i : 0]));
        fbar[i] = Store<S>::dev ? v + pop_offset<L, S, C>(i, g.off) : v;
      }
      Pp = rP;
#pragma unroll
      for (int q = 0; q < L::NDEV; ++q) dAFp[q] = rA[RP ? q : 0];
      is_forced = rfl != 0;
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) fbar[i] = load_pop<L, S, C, Ix>(a.f_in, i, N, n, g.off);
      Pp = a.Pp[n];
#pragma unroll
      for (int q = 0; q < L::NDEV; ++q) dAFp[q] = a.Ap[q * N + n];
      is_forced = a.forced && a.forced[n];
    }
    C fu[3] = {C(0), C(0), C(0)};
    if (is_forced) {
      // the node's CSR row: from the per-node map when there is one (one
      // load), else by binary search over the ascending row nodes
      const int r = a.row_of_node ? a.row_of_node[n] : find_row_dev(a.cell_id, a.n_rows, (int)n);
      if (r >= 0) {
#pragma unroll
        for (int d = 0; d < D; ++d) fu[d] = C(a.FU[(long long)r * D + d]);
      }
    }
    C fcol[Q], Pn, dAFn[L::NDEV];
    if constexpr (exact) {
      collide<L, C>(fbar, m, du, aC, Pp, dAFp, fu, ph, fcol, Pn, dAFn);
    } else {
      collide_fast<L, C>(fbar, m, du, aC, Pp, dAFp, fu, ph, fcol, Pn, dAFn);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[i * NH1 + t] = fcol[i];
    if (interior && z >= z0 && z < z1) {
      a.Pn[n] = Pn;
#pragma unroll
      for (int q = 0; q < L::NDEV; ++q) a.An[q * N + n] = dAFn[q];
    }
  };
  auto fcol_at = [&](int i, int z, int kx, int ky) { return fr[((size_t)fslot(z) * Q + i) * NH1 + ky * HX1 + kx]; };
  // x-face role of this thread's node: xeq = equilibrium face node; xs = -1
  // / +1 = outlet face node that takes the values of its inner neighbour
  // at x + xs (same tile: the host checks the tile alignment)
  bool xeq = false;
  int xs = 0;
  if (a.bc_fused) {
    const bool lo = gx == 0, hi = gx == g.n[0] - 1;
    const int t0 = a.bct[0], t1 = a.bct[1];
    xeq = (lo && (t0 == 1 || t0 == 3)) || (hi && (t1 == 1 || t1 == 3));
    if (lo && t0 == 2) xs = 1;
    if (hi && t1 == 2) xs = -1;
  }
  const int sx = cx + xs;  // the node whose stream, faces and energy this thread computes
  const int st = t + xs;
  // energy flux through the + face (axis AX) of plane bz of the node at
  // x offset sh from this thread's node
  auto face = [&](auto AXc, int bz, int sh) {
    constexpr int AX = decltype(AXc)::value;
    auto MAl = [&](int k) {
      return macro_at(bz + (AX == 2 ? k : 0), hx + sh + (AX == 0 ? k : 0), hy + (AX == 1 ? k : 0));
    };
    auto FCl = [&](int i, int dx, int dy, int dz) { return fcol_at(i, bz + dz, cx + sh + dx, cy + dy); };
    return energy_face_flux<L, C, AX>(MAl, FCl, ph);
  };

  // prologue: macros of planes z0-2..z0+2, collisions of planes z0-1 and z0
  if constexpr (D == 3) {
    for (int z = z0 - 2; z <= z0 + 2; ++z) load_macros(z);
    __syncthreads();
    collide_plane(z0 - 1, false);
    collide_plane(z0, false);
    prefetch_regs(z0 + 1, std::integral_constant<int, 0>{}, std::integral_constant<int, Q>{}, true);
    prefetch_moments(z0 + 3);
    __syncthreads();
  }
  // the -z face of plane z is the +z face of plane z-1: carried in a register
  C Fz_prev = C(0);
  if constexpr (D == 3) {
    if (interior) Fz_prev = face(std::integral_constant<int, 2>{}, z0 - 1, xs);
  }
  const bool xface = cx <= TX && cy >= 1 && cy <= TY;  // +x faces of nodes cx = 0..TX
  const bool yface = cy <= TY && cx >= 1 && cx <= TX;  // +y faces of nodes cy = 0..TY
  // energy update of plane zp, one iteration late (after the barrier that
  // makes its face fluxes visible):
  // rho E^{n+1} = rho E' - sum_a (F_{+a/2}(x) - F_{+a/2}(x - e_a))
  C Fz_pend = C(0);
  auto finish = [&](int zp) {
    if (interior) {
      const C* fx = Fx + (zp & 1) * NH1;
      const C* fy = Fy + (zp & 1) * NH1;
      C E = macro_at(zp, hx + xs, hy).E;
      E = E - (fx[st] - fx[st - 1]);
      E = E - (fy[st] - fy[st - HX1]);
      if constexpr (D == 3) {
        E = E - (Fz_pend - Fz_prev);
        Fz_prev = Fz_pend;
      }
      if (xeq) E = a.E_inf;
      a.M_out[(1 + D) * N + lin(gx, gy, zp)] = E;
    }
  };
  for (int z = z0; z < z1; ++z) {
    __syncthreads();
    if (z > z0) finish(z - 1);
    if constexpr (D == 3) {
      // the macros of plane z+3 go to a slot no one reads in this
      // iteration; the collision of plane z+1 reads planes z..z+2, filled
      // in earlier iterations: one barrier covers both
      load_macros(z + 3, true);
      collide_plane(z + 1, true);
      __syncthreads();
      prefetch_regs(z + 2, std::integral_constant<int, 0>{}, std::integral_constant<int, QA>{}, false);
      prefetch_moments(z + 4);
    } else {
      load_macros(0);
      __syncthreads();
      collide_plane(0, false);
      __syncthreads();
    }
    C rho = C(0), j[3] = {C(0), C(0), C(0)};
    Ix n = 0;
    if (interior) {
      n = lin(gx, gy, z);
      // Eq. LB pull streaming and the predicted moments of step n+1
      sfor<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const C v = fcol_at(i, z - L::c(i, 2), sx - L::c(i, 0), cy - L::c(i, 1));
        store_pop<L, S, C, Ix>(a.f_out, i, N, n, v, g.off);
        rho += v;
        sfor<0, D>([&](auto A) {
          constexpr int d = decltype(A)::value;
          if constexpr (L::c(i, d) != 0) j[d] += C(L::c(i, d)) * v;
        });
      });
      if (xeq) {
        // free-stream equilibrium and its moments, as stored
        rho = C(0);
        j[0] = j[1] = j[2] = C(0);
        sfor<0, Q>([&](auto I) {
          constexpr int i = decltype(I)::value;
          store_pop<L, S, C, Ix>(a.f_out, i, N, n, a.feq_inf[i], g.off);
          const C v = roundtrip_pop<L, S, C>(i, a.feq_inf[i], g.off);
          rho += v;
          sfor<0, D>([&](auto A) {
            constexpr int d = decltype(A)::value;
            if constexpr (L::c(i, d) != 0) j[d] += C(L::c(i, d)) * v;
          });
        });
      }
    }
    if constexpr (D == 3) {
      prefetch_regs(z + 2, std::integral_constant<int, QA>{}, std::integral_constant<int, QB>{}, false);
    }
    // Eq. energy face fluxes, each face once
    if (xface) Fx[(z & 1) * NH1 + t] = face(std::integral_constant<int, 0>{}, z, 0);
    if constexpr (D == 3) {
      prefetch_regs(z + 2, std::integral_constant<int, QB>{}, std::integral_constant<int, Q>{}, true);
    }
    if (yface) Fy[(z & 1) * NH1 + t] = face(std::integral_constant<int, 1>{}, z, 0);
    // the predicted moments of step n+1, stored late so that the stores
    // overlap the z face flux
    if (interior) {
      a.M_out[n] = rho;
#pragma unroll
      for (int d = 0; d < D; ++d) a.M_out[(1 + d) * N + n] = j[d];
    }
    if constexpr (D == 3) {
      if (interior) Fz_pend = face(std::integral_constant<int, 2>{}, z, xs);
    }
  }
  __syncthreads();
  finish(z1 - 1);
}

template <class L, class S, class C, int HY, bool NARROW>
__global__ void __launch_bounds__(FusedLayout<L, S, C, HY>::NT, FusedLayout<L, S, C, HY>::min_blocks)
    k_fused(Grid g, FusedArgs<S, C> a, Phys<C> ph, int zchunk) {
  fused_body<L, S, C, HY, NARROW>(g, a, ph, zchunk, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Several cases in one launch: work item k = (case, tile x, tile y, z-chunk)
// from a schedule table; each block reads its case's descriptor.
template <class S, class C>
struct CaseDesc {
  Grid g;
  FusedArgs<S, C> a;
  Phys<C> ph;
  int zchunk;
};

template <class L, class S, class C, int HY, bool NARROW>
__global__ void __launch_bounds__(FusedLayout<L, S, C, HY>::NT, FusedLayout<L, S, C, HY>::min_blocks)
    k_fused_batched(const CaseDesc<S, C>* descs, const int4* work) {
  const int4 w = work[blockIdx.x];
  const CaseDesc<S, C>& d = descs[w.x];
  fused_body<L, S, C, HY, NARROW>(d.g, d.a, d.ph, d.zchunk, w.y, w.z, w.w);
}

// 32-bit element offsets reach every array of a case with Q N < 2^32
template <class L>
inline bool narrow_index(long long N) {
  return (long long)L::Q * N < (1LL << 32);
}

// the dynamic shared-memory limit of a kernel is a per-device attribute:
// set it once on each device that launches the kernel (one flag array per
// kernel: the template takes the kernel itself, not its type)
template <auto kernel>
inline void smem_attr_once(int bytes) {
  constexpr int kMaxDev = 64;
  static bool done[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return;
  }
  if (!done[dev]) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done[dev] = true;
  }
}

template <class L, class S, class C, int HY>
inline void launch_fused_tile(const Grid& g, const FusedArgs<S, C>& a, const Phys<C>& ph, cudaStream_t st,
                              int zchunk) {
  using Lay = FusedLayout<L, S, C, HY>;
  dim3 grid((g.n[0] + Lay::TX - 1) / Lay::TX, (g.n[1] + Lay::TY - 1) / Lay::TY,
            L::D == 3 ? (g.n[2] + zchunk - 1) / zchunk : 1);
  if (narrow_index<L>(g.N)) {
    smem_attr_once<k_fused<L, S, C, HY, true>>((int)Lay::bytes);
    k_fused<L, S, C, HY, true><<<grid, Lay::NT, Lay::bytes, st>>>(g, a, ph, zchunk);
  } else {
    smem_attr_once<k_fused<L, S, C, HY, false>>((int)Lay::bytes);
    k_fused<L, S, C, HY, false><<<grid, Lay::NT, Lay::bytes, st>>>(g, a, ph, zchunk);
  }
}

// zchunk: planes per CTA along z (3D); tile_rows selects the halo-1 tile
// height of the 2D FP32 step: 0 = 8, 16 or 32 (1024 threads); other forms
// have one tile
template <class L, class S, class C>
inline void launch_fused(const Grid& g, const FusedArgs<S, C>& a, const Phys<C>& ph, cudaStream_t st,
                         int zchunk, int tile_rows) {
  if constexpr (L::D == 2 && sizeof(C) == 4) {
    if (tile_rows == 16) return launch_fused_tile<L, S, C, 16>(g, a, ph, st, zchunk);
    if (tile_rows == 32) return launch_fused_tile<L, S, C, 32>(g, a, ph, st, zchunk);
  }
  launch_fused_tile<L, S, C, 0>(g, a, ph, st, zchunk);
}

// predicted moments rho, rho u, rho E of every node from populations and E
template <class L, class S, class C>
__global__ void k_moments(Grid g, const S* f, const C* E, C* M) {
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
  M[n] = r;
#pragma unroll
  for (int a = 0; a < D; ++a) M[(1 + a) * g.N + n] = j[a];
  M[(1 + D) * g.N + n] = E[n];
}

// All domain faces in one launch (reading Q24); the faces also refresh the
// predicted moments of the nodes they set: a node on an inlet or far-field
// face takes the free-stream equilibrium; a node on an outlet face and on no
// equilibrium face copies its inner neighbour along the outlet axis.  This is
// the outlet-copy-then-equilibrium order with the edges resolved up front.
struct BCFaces {
  int type[6];  // LBM_BC_* per face: 0 periodic, 1 inlet, 2 outlet, 3 far field, 4 slab ghost face,
                // 5 characteristic far field
  // free stream and gas constants of the characteristic faces
  double rho_inf, u_inf[3], p_inf, gamma, R, Cv;
};

// boundary node t of face `face` (see k_bc_all_m)
template <class L, class S, class C>
__device__ __forceinline__ void bc_node(const Grid& g, S* f, C* M, const BCFaces& bf, const C* feq_inf, C E_inf,
                                        int skip_x, int face, int t) {
  constexpr int D = L::D;
  const int axis = face / 2, side = face % 2;
  const int ft = bf.type[face];
  if (ft == 0 || ft == kBCGhostFace || (skip_x && axis == 0)) return;
  const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
  if (t >= g.n[a1] * g.n[a2]) return;
  int c[3];
  c[a1] = t % g.n[a1];
  c[a2] = t / g.n[a1];
  c[axis] = side ? g.n[axis] - 1 : 0;
  auto on_eq_face = [&](int b) {
    for (int s2 = 0; s2 < 2; ++s2) {
      const int t2 = bf.type[2 * b + s2];
      if ((t2 == 1 || t2 == 3) && c[b] == (s2 ? g.n[b] - 1 : 0)) return true;
    }
    return false;
  };
  bool eq = false;
  for (int b = 0; b < D; ++b) eq = eq || on_eq_face(b);
  const long long dst = g.lin(c[0], c[1], c[2]);
  if (eq) {
    if (ft != 1 && ft != 3) return;  // written by the equilibrium face's own thread
    C r = C(0), j[3] = {C(0), C(0), C(0)};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      store_pop<L, S, C>(f, i, g.N, dst, feq_inf[i], g.off);
      const C v = roundtrip_pop<L, S, C>(i, feq_inf[i], g.off);
      r += v;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (L::c(i, a) != 0) j[a] += C(L::c(i, a)) * v;
    }
    M[dst] = r;
#pragma unroll
    for (int a = 0; a < D; ++a) M[(1 + a) * g.N + dst] = j[a];
    M[(1 + D) * g.N + dst] = E_inf;
    return;
  }
  // free-stream equilibrium at dst with its moments, as stored
  auto put_state = [&](auto feq_of, C E) {
    C r = C(0), j[3] = {C(0), C(0), C(0)};
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const C fe = feq_of(I);
      store_pop<L, S, C>(f, i, g.N, dst, fe, g.off);
      const C v = roundtrip_pop<L, S, C>(i, fe, g.off);
      r += v;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (L::c(i, a) != 0) j[a] += C(L::c(i, a)) * v;
    });
    M[dst] = r;
#pragma unroll
    for (int a = 0; a < D; ++a) M[(1 + a) * g.N + dst] = j[a];
    M[(1 + D) * g.N + dst] = E;
  };
  if (ft == kBCChar) {
    // a node on two or more characteristic faces (an edge between them)
    // takes the free stream, written by the first of those faces
    int nchar = 0, first = -1;
    for (int b = 0; b < D; ++b)
      for (int s2 = 0; s2 < 2; ++s2)
        if (bf.type[2 * b + s2] == kBCChar && c[b] == (s2 ? g.n[b] - 1 : 0)) {
          ++nchar;
          if (first < 0) first = 2 * b + s2;
        }
    if (nchar >= 2) {
      if (face == first) put_state([&](auto I) { return feq_inf[decltype(I)::value]; }, E_inf);
      return;
    }
    // the state of the linearized one-dimensional Riemann invariants normal
    // to the face: W+ = p + rho c u_n, W- = p - rho c u_n, W0 = rho - p/c^2
    // and u_t, each from the interior neighbour when its characteristic
    // leaves the domain and from the free stream when it enters (the
    // neighbour's carried moments are this step's streamed values)
    int ci[3] = {c[0], c[1], c[2]};
    ci[axis] = side ? g.n[axis] - 2 : 1;
    const long long src = g.lin(ci[0], ci[1], ci[2]);
    const C rho = M[src];
    C u[3] = {C(0), C(0), C(0)}, uu = C(0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      u[b] = M[(1 + b) * g.N + src] / rho;
      uu = uu + u[b] * u[b];
    }
    const C Rg = C(bf.R), Cv = C(bf.Cv);
    const C th = (M[(1 + D) * g.N + src] / rho - C(0.5) * uu) / Cv;
    const C p = rho * Rg * th;
    const C cs = sqrt(C(bf.gamma) * Rg * th);
    const C sgn = side ? C(1) : C(-1);
    const C un = sgn * u[axis];
    const C un_inf = sgn * C(bf.u_inf[axis]);
    const C p_inf = C(bf.p_inf);
    const C rc = rho * cs;
    const C c2 = cs * cs;
    const C Wp = (un + cs > C(0)) ? p + rc * un : p_inf + rc * un_inf;
    const C Wm = (un - cs < C(0)) ? p_inf - rc * un_inf : p - rc * un;
    const bool out = un > C(0);
    const C W0 = out ? rho - p / c2 : C(bf.rho_inf) - p_inf / c2;
    const C pb = C(0.5) * (Wp + Wm);
    const C unb = (Wp - Wm) / (C(2) * rc);
    const C rb = W0 + pb / c2;
    C ub[3] = {C(0), C(0), C(0)};
#pragma unroll
    for (int b = 0; b < D; ++b) ub[b] = b == axis ? sgn * unb : (out ? u[b] : C(bf.u_inf[b]));
    const C thb = pb / (rb * Rg);
    C kb = C(0);
#pragma unroll
    for (int b = 0; b < D; ++b) kb = kb + ub[b] * ub[b];
    const C Eb = rb * (C(0.5) * kb + Cv * thb);
    put_state([&](auto I) { return feq_i<L, C, decltype(I)::value>(rb, ub, thb); }, Eb);
    return;
  }
  if (ft != 2) return;
  c[axis] = side ? g.n[axis] - 2 : 1;
  const long long src = g.lin(c[0], c[1], c[2]);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) f[(long long)i * g.N + dst] = f[(long long)i * g.N + src];
#pragma unroll
  for (int k = 0; k < L::D + 2; ++k) M[k * g.N + dst] = M[k * g.N + src];
}

template <class L, class S, class C>
__global__ void k_bc_all_m(Grid g, S* f, C* M, BCFaces bf, const C* feq_inf, C E_inf, int skip_x) {
  bc_node<L, S, C>(g, f, M, bf, feq_inf, E_inf, skip_x, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x);
}

// Several cases in one launch.
template <class S, class C>
struct BCCaseDesc {
  Grid g;
  S* f;
  C* M;
  BCFaces bf;
  const C* feq_inf;
  C E_inf;
  int skip_x;
};

// work item = (case, face, block of that face's nodes)
template <class L, class S, class C>
__global__ void k_bc_batched(const BCCaseDesc<S, C>* d, const int4* work) {
  const int4 w = work[blockIdx.x];
  const BCCaseDesc<S, C>& c = d[w.x];
  bc_node<L, S, C>(c.g, c.f, c.M, c.bf, c.feq_inf, c.E_inf, c.skip_x, w.y, w.z * blockDim.x + threadIdx.x);
}


}  // namespace lbmib
