// Device arithmetic of the hybrid LBM time step (arXiv 2607.07432,
// Sec. 2.2 and App. A): equilibrium (Eq. feq), HRR regularized collision
// (Eqs. fneq, pi2, pi3) with the force populations (Eqs. fi, af2), the
// finite-difference quantities it needs, and the face flux of the total
// energy (Eq. energy with Eqs. fluxx-z and the MUSCL-Hancock face values of
// Eq. linear).  The functions are templated on the lattice L and the
// compute type C and take accessors for neighbouring data, so that the
// same arithmetic serves the global-memory and the shared-memory kernels.
#pragma once
#include "lattice.cuh"

namespace lbmib {

template <class C>
struct Phys {
  C cs2, Cv, Cp, mu, lam, sigma;
  C gcs2;         // gamma c_s^2: the squared sound speed over theta
  C mub2;         // twice the artificial bulk viscosity mu_b
  int theta_tau;  // 1: tau_LB = mu / (rho c_s^2 theta)
  int use_ac;
};

// corrected macroscopic state of one node (after the IB forcing)
template <class C>
struct Macro {
  C rho, u[3], th, E;
};

// Eq. feq for population I (compile-time index)
template <class L, class C, int I>
__device__ __forceinline__ C feq_i(C rho, const C* u, C th) {
  constexpr int D = L::D;
  const C cs2 = C(kCs2);
  C t1 = C(0);
  sfor<0, D>([&](auto A) {
    constexpr int a = decltype(A)::value;
    if constexpr (L::c(I, a) != 0) t1 += C(L::c(I, a)) * rho * u[a];
  });
  t1 = t1 / cs2;
  C t2 = C(0);
  sfor<0, D>([&](auto A) {
    sfor<0, D>([&](auto B) {
      constexpr int a = decltype(A)::value, b = decltype(B)::value;
      constexpr double h = H2<L>(I, a, b);
      if constexpr (h != 0.0) t2 += C(h) * rho * u[a] * u[b];
    });
  });
  t2 = t2 / (C(2) * cs2 * cs2);
  C t3 = C(0);
  sfor<0, L::N3>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr double h = H3r<L>(k, I);
    if constexpr (h != 0.0) {
      constexpr double nk = N3r<L>(k);
      C A = C(0);
      sfor<0, L::h3terms(k)>([&](auto T) {
        constexpr int t = decltype(T)::value;
        constexpr int a = L::h3idx(k, t, 0), b = L::h3idx(k, t, 1), g = L::h3idx(k, t, 2);
        A += C(L::h3sign(k, t)) * (rho * u[a] * u[b] * u[g]);
      });
      t3 += C(h) * A / C(nk);
    }
  });
  constexpr double wi = L::w(I);
  constexpr double cth = (L::w(I) - (I == 0 ? 1.0 : 0.0)) / L::w(I);
  const C tth = C(cth) * rho * (th - C(1));
  return C(wi) * (rho + tth + t1 + t2 + t3);
}

// Largest upstream weight of the a^C differences under use_ac = 3.
constexpr double kAcUpwindCap = 1.5;

// Velocity gradient du[a][b] = d u_a / d x_b and a^C, the lattice-dependent
// part of Eq. af2 (only cited by the paper), read from the Chapman-Enskog
// expansion of the lattice's third moment:
//   a^C_ab = c_s^2 (u_a d_b P + u_b d_a P) - d_ab d_a(rho u_a^3),
// P = rho(1-theta) (use_ac = 2; use_ac = 1 keeps the cubic part only,
// 0 none).  Central differences, except for a^C under use_ac = 3: each
// difference along b leans to the node's upstream side in proportion to its
// Mach number along b, D_b g = (g+ - g-)/2 - (alpha_b/2)(g+ - 2g + g-),
// alpha_b = clamp(u_b / c, -kAcUpwindCap, kAcUpwindCap), c^2 = gamma c_s^2
// theta, which keeps streams faster than the sound speed stable (central
// differences cannot see their growing odd-even mode).  MacroAt(dx,dy,dz)
// returns the neighbour's Macro, mc is the node's own.  In FP64 the
// operations follow the oracle's order.
template <class L, class C, class MacroAt>
__device__ __forceinline__ void gradients(const MacroAt& M, const Macro<C>& mc, C du[3][3], C aC[3][3],
                                          int use_ac, C gcs2) {
  constexpr int D = L::D;
  const C* uc = mc.u;
  C dP[3];
  C c = C(1);
  if (use_ac == 3) c = sqrt(gcs2 * mc.th);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    const Macro<C> p = M(b == 0 ? 1 : 0, b == 1 ? 1 : 0, b == 2 ? 1 : 0);
    const Macro<C> m = M(b == 0 ? -1 : 0, b == 1 ? -1 : 0, b == 2 ? -1 : 0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      du[a][b] = (p.u[a] - m.u[a]) * C(0.5);
      aC[a][b] = C(0);
    }
    const C gp = p.rho * (p.u[b] * p.u[b] * p.u[b]);
    const C gm = m.rho * (m.u[b] * m.u[b] * m.u[b]);
    const C Pp = p.rho * (C(1) - p.th);
    const C Pm = m.rho * (C(1) - m.th);
    if (use_ac == 3) {
      // comparisons keep a NaN weight NaN, as the oracle's clip does
      C al = uc[b] / c;
      al = al > C(kAcUpwindCap) ? C(kAcUpwindCap) : (al < C(-kAcUpwindCap) ? C(-kAcUpwindCap) : al);
      const C hw = C(0.5) * al;
      const C g0 = mc.rho * (uc[b] * uc[b] * uc[b]);
      const C P0 = mc.rho * (C(1) - mc.th);
      aC[b][b] = -(C(0.5) * (gp - gm) - hw * (gp - C(2) * g0 + gm));
      dP[b] = C(0.5) * (Pp - Pm) - hw * (Pp - C(2) * P0 + Pm);
    } else {
      if (use_ac) aC[b][b] = -((gp - gm) * C(0.5));
      dP[b] = (Pp - Pm) * C(0.5);
    }
  }
  if (use_ac >= 2) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) aC[a][b] = aC[a][b] + C(kCs2) * (uc[a] * dP[b] + uc[b] * dP[a]);
  }
}

// expand stored deviator slots to a full symmetric traceless tensor
template <class L, class C>
__device__ __forceinline__ void dev_expand(const C* s, C T[3][3]) {
  constexpr int D = L::D;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const int k = dev_slot<L>(a, b);
      if (k >= 0) T[a][b] = s[k];
    }
  if (D == 2) {
    T[1][1] = -s[0];
  } else {
    T[2][2] = -s[0] - s[1];
  }
}

// quotient a / b: the hardware approximation (2 ulp) in FP32, exact otherwise
template <class C>
__device__ __forceinline__ C fdiv(C a, C b) {
  if constexpr (sizeof(C) == 4) {
    return __fdividef(a, b);
  } else {
    return a / b;
  }
}

// HRR collision at one node (Eq. LB with dt = 1, Eqs. fi, af2, fneq, pi2,
// pi3).  fbar: post-stream populations of the node; m: corrected macros;
// du, aC: gradients; P_prev, dAFp: rho(1-theta) and the deviator of a^F of
// the previous step; fu: IB force density at the node.  Outputs f^col, the
// new rho(1-theta) and the deviator of a^F (NDEV slots).
template <class L, class C>
__device__ __forceinline__ void collide(const C* fbar, const Macro<C>& m, const C du[3][3],
                                        const C aC[3][3], C P_prev, const C* dAFp, const C* fu,
                                        const Phys<C>& ph, C* fcol, C& P_new, C* dAF_new) {
  constexpr int D = L::D;
  constexpr int Q = L::Q;
  const C cs2 = C(kCs2);
  C div = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) div += du[a][a];
  const C P = m.rho * (C(1) - m.th);
  const C dPdt = P - P_prev;
  C aF[3][3];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      C v = aC[a][b] + fu[a] * m.u[b] + fu[b] * m.u[a];
      if (a == b) v = v + (C(2) / C(D)) * m.rho * cs2 * div - cs2 * dPdt - ph.mub2 * div;
      aF[a][b] = v;
    }
  C feq[Q];
  sfor<0, Q>([&](auto I) { feq[decltype(I)::value] = feq_i<L, C, decltype(I)::value>(m.rho, m.u, m.th); });
  const C th_m = ph.theta_tau ? m.th : C(1);
  const C tau_lb = ph.mu / (m.rho * cs2 * th_m);
  const C tau_bar = tau_lb + C(0.5);
  C Fp[3][3];
  dev_expand<L, C>(dAFp, Fp);
  C Pi[3][3];
  sfor<0, D>([&](auto A) {
    sfor<decltype(A)::value, D>([&](auto B) {
      constexpr int a = decltype(A)::value, b = decltype(B)::value;
      C s = C(0);
      sfor<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr double proj = double(L::c(i, a) * L::c(i, b)) - (a == b ? double(c2<L>(i)) / D : 0.0);
        if constexpr (proj != 0.0) s = s + C(proj) * (fbar[i] - feq[i]);
      });
      s = s + C(0.5) * Fp[a][b];
      const C S = du[a][b] + du[b][a] - (a == b ? (C(2) / C(D)) * div : C(0));
      Pi[a][b] = ph.sigma * s - (C(1) - ph.sigma) * m.rho * cs2 * th_m * tau_bar * S;
      Pi[b][a] = Pi[a][b];
    });
  });
  // third-order combinations of Eq. pi3
  C A3[L::N3];
  sfor<0, L::N3>([&](auto K) {
    constexpr int k = decltype(K)::value;
    C A = C(0);
    sfor<0, L::h3terms(k)>([&](auto T) {
      constexpr int t = decltype(T)::value;
      constexpr int a = L::h3idx(k, t, 0), b = L::h3idx(k, t, 1), g = L::h3idx(k, t, 2);
      A += C(L::h3sign(k, t)) * (m.u[a] * Pi[b][g] + m.u[b] * Pi[g][a] + m.u[g] * Pi[a][b]);
    });
    A3[k] = A;
  });
  const C omega = C(1) - C(1) / tau_bar;
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    C t2 = C(0);
    sfor<0, D>([&](auto A) {
      sfor<0, D>([&](auto B) {
        constexpr int a = decltype(A)::value, b = decltype(B)::value;
        constexpr double h = H2<L>(i, a, b);
        if constexpr (h != 0.0) t2 += C(h) * Pi[a][b];
      });
    });
    t2 = t2 / (C(2) * cs2 * cs2);
    C t3 = C(0);
    sfor<0, L::N3>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr double h = H3r<L>(k, i);
      constexpr double nk = N3r<L>(k);
      if constexpr (h != 0.0) t3 += C(h) * A3[k] / C(nk);
    });
    const C fneq = C(L::w(i)) * (t2 + t3);
    C f1 = C(0);
    sfor<0, D>([&](auto A) {
      constexpr int a = decltype(A)::value;
      if constexpr (L::c(i, a) != 0) f1 += C(L::c(i, a)) * fu[a];
    });
    f1 = f1 / cs2;
    C f2 = C(0);
    sfor<0, D>([&](auto A) {
      sfor<0, D>([&](auto B) {
        constexpr int a = decltype(A)::value, b = decltype(B)::value;
        constexpr double h = H2<L>(i, a, b);
        if constexpr (h != 0.0) f2 += C(h) * aF[a][b];
      });
    });
    const C Fi = C(L::w(i)) * (f1 + f2 / (C(2) * cs2 * cs2));
    fcol[i] = feq[i] + omega * fneq + C(0.5) * Fi;
  });
  P_new = P;
  C tr = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) tr += aF[a][a];
  sfor<0, D>([&](auto A) {
    sfor<decltype(A)::value, D>([&](auto B) {
      constexpr int a = decltype(A)::value, b = decltype(B)::value;
      constexpr int k = dev_slot<L>(a, b);
      if constexpr (k >= 0) dAF_new[k] = aF[a][b] - (a == b ? tr / C(D) : C(0));
    });
  });
}

// Same collision in Hermite-coefficient form (FP32 path): with
// a1 = rho u + f_u/2, a2 = rho u u + (1 - 1/tau) Pi + a^F/2 and
// a3_k = A^eq_k + (1 - 1/tau) A^neq_k,
// f^col_i = w_i [rho + c_i.a1/c_s^2 + H2_i:a2/(2 c_s^4) + sum_k H3r_k,i a3_k/N_k]
//         + (w_i - delta_0i) rho (theta - 1),
// algebraically identical to f^eq + (1 - 1/tau) f^neq + F/2 but with about a
// third of the arithmetic (every population reuses the same coefficients).
// Divisions by the constants c_s^2 and D are products with their
// reciprocals, and the two data-dependent quotients (tau, 1/tau) use the
// hardware division (2 ulp), which avoids the checked IEEE division.
template <class L, class C>
__device__ __forceinline__ void collide_fast(const C* fbar, const Macro<C>& m, const C du[3][3],
                                             const C aC[3][3], C P_prev, const C* dAFp, const C* fu,
                                             const Phys<C>& ph, C* fcol, C& P_new, C* dAF_new) {
  constexpr int D = L::D;
  constexpr int Q = L::Q;
  const C cs2 = C(kCs2);
  C div = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) div += du[a][a];
  const C P = m.rho * (C(1) - m.th);
  const C dPdt = P - P_prev;
  const C trace_term = (C(2) / C(D)) * m.rho * cs2 * div - cs2 * dPdt - ph.mub2 * div;
  C aF[3][3];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) aF[a][b] = aC[a][b] + fu[a] * m.u[b] + fu[b] * m.u[a] + (a == b ? trace_term : C(0));
  const C th_m = ph.theta_tau ? m.th : C(1);
  const C tau_bar = fdiv(ph.mu, m.rho * cs2 * th_m) + C(0.5);
  const C omega = C(1) - fdiv(C(1), tau_bar);
  const C fd = (C(1) - ph.sigma) * m.rho * cs2 * th_m * tau_bar;
  C Fp[3][3];
  dev_expand<L, C>(dAFp, Fp);
  // raw second moments of f-bar from the even parts f_i + f_opp(i) of the
  // opposite pairs (c_a c_b is even in c, so each pair enters once)
  C ev[Q];
  sfor<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int o = opposite<L>(i);
    if constexpr (i < o) ev[i] = fbar[i] + fbar[o];
  });
  C S2[3][3];
  sfor<0, D>([&](auto A) {
    sfor<decltype(A)::value, D>([&](auto B) {
      constexpr int a = decltype(A)::value, b = decltype(B)::value;
      C s = C(0);
      bool first = true;
      sfor<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int o = opposite<L>(i);
        constexpr int cc = L::c(i, a) * L::c(i, b);
        if constexpr (i < o && cc == 1) {
          s = first ? ev[i] : s + ev[i];
          first = false;
        }
        if constexpr (i < o && cc == -1) {
          s = first ? -ev[i] : s - ev[i];
          first = false;
        }
      });
      S2[a][b] = s;
    });
  });
  C trS = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) trS += S2[a][a] - m.rho * m.u[a] * m.u[a];
  C Pi[3][3];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = a; b < D; ++b) {
      C dev = S2[a][b] - m.rho * m.u[a] * m.u[b] - (a == b ? trS * C(1.0 / D) : C(0));
      const C S = du[a][b] + du[b][a] - (a == b ? (C(2) / C(D)) * div : C(0));
      Pi[a][b] = ph.sigma * (dev + C(0.5) * Fp[a][b]) - fd * S;
      Pi[b][a] = Pi[a][b];
    }
  // coefficients
  C A1[3], B2[3][3];
#pragma unroll
  for (int a = 0; a < D; ++a) A1[a] = (m.rho * m.u[a] + C(0.5) * fu[a]) * C(1.0 / kCs2);
  const C inv2cs4 = C(1) / (C(2) * cs2 * cs2);
  C trB = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = a; b < D; ++b) {
      B2[a][b] = (m.rho * m.u[a] * m.u[b] + omega * Pi[a][b] + C(0.5) * aF[a][b]) * inv2cs4;
      if (a == b) trB += B2[a][b];
    }
  C A3[L::N3];
  sfor<0, L::N3>([&](auto K) {
    constexpr int k = decltype(K)::value;
    C A = C(0);
    sfor<0, L::h3terms(k)>([&](auto T) {
      constexpr int t = decltype(T)::value;
      constexpr int a = L::h3idx(k, t, 0), b = L::h3idx(k, t, 1), g = L::h3idx(k, t, 2);
      A += C(L::h3sign(k, t)) * (m.rho * m.u[a] * m.u[b] * m.u[g] +
                                 omega * (m.u[a] * Pi[b][g] + m.u[b] * Pi[g][a] + m.u[g] * Pi[a][b]));
    });
    A3[k] = A * C(1.0 / N3r<L>(k));
  });
  const C R1 = m.rho * (m.th - C(1));
  const C base = m.rho + R1 - cs2 * trB;
  // f_i = w_i (E_i + O_i) and f_opp(i) = w_i (E_i - O_i): the even (zeroth and
  // second order) part is shared by a direction and its opposite, the odd
  // (first and third order) part changes sign
  fcol[0] = C(L::w(0)) * base - R1;
  sfor<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int o = opposite<L>(i);
    if constexpr (i < o) {
      C E = base, O = C(0);
      sfor<0, D>([&](auto A) {
        constexpr int a = decltype(A)::value;
        if constexpr (L::c(i, a) != 0) E += B2[a][a];
        if constexpr (L::c(i, a) == 1) O += A1[a];
        if constexpr (L::c(i, a) == -1) O -= A1[a];
        sfor<decltype(A)::value + 1, D>([&](auto B) {
          constexpr int b = decltype(B)::value;
          constexpr int cc = L::c(i, a) * L::c(i, b);
          if constexpr (cc == 1) E += C(2) * B2[a][b];
          if constexpr (cc == -1) E -= C(2) * B2[a][b];
        });
      });
      sfor<0, L::N3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        constexpr double h = H3r<L>(k, i);
        if constexpr (h != 0.0) O += C(h) * A3[k];
      });
      const C wE = C(L::w(i)) * E, wO = C(L::w(i)) * O;
      fcol[i] = wE + wO;
      fcol[o] = wE - wO;
    }
  });
  P_new = P;
  C tr = C(0);
#pragma unroll
  for (int a = 0; a < D; ++a) tr += aF[a][a];
  sfor<0, D>([&](auto A) {
    sfor<decltype(A)::value, D>([&](auto B) {
      constexpr int a = decltype(A)::value, b = decltype(B)::value;
      constexpr int k = dev_slot<L>(a, b);
      if constexpr (k >= 0) dAF_new[k] = aF[a][b] - (a == b ? tr * C(1.0 / D) : C(0));
    });
  });
}

// x / 3: exact division in FP64 (bitwise parity form), a multiply in FP32
template <class C>
__device__ __forceinline__ C third(C x) {
  if constexpr (sizeof(C) == 8) {
    return x / C(3);
  } else {
    return x * C(1.0 / 3.0);
  }
}

// MUSCL-Hancock face value of Eq. linear from the upwind stencil: B is the
// reconstructing cell (x if u~ >= 0, else x + e), A and Cc its neighbours
// behind and ahead along the axis, uB its axial velocity; plus selects the
// x + e/2 face value of cell x (phi_+ branch) or the x - e/2 value of cell
// x + e (phi_- branch).
template <class C>
__device__ __forceinline__ C muscl3(C A, C B, C Cc, C uB, bool plus) {
  const C sg = uB > C(0) ? C(1) : (uB < C(0) ? C(-1) : C(0));
  const C eta = third<C>(C(2) * uB - sg);
  const C delta = C(0.5) * ((C(1) + eta) * (B - A) + (C(1) - eta) * (Cc - B));
  const C pp = B + C(0.5) * delta;
  const C pm = B - C(0.5) * delta;
  return (plus ? pp : pm) + C(0.5) * uB * (pm - pp);
}

// FP32 form of the face flux below, algebraically the same: the LB mass
// and momentum fluxes are sums over the crossing populations grouped by
// direction (the transverse pairs of a diagonal population are added before
// the common 1/2 is applied), and the MUSCL-Hancock face value
// B +- delta/2 - uB delta/2 of Eq. linear is written as
// B + alpha (B - A) + beta (Cc - B) with the weights computed once per face.
template <class L, class C, int AX, class MacroAlong, class FcolAt>
__device__ __forceinline__ C energy_face_flux_fast(const MacroAlong& MA, const FcolAt& FC, const Phys<C>& ph) {
  constexpr int D = L::D;
  const C cs2 = C(kCs2);
  C Ps = C(0), Ns = C(0), Pd = C(0), Nd = C(0);
  C Tm[3] = {C(0), C(0), C(0)};
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ca = L::c(i, AX);
    if constexpr (ca != 0) {
      constexpr int b0 = (ca < 0 && AX == 0) ? 1 : 0;
      constexpr int b1 = (ca < 0 && AX == 1) ? 1 : 0;
      constexpr int b2 = (ca < 0 && AX == 2) ? 1 : 0;
      constexpr int t = transverse_axis<L>(i, AX);
      if constexpr (t < 0) {
        if constexpr (ca > 0) Ps += FC(i, b0, b1, b2);
        else Ns += FC(i, b0, b1, b2);
      } else {
        constexpr int o0 = b0 - (t == 0 ? L::c(i, 0) : 0);
        constexpr int o1 = b1 - (t == 1 ? L::c(i, 1) : 0);
        constexpr int o2 = b2 - (t == 2 ? L::c(i, 2) : 0);
        const C u = FC(i, b0, b1, b2) + FC(i, o0, o1, o2);
        if constexpr (ca > 0) Pd += u;
        else Nd += u;
        constexpr int sgn = L::c(i, t) * ca;
        if constexpr (sgn > 0) Tm[t] += u;
        else Tm[t] -= u;
      }
    }
  });
  const C Frho = (Ps - Ns) + C(0.5) * (Pd - Nd);
  C Fm[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) Fm[b] = C(0.5) * Tm[b];
  Fm[AX] = (Ps + Ns) + C(0.5) * (Pd + Nd);
  const Macro<C> m1 = MA(0), m2 = MA(1);
  const bool plus = C(0.5) * (m1.u[AX] + m2.u[AX]) >= C(0);
  const Macro<C> mo = MA(plus ? -1 : 2);
  const C uB = plus ? m1.u[AX] : m2.u[AX];
  const C sg = uB > C(0) ? C(1) : (uB < C(0) ? C(-1) : C(0));
  const C eta = third<C>(C(2) * uB - sg);
  const C kap = C(0.25) * ((plus ? C(1) : C(-1)) - uB);
  const C al = kap * (C(1) + eta), be = kap * (C(1) - eta);
  // the face value B + al (B - A) + be (Cc - B) as weights of the cells
  // (outer, x, x + e): (A, B, Cc) = (outer, x, x + e) upwind of +, else
  // (x, x + e, outer)
  const C wB = C(1) + al - be;
  const C wo = plus ? -al : be;
  const C w1 = plus ? wB : -al;
  const C w2 = plus ? be : wB;
  auto rec = [&](C fo, C f1, C f2) { return wo * fo + w1 * f1 + w2 * f2; };
  const C po = mo.rho * cs2 * mo.th, p1 = m1.rho * cs2 * m1.th, p2 = m2.rho * cs2 * m2.th;
  const C FH = rec((mo.E + po) * mo.u[AX], (m1.E + p1) * m1.u[AX], (m2.E + p2) * m2.u[AX]);
  const C ro = mo.rho * mo.u[AX], r1 = m1.rho * m1.u[AX], r2 = m2.rho * m2.u[AX];
  const C Fr = rec(ro, r1, r2);
  C k1 = C(0), k2 = C(0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    k1 += m1.u[b] * m1.u[b];
    k2 += m2.u[b] * m2.u[b];
  }
  const C hk = C(0.5) * ((ph.Cp * m1.th + ph.Cp * m2.th) - C(0.5) * (k1 + k2));
  C FE = FH + hk * (Frho - Fr);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    const C Fb = rec(ro * mo.u[b] + (AX == b ? po : C(0)), r1 * m1.u[b] + (AX == b ? p1 : C(0)),
                     r2 * m2.u[b] + (AX == b ? p2 : C(0)));
    const C ub = C(0.5) * (m1.u[b] + m2.u[b]);
    FE = FE + ub * (Fm[b] - Fb);
  }
  FE = FE - ph.lam * (m2.th - m1.th);
  return FE;
}

// Total-energy flux F^{rhoE}_{+axis/2} through the face x + e_axis/2
// (Eq. energy).  MacroAlong(k) returns the Macro of cell x + k e_axis
// (k = -1..2); FcolAt(i, dx, dy, dz) returns f^col_i at x + (dx,dy,dz).
template <class L, class C, int AX, class MacroAlong, class FcolAt>
__device__ __forceinline__ C energy_face_flux(const MacroAlong& MA, const FcolAt& FC, const Phys<C>& ph) {
  if constexpr (sizeof(C) == 4) return energy_face_flux_fast<L, C, AX>(MA, FC, ph);
  constexpr int D = L::D;
  const C cs2 = C(kCs2);
  // LB mass and momentum fluxes (Eqs. fluxx-z and the rule below them)
  C Frho = C(0);
  C Fm[3] = {C(0), C(0), C(0)};
  auto add = [&](C v, auto I) {
    constexpr int i = decltype(I)::value;
    Frho = Frho + v;
    sfor<0, D>([&](auto B) {
      constexpr int b = decltype(B)::value;
      if constexpr (L::c(i, b) != 0) Fm[b] = Fm[b] + C(L::c(i, b)) * v;
    });
  };
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ca = L::c(i, AX);
    if constexpr (ca != 0) {
      constexpr int b0 = (ca < 0 && AX == 0) ? 1 : 0;
      constexpr int b1 = (ca < 0 && AX == 1) ? 1 : 0;
      constexpr int b2 = (ca < 0 && AX == 2) ? 1 : 0;
      constexpr int t = transverse_axis<L>(i, AX);
      if constexpr (t < 0) {
        add(C(ca) * FC(i, b0, b1, b2), I);
      } else {
        constexpr int o0 = b0 - (t == 0 ? L::c(i, 0) : 0);
        constexpr int o1 = b1 - (t == 1 ? L::c(i, 1) : 0);
        constexpr int o2 = b2 - (t == 2 ? L::c(i, 2) : 0);
        add(C(0.5 * ca) * FC(i, b0, b1, b2), I);
        add(C(0.5 * ca) * FC(i, o0, o1, o2), I);
      }
    }
  });
  // upwind stencil of the MUSCL reconstruction: only three cells are read
  const Macro<C> m1 = MA(0), m2 = MA(1);
  const bool plus = C(0.5) * (m1.u[AX] + m2.u[AX]) >= C(0);
  const Macro<C> mo = MA(plus ? -1 : 2);
  const Macro<C>& A = plus ? mo : m1;
  const Macro<C>& B = plus ? m1 : m2;
  const Macro<C>& Cc = plus ? m2 : mo;
  const C pA = A.rho * cs2 * A.th, pB = B.rho * cs2 * B.th, pC = Cc.rho * cs2 * Cc.th;
  const C uB = B.u[AX];
  const C FH = muscl3<C>((A.E + pA) * A.u[AX], (B.E + pB) * B.u[AX], (Cc.E + pC) * Cc.u[AX], uB, plus);
  const C Fr = muscl3<C>(A.rho * A.u[AX], B.rho * B.u[AX], Cc.rho * Cc.u[AX], uB, plus);
  C k1 = C(0), k2 = C(0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    k1 += m1.u[b] * m1.u[b];
    k2 += m2.u[b] * m2.u[b];
  }
  k1 = C(0.5) * k1;
  k2 = C(0.5) * k2;
  const C hk = C(0.5) * ((ph.Cp * m1.th - k1) + (ph.Cp * m2.th - k2));
  C FE = FH + hk * (Frho - Fr);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    const C Fb = muscl3<C>(A.rho * A.u[AX] * A.u[b] + (AX == b ? pA : C(0)),
                           B.rho * B.u[AX] * B.u[b] + (AX == b ? pB : C(0)),
                           Cc.rho * Cc.u[AX] * Cc.u[b] + (AX == b ? pC : C(0)), uB, plus);
    const C ub = C(0.5) * (m1.u[b] + m2.u[b]);
    FE = FE + ub * (Fm[b] - Fb);
  }
  FE = FE - ph.lam * (m2.th - m1.th);
  return FE;
}

}  // namespace lbmib
