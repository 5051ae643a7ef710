// Device building blocks of the fused lattice Boltzmann step: storage codecs,
// the pulled gather, the moments of Eq. 4.5 in deviation form, the
// equations of state, and the Hermite-space collision polynomial.
//
// Stored variable.  Populations are kept as Hermite-normalised deviations
//     g_i = (f^_i - w_i rho0) / w_i,
// so that f^eq_i and S_i, both of the form w_i sum_n A^(n) : H^(n)(xi_i) / n!
// (Eqs. 2.4-2.5), lose their weight factor, the stored numbers stay O(signal)
// (no cancellation against w_i rho0 in FP32, no FP16 subnormals for the small
// weights), and the update of Eq. 4.4 reads
//     g*_i = (1 - omega) g_i + sum_n B^(n) : H^(n)(xi_i) / n!,
//     B^(n) = omega a^(n,eq) + beta s^(n),  omega = 1/tau^, beta = 1 - 1/(2 tau^),
// with a^(0,eq) replaced by rho - rho0.
//
// Hermite coefficients (xi = c / c0, velocities and forces divided by c0).
// The Cartesian Hermite tensors factor per axis into probabilists' Hermite
// polynomials He_a, so a coefficient is indexed by its number of x, y (, z)
// indices (a, b (, c)) and the expansion is sum B_ab He_a(xi_x) He_b(xi_y) / (a! b!).
//  * Equilibrium (Eq. 2.6): the Hermite coefficients of the Maxwellian factor
//    into 1D Gaussian moments, a_ab = rho m_a(u_x) m_b(u_y) with
//    m_0 = 1, m_1 = u, m_2 = u^2 + tb, m_3 = u^3 + 3 u tb, m_4 = u^4 + 6 u^2 tb + 3 tb^2
//    (tb = theta - 1), truncated at order 4 (D2Q37) or 3 (D3Q39).
//  * Body force (Eq. 3.2): s^(1) = F, s^(2) = [F u], s^(3) = [F u u] + tb [F delta]
//    are exactly F . d/du of the equilibrium coefficients of orders 1-3 divided
//    by rho, so s_ab = F_x a m_{a-1}(u_x) m_b(u_y) + F_y b m_a(u_x) m_{b-1}(u_y).
//  * Thermal diffusion (Eq. 3.6): s^(3) += rho theta (1 - 1/Pr) [delta grad_xi theta].
//  * Pressure tensor (Eq. 3.12): s^(2) += sigma delta (trace only).
// The sum over n is then rewritten once per node as a polynomial in the
// integer velocity components, P(c) = sum_pq K_pq c_x^p c_y^q, whose monomials
// are compile-time constants per velocity; opposite velocities share the even
// part of P.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "lattice.cuh"

namespace hlbm {

// ------------------------------------------------------------------ codecs
template <int S> struct Codec;
template <> struct Codec<ST_F32> {
  using T = float;
  __device__ static __forceinline__ float ld(const T* p) { return __ldg(p); }
  __device__ static __forceinline__ void st(T* p, float v) { *p = v; }
};
template <> struct Codec<ST_F16> {
  using T = __half;
  __device__ static __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)); }
  __device__ static __forceinline__ void st(T* p, float v) { *p = __float2half_rn(v); }
};
template <> struct Codec<ST_BF16> {
  using T = __nv_bfloat16;
  __device__ static __forceinline__ float ld(const T* p) { return __bfloat162float(__ldg(p)); }
  __device__ static __forceinline__ void st(T* p, float v) { *p = __float2bfloat16_rn(v); }
};

// ----------------------------------------------------- compile-time helpers
__host__ __device__ constexpr int ipow_i(int x, int n) { return n == 0 ? 1 : x * ipow_i(x, n - 1); }
__host__ __device__ constexpr double ipow_d(double x, int n) { return n == 0 ? 1.0 : x * ipow_d(x, n - 1); }
__host__ __device__ constexpr double fact_d(int n) { return n <= 1 ? 1.0 : n * fact_d(n - 1); }
// coefficient of x^p in He_a(x) (a <= 4): He_2 = x^2 - 1, He_3 = x^3 - 3x, He_4 = x^4 - 6x^2 + 3
__host__ __device__ constexpr int he(int a, int p) {
  return a == 0   ? (p == 0 ? 1 : 0)
         : a == 1 ? (p == 1 ? 1 : 0)
         : a == 2 ? (p == 2 ? 1 : p == 0 ? -1 : 0)
         : a == 3 ? (p == 3 ? 1 : p == 1 ? -3 : 0)
                  : (p == 4 ? 1 : p == 2 ? -6 : p == 0 ? 3 : 0);
}

// 2D monomials c_x^p c_y^q, p + q <= 4
__host__ __device__ constexpr int mono2(int m, int axis) {
  constexpr int t[15][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}, {3, 0}, {2, 1},
                            {1, 2}, {0, 3}, {4, 0}, {3, 1}, {2, 2}, {1, 3}, {0, 4}};
  return t[m][axis];
}
// 3D monomials c_x^p c_y^q c_z^r, p + q + r <= 3
__host__ __device__ constexpr int mono3(int m, int axis) {
  constexpr int t[20][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
                            {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {3, 0, 0}, {0, 3, 0}, {0, 0, 3}, {2, 1, 0},
                            {2, 0, 1}, {1, 2, 0}, {0, 2, 1}, {1, 0, 2}, {0, 1, 2}, {1, 1, 1}};
  return t[m][axis];
}
__host__ __device__ constexpr int mono2_index(int p, int q) {
  for (int m = 0; m < 15; ++m)
    if (mono2(m, 0) == p && mono2(m, 1) == q) return m;
  return -1;
}
__host__ __device__ constexpr int mono3_index(int p, int q, int r) {
  for (int m = 0; m < 20; ++m)
    if (mono3(m, 0) == p && mono3(m, 1) == q && mono3(m, 2) == r) return m;
  return -1;
}

// ------------------------------------------------------------- index wrap
__device__ __forceinline__ int wrap1(int v, int n) {  // v in [-n, 2n)
  v += (v < 0) ? n : 0;
  v -= (v >= n) ? n : 0;
  return v;
}
__device__ __forceinline__ int wrapm(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// ------------------------------------------------------------------ gather
// g_i(x) = stored_i(x - c_i), periodic.  x in [0,nx), y in [0,ny), z in [0,nz).
template <class L, class C>
__device__ __forceinline__ void gather(const typename C::T* __restrict__ f, long long N, int nx, int ny,
                                       int nz, int x, int y, int z, float (&g)[L::Q]) {
  int xs[7], ys[7], zs[7];
#pragma unroll
  for (int d = -3; d <= 3; ++d) {
    xs[d + 3] = wrap1(x - d, nx);
    ys[d + 3] = wrap1(y - d, ny) * nx;
    if constexpr (L::D == 3) zs[d + 3] = wrap1(z - d, nz) * nx * ny;
  }
  static_for<L::Q>([&](auto I) {
    constexpr int i = I;
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    int off = ys[cy + 3] + xs[cx + 3];
    if constexpr (L::D == 3) off += zs[cz + 3];
    g[i] = C::ld(f + (size_t)i * (size_t)N + off);
  });
}

// ----------------------------------------------------------------- moments
// dr = sum w g (= rho - rho0), J = sum w c g (= sum c f^), Pi = sum w |c|^2 g
// (= sum |c|^2 f^ - rho0 D c0^2); opposite pairs share the sum and difference.
template <class L>
__device__ __forceinline__ void moments(const float (&g)[L::Q], float& dr, float (&J)[3], float& Pi) {
  dr = (float)L::w(0) * g[0];
  J[0] = J[1] = J[2] = 0.f;
  Pi = 0.f;
  static_for<L::NPAIR>([&](auto P) {
    constexpr int i = 2 * P + 1, j = 2 * P + 2;
    const float s = g[i] + g[j], d = g[i] - g[j];
    dr = fmaf((float)L::w(i), s, dr);
    Pi = fmaf((float)(L::w(i) * L::norm2(i)), s, Pi);
    static_for<L::D>([&](auto A) {
      constexpr int a = A;
      if constexpr (L::c(i, a) != 0) J[a] = fmaf((float)(L::w(i) * L::c(i, a)), d, J[a]);
    });
  });
}

template <class L>
__device__ __forceinline__ float sum_w(const float (&g)[L::Q]) {
  float dr = (float)L::w(0) * g[0];
  static_for<L::NPAIR>([&](auto P) {
    constexpr int i = 2 * P + 1, j = 2 * P + 2;
    dr = fmaf((float)L::w(i), g[i] + g[j], dr);
  });
  return dr;
}

// ---------------------------------------------------------- pseudopotential
// psi = sqrt(2 (p_EOS - rho c0^2) / (G c0^2)), G = -1, theta = 1 (Eq. 3.8)
template <class L>
__device__ __forceinline__ float psi_of(const StepArgs& a, float rho) {
  float p;
  if (a.eos == 0) {
    p = rho * a.eos_T / (1.f - a.eos_b * rho) - a.eos_a * rho * rho;
  } else {
    const float e = 0.25f * a.eos_b * rho;
    const float om = 1.f - e;
    p = rho * a.eos_T * (1.f + e + e * e - e * e * e) / (om * om * om) - a.eos_a * rho * rho;
  }
  const float s = (2.f / (float)L::cs2) * (rho * (float)L::cs2 - p);
  return sqrtf(fmaxf(s, 0.f));
}

// ---------------------------------------------------------- body acceleration
template <int D>
__device__ __forceinline__ void accel(const StepArgs& a, int node, int y, float (&g)[3]) {
  g[0] = g[1] = g[2] = 0.f;
  if (a.force_mode == FORCE_UNIFORM) {
#pragma unroll
    for (int d = 0; d < D; ++d) g[d] = a.g[d];
  } else if (a.force_mode == FORCE_FIELD) {
#pragma unroll
    for (int d = 0; d < D; ++d) g[d] = __ldg(a.gfield + (size_t)d * (size_t)a.N + node);
  } else if (a.force_mode == FORCE_PROFILE_Y) {
#pragma unroll
    for (int d = 0; d < D; ++d) g[d] = __ldg(a.gfield + (size_t)d * a.ny + y);
  }
}

// ------------------------------------------------------ collision polynomial
// Per-node inputs in xi units: u, F divided by c0; hG = rho theta (1 - 1/Pr)
// c0 grad theta; sigma the trace coefficient of P_i.
struct NodeSrc {
  float dr, rho, tb;
  float u[3], F[3], hG[3];
  float sigma;
};

// Hermite moments of a unit-variance-plus-tb Gaussian, m_0..m_4.
__device__ __forceinline__ void gauss_moments(float u, float tb, float (&m)[5]) {
  const float u2 = u * u;
  m[0] = 1.f;
  m[1] = u;
  m[2] = u2 + tb;
  m[3] = u * (u2 + 3.f * tb);
  m[4] = u2 * (u2 + 6.f * tb) + 3.f * tb * tb;
}

// K[m] (monomial m of mono2) for D2Q37: 4th-order equilibrium + sources.
template <class L>
__device__ __forceinline__ void poly2(const NodeSrc& s, float omega, float beta, float (&K)[15]) {
  float mx[5], my[5];
  gauss_moments(s.u[0], s.tb, mx);
  gauss_moments(s.u[1], s.tb, my);
#pragma unroll
  for (int m = 0; m < 15; ++m) K[m] = 0.f;
  static_for<5>([&](auto A) {
    static_for<5>([&](auto Bq) {
      constexpr int a = A, b = Bq;
      if constexpr (a + b <= L::FEQ_ORDER) {
        float eq = (a == 0 && b == 0) ? s.dr : s.rho * mx[a] * my[b];
        float src = 0.f;
        if constexpr (a + b >= 1 && a + b <= 3) {
          if constexpr (a > 0) src = fmaf(s.F[0] * (float)a, mx[a > 0 ? a - 1 : 0] * my[b], src);
          if constexpr (b > 0) src = fmaf(s.F[1] * (float)b, mx[a] * my[b > 0 ? b - 1 : 0], src);
        }
        if constexpr ((a == 2 && b == 0) || (a == 0 && b == 2)) src += s.sigma;
        if constexpr (a == 3 && b == 0) src = fmaf(3.f, s.hG[0], src);
        if constexpr (a == 2 && b == 1) src += s.hG[1];
        if constexpr (a == 1 && b == 2) src += s.hG[0];
        if constexpr (a == 0 && b == 3) src = fmaf(3.f, s.hG[1], src);
        const float Bab = fmaf(omega, eq, beta * src);
        // He_a(cx / c0) He_b(cy / c0) / (a! b!) -> monomials c_x^p c_y^q
        static_for<5>([&](auto Pp) {
          static_for<5>([&](auto Qq) {
            constexpr int p = Pp, q = Qq;
            if constexpr (p <= a && q <= b && he(a, p) != 0 && he(b, q) != 0) {
              constexpr float cf = (float)((double)(he(a, p) * he(b, q)) /
                                           (fact_d(a) * fact_d(b) * ipow_d(L::c0, p + q)));
              constexpr int m = mono2_index(p, q);
              K[m] = fmaf(cf, Bab, K[m]);
            }
          });
        });
      }
    });
  });
}

// K[m] (monomial m of mono3) for D3Q39: 3rd-order equilibrium + body force.
template <class L>
__device__ __forceinline__ void poly3(const NodeSrc& s, float omega, float beta, float (&K)[20]) {
  float mx[5], my[5], mz[5];
  gauss_moments(s.u[0], s.tb, mx);
  gauss_moments(s.u[1], s.tb, my);
  gauss_moments(s.u[2], s.tb, mz);
#pragma unroll
  for (int m = 0; m < 20; ++m) K[m] = 0.f;
  static_for<4>([&](auto A) {
    static_for<4>([&](auto Bq) {
      static_for<4>([&](auto Cr) {
        constexpr int a = A, b = Bq, c = Cr;
        if constexpr (a + b + c <= L::FEQ_ORDER) {
          float eq = (a == 0 && b == 0 && c == 0) ? s.dr : s.rho * mx[a] * my[b] * mz[c];
          float src = 0.f;
          if constexpr (a + b + c >= 1) {
            if constexpr (a > 0) src = fmaf(s.F[0] * (float)a, mx[a > 0 ? a - 1 : 0] * my[b] * mz[c], src);
            if constexpr (b > 0) src = fmaf(s.F[1] * (float)b, mx[a] * my[b > 0 ? b - 1 : 0] * mz[c], src);
            if constexpr (c > 0) src = fmaf(s.F[2] * (float)c, mx[a] * my[b] * mz[c > 0 ? c - 1 : 0], src);
          }
          if constexpr ((a == 2 && b == 0 && c == 0) || (a == 0 && b == 2 && c == 0) ||
                        (a == 0 && b == 0 && c == 2))
            src += s.sigma;
          // [delta hG] components: (3,0,0) -> 3 hGx, (2,1,0) -> hGy, (1,2,0) -> hGx, ...
          if constexpr (a + b + c == 3) {
            if constexpr (a == 3) src = fmaf(3.f, s.hG[0], src);
            if constexpr (b == 3) src = fmaf(3.f, s.hG[1], src);
            if constexpr (c == 3) src = fmaf(3.f, s.hG[2], src);
            if constexpr (a == 2 && b == 1) src += s.hG[1];
            if constexpr (a == 2 && c == 1) src += s.hG[2];
            if constexpr (b == 2 && a == 1) src += s.hG[0];
            if constexpr (b == 2 && c == 1) src += s.hG[2];
            if constexpr (c == 2 && a == 1) src += s.hG[0];
            if constexpr (c == 2 && b == 1) src += s.hG[1];
          }
          const float Babc = fmaf(omega, eq, beta * src);
          static_for<4>([&](auto Pp) {
            static_for<4>([&](auto Qq) {
              static_for<4>([&](auto Rr) {
                constexpr int p = Pp, q = Qq, r = Rr;
                if constexpr (p <= a && q <= b && r <= c && he(a, p) != 0 && he(b, q) != 0 && he(c, r) != 0) {
                  constexpr float cf = (float)((double)(he(a, p) * he(b, q) * he(c, r)) /
                                               (fact_d(a) * fact_d(b) * fact_d(c) * ipow_d(L::c0, p + q + r)));
                  constexpr int m = mono3_index(p, q, r);
                  K[m] = fmaf(cf, Babc, K[m]);
                }
              });
            });
          });
        }
      });
    });
  });
}

// Evaluates P(c_i) for all velocities and applies g*_i = (1 - omega) g_i + P(c_i)
// in place; the even part of P is shared by each opposite pair.
template <class L, int NM>
__device__ __forceinline__ void apply_poly(float (&g)[L::Q], const float (&K)[NM], float om1) {
  g[0] = fmaf(om1, g[0], K[0]);
  static_for<L::NPAIR>([&](auto P) {
    constexpr int i = 2 * P + 1, j = 2 * P + 2;
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    float E = K[0], O = 0.f;
    static_for<NM>([&](auto M) {
      constexpr int m = M;
      if constexpr (m > 0) {
        constexpr int px = (NM == 15) ? mono2(m, 0) : mono3(m, 0);
        constexpr int py = (NM == 15) ? mono2(m, 1) : mono3(m, 1);
        constexpr int pz = (NM == 15) ? 0 : mono3(m, 2);
        constexpr int mv = ipow_i(cx, px) * ipow_i(cy, py) * ipow_i(cz, pz);
        if constexpr (mv != 0) {
          if constexpr ((px + py + pz) % 2 == 0) {
            if constexpr (mv == 1) E += K[m];
            else E = fmaf((float)mv, K[m], E);
          } else {
            if constexpr (mv == 1) O += K[m];
            else if constexpr (mv == -1) O -= K[m];
            else O = fmaf((float)mv, K[m], O);
          }
        }
      }
    });
    g[i] = fmaf(om1, g[i], E + O);
    g[j] = fmaf(om1, g[j], E - O);
  });
}

}  // namespace hlbm
