// D2Q37 step between two Tamm-Mott-Smith walls (Sec. 4.3, Eqs. 4.7-4.8),
// periodic in x: the wall-bounded cases of Sec. 5.1-5.3 (thermal Couette and
// Poiseuille flow, Rayleigh-Benard convection).
//
// Geometry: rows 0 and ny - 1 are the wall nodes; the solid-liquid interfaces
// lie half a cell inside them (y = 1/2 and ny - 3/2), so the fluid layer is
// H = ny - 2 high.  A node whose pull source y - c_iy lies outside the rows
// has an unknown population i (the wall rows and the two rows next to each).
//
// Completion of the unknowns at a node r rows from its wall node, with the
// node's moments of the previous step (rho_p, u_p, theta_p) and those of the
// first fluid row of its column (u_1, theta_1):
//   f_i = f*_ibar(x) + s f^eq_i(rho_p, u_i, theta_i) - f^eq_ibar(rho_p, u_p, theta_p)
// (Eq. 4.7).  f*_ibar(x) is the population that left x in the opposite
// direction at the last streaming: in the pull layout it is still stored at x.
// u_i, theta_i are the wall's velocity and temperature extrapolated linearly
// from the interface through (u_1, theta_1) to the point where population i
// turned back, r - |c_iy| / 2 rows from the wall node.  s makes the unknowns
// carry exactly the mass that left (impermeable wall):
//   s = sum_U f^eq_ibar(p) / sum_U f^eq_i(targets).
// In stored units g = f / w - rho0 (w_i = w_ibar):
//   g_i = g*_ibar + rho_p (s P_i - P_ibar),   f^eq_i = w_i rho P_i.
//
// Stored values are deviations from the rest equilibrium at a reference
// temperature theta_r (the mean of the wall temperatures):
//   h_i = f_i / w_i - rho0 P_i(0, theta_r),
// so a fluid near theta_r stores small numbers (with the reference theta = 1
// of the periodic kernels, a fluid at theta = 0.8 stores O(1) values and the
// FP32 collision loses a decimal digit).  The offset r_i = rho0 (P_i(0,
// theta_r) - 1) has zero mass and momentum and energy sum_i w_i |c_i|^2 r_i =
// rho0 D c0^2 (theta_r - 1); the collision subtracts omega r_i
// (h* = (1 - omega) h + omega (g^eq - r) + beta S), and the completion is
// the same in h as in g (r_i = r_ibar).
//
// Each step is three launches: wall_complete_kernel completes the unknowns of
// the six wall rows in FP64 into a small buffer; wall_moments_kernel pulls
// every node's populations (the unknowns from that buffer) and writes its
// moments (rho, u, theta - 1) of time t, which are the next step's targets and
// the neighbour temperatures of grad theta; wall_collide_kernel pulls again,
// collides (Eq. 4.4 with F_i and H_i) and stores.  grad theta is a
// second-order central difference, one-sided into the fluid at the wall rows.
// Two reads of the populations per step: these domains are the paper's
// validation cases, a few thousand to a few hundred thousand nodes.
#include "internal.h"
#include "lattice.cuh"
#include "step_common.cuh"

#include <type_traits>

namespace hlbm {
namespace {

using L = D2Q37;
constexpr int kBX = 32, kBY = 8;

__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : (((i - 1) & 1) ? i - 1 : i + 1); }

__device__ __forceinline__ int wrapx(int v, int n) {
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

// P_i - 1 for f^eq_i = w_i rho P_i (Eq. 2.2): the Hermite expansion
// sum_{a+b<=4} m_a(u_x) m_b(u_y) He_a(xi_x) He_b(xi_y) / (a! b!), without the
// (0, 0) term, u in units of c0, m_a the Hermite moments of a Gaussian of
// variance 1 + tb.  FP64: the completion differences two such values whose
// difference is O(u), which FP32 would leave with O(1e-7) absolute error at
// every wall node and step (a drift in mass and momentum at the walls).
__device__ __forceinline__ void gauss_moments_d(double u, double tb, double (&m)[5]) {
  const double u2 = u * u;
  m[0] = 1.0;
  m[1] = u;
  m[2] = u2 + tb;
  m[3] = u * (u2 + 3.0 * tb);
  m[4] = u2 * (u2 + 6.0 * tb) + 3.0 * tb * tb;
}
// P_i - 1 from precomputed products: hp[k] = m_a(u_x) m_b(u_y) for
// the 14 index pairs (a, b) with 1 <= a + b <= 4 (k = hk(a, b)), so that the
// completion forms the products once per state (the node's previous moments,
// and one wall target per |c_y|) and then costs 14 FP64 multiply-adds per
// population instead of a whole expansion.
__host__ __device__ constexpr int hk(int a, int b) {
  return (a + b == 1) ? a : (a + b == 2) ? 2 + a : (a + b == 3) ? 5 + a : 9 + a;
}
__device__ __forceinline__ void herm_prod(double ux, double uy, double tb, double (&hp)[14]) {
  double mx[5], my[5];
  gauss_moments_d(ux * (1.0 / L::c0), tb, mx);
  gauss_moments_d(uy * (1.0 / L::c0), tb, my);
  static_for<5>([&](auto A) {
    static_for<5>([&](auto B) {
      constexpr int a = A, b = B;
      if constexpr (a + b >= 1 && a + b <= L::FEQ_ORDER) hp[hk(a, b)] = mx[a] * my[b];
    });
  });
}
template <int I>
__device__ __forceinline__ double peq_m1_hp(const double (&hp)[14]) {
  constexpr int cx = L::c(I, 0), cy = L::c(I, 1);
  double acc = 0.0;
  static_for<5>([&](auto A) {
    static_for<5>([&](auto B) {
      constexpr int a = A, b = B;
      if constexpr (a + b >= 1 && a + b <= L::FEQ_ORDER) {
        constexpr double hx = [] {
          double s = 0.0;
          for (int p = 0; p <= a; ++p) s += he(a, p) * ipow_d((double)cx / L::c0, p);
          return s;
        }();
        constexpr double hy = [] {
          double s = 0.0;
          for (int q = 0; q <= b; ++q) s += he(b, q) * ipow_d((double)cy / L::c0, q);
          return s;
        }();
        constexpr double cf = hx * hy / (fact_d(a) * fact_d(b));
        if constexpr (cf != 0.0) acc = fma(cf, hp[hk(a, b)], acc);
      }
    });
  });
  return acc;
}

template <int ST>
__device__ __forceinline__ float ldpop(const WallArgs& a, int i, int x, int y) {
  using T = typename Codec<ST>::T;
  return Codec<ST>::ld(static_cast<const T*>(a.fin) +
                       HLBM_IDX((long long)i * a.N + (long long)y * a.nx + x, 37 * a.N, DBG_GATHER));
}

__device__ __forceinline__ void wall_accel(const WallArgs& a, int node, int y, float& gx, float& gy) {
  gx = gy = 0.f;
  if (a.force_mode == FORCE_UNIFORM) {
    gx = a.g[0];
    gy = a.g[1];
  } else if (a.force_mode == FORCE_FIELD) {
    gx = __ldg(a.gfield + node);
    gy = __ldg(a.gfield + (size_t)a.N + node);
  } else if (a.force_mode == FORCE_PROFILE_Y) {
    gx = __ldg(a.gfield + y);
    gy = __ldg(a.gfield + a.ny + y);
  }
}

// Completion of the unknowns of a wall-row node (x, y), r = 0, 1, 2 rows from
// its wall node: written to a.comp[slot][i][x] (slot = 3 side + r) for every
// unknown i.  It runs once per step, before the two launches that read the
// populations, in a launch of its own over the six wall rows, so that its
// FP64 arithmetic neither stalls the blocks of the full-domain launches nor
// is done twice.
template <int ST>
__device__ __forceinline__ void wall_complete(const WallArgs& a, int x, int y) {
  const int nx = a.nx, ny = a.ny;
  const int side = (y < ny / 2) ? 0 : 1;
  const int r = side == 0 ? y : ny - 1 - y;
  const size_t N = (size_t)a.N;
  const int node = y * nx + x;
  const int node1 = (side == 0 ? 1 : ny - 2) * nx + x;
  const double rp = __ldg(a.mprev + node);
  const double upx = __ldg(a.mprev + N + node), upy = __ldg(a.mprev + 2 * N + node);
  const double tbp = __ldg(a.mprev + 3 * N + node);
  const double u1x = __ldg(a.mprev + N + node1), u1y = __ldg(a.mprev + 2 * N + node1);
  const double tb1 = __ldg(a.mprev + 3 * N + node1);
  const double uwx = a.wall_u[side][0], uwy = a.wall_u[side][1], tbw = a.wall_tb[side];
  // Hermite products of the previous moments and of the wall target of each
  // |c_y| = 1, 2, 3 (extrapolated to the turning point)
  double hpp[14], hpt[3][14];
  herm_prod(upx, upy, tbp, hpp);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double wgt = (double)(2 + k - 2 * r);   // (1/2 - turning point) / (1/2), |c_y| = k + 1
    herm_prod(fma(wgt, uwx - u1x, uwx), fma(wgt, uwy - u1y, uwy), fma(wgt, tbw - tb1, tbw), hpt[k]);
  }
  // sums over the unknowns of w P_i(targets) - w and w P_ibar(p) - w
  double W = 0.0, A = 0.0, B = 0.0;
  static_for<37>([&](auto I) {
    constexpr int i = I;
    constexpr int cy = L::c(i, 1), ab = cy < 0 ? -cy : cy;
    constexpr int b = opp_of(i);
    if constexpr (ab > 0) {
      if (y - cy < 0 || y - cy >= ny) {
        constexpr double w = L::w(i);
        W += w;
        A = fma(w, peq_m1_hp<i>(hpt[ab - 1]), A);
        B = fma(w, peq_m1_hp<b>(hpp), B);
      }
    }
  });
  const double sm1 = (B - A) / (W + A);            // s - 1
  float* comp = a.comp + (size_t)(3 * side + r) * 37 * nx + x;
  static_for<37>([&](auto I) {
    constexpr int i = I;
    constexpr int cy = L::c(i, 1), ab = cy < 0 ? -cy : cy;
    constexpr int b = opp_of(i);
    if constexpr (ab > 0) {
      if (y - cy < 0 || y - cy >= ny) {
        const double pi = peq_m1_hp<i>(hpt[ab - 1]), pb = peq_m1_hp<b>(hpp);
        // s P_i - P_ibar = (s - 1) + s (P_i - 1) - (P_ibar - 1)
        comp[(size_t)i * nx] = (float)fma(rp, sm1 + fma(sm1, pi, pi) - pb, (double)ldpop<ST>(a, b, x, y));
      }
    }
  });
}

// The 37 populations of node (x, y) at time t after streaming, the unknowns
// at the walls taken from the completion launch.
template <int ST>
__device__ __forceinline__ void wall_gather(const WallArgs& a, int x, int y, float (&g)[37]) {
  const int nx = a.nx, ny = a.ny;
  const int side = (y < ny / 2) ? 0 : 1;
  const int r = side == 0 ? y : ny - 1 - y;
  const float* comp = a.comp + (size_t)(3 * side + (r < 3 ? r : 0)) * 37 * nx + x;
  static_for<37>([&](auto I) {
    constexpr int i = I;
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1);
    const int ys = y - cy;
    g[i] = (ys >= 0 && ys < ny) ? ldpop<ST>(a, i, wrapx(x - cx, nx), ys) : __ldg(comp + (size_t)i * nx);
  });
}

// Collision polynomial relative to the reference rest equilibrium: the
// coefficients of poly2 (step_common.cuh) with each equilibrium Hermite
// coefficient rho m_a(u_x) m_b(u_y) replaced by
//   rho m_a m_b - rho0 m_a(0, tr) m_b(0, tr),   m(0, tr) = (1, 0, tr, 0, 3 tr^2),
// written in terms that are all small near the reference state
// (d = theta - theta_r, dr = rho - rho0, t = tr + d):
//   (2,0): rho u_x^2 + rho d + dr tr
//   (4,0): rho u_x^4 + 6 rho u_x^2 t + 3 (dr tr^2 + rho d (2 tr + d))
//   (2,2): rho (u_x^2 u_y^2 + t (u_x^2 + u_y^2)) + dr tr^2 + rho d (2 tr + d)
// and the odd ones unchanged (they carry a factor u).  Forming rho m_a m_b
// (O(theta - 1)) and then subtracting the reference would leave an FP32
// residual that is the same at every node: a systematic drift of mass and
// energy.  u, F in units of c0; s.tb holds d.
__device__ __forceinline__ void poly2_ref(const NodeSrcT<float>& s, float dr, float tr, float omega, float beta,
                                          float (&K)[15]) {
  const float X = s.u[0], Y = s.u[1], d = s.tb, t = tr + d, rho = s.rho;
  float mx[5], my[5];
  gauss_moments(X, t, mx);
  gauss_moments(Y, t, my);
  const float X2 = X * X, Y2 = Y * Y;
  const float c2 = fmaf(rho, d, dr * tr);                              // rho t - rho0 tr
  const float c4 = 3.f * fmaf(dr, tr * tr, rho * d * (2.f * tr + d));    // 3 (rho t^2 - rho0 tr^2)
  float EQ[5][5];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) EQ[a][b] = rho * mx[a] * my[b];
  EQ[2][0] = fmaf(rho, X2, c2);
  EQ[0][2] = fmaf(rho, Y2, c2);
  EQ[4][0] = fmaf(rho, X2 * X2, fmaf(6.f * rho, X2 * t, c4));
  EQ[0][4] = fmaf(rho, Y2 * Y2, fmaf(6.f * rho, Y2 * t, c4));
  EQ[2][2] = fmaf(rho, fmaf(X2, Y2, t * (X2 + Y2)), c4 * (1.f / 3.f));
#pragma unroll
  for (int m = 0; m < 15; ++m) K[m] = 0.f;
  static_for<5>([&](auto A) {
    static_for<5>([&](auto Bq) {
      constexpr int a = A, b = Bq;
      if constexpr (a + b <= L::FEQ_ORDER && a + b >= 1) {
        float src = 0.f;
        if constexpr (a + b <= 3) {
          if constexpr (a > 0) src = fmaf(s.F[0] * (float)a, mx[a > 0 ? a - 1 : 0] * my[b], src);
          if constexpr (b > 0) src = fmaf(s.F[1] * (float)b, mx[a] * my[b > 0 ? b - 1 : 0], src);
        }
        if constexpr (a == 3 && b == 0) src = fmaf(3.f, s.hG[0], src);
        if constexpr (a == 2 && b == 1) src += s.hG[1];
        if constexpr (a == 1 && b == 2) src += s.hG[0];
        if constexpr (a == 0 && b == 3) src = fmaf(3.f, s.hG[1], src);
        const float Bab = fmaf(omega, EQ[a][b], beta * src);
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

// Moments of Eq. 4.5 (thermal mode, F = rho g) of completed populations; h is
// left in the local-deviation form of moments_h.
struct WallMoments {
  float dr, acc, rho, ux, uy, tb, dth, Fx, Fy, Pih, G2;
};
__device__ __forceinline__ WallMoments wall_moments(const WallArgs& a, float (&g)[37], int node, int y) {
  WallMoments m;
  float J[3];
  moments_h<L>(g, m.dr, m.acc, J, m.Pih);
  m.rho = a.rho0 + m.dr;
  float gx, gy;
  wall_accel(a, node, y, gx, gy);
  m.Fx = m.rho * gx;
  m.Fy = m.rho * gy;
  const float inv = rcp_nr(m.rho);
  m.ux = fmaf(0.5f, m.Fx, J[0]) * inv;
  m.uy = fmaf(0.5f, m.Fy, J[1]) * inv;
  m.G2 = 2.f * fmaf(m.ux, m.Fx, m.uy * m.Fy);
  constexpr float Dc = (float)(2.0 * L::cs2);
  // theta - theta_r = (Pih_h - rho |u|^2 + G2 / 2 - dr D c0^2 tr) / (rho D c0^2),
  // Pih_h = sum_i w_i |c_i|^2 (h_i - dr) (the reference offset's energy
  // rho0 D c0^2 tr taken out exactly)
  m.dth = (fmaf(0.5f, m.G2, fmaf(-m.dr * Dc, a.tb_ref, m.Pih - m.rho * fmaf(m.ux, m.ux, m.uy * m.uy))) * inv) *
          (1.f / Dc);
  m.tb = a.tb_ref + m.dth;
  m.Pih += a.e_ref;                                // sum_i |c_i|^2 f_i - rho D c0^2
  return m;
}

template <int ST>
__global__ void __launch_bounds__(kBX * kBY, 4) wall_moments_kernel(const __grid_constant__ WallArgs a) {
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const bool active = x < a.nx && y < a.ny;
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (active) {
    float g[37];
    wall_gather<ST>(a, x, y, g);
    const int node = y * a.nx + x;
    const WallMoments m = wall_moments(a, g, node, y);
    const size_t N = (size_t)a.N;
    if (a.mcur) {
      a.mcur[node] = m.rho;
      a.mcur[N + node] = m.ux;
      a.mcur[2 * N + node] = m.uy;
      a.mcur[3 * N + node] = m.tb;
    }
    if (a.rho_out) a.rho_out[node] = m.rho;
    if (a.u_out) {
      a.u_out[node] = m.ux;
      a.u_out[N + node] = m.uy;
    }
    if (a.theta_out) a.theta_out[node] = 1.f + m.tb;
    constexpr float Dc = (float)(2.0 * L::cs2);
    const bool bad = !(isfinite(m.rho) && m.rho > 0.f && isfinite(m.ux) && isfinite(m.uy) && isfinite(m.tb));
    v[0] = m.dr;
    v[1] = (double)m.rho * m.ux;
    v[2] = (double)m.rho * m.uy;
    v[4] = 0.5 * ((double)m.Pih + (double)Dc * m.dr + 0.5 * (double)m.G2);
    v[5] = bad ? 1.0 : 0.0;
  }
  if (a.partials) {
    __shared__ double red[kBY][6];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < 6; ++k) red[threadIdx.y][k] = v[k];
    __syncthreads();
    const int tid = threadIdx.y * kBX + threadIdx.x;
    if (tid < 6) {
      double s = 0.0;
      for (int w = 0; w < kBY; ++w) s += red[w][tid];
      a.partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + tid] = s;
    }
  }
}

template <int ST, bool THERMAL>
__global__ void __launch_bounds__(kBX * kBY, 3) wall_collide_kernel(const __grid_constant__ WallArgs a) {
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const int nx = a.nx, ny = a.ny;
  const size_t N = (size_t)a.N;
  const int node = y * nx + x;
  float g[37];
  wall_gather<ST>(a, x, y, g);
  const WallMoments m = wall_moments(a, g, node, y);
  NodeSrcT<float> s;
  s.hG[0] = s.hG[1] = s.hG[2] = 0.f;
  if constexpr (THERMAL) {
    const float* tb = a.mcur + 3 * N;
    const float gtx = 0.5f * (tb[y * nx + wrapx(x + 1, nx)] - tb[y * nx + wrapx(x - 1, nx)]);
    float gty;
    if (y == 0)
      gty = 0.5f * (-3.f * tb[node] + 4.f * tb[node + nx] - tb[node + 2 * nx]);
    else if (y == ny - 1)
      gty = -0.5f * (-3.f * tb[node] + 4.f * tb[node - nx] - tb[node - 2 * nx]);
    else
      gty = 0.5f * (tb[node + nx] - tb[node - nx]);
    // s^(3) += rho theta (1 - 1/Pr) [delta grad_xi theta], grad_xi = c0 grad
    const float hc = m.rho * (1.f + m.tb) * (a.h_coef * (float)L::c0);
    s.hG[0] = hc * gtx;
    s.hG[1] = hc * gty;
  }
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  s.dr = 0.f;
  s.rho = m.rho;
  s.tb = m.dth;
  s.u[0] = m.ux * inv_c0;
  s.u[1] = m.uy * inv_c0;
  s.u[2] = 0.f;
  s.F[0] = m.Fx * inv_c0;
  s.F[1] = m.Fy * inv_c0;
  s.F[2] = 0.f;
  s.sigma = 0.f;
  float K[15];
  poly2_ref(s, m.dr, a.tb_ref, a.omega, a.beta, K);
  const float om1 = 1.f - a.omega;
  K[0] = fmaf(-om1, m.acc, K[0]);
  apply_poly_h<L, 15>(g, K, om1, m.dr);
  using T = typename Codec<ST>::T;
  if (!HLBM_IN(node, a.N, DBG_STORE)) return;
  T* __restrict__ fout = static_cast<T*>(a.fout) + node;
  const uint32_t salt = std::is_same<T, float>::value ? 0u : node_salt(node, g[0]);
  static_for<37>([&](auto I) {
    constexpr int i = I;
    fout[(size_t)i * N] = round_store<T>(g[i], pop_bits(salt, i));
  });
}

// Initial state: h_i = f^eq_i(rho, u, theta) / w_i - rho0 P_i(0, theta_r),
// stored where the first step pulls it from (x - c_i, periodic like the
// periodic initialisation), and the previous-step moments = the initial fields.
template <int ST>
__global__ void __launch_bounds__(256) wall_init_kernel(const __grid_constant__ WallArgs a, const float* __restrict__ rho,
                                                        const float* __restrict__ u, const float* __restrict__ theta,
                                                        float* m) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = a.N;
  if (n >= N) return;
  const int x = (int)(n % a.nx), y = (int)(n / a.nx);
  m[n] = rho[n];
  m[N + n] = u[n];
  m[2 * N + n] = u[N + n];
  m[3 * N + n] = theta[n] - 1.f;
  NodeSrcT<float> s;
  const float dr = rho[n] - a.rho0;
  s.dr = 0.f;
  s.rho = rho[n];
  s.tb = (theta[n] - 1.f) - a.tb_ref;
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  s.u[0] = u[n] * inv_c0;
  s.u[1] = u[N + n] * inv_c0;
  s.u[2] = 0.f;
  s.F[0] = s.F[1] = s.F[2] = 0.f;
  s.hG[0] = s.hG[1] = s.hG[2] = 0.f;
  s.sigma = 0.f;
  float K[15], h[37];
  poly2_ref(s, dr, a.tb_ref, 1.f, 0.f, K);
  K[0] += dr;
#pragma unroll
  for (int i = 0; i < 37; ++i) h[i] = 0.f;
  apply_poly<L, 15>(h, K, 0.f);
  using T = typename Codec<ST>::T;
  T* __restrict__ fout = static_cast<T*>(a.fout);
  static_for<37>([&](auto I) {
    constexpr int i = I;
    const int xs = wrap1(x - L::c(i, 0), a.nx), ys = wrap1(y - L::c(i, 1), a.ny);
    Codec<ST>::st(fout + (size_t)i * (size_t)N + (size_t)ys * a.nx + xs, h[i]);
  });
}

// One thread per node of the six wall rows (rows 0, 1, 2 and ny - 1, ny - 2,
// ny - 3), one warp per block so that the FP64 work spreads over the SMs.
template <int ST>
__global__ void __launch_bounds__(32) wall_complete_kernel(const __grid_constant__ WallArgs a) {
  const int t = blockIdx.x * 32 + threadIdx.x;
  if (t >= 6 * a.nx) return;
  const int slot = t / a.nx, x = t - slot * a.nx;
  const int y = slot < 3 ? slot : a.ny - 1 - (slot - 3);
  wall_complete<ST>(a, x, y);
}

template <int ST>
cudaError_t launch_walls_st(const WallArgs& a, int mode, bool thermal, cudaStream_t s) {
  if (mode == 2) {
    wall_complete_kernel<ST><<<(6 * a.nx + 31) / 32, 32, 0, s>>>(a);
    return cudaGetLastError();
  }
  const bool collide = mode == 1;
  const dim3 block(kBX, kBY), grid((a.nx + kBX - 1) / kBX, (a.ny + kBY - 1) / kBY);
  if (!collide)
    wall_moments_kernel<ST><<<grid, block, 0, s>>>(a);
  else if (thermal)
    wall_collide_kernel<ST, true><<<grid, block, 0, s>>>(a);
  else
    wall_collide_kernel<ST, false><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wall_init(const WallArgs& a, int storage, const float* rho, const float* u, const float* theta,
                             float* m, cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.N + 255) / 256);
  switch (storage) {
    case ST_F32: wall_init_kernel<ST_F32><<<blocks, 256, 0, s>>>(a, rho, u, theta, m); break;
    case ST_F16: wall_init_kernel<ST_F16><<<blocks, 256, 0, s>>>(a, rho, u, theta, m); break;
    default: wall_init_kernel<ST_BF16><<<blocks, 256, 0, s>>>(a, rho, u, theta, m); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_walls(const WallArgs& a, int storage, int mode, bool thermal, cudaStream_t s) {
  switch (storage) {
    case ST_F32: return launch_walls_st<ST_F32>(a, mode, thermal, s);
    case ST_F16: return launch_walls_st<ST_F16>(a, mode, thermal, s);
    default: return launch_walls_st<ST_BF16>(a, mode, thermal, s);
  }
}

}  // namespace hlbm
