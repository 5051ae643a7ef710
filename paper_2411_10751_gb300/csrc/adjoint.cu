// Discrete adjoint of the fused step with a body-force field, with
// checkpoint-and-recompute, for the gradient of the kinetic energy
// L = sum_x rho |u|^2 / 2 at step T with respect to the acceleration field g.
//
// Notation (pull scheme): f_n are the populations after streaming at time n,
// C the local collision of Eq. 4.4 (equilibrium of Eq. 2.2 and body force of
// Eq. 3.3 with F = rho g), G the streaming, f_{n+1} = G(C(f_n, g)).
//   seed:    lambda_T,i = dL/df_T,i = |u|^2/2 - u.j/rho + c_i.u,  dL/dg = rho u / 2
//   step:    mu_i(x) = lambda_{n+1,i}(x + c_i)                      (reverse streaming)
//            lambda_n = (1 - omega) mu + dPhi/df,  dL/dg(x) += dPhi/dg
// where Phi = sum_i mu_i (C_i - (1 - omega) f_i) = sum_ab B_ab M_ab / (a! b!)
// (M the weighted Hermite moments of mu, B = omega a^eq + beta s the
// coefficients of the collision), a polynomial in (rho, u, theta-bar, F).
// Its partial derivatives come from a forward-mode dual-number evaluation;
// the chain rule through u = j/rho + g/2, theta-bar(e, rho, u, g) and F = rho g
// then gives the derivatives with respect to rho = sum f, j = sum c f,
// e = sum |c|^2 f and g.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "hlbm.h"
#include "internal.h"
#include "step_common.cuh"

namespace hlbm {
namespace {

// value and NV partial derivatives
template <int NV>
struct Dual {
  float v;
  float d[NV];
};
template <int NV>
__device__ __forceinline__ Dual<NV> dconst(float c) {
  Dual<NV> r;
  r.v = c;
#pragma unroll
  for (int k = 0; k < NV; ++k) r.d[k] = 0.f;
  return r;
}
template <int NV>
__device__ __forceinline__ Dual<NV> dvar(float v, int k0) {
  Dual<NV> r = dconst<NV>(v);
#pragma unroll
  for (int k = 0; k < NV; ++k) r.d[k] = (k == k0) ? 1.f : 0.f;
  return r;
}
template <int NV>
__device__ __forceinline__ Dual<NV> operator+(const Dual<NV>& a, const Dual<NV>& b) {
  Dual<NV> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < NV; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int NV>
__device__ __forceinline__ Dual<NV> operator*(const Dual<NV>& a, const Dual<NV>& b) {
  Dual<NV> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < NV; ++k) r.d[k] = fmaf(a.v, b.d[k], a.d[k] * b.v);
  return r;
}
template <int NV>
__device__ __forceinline__ Dual<NV> operator*(float s, const Dual<NV>& a) {
  Dual<NV> r;
  r.v = s * a.v;
#pragma unroll
  for (int k = 0; k < NV; ++k) r.d[k] = s * a.d[k];
  return r;
}

// He_n(c / c0) (n <= 4) at integer c, as a compile-time constant
template <class L>
__host__ __device__ constexpr double he_at(int n, int c) {
  double r = 0.0;
  for (int p = 0; p <= n; ++p) r += he(n, p) * ipow_d((double)c / L::c0, p);
  return r;
}

template <class L>
struct AdjCfg {
  static constexpr int D = L::D;
  static constexpr int NM = (D == 2) ? 15 : 20;
  static constexpr int NV = 2 * D + 2;  // rho, u (D), theta-bar, F (D)
  __host__ __device__ static constexpr int mono(int m, int ax) { return D == 2 ? (ax < 2 ? mono2(m, ax) : 0) : mono3(m, ax); }
};

// Phi(rho, u, tb, F) = sum_m B_m M_m / (a! b! c!) with dual inputs in lattice units.
template <class L>
__device__ __forceinline__ Dual<AdjCfg<L>::NV> phi_dual(const float (&M)[AdjCfg<L>::NM], float rho, const float (&u)[3],
                                                       float tb, const float (&F)[3], bool thermal, float omega,
                                                       float beta) {
  using A = AdjCfg<L>;
  constexpr int D = A::D, NV = A::NV;
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  const Dual<NV> r = dvar<NV>(rho, 0);
  Dual<NV> ux[3], fx[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ux[a] = (a < D) ? inv_c0 * dvar<NV>(u[a], 1 + a) : dconst<NV>(0.f);
    fx[a] = (a < D) ? inv_c0 * dvar<NV>(F[a], 2 + D + a) : dconst<NV>(0.f);
  }
  const Dual<NV> t = thermal ? dvar<NV>(tb, 1 + D) : dconst<NV>(0.f);
  // per-axis Gaussian Hermite moments m_0..m_4 of N(u, 1 + tb)
  Dual<NV> m[3][5];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Dual<NV> u2 = ux[a] * ux[a];
    m[a][0] = dconst<NV>(1.f);
    m[a][1] = ux[a];
    m[a][2] = u2 + t;
    m[a][3] = ux[a] * (u2 + 3.f * t);
    m[a][4] = u2 * (u2 + 6.f * t) + 3.f * (t * t);
  }
  Dual<NV> phi = dconst<NV>(0.f);
  static_for<A::NM>([&](auto Mi) {
    constexpr int mi = Mi;
    constexpr int a = A::mono(mi, 0), b = A::mono(mi, 1), c = A::mono(mi, 2);
    constexpr int n = a + b + c;
    // equilibrium coefficient (a_000 = rho)
    Dual<NV> eq = r * (m[0][a] * (m[1][b] * m[2][c]));
    Dual<NV> B = omega * eq;
    if constexpr (n >= 1 && n <= 3) {
      // body force: F . d/du of the equilibrium coefficient / rho
      Dual<NV> src = dconst<NV>(0.f);
      if constexpr (a > 0) src = src + ((float)a * fx[0]) * (m[0][a > 0 ? a - 1 : 0] * (m[1][b] * m[2][c]));
      if constexpr (b > 0) src = src + ((float)b * fx[1]) * (m[0][a] * (m[1][b > 0 ? b - 1 : 0] * m[2][c]));
      if constexpr (c > 0) src = src + ((float)c * fx[2]) * (m[0][a] * (m[1][b] * m[2][c > 0 ? c - 1 : 0]));
      B = B + beta * src;
    }
    constexpr float inv_fact = (float)(1.0 / (fact_d(a) * fact_d(b) * fact_d(c)));
    phi = phi + (inv_fact * M[mi]) * B;
  });
  return phi;
}

// Weighted Hermite moments M_m = sum_i w_i mu_i He_a(cx/c0) He_b(cy/c0) He_c(cz/c0).
template <class L>
__device__ __forceinline__ void hermite_moments(const float (&mu)[L::Q], float (&M)[AdjCfg<L>::NM]) {
  using A = AdjCfg<L>;
#pragma unroll
  for (int m = 0; m < A::NM; ++m) M[m] = 0.f;
  static_for<L::Q>([&](auto I) {
    constexpr int i = I;
    static_for<A::NM>([&](auto Mi) {
      constexpr int mi = Mi;
      constexpr int a = A::mono(mi, 0), b = A::mono(mi, 1), c = A::mono(mi, 2);
      constexpr double h = L::w(i) * he_at<L>(a, L::c(i, 0)) * he_at<L>(b, L::c(i, 1)) * he_at<L>(c, L::c(i, 2));
      // He_odd(0) = 0 exactly; skip by the integer structure
      constexpr bool zero = ((a % 2) && L::c(i, 0) == 0) || ((b % 2) && L::c(i, 1) == 0) || ((c % 2) && L::c(i, 2) == 0);
      if constexpr (!zero) M[mi] = fmaf((float)h, mu[i], M[mi]);
    });
  });
}

struct AdjArgs {
  const void* fwd;        // forward state S_{n-1}: gathering it gives f_n
  const float* lam_in;    // lambda_{n+1} [Q][N]
  float* lam_out;         // lambda_n [Q][N]
  const float* gfield;    // [D][N] acceleration
  float* dLdg;            // [D][N] accumulated gradient
  double* partials;       // seed: per-block loss sums (stride 8)
  long long N;
  int nx, ny, nz;
  float rho0, omega, beta;
  int thermal;
};

// node quantities of f_n(x): rho, j, e, u, tb, F with the forward kernel's arithmetic
template <class L>
struct NodeQ {
  float rho, j[3], e, u[3], tb, F[3], g[3];
};

template <class L, class C>
__device__ __forceinline__ NodeQ<L> node_q(const AdjArgs& a, int x, int y, int z, int node) {
  constexpr int D = L::D;
  constexpr float Dc = (float)(D * L::cs2);
  float gv[L::Q];
  gather<L, C>(static_cast<const typename C::T*>(a.fwd), a.N, a.nx, a.ny, a.nz, x, y, z, gv);
  float dr, acc, J[3], Pih;
  moments_h<L>(gv, dr, acc, J, Pih);
  NodeQ<L> q;
  q.rho = a.rho0 + dr;
  q.e = fmaf(Dc, q.rho, Pih);
  float uu = 0.f, ug = 0.f;
  for (int d = 0; d < 3; ++d) {
    q.g[d] = (d < D) ? __ldg(a.gfield + (size_t)d * a.N + node) : 0.f;
    q.j[d] = (d < D) ? J[d] : 0.f;
    q.F[d] = q.rho * q.g[d];
    q.u[d] = fmaf(0.5f, q.F[d], q.j[d]) / q.rho;
    uu = fmaf(q.u[d], q.u[d], uu);
    ug = fmaf(q.u[d], q.g[d], ug);
  }
  // theta-bar = (e - rho |u|^2 + rho u.g) / (rho D c0^2) - 1 (Eq. 4.5, G2 = 2 u.F)
  q.tb = a.thermal ? (Pih - q.rho * uu + q.rho * ug) / (q.rho * Dc) : 0.f;
  return q;
}

template <class L>
__device__ __forceinline__ void coords(const AdjArgs& a, long long n, int& x, int& y, int& z) {
  x = (int)(n % a.nx);
  y = (int)((n / a.nx) % a.ny);
  z = (int)(n / ((long long)a.nx * a.ny));
}

// lambda_T and dL/dg at T, plus per-block sums of rho |u|^2 / 2 (one CTA per 256 nodes)
template <class L, int ST>
__global__ void __launch_bounds__(256) adjoint_seed_kernel(const __grid_constant__ AdjArgs a) {
  using C = Codec<ST>;
  constexpr int D = L::D;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double ke = 0.0;
  if (n < a.N) {
    int x, y, z;
    coords<L>(a, n, x, y, z);
    const NodeQ<L> q = node_q<L, C>(a, x, y, z, (int)n);
    float uu = 0.f, uj = 0.f;
    for (int d = 0; d < D; ++d) {
      uu = fmaf(q.u[d], q.u[d], uu);
      uj = fmaf(q.u[d], q.j[d], uj);
    }
    const float dl_drho = 0.5f * uu - uj / q.rho;
    static_for<L::Q>([&](auto I) {
      constexpr int i = I;
      float v = dl_drho;
      static_for<D>([&](auto A) {
        constexpr int ax = A;
        if constexpr (L::c(i, ax) != 0) v = fmaf((float)L::c(i, ax), q.u[ax], v);
      });
      a.lam_out[(size_t)i * a.N + n] = v;
    });
    for (int d = 0; d < D; ++d) a.dLdg[(size_t)d * a.N + n] = 0.5f * q.rho * q.u[d];
    ke = 0.5 * (double)q.rho * (double)uu;
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ke;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    a.partials[(size_t)blockIdx.x * 8] = s;
  }
}

// one reverse step: lambda_n from lambda_{n+1}, accumulating dL/dg
template <class L, int ST>
__global__ void __launch_bounds__(128) adjoint_step_kernel(const __grid_constant__ AdjArgs a) {
  using C = Codec<ST>;
  using A = AdjCfg<L>;
  constexpr int D = L::D, NV = A::NV;
  constexpr float Dc = (float)(D * L::cs2);
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  int x, y, z;
  coords<L>(a, n, x, y, z);
  const NodeQ<L> q = node_q<L, C>(a, x, y, z, (int)n);
  // mu_i = lambda_{n+1,i}(x + c_i)
  float mu[L::Q];
  {
    int xs[7], ys[7], zs[7];
#pragma unroll
    for (int d = -3; d <= 3; ++d) {
      xs[d + 3] = wrap1(x + d, a.nx);
      ys[d + 3] = wrap1(y + d, a.ny) * a.nx;
      zs[d + 3] = (D == 3) ? wrap1(z + d, a.nz) * a.nx * a.ny : 0;
    }
    static_for<L::Q>([&](auto I) {
      constexpr int i = I;
      const int off = zs[L::c(i, 2) + 3] + ys[L::c(i, 1) + 3] + xs[L::c(i, 0) + 3];
      mu[i] = __ldg(a.lam_in + (size_t)i * a.N + off);
    });
  }
  float M[A::NM];
  hermite_moments<L>(mu, M);
  const Dual<NV> phi = phi_dual<L>(M, q.rho, q.u, q.tb, q.F, a.thermal != 0, a.omega, a.beta);
  const float Prho = phi.d[0], Pt = a.thermal ? phi.d[1 + D] : 0.f;
  float qv[3], PF[3];
  for (int d = 0; d < 3; ++d) {
    PF[d] = (d < D) ? phi.d[2 + D + d] : 0.f;
    qv[d] = (d < D) ? fmaf(Pt, (-2.f * q.u[d] + q.g[d]) / Dc, phi.d[1 + d]) : 0.f;
  }
  const float inv_rho = 1.f / q.rho;
  float dj[3], dg[3], qj = 0.f, Fg = 0.f;
  for (int d = 0; d < 3; ++d) {
    dj[d] = qv[d] * inv_rho;
    qj = fmaf(qv[d], q.j[d], qj);
    Fg = fmaf(PF[d], q.g[d], Fg);
    dg[d] = q.rho * PF[d] + 0.5f * qv[d] + Pt * q.u[d] / Dc;
  }
  const float de = Pt * inv_rho / Dc;
  const float drho = Prho + Fg - qj * inv_rho * inv_rho - Pt * q.e * inv_rho * inv_rho / Dc;
  const float om1 = 1.f - a.omega;
  static_for<L::Q>([&](auto I) {
    constexpr int i = I;
    float v = fmaf(om1, mu[i], drho);
    static_for<D>([&](auto Ax) {
      constexpr int ax = Ax;
      if constexpr (L::c(i, ax) != 0) v = fmaf((float)L::c(i, ax), dj[ax], v);
    });
    if constexpr (L::norm2(i) != 0) v = fmaf((float)L::norm2(i), de, v);
    a.lam_out[(size_t)i * a.N + n] = v;
  });
  for (int d = 0; d < D; ++d) a.dLdg[(size_t)d * a.N + n] += dg[d];
}

template <class L>
cudaError_t launch_adj(int storage, bool seed, const AdjArgs& a, cudaStream_t s) {
  const unsigned b256 = (unsigned)((a.N + 255) / 256), b128 = (unsigned)((a.N + 127) / 128);
  switch (storage) {
    case ST_F32:
      if (seed) adjoint_seed_kernel<L, ST_F32><<<b256, 256, 0, s>>>(a);
      else adjoint_step_kernel<L, ST_F32><<<b128, 128, 0, s>>>(a);
      break;
    case ST_F16:
      if (seed) adjoint_seed_kernel<L, ST_F16><<<b256, 256, 0, s>>>(a);
      else adjoint_step_kernel<L, ST_F16><<<b128, 128, 0, s>>>(a);
      break;
    default:
      if (seed) adjoint_seed_kernel<L, ST_BF16><<<b256, 256, 0, s>>>(a);
      else adjoint_step_kernel<L, ST_BF16><<<b128, 128, 0, s>>>(a);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint(int lattice, int storage, bool seed, const void* fwd, const float* lam_in, float* lam_out,
                           const float* gfield, float* dLdg, double* partials, long long N, int nx, int ny, int nz,
                           float rho0, float omega, float beta, int thermal, cudaStream_t s) {
  AdjArgs a{};
  a.fwd = fwd;
  a.lam_in = lam_in;
  a.lam_out = lam_out;
  a.gfield = gfield;
  a.dLdg = dLdg;
  a.partials = partials;
  a.N = N;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.rho0 = rho0;
  a.omega = omega;
  a.beta = beta;
  a.thermal = thermal;
  return lattice == 0 ? launch_adj<D2Q37>(storage, seed, a, s) : launch_adj<D3Q39>(storage, seed, a, s);
}

int adjoint_seed_blocks(long long N) { return (int)((N + 255) / 256); }

}  // namespace hlbm
