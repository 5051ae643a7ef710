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
// Its partial derivatives are contractions of M shifted by one or two indices
// (phi_grad below); the chain rule through u = j/rho + g/2,
// theta-bar(e, rho, u, g) and F = rho g then gives the derivatives with
// respect to rho = sum f, j = sum c f, e = sum |c|^2 f and g.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "hlbm.h"
#include "internal.h"
#include "step_common.cuh"

namespace hlbm {
namespace {

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
  __host__ __device__ static constexpr int mono(int m, int ax) { return D == 2 ? (ax < 2 ? mono2(m, ax) : 0) : mono3(m, ax); }
  __host__ __device__ static constexpr int index(int a, int b, int c) {
    return D == 2 ? (c == 0 ? mono2_index(a, b) : -1) : mono3_index(a, b, c);
  }
};

// sum over the monomials (a, b, c) of order <= LIM of M[(a, b, c) + (SX, SY, SZ)] P_abc / (a! b! c!)
template <class L, int SX, int SY, int SZ, int LIM>
__device__ __forceinline__ float hshift(const float (&M)[AdjCfg<L>::NM], const float (&P)[AdjCfg<L>::NM]) {
  using A = AdjCfg<L>;
  float s = 0.f;
  static_for<A::NM>([&](auto Mi) {
    constexpr int mi = Mi;
    constexpr int a = A::mono(mi, 0), b = A::mono(mi, 1), c = A::mono(mi, 2);
    if constexpr (a + b + c <= LIM) {
      constexpr int j = A::index(a + SX, b + SY, c + SZ);
      static_assert(j >= 0, "shifted monomial outside the moment set");
      constexpr float cf = (float)(1.0 / (fact_d(a) * fact_d(b) * fact_d(c)));
      s = fmaf(M[j] * cf, P[mi], s);
    }
  });
  return s;
}

// Partial derivatives of Phi(rho, u, tb, F) = sum_m B_m M_m / (a! b! c!) with
// B_abc = omega rho P_abc + beta sum_d (F_d / c0) idx_d P_{abc - e_d} (the
// body force for orders 1..3), P_abc = m_a(u_x/c0) m_b(u_y/c0) m_c(u_z/c0) and
// m_k the Gaussian Hermite moments of N(u, 1 + tb).  Since dm_k/du~ = k m_{k-1}
// and dm_k/dtb = k (k - 1) / 2 m_{k-2}, each derivative is the contraction of
// M shifted by one or two indices with P:
//   dPhi/drho = omega S,  S = sum_{n <= E} M_m P_m / m!          (E: equilibrium order)
//   dPhi/dF_d = beta S_d / c0,  S_d = sum_{n <= 2} M_{m + e_d} P_m / m!
//   dPhi/du_e = (omega rho sum_{n <= E-1} M_{m+e_e} P_m / m! + beta sum_d F~_d U_de) / c0,
//               U_de = sum_{n <= 1} M_{m + e_d + e_e} P_m / m!
//   dPhi/dtb  = omega rho / 2 sum_d sum_{n <= E-2} M_{m + 2 e_d} P_m / m!
//               + beta / 2 sum_d F~_d sum_e M_{e_d + 2 e_e}
template <class L>
__device__ __forceinline__ void phi_grad(const float (&M)[AdjCfg<L>::NM], float rho, const float (&u)[3], float tb,
                                         const float (&F)[3], bool thermal, float omega, float beta, float& Prho,
                                         float (&Pu)[3], float& Pt, float (&PF)[3]) {
  using A = AdjCfg<L>;
  constexpr int D = A::D, NM = A::NM, E = L::FEQ_ORDER;
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  const float t = thermal ? tb : 0.f;
  float m[3][5];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float x = (a < D) ? u[a] * inv_c0 : 0.f;
    const float x2 = x * x;
    m[a][0] = 1.f;
    m[a][1] = x;
    m[a][2] = x2 + t;
    m[a][3] = x * fmaf(3.f, t, x2);
    m[a][4] = fmaf(x2, fmaf(6.f, t, x2), 3.f * t * t);
  }
  float P[NM];
  static_for<NM>([&](auto Mi) {
    constexpr int mi = Mi;
    P[mi] = m[0][A::mono(mi, 0)] * (m[1][A::mono(mi, 1)] * m[2][A::mono(mi, 2)]);
  });
  const float Ft[3] = {F[0] * inv_c0, F[1] * inv_c0, D == 3 ? F[2] * inv_c0 : 0.f};
  const float orho = omega * rho;
  Prho = omega * hshift<L, 0, 0, 0, E>(M, P);
  // first shifts: equilibrium (order E - 1) and body force (order 2)
  float Eq[3] = {0.f, 0.f, 0.f}, Sd[3] = {0.f, 0.f, 0.f};
  Eq[0] = hshift<L, 1, 0, 0, E - 1>(M, P);
  Eq[1] = hshift<L, 0, 1, 0, E - 1>(M, P);
  Sd[0] = (E - 1 == 2) ? Eq[0] : hshift<L, 1, 0, 0, 2>(M, P);
  Sd[1] = (E - 1 == 2) ? Eq[1] : hshift<L, 0, 1, 0, 2>(M, P);
  if constexpr (D == 3) {
    Eq[2] = hshift<L, 0, 0, 1, E - 1>(M, P);
    Sd[2] = (E - 1 == 2) ? Eq[2] : hshift<L, 0, 0, 1, 2>(M, P);
  }
  // second shifts of the body force (order 1), symmetric in (d, e)
  float U[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  U[0][0] = hshift<L, 2, 0, 0, 1>(M, P);
  U[1][1] = hshift<L, 0, 2, 0, 1>(M, P);
  U[0][1] = U[1][0] = hshift<L, 1, 1, 0, 1>(M, P);
  if constexpr (D == 3) {
    U[2][2] = hshift<L, 0, 0, 2, 1>(M, P);
    U[0][2] = U[2][0] = hshift<L, 1, 0, 1, 1>(M, P);
    U[1][2] = U[2][1] = hshift<L, 0, 1, 1, 1>(M, P);
  }
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    float s = orho * Eq[e];
#pragma unroll
    for (int d = 0; d < D; ++d) s = fmaf(beta * Ft[d], U[d][e], s);
    Pu[e] = (e < D) ? s * inv_c0 : 0.f;
    PF[e] = (e < D) ? beta * Sd[e] * inv_c0 : 0.f;
  }
  Pt = 0.f;
  if (thermal) {
    // equilibrium: second shifts in one axis (order E - 2)
    float q = hshift<L, 2, 0, 0, E - 2>(M, P) + hshift<L, 0, 2, 0, E - 2>(M, P);
    if constexpr (D == 3) q += hshift<L, 0, 0, 2, E - 2>(M, P);
    // body force: sum_e M_{e_d + 2 e_e} (order 3, P_000 = 1)
    float src = 0.f;
    static_for<D>([&](auto Dd) {
      constexpr int d = Dd;
      float md = 0.f;
      static_for<D>([&](auto Ee) {
        constexpr int e = Ee;
        constexpr int j = A::index((d == 0) + 2 * (e == 0), (d == 1) + 2 * (e == 1), (d == 2) + 2 * (e == 2));
        md += M[j];
      });
      src = fmaf(Ft[d], md, src);
    });
    Pt = 0.5f * fmaf(orho, q, beta * src);
  }
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
  constexpr int D = L::D;
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
  float Prho, Pu[3], Pt, PF[3];
  phi_grad<L>(M, q.rho, q.u, q.tb, q.F, a.thermal != 0, a.omega, a.beta, Prho, Pu, Pt, PF);
  float qv[3];
  for (int d = 0; d < 3; ++d) qv[d] = (d < D) ? fmaf(Pt, (-2.f * q.u[d] + q.g[d]) / Dc, Pu[d]) : 0.f;
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
