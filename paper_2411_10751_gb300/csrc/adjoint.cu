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
#include "tma.cuh"

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
  int* status;                  // whole-row kernel: HLBM_ETIMEOUT when a copy wait gives up
  unsigned long long wait_ns;   // bound of each copy wait
  unsigned long long* ctr;      // whole-row kernel: tile counter; each launch takes tiles + CTAs values
};

// node quantities of f_n(x): rho, j, e, u, tb, F with the forward kernel's arithmetic
template <class L>
struct NodeQ {
  float rho, j[3], e, u[3], tb, F[3], g[3];
};

// from the node's pulled populations gv (overwritten) and its acceleration
// (component d: gn(d), read after the moments)
template <class L, class GN>
__device__ __forceinline__ NodeQ<L> node_q_from(const AdjArgs& a, float (&gv)[L::Q], GN&& gn) {
  constexpr int D = L::D;
  constexpr float Dc = (float)(D * L::cs2);
  float dr, acc, J[3], Pih;
  moments_h<L>(gv, dr, acc, J, Pih);
  NodeQ<L> q;
  q.rho = a.rho0 + dr;
  q.e = fmaf(Dc, q.rho, Pih);
  float uu = 0.f, ug = 0.f;
  for (int d = 0; d < 3; ++d) {
    q.g[d] = (d < D) ? gn(d) : 0.f;
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

template <class L, class C>
__device__ __forceinline__ NodeQ<L> node_q(const AdjArgs& a, int x, int y, int z, int node) {
  float gv[L::Q];
  gather<L, C>(static_cast<const typename C::T*>(a.fwd), a.N, a.nx, a.ny, a.nz, x, y, z, gv);
  return node_q_from<L>(a, gv, [&](int d) { return __ldg(a.gfield + (size_t)d * a.N + node); });
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

// lambda_n (stored) and the dL/dg increment dg at one node from its forward
// quantities q and mu_i = lambda_{n+1,i}(x + c_i)
template <class L>
__device__ __forceinline__ void reverse_node(const AdjArgs& a, const NodeQ<L>& q, const float (&mu)[L::Q], long long n,
                                             float (&dg)[3]) {
  using A = AdjCfg<L>;
  constexpr int D = L::D;
  constexpr float Dc = (float)(D * L::cs2);
  float M[A::NM];
  hermite_moments<L>(mu, M);
  float Prho, Pu[3], Pt, PF[3];
  phi_grad<L>(M, q.rho, q.u, q.tb, q.F, a.thermal != 0, a.omega, a.beta, Prho, Pu, Pt, PF);
  float qv[3];
  for (int d = 0; d < 3; ++d) qv[d] = (d < D) ? fmaf(Pt, (-2.f * q.u[d] + q.g[d]) / Dc, Pu[d]) : 0.f;
  const float inv_rho = 1.f / q.rho;
  float dj[3], qj = 0.f, Fg = 0.f;
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
  float dg[3];
  reverse_node<L>(a, q, mu, n, dg);
  for (int d = 0; d < D; ++d) a.dLdg[(size_t)d * a.N + n] += dg[d];
}

// Persistent D3Q39 reverse step on tiles of 256 nodes spanning whole x-rows
// (a tile is 256 / nx rows of one z-plane).  Plane i of the forward state
// (pulled: f_i(x) = S_i(x - c_i)) is the 4D box at (0, y0 - c_y, z - c_z) and
// plane i of lambda_{n+1} (mu_i(x) = lambda_i(x + c_i)) the box at
// (0, y0 + c_y, z + c_z); the x shifts are index masks in shared memory, the
// z wrap a wrapped coordinate, and a plane whose rows cross the y-edge is
// copied row by row.  The tile's acceleration comes with the same barrier,
// and its dL/dg increment goes back as one bulk reduce-add per component, so
// the arithmetic waits on no global load.  Tiles come in order from the
// device counter; once a tile is in registers the CTA takes the next index
// and issues its copies (threads 0..38 the forward planes, 128..166 the
// lambda planes, 64..66 the acceleration), so they overlap the arithmetic and
// the stores.  One node per thread.
constexpr int kAdjRowNodes = 256;

template <int ST>
struct AdjRowsSmem {
  static constexpr int TN = kAdjRowNodes, Q = D3Q39::Q;
  static constexpr int LAM = 0;                                                // lambda_{n+1} planes (FP32)
  static constexpr int FWD = LAM + Q * TN * 4;                                 // forward-state planes
  static constexpr int G = FWD + Q * TN * (int)sizeof(typename Codec<ST>::T);  // acceleration [3][TN]
  static constexpr int DG = G + 3 * TN * 4;                                    // dL/dg increment [3][TN]
  static constexpr int BAR = DG + 3 * TN * 4;
  static constexpr int BYTES = BAR + 16;
  static constexpr uint32_t TX = (uint32_t)DG;                                 // bytes landing per tile
};

template <int ST>
__global__ void __launch_bounds__(256, 2)
    adjoint_rows_kernel(const __grid_constant__ AdjArgs a, const __grid_constant__ CUtensorMap tm_fb,
                        const __grid_constant__ CUtensorMap tm_fr, const __grid_constant__ CUtensorMap tm_lb,
                        const __grid_constant__ CUtensorMap tm_lr, const __grid_constant__ CUtensorMap tm_g,
                        const __grid_constant__ CUtensorMap tm_dg) {
  using L = D3Q39;
  using T = typename Codec<ST>::T;
  using S = AdjRowsSmem<ST>;
  constexpr int TN = kAdjRowNodes;
  constexpr int RED = 96;   // the thread that issues the dL/dg reductions
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_next[2];
  float* sl = reinterpret_cast<float*>(smem + S::LAM);
  T* sf = reinterpret_cast<T*>(smem + S::FWD);
  float* sg = reinterpret_cast<float*>(smem + S::G);
  float* sdg = reinterpret_cast<float*>(smem + S::DG);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::BAR);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int by = TN / nx;
  const int nty = (ny + by - 1) / by;
  const int ntiles = nty * nz;
  const unsigned long long period = (unsigned long long)ntiles + gridDim.x;
  const int tid = threadIdx.x, xm = nx - 1;
  if (!HLBM_IN(smem_u32(smem) & 127u, 1, DBG_SMEM)) return;   // TMA destinations need 128-byte alignment
  const int xk = tid & xm, rk = tid / nx;
  const bool isf = tid < L::Q, isl = tid >= 128 && tid < 128 + L::Q, isg = tid >= 64 && tid < 67;
  const int p = isf ? tid : (isl ? tid - 128 : tid - 64);   // the plane this thread copies
  int pcy = 0, pcz = 0;
  if (isf || isl) d3_cyz(p, pcy, pcz, typename make_iseq<L::Q>::type{});
  // this thread's plane of tile t into shared memory (the barrier is armed)
  auto issue_plane = [&](int t) {
    const int z = t / nty, y0 = (t - z * nty) * by;
    fence_proxy_async_smem();
    if (isf) {
      const int zz = wrap_near3(z - pcz, nz), ys = y0 - pcy;
      if (ys >= 0 && ys + by <= ny) {
        tma_load_4d(sf + p * TN, &tm_fb, 0, ys, zz, p, bar);
      } else {
        for (int r = 0; r < by; ++r)
          tma_load_4d(sf + p * TN + r * nx, &tm_fr, 0, ((ys + r) % ny + ny) % ny, zz, p, bar);
      }
    } else if (isl) {
      const int zz = wrap_near3(z + pcz, nz), ys = y0 + pcy;
      if (ys >= 0 && ys + by <= ny) {
        tma_load_4d(sl + p * TN, &tm_lb, 0, ys, zz, p, bar);
      } else {
        for (int r = 0; r < by; ++r)
          tma_load_4d(sl + p * TN + r * nx, &tm_lr, 0, ((ys + r) % ny + ny) % ny, zz, p, bar);
      }
    } else if (isg) {
      tma_load_4d(sg + p * TN, &tm_g, 0, y0, z, p, bar);   // rows past the y-edge read as zero
    }
  };
  // tid 0: takes the next tile index into slot `slot` and arms the barrier for it
  auto take = [&](int slot) {
    const int t = (int)(atomicAdd(a.ctr, 1ull) % period);
    s_next[slot] = t;
    if (t < ntiles) mbar_arrive_expect_tx(bar, S::TX);
  };
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    take(0);
  }
  __syncthreads();
  int t = s_next[0];
  if (t < ntiles && (isf || isl || isg)) issue_plane(t);
  uint32_t phase = 0;
  for (int it = 1; t < ntiles; ++it) {
    const int z = t / nty, y0 = (t - z * nty) * by;
    const bool ok = mbar_wait_bounded(bar, phase, a.wait_ns);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(a.status, (int)5 /* HLBM_ETIMEOUT */);
      mbar_wait_bounded(bar, phase, a.wait_ns);
      if (tid == RED) bulk_wait_all();
      __syncthreads();
      return;
    }
    phase ^= 1u;
    if (tid == 0) take(it & 1);   // the barrier's next phase belongs to the next tile
    float gv[L::Q], mu[L::Q], gn[3];
    static_for<L::Q>([&](auto I) {
      constexpr int i = I;
      constexpr int cx = L::c(i, 0);
      gv[i] = to_float(sf[i * TN + rk * nx + ((xk - cx) & xm)]);
      mu[i] = sl[i * TN + rk * nx + ((xk + cx) & xm)];
    });
#pragma unroll
    for (int d = 0; d < 3; ++d) gn[d] = sg[d * TN + tid];
    if (tid == RED) bulk_wait_read_all();   // the previous tile's reductions have read their source
    __syncthreads();  // the staging buffers are free and the next index is published
    const int tn = s_next[it & 1];
    if (tn < ntiles && (isf || isl || isg)) issue_plane(tn);
    const int y = y0 + rk;
    float dg[3] = {0.f, 0.f, 0.f};
    if (y < ny) {
      const long long n = ((long long)z * ny + y) * nx + xk;
      const NodeQ<L> q = node_q_from<L>(a, gv, [&](int d) { return gn[d]; });
      reverse_node<L>(a, q, mu, n, dg);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) sdg[d * TN + tid] = dg[d];
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == RED) {
#pragma unroll
      for (int d = 0; d < 3; ++d) tma_reduce_add_4d(&tm_dg, sdg + d * TN, 0, y0, z, d);   // rows past the edge are skipped
      bulk_commit();
    }
    t = tn;
  }
  if (tid == RED) bulk_wait_read_all();   // the reductions have read their source; they complete with the grid
}

// Whether the whole-row kernel serves this domain (rows of the stored type
// fill 128 bytes, so single-row copies land on 128-byte aligned addresses).
template <int ST>
bool adj_rows_eligible(const AdjArgs& a) {
  return (a.nx == 32 || a.nx == 64 || a.nx == 128 || a.nx == 256) &&
         a.nx * (int)sizeof(typename Codec<ST>::T) >= 128;
}

template <int ST>
int adj_rows_ctas() {
  static std::atomic<int> cache[kMaxDevicesCached];
  return per_device_cached(cache, [](int dev) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(adjoint_rows_kernel<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, AdjRowsSmem<ST>::BYTES);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, adjoint_rows_kernel<ST>, 256, AdjRowsSmem<ST>::BYTES);
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  });
}

template <int ST>
cudaError_t launch_adj_step(const AdjArgs& a, const CUtensorMap* tm, cudaStream_t s) {
  if (tm && a.ctr && adj_rows_eligible<ST>(a)) {
    const int tiles = ((a.ny + kAdjRowNodes / a.nx - 1) / (kAdjRowNodes / a.nx)) * a.nz;
    const int ctas = std::min(tiles, adj_rows_ctas<ST>());
    adjoint_rows_kernel<ST><<<ctas, 256, AdjRowsSmem<ST>::BYTES, s>>>(a, tm[0], tm[1], tm[2], tm[3], tm[4], tm[5]);
  } else {
    adjoint_step_kernel<D3Q39, ST><<<(unsigned)((a.N + 127) / 128), 128, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <class L>
cudaError_t launch_adj(int storage, bool seed, const AdjArgs& a, const CUtensorMap* tm, cudaStream_t s) {
  const unsigned b256 = (unsigned)((a.N + 255) / 256), b128 = (unsigned)((a.N + 127) / 128);
  if constexpr (L::D == 3) {
    if (!seed) {
      if (storage == ST_F32) return launch_adj_step<ST_F32>(a, tm, s);
      if (storage == ST_F16) return launch_adj_step<ST_F16>(a, tm, s);
      return launch_adj_step<ST_BF16>(a, tm, s);
    }
  }
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
                           float rho0, float omega, float beta, int thermal, const AdjRows& rows, cudaStream_t s) {
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
  a.status = rows.status;
  a.wait_ns = rows.wait_ns;
  a.ctr = rows.ctr;
  return lattice == 0 ? launch_adj<D2Q37>(storage, seed, a, nullptr, s)
                      : launch_adj<D3Q39>(storage, seed, a, rows.tmaps, s);
}

int adjoint_seed_blocks(long long N) { return (int)((N + 255) / 256); }

}  // namespace hlbm
