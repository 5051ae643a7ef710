// In-place D2Q37 step (AA pattern) with single-pass neighbour fields: one
// population buffer instead of two, and one read and one write of every
// population per step with no frame of populations.
//
// AA pattern.  Before an even step, slot i of node x holds f_i(x, t) (after
// streaming).  The even step reads node x's own 37 slots, collides, and writes
// f*_i into slot ibar of the same node.  Before an odd step, f_i(x, t) is
// therefore in slot ibar of node x - c_i; the odd step reads those, collides,
// and writes f*_i into slot i of node x + c_i, which is where the next even
// step finds f_i(x + c_i, t + 1).  In both steps the slots a node writes are
// exactly the slots it read (slot i of x + c_i is slot (ibar)bar of
// x - c_ibar), so the update is in place without any ordering between nodes.
//
// Neighbour fields.  grad theta (H_i) and the pseudopotential of F^SC and
// P_i would need the populations of the neighbours at time t, which other
// threads may already have overwritten; they are taken from the previous
// step instead (the single-pass variant of the method): each step writes its
// nodes' theta - 1 (thermal kind) or psi (pseudopotential kind) into one of
// two auxiliary fields and reads the neighbours' from the other.  The frame
// of the auxiliary field (1 or 3 nodes around the 32 x 8 tile) is staged in
// shared memory.
//
// Bytes per node and step: 37 x elem read + 37 x elem write + 4 (own field
// written) + about 4 (the staged field, neighbours served by L2): 304 B FP32.
#include "internal.h"
#include "lattice.cuh"
#include "step_common.cuh"

#include <type_traits>

namespace hlbm {
namespace {

using L = D2Q37;
constexpr int kBX = 32, kBY = 8;

__host__ __device__ constexpr int aa_opp(int i) { return i == 0 ? 0 : (((i - 1) & 1) ? i - 1 : i + 1); }

template <int KIND>
constexpr int frame_of() {
  return KIND == KIND_SC ? 3 : (KIND == KIND_THERMAL ? 1 : 0);
}

// ODD: the step's parity; MOM: moments readout (no store).  NPT nodes per
// thread: lane k of thread (tx, ty) is tile row ty + k kBY / NPT, and with
// NPT = 2 the node arithmetic runs on paired FP32 lanes (float2), rounding
// exactly like the one-node form.
template <int ST, int KIND, bool ODD, bool MOM, int NPT>
__global__ void __launch_bounds__(kBX * kBY / NPT, 2 * NPT) aa_step_kernel(const __grid_constant__ StepArgs a) {
  using T = typename Codec<ST>::T;
  using V = typename std::conditional<NPT == 2, float2, float>::type;
  constexpr int H = frame_of<KIND>();
  constexpr int SW = kBX + 2 * H, SH = kBY + 2 * H;
  constexpr int TR = kBY / NPT, NT = kBX * TR;   // thread rows, threads
  __shared__ float aux[(H > 0) ? SW * SH : 1];
  __shared__ double red[TR][6];
  const int nx = a.nx, ny = a.ny;
  const size_t N = (size_t)a.N;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kBX + tx;
  const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY;
  const int x = x0 + tx;
  const int xc = x < nx ? x : x % nx;   // inactive lanes still compute (the frame is shared)
  int yck[NPT], nodek[NPT];
  bool activek[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int y = y0 + ty + k * TR;
    activek[k] = x < nx && y < ny;
    yck[k] = y < ny ? y : y % ny;
    nodek[k] = yck[k] * nx + xc;
  }

  // the previous step's neighbour field, on the tile and its frame
  if constexpr (H > 0) {
    for (int k = tid; k < SW * SH; k += NT) {
      const int j = k / SW, i = k - j * SW;
      const int X = wrapm(x0 - H + i, nx), Y = wrapm(y0 - H + j, ny);
      aux[k] = __ldg(a.aux_rd + HLBM_IDX((long long)Y * nx + X, a.N, DBG_AUX));
    }
    __syncthreads();
  }

  // the nodes' populations at time t
  const T* __restrict__ f = static_cast<const T*>(a.fin);
  V g[37];
  int xs[7], ys[NPT][7];
#pragma unroll
  for (int d = -3; d <= 3; ++d) {
    xs[d + 3] = wrap1(xc - d, nx);
#pragma unroll
    for (int k = 0; k < NPT; ++k) ys[k][d + 3] = wrap1(yck[k] - d, ny) * nx;
  }
  static_for<37>([&](auto I) {
    constexpr int i = I;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if constexpr (!ODD) {
        set_lane(g[i], k, to_float(f[HLBM_IDX((long long)i * N + nodek[k], 37 * a.N, DBG_GATHER)]));
      } else {
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), b = aa_opp(i);
        set_lane(g[i], k, to_float(f[HLBM_IDX((long long)b * N + ys[k][cy + 3] + xs[cx + 3], 37 * a.N, DBG_GATHER)]));
      }
    }
  });

  V dr, dr_l, acc, J[3], Pih;
  moments_h<L>(g, dr, dr_l, acc, J, Pih);
  const V rho = vadd(splat<V>(a.rho0), dr);
  V gax, gay;
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    float ga[3];
    accel<2>(a, nodek[k], yck[k], ga);
    set_lane(gax, k, ga[0]);
    set_lane(gay, k, ga[1]);
  }
  V Fx = vmul(rho, gax), Fy = vmul(rho, gay);
  V sigma = splat<V>(0.f), psi_now = splat<V>(0.f);
  if constexpr (KIND == KIND_SC) {
    // F^SC = -G psi(x) sum_i w_i psi(x + c_i) c_i, G = -1, psi of the previous step
    V sx = splat<V>(0.f), sy = splat<V>(0.f), ps;
    static_for<L::NPAIR>([&](auto P) {
      constexpr int i = 2 * P + 1;
      constexpr int cx = L::c(i, 0), cy = L::c(i, 1);
      V dpsi;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const float* ap = aux + (ty + k * TR + H) * SW + tx + H;
        set_lane(dpsi, k, ap[cy * SW + cx] - ap[-cy * SW - cx]);
      }
      if constexpr (cx != 0) sx = vfma(splat<V>((float)(L::w(i) * cx)), dpsi, sx);
      if constexpr (cy != 0) sy = vfma(splat<V>((float)(L::w(i) * cy)), dpsi, sy);
    });
#pragma unroll
    for (int k = 0; k < NPT; ++k) set_lane(ps, k, aux[(ty + k * TR + H) * SW + tx + H]);
    const V fsx = vmul(ps, sx), fsy = vmul(ps, sy);
    Fx = vadd(Fx, fsx);
    Fy = vadd(Fy, fsy);
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const float p1 = lane(ps, k), f1 = lane(fsx, k), f2 = lane(fsy, k);
      set_lane(sigma, k, (p1 > 0.f) ? a.p_coef * (f1 * f1 + f2 * f2) * rcp_nr(p1 * p1) : 0.f);
      set_lane(psi_now, k, psi_of<L>(a, lane(dr, k), lane(dr_l, k)));
    }
  }
  constexpr float Dc = (float)(2.0 * L::cs2);
  const V inv_rho = vmap(rho, [](float r) { return rcp_nr(r); });
  const V ux = vmul(vfma(splat<V>(0.5f), Fx, J[0]), inv_rho);
  const V uy = vmul(vfma(splat<V>(0.5f), Fy, J[1]), inv_rho);
  const V uu = vfma(ux, ux, vmul(uy, uy));
  const V G2 = vfma(splat<V>(Dc), sigma, vmul(splat<V>(2.f), vfma(ux, Fx, vmul(uy, Fy))));
  const V tb = vmul(vmul(vfma(splat<V>(0.5f), G2, vsub(Pih, vmul(rho, uu))), inv_rho), splat<V>(1.f / Dc));

  if constexpr (MOM) {
    double v[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (!activek[k]) continue;
      const int node = nodek[k];
      const float r = lane(rho, k), vx = lane(ux, k), vy = lane(uy, k), t = lane(tb, k);
      if (a.rho_out) a.rho_out[node] = r;
      if (a.u_out) {
        a.u_out[node] = vx;
        a.u_out[N + node] = vy;
      }
      if (a.theta_out) a.theta_out[node] = 1.f + t;
      const bool bad = !(isfinite(r) && r > 0.f && isfinite(vx) && isfinite(vy) && isfinite(t));
      v[0] += lane(dr, k);
      v[1] += (double)r * vx;
      v[2] += (double)r * vy;
      v[4] += 0.5 * ((double)lane(Pih, k) + (double)Dc * lane(dr, k) + 0.5 * (double)lane(G2, k));
      v[5] += bad ? 1.0 : 0.0;
    }
    if (a.partials) {
#pragma unroll
      for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
      if (tx == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) red[ty][k] = v[k];
      __syncthreads();
      if (tid < 6) {
        double sum = 0.0;
        for (int w = 0; w < TR; ++w) sum += red[w][tid];
        a.partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + tid] = sum;
      }
    }
    return;
  } else {
    // this step's field for the next step's neighbours
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (!activek[k]) continue;
      if constexpr (KIND == KIND_SC) a.aux_wr[nodek[k]] = lane(psi_now, k);
      if constexpr (KIND == KIND_THERMAL) a.aux_wr[nodek[k]] = lane(tb, k);
    }
    NodeSrcT<V> s;
    s.hG[0] = s.hG[1] = s.hG[2] = splat<V>(0.f);
    if constexpr (KIND == KIND_THERMAL) {
      V gtx, gty;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const float* ap = aux + (ty + k * TR + 1) * SW + tx + 1;
        set_lane(gtx, k, 0.5f * (ap[1] - ap[-1]));
        set_lane(gty, k, 0.5f * (ap[SW] - ap[-SW]));
      }
      // s^(3) += rho theta (1 - 1/Pr) [delta grad_xi theta], grad_xi = c0 grad
      const V hc = vmul(vmul(rho, vadd(splat<V>(1.f), tb)), splat<V>(a.h_coef * (float)L::c0));
      s.hG[0] = vmul(hc, gtx);
      s.hG[1] = vmul(hc, gty);
    }
    constexpr float inv_c0 = (float)(1.0 / L::c0);
    s.dr = splat<V>(0.f);
    s.rho = rho;
    s.tb = a.isothermal ? splat<V>(0.f) : tb;
    s.u[0] = vmul(ux, splat<V>(inv_c0));
    s.u[1] = vmul(uy, splat<V>(inv_c0));
    s.u[2] = splat<V>(0.f);
    s.F[0] = vmul(Fx, splat<V>(inv_c0));
    s.F[1] = vmul(Fy, splat<V>(inv_c0));
    s.F[2] = splat<V>(0.f);
    s.sigma = sigma;
    V K[15];
    poly2<L>(s, a.omega, a.beta, K);
    const float om1 = 1.f - a.omega;
    K[0] = vfma(splat<V>(-om1), acc, K[0]);
    if constexpr (KIND == KIND_SC) K[0] = vadd(K[0], dr_l);
    apply_poly_h<L, 15>(g, K, om1, dr);
    T* __restrict__ fo = static_cast<T*>(a.fout);
    // the odd step's store offsets are recomputed here from a copy of x that
    // the compiler cannot match with the load offsets, so that the loads'
    // offset arrays need not stay live across the collision
    int xl = xc;
    asm volatile("" : "+r"(xl));
    int xt[7];
#pragma unroll
    for (int d = -3; d <= 3; ++d) xt[d + 3] = ODD ? wrap1(xl + d, nx) : 0;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (!activek[k] || !HLBM_IN(nodek[k], a.N, DBG_STORE)) continue;
      const int node = nodek[k];
      int yl = yck[k];
      asm volatile("" : "+r"(yl));
      int yt[7];
#pragma unroll
      for (int d = -3; d <= 3; ++d) yt[d + 3] = ODD ? wrap1(yl + d, ny) * nx : 0;
      // 16-bit storage: stochastic rounding keyed by node and result (step_common.cuh)
      const uint32_t salt = std::is_same<T, float>::value ? 0u : node_salt(node, lane(g[0], k));
      static_for<37>([&](auto I) {
        constexpr int i = I;
        constexpr int b = aa_opp(i);
        const T v = round_store<T>(lane(g[i], k), pop_bits(salt, i));
        if constexpr (!ODD) {
          fo[(size_t)b * N + node] = v;                             // slot ibar of x
        } else {
          constexpr int cx = L::c(i, 0), cy = L::c(i, 1);
          const long long o = (long long)i * N + yt[cy + 3] + xt[cx + 3];
          if (HLBM_IN(o, 37 * a.N, DBG_STORE)) fo[o] = v;           // slot i of x + c_i
        }
      });
    }
  }
}

// Initial state in the even layout: slot i of node x = f^eq_i(x); the
// neighbour field the first step reads (theta - 1, or psi of the density).
template <int ST, int KIND>
__global__ void __launch_bounds__(256) aa_init_kernel(const __grid_constant__ StepArgs a, const float* __restrict__ rho,
                                                      const float* __restrict__ u, const float* __restrict__ theta) {
  using T = typename Codec<ST>::T;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const size_t N = (size_t)a.N;
  NodeSrcT<float> s;
  s.dr = rho[n] - a.rho0;
  s.rho = rho[n];
  s.tb = theta[n] - 1.f;
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  s.u[0] = u[n] * inv_c0;
  s.u[1] = u[N + n] * inv_c0;
  s.u[2] = 0.f;
  s.F[0] = s.F[1] = s.F[2] = 0.f;
  s.hG[0] = s.hG[1] = s.hG[2] = 0.f;
  s.sigma = 0.f;
  float g[37], K[15];
#pragma unroll
  for (int i = 0; i < 37; ++i) g[i] = 0.f;
  poly2<L>(s, 1.f, 0.f, K);
  apply_poly<L, 15>(g, K, 0.f);
  T* __restrict__ fo = static_cast<T*>(a.fout);
  static_for<37>([&](auto I) {
    constexpr int i = I;
    Codec<ST>::st(fo + (size_t)i * N + n, g[i]);
  });
  if constexpr (KIND == KIND_THERMAL) a.aux_wr[n] = theta[n] - 1.f;
  if constexpr (KIND == KIND_SC) a.aux_wr[n] = psi_of<L>(a, rho[n] - a.rho0, 0.f);
}

// steps: two nodes per thread (paired FP32 lanes); the moments readout: one
template <int ST, int KIND>
cudaError_t launch_kind(const StepArgs& a, bool odd, bool mom, cudaStream_t s) {
  const dim3 grid((a.nx + kBX - 1) / kBX, (a.ny + kBY - 1) / kBY);
  if (mom) {
    const dim3 block(kBX, kBY);
    if (odd) aa_step_kernel<ST, KIND, true, true, 1><<<grid, block, 0, s>>>(a);
    else aa_step_kernel<ST, KIND, false, true, 1><<<grid, block, 0, s>>>(a);
  } else {
    const dim3 block(kBX, kBY / 2);
    if (odd) aa_step_kernel<ST, KIND, true, false, 2><<<grid, block, 0, s>>>(a);
    else aa_step_kernel<ST, KIND, false, false, 2><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <int ST>
cudaError_t launch_st(const StepArgs& a, int kind, bool odd, bool mom, cudaStream_t s) {
  if (kind == KIND_SC) return launch_kind<ST, KIND_SC>(a, odd, mom, s);
  if (kind == KIND_THERMAL) return launch_kind<ST, KIND_THERMAL>(a, odd, mom, s);
  return launch_kind<ST, KIND_LOCAL>(a, odd, mom, s);
}

template <int ST>
cudaError_t init_st(const StepArgs& a, int kind, const float* rho, const float* u, const float* theta,
                    cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.N + 255) / 256);
  if (kind == KIND_SC) aa_init_kernel<ST, KIND_SC><<<blocks, 256, 0, s>>>(a, rho, u, theta);
  else if (kind == KIND_THERMAL) aa_init_kernel<ST, KIND_THERMAL><<<blocks, 256, 0, s>>>(a, rho, u, theta);
  else aa_init_kernel<ST, KIND_LOCAL><<<blocks, 256, 0, s>>>(a, rho, u, theta);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_aa(const StepArgs& a, int kind, int storage, bool odd, bool mom, cudaStream_t s) {
  switch (storage) {
    case ST_F32: return launch_st<ST_F32>(a, kind, odd, mom, s);
    case ST_F16: return launch_st<ST_F16>(a, kind, odd, mom, s);
    default: return launch_st<ST_BF16>(a, kind, odd, mom, s);
  }
}

cudaError_t launch_aa_init(const StepArgs& a, int kind, int storage, const float* rho, const float* u,
                           const float* theta, cudaStream_t s) {
  switch (storage) {
    case ST_F32: return init_st<ST_F32>(a, kind, rho, u, theta, s);
    case ST_F16: return init_st<ST_F16>(a, kind, rho, u, theta, s);
    default: return init_st<ST_BF16>(a, kind, rho, u, theta, s);
  }
}

}  // namespace hlbm
