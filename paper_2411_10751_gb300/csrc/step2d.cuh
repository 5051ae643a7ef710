// Fused pull-collide-source step on D2Q37 (Eq. 4.4), one node per thread.
//
// CTA tile: 32 x BY nodes (a warp spans 32 consecutive x, so every pulled
// load and every store of a warp covers one contiguous row segment).
// Population planes are [Q][ny][nx] (structure of arrays), periodic by index
// wrap with no halo cells in memory.
//
// Neighbour fields of time t (no lag, as the sources of Eq. 4.4 are all taken
// at time t):
//   KIND_THERMAL  grad theta for H_i needs theta at the four nearest
//                 neighbours: each CTA recomputes theta on a one-node frame
//                 around its tile from pulled populations into shared memory.
//   KIND_SC       F^SC (Eq. 3.8) needs psi(rho) on the reach-3 neighbourhood:
//                 psi on a three-node frame is recomputed the same way.
// The frame's populations come mostly from L2 (neighbouring CTAs read them
// too), so HBM traffic stays one read and one write of every population.
//
// Threads whose node lies past the domain edge (ragged last tile) compute the
// aux value of the periodic image of their position so that the shared tile
// is exact, and skip the store.
#pragma once

#include "step_common.cuh"

namespace hlbm {

template <int BX, int BY, int H>
struct Frame2 {
  static constexpr int SW = BX + 2 * H;
  static constexpr int SH = BY + 2 * H;
  // nodes on the frame around the tile: the 4-neighbour ring for H == 1
  // (no corners), the full ring for H == 3
  static constexpr int count = (H == 1) ? 2 * BX + 2 * BY : SW * SH - BX * BY;
  __device__ static __forceinline__ void pos(int k, int& i, int& j) {
    if constexpr (H == 1) {
      if (k < BX) { i = k + 1; j = 0; }
      else if (k < 2 * BX) { i = k - BX + 1; j = BY + 1; }
      else if (k < 2 * BX + BY) { i = 0; j = k - 2 * BX + 1; }
      else { i = BX + 1; j = k - 2 * BX - BY + 1; }
    } else {
      if (k < H * SW) { i = k % SW; j = k / SW; }
      else if (k < 2 * H * SW) { const int kk = k - H * SW; i = kk % SW; j = BY + H + kk / SW; }
      else {
        const int m = k - 2 * H * SW;
        const int r = m / (2 * H), c = m % (2 * H);
        j = H + r;
        i = (c < H) ? c : BX + c;
      }
    }
  }
};

// theta - 1 of a node from its pulled populations (Eq. 4.5), local force only
template <class L>
__device__ __forceinline__ float theta_bar_local(const StepArgs& a, const float (&g)[L::Q], int node, int y) {
  float dr, J[3], Pi;
  moments<L>(g, dr, J, Pi);
  const float rho = a.rho0 + dr;
  float acc[3];
  accel<2>(a, node, y, acc);
  const float inv = 1.f / rho;
  const float ux = fmaf(0.5f * rho, acc[0], J[0]) * inv;
  const float uy = fmaf(0.5f * rho, acc[1], J[1]) * inv;
  const float G2 = 2.f * rho * (ux * acc[0] + uy * acc[1]);
  constexpr float Dc = (float)(2.0 * L::cs2);
  return (Pi - dr * Dc - rho * (ux * ux + uy * uy) + 0.5f * G2) * inv * (1.f / Dc);
}

template <int ST, int KIND, bool MOM, int BY>
__global__ void __launch_bounds__(32 * BY, (BY <= 8) ? 2 : 1) step2d_kernel(const __grid_constant__ StepArgs a) {
  using L = D2Q37;
  using C = Codec<ST>;
  using T = typename C::T;
  constexpr int BX = 32;
  constexpr int NT = BX * BY;
  constexpr int H = (KIND == KIND_SC) ? 3 : ((KIND == KIND_THERMAL && !MOM) ? 1 : 0);
  using Fr = Frame2<BX, BY, (H > 0 ? H : 1)>;
  constexpr float Dc = (float)(2.0 * L::cs2);
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  __shared__ float aux[(H > 0) ? Fr::SW * Fr::SH : 1];
  __shared__ double red[MOM ? (NT / 32) * 6 : 1];

  const T* __restrict__ fin = static_cast<const T*>(a.fin);
  const int nx = a.nx, ny = a.ny;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int gxp = x0 + tx, gyp = y0 + ty;
  const bool active = gxp < nx && gyp < ny;
  const int x = gxp < nx ? gxp : gxp % nx;
  const int y = gyp < ny ? gyp : gyp % ny;
  const int node = y * nx + x;

  float g[L::Q];
  gather<L, C>(fin, a.N, nx, ny, 1, x, y, 0, g);
  float dr, J[3], Pi;
  moments<L>(g, dr, J, Pi);
  const float rho = a.rho0 + dr;
  float acc[3];
  accel<2>(a, node, y, acc);
  float Fx = rho * acc[0], Fy = rho * acc[1];
  float sigma = 0.f;

  if constexpr (KIND == KIND_SC) {
    const float psi = psi_of<L>(a, rho);
    aux[(ty + H) * Fr::SW + tx + H] = psi;
    for (int k = tid; k < Fr::count; k += NT) {
      int i, j;
      Fr::pos(k, i, j);
      const int hx = wrapm(x0 - H + i, nx), hy = wrapm(y0 - H + j, ny);
      float gh[L::Q];
      gather<L, C>(fin, a.N, nx, ny, 1, hx, hy, 0, gh);
      aux[j * Fr::SW + i] = psi_of<L>(a, a.rho0 + sum_w<L>(gh));
    }
    __syncthreads();
    // F^SC = -G psi(x) sum_i w_i psi(x + c_i) c_i with G = -1
    float sx = 0.f, sy = 0.f;
    static_for<L::NPAIR>([&](auto P) {
      constexpr int i = 2 * P + 1;
      constexpr int cx = L::c(i, 0), cy = L::c(i, 1);
      const float dpsi = aux[(ty + H + cy) * Fr::SW + tx + H + cx] - aux[(ty + H - cy) * Fr::SW + tx + H - cx];
      if constexpr (cx != 0) sx = fmaf((float)(L::w(i) * cx), dpsi, sx);
      if constexpr (cy != 0) sy = fmaf((float)(L::w(i) * cy), dpsi, sy);
    });
    const float fsx = psi * sx, fsy = psi * sy;
    Fx += fsx;
    Fy += fsy;
    // P_i trace coefficient (Eq. 3.12): sigma = p_coef |F^SC|^2 / psi^2
    sigma = (psi > 0.f) ? a.p_coef * (fsx * fsx + fsy * fsy) / (psi * psi) : 0.f;
  }

  const float inv_rho = 1.f / rho;
  const float ux = fmaf(0.5f, Fx, J[0]) * inv_rho;
  const float uy = fmaf(0.5f, Fy, J[1]) * inv_rho;
  const float uu = ux * ux + uy * uy;
  const float G2 = 2.f * (ux * Fx + uy * Fy) + Dc * sigma;
  const float tb_m = (Pi - dr * Dc - rho * uu + 0.5f * G2) * inv_rho * (1.f / Dc);

  if constexpr (MOM) {
    if (active) {
      if (a.rho_out) a.rho_out[node] = rho;
      if (a.u_out) {
        a.u_out[node] = ux;
        a.u_out[(size_t)a.N + node] = uy;
      }
      if (a.theta_out) a.theta_out[node] = 1.f + tb_m;
    }
    if (a.partials) {
      // FP64 block sums: d rho, rho u, (Pi + G2/2)/2, non-finite count
      double v[6] = {0, 0, 0, 0, 0, 0};
      if (active) {
        const bool bad = !(isfinite(rho) && rho > 0.f && isfinite(ux) && isfinite(uy) && isfinite(tb_m));
        v[0] = dr;
        v[1] = (double)rho * ux;
        v[2] = (double)rho * uy;
        v[4] = 0.5 * ((double)Pi + 0.5 * (double)G2);
        v[5] = bad ? 1.0 : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
      if ((tid & 31) == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) red[(tid >> 5) * 6 + k] = v[k];
      __syncthreads();
      if (tid < 6) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w * 6 + tid];
        a.partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + tid] = s;
      }
    }
  } else {
    NodeSrc s;
    s.hG[0] = s.hG[1] = s.hG[2] = 0.f;
    if constexpr (KIND == KIND_THERMAL) {
      // theta - 1 on the tile and its 4-neighbour frame, then grad theta
      aux[(ty + 1) * Fr::SW + tx + 1] = tb_m;
      for (int k = tid; k < Fr::count; k += NT) {
        int i, j;
        Fr::pos(k, i, j);
        const int hx = wrapm(x0 - 1 + i, nx), hy = wrapm(y0 - 1 + j, ny);
        float gh[L::Q];
        gather<L, C>(fin, a.N, nx, ny, 1, hx, hy, 0, gh);
        aux[j * Fr::SW + i] = theta_bar_local<L>(a, gh, hy * nx + hx, hy);
      }
      __syncthreads();
      const float gtx = 0.5f * (aux[(ty + 1) * Fr::SW + tx + 2] - aux[(ty + 1) * Fr::SW + tx]);
      const float gty = 0.5f * (aux[(ty + 2) * Fr::SW + tx + 1] - aux[ty * Fr::SW + tx + 1]);
      // s^(3) += rho theta (1 - 1/Pr) [delta grad_xi theta], grad_xi = c0 grad
      const float hc = rho * (1.f + tb_m) * a.h_coef * (float)L::c0;
      s.hG[0] = hc * gtx;
      s.hG[1] = hc * gty;
    }
    s.dr = dr;
    s.rho = rho;
    s.tb = a.isothermal ? 0.f : tb_m;
    s.u[0] = ux * inv_c0;
    s.u[1] = uy * inv_c0;
    s.u[2] = 0.f;
    s.F[0] = Fx * inv_c0;
    s.F[1] = Fy * inv_c0;
    s.F[2] = 0.f;
    s.sigma = sigma;
    float K[15];
    poly2<L>(s, a.omega, a.beta, K);
    apply_poly<L, 15>(g, K, 1.f - a.omega);
    if (active) {
      T* __restrict__ fout = static_cast<T*>(a.fout);
      static_for<L::Q>([&](auto I) {
        constexpr int i = I;
        C::st(fout + (size_t)i * (size_t)a.N + node, g[i]);
      });
    }
  }
}

template <int ST>
cudaError_t launch_step2d_st(const StepArgs& a, int kind, bool mom, int rows, cudaStream_t s) {
  const int by = (rows == 4 || rows == 16) ? rows : 8;
  const dim3 grid((a.nx + 31) / 32, (a.ny + by - 1) / by, 1);
  const dim3 block(32, by, 1);
#define HLBM_L2(K, M, R) step2d_kernel<ST, K, M, R><<<grid, block, 0, s>>>(a)
  if (mom) {
    const dim3 g8((a.nx + 31) / 32, (a.ny + 7) / 8, 1);
    if (kind == KIND_SC) step2d_kernel<ST, KIND_SC, true, 8><<<g8, dim3(32, 8), 0, s>>>(a);
    else step2d_kernel<ST, KIND_LOCAL, true, 8><<<g8, dim3(32, 8), 0, s>>>(a);
  } else if (by == 4) {
    if (kind == KIND_SC) HLBM_L2(KIND_SC, false, 4);
    else if (kind == KIND_THERMAL) HLBM_L2(KIND_THERMAL, false, 4);
    else HLBM_L2(KIND_LOCAL, false, 4);
  } else if (by == 8) {
    if (kind == KIND_SC) HLBM_L2(KIND_SC, false, 8);
    else if (kind == KIND_THERMAL) HLBM_L2(KIND_THERMAL, false, 8);
    else HLBM_L2(KIND_LOCAL, false, 8);
  } else {
    if (kind == KIND_SC) HLBM_L2(KIND_SC, false, 16);
    else if (kind == KIND_THERMAL) HLBM_L2(KIND_THERMAL, false, 16);
    else HLBM_L2(KIND_LOCAL, false, 16);
  }
#undef HLBM_L2
  return cudaGetLastError();
}

}  // namespace hlbm
