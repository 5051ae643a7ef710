// Fused pull-collide-source step on D3Q39 (Eq. 4.4 with the third-order
// equilibrium that the degree-7 quadrature supports), one node per thread,
// CTA tile 32 x BY x 1 nodes, population planes [Q][nz][ny][nx], periodic.
// Sources: body force F_i (Eq. 3.3) from a uniform, per-row or full
// acceleration field.
#pragma once

#include "step_common.cuh"

namespace hlbm {

template <int ST, bool MOM, int BY>
__global__ void __launch_bounds__(32 * BY, 2) step3d_kernel(const __grid_constant__ StepArgs a) {
  using L = D3Q39;
  using C = Codec<ST>;
  using T = typename C::T;
  constexpr int NT = 32 * BY;
  constexpr float Dc = (float)(3.0 * L::cs2);
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  __shared__ double red[MOM ? (NT / 32) * 6 : 1];

  const T* __restrict__ fin = static_cast<const T*>(a.fin);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int gxp = blockIdx.x * 32 + tx, gyp = blockIdx.y * BY + ty, z = blockIdx.z;
  const bool active = gxp < nx && gyp < ny;
  const int x = gxp < nx ? gxp : gxp % nx;
  const int y = gyp < ny ? gyp : gyp % ny;
  const int node = (z * ny + y) * nx + x;

  float g[L::Q];
  gather<L, C>(fin, a.N, nx, ny, nz, x, y, z, g);
  float dr, acc, J[3], Pih;
  moments_h<L>(g, dr, acc, J, Pih);
  const float rho = a.rho0 + dr;
  float gacc[3];
  accel<3>(a, node, y, gacc);
  const float F0 = rho * gacc[0], F1 = rho * gacc[1], F2 = rho * gacc[2];
  const float inv_rho = 1.f / rho;
  const float ux = fmaf(0.5f, F0, J[0]) * inv_rho;
  const float uy = fmaf(0.5f, F1, J[1]) * inv_rho;
  const float uz = fmaf(0.5f, F2, J[2]) * inv_rho;
  const float uu = ux * ux + uy * uy + uz * uz;
  const float G2 = 2.f * (ux * F0 + uy * F1 + uz * F2);
  const float tb_m = (Pih - rho * uu + 0.5f * G2) * inv_rho * (1.f / Dc);

  if constexpr (MOM) {
    if (active) {
      if (a.rho_out) a.rho_out[node] = rho;
      if (a.u_out) {
        a.u_out[node] = ux;
        a.u_out[(size_t)a.N + node] = uy;
        a.u_out[2 * (size_t)a.N + node] = uz;
      }
      if (a.theta_out) a.theta_out[node] = 1.f + tb_m;
    }
    if (a.partials) {
      double v[6] = {0, 0, 0, 0, 0, 0};
      if (active) {
        const bool bad = !(isfinite(rho) && rho > 0.f && isfinite(ux) && isfinite(uy) && isfinite(uz) &&
                           isfinite(tb_m));
        v[0] = dr;
        v[1] = (double)rho * ux;
        v[2] = (double)rho * uy;
        v[3] = (double)rho * uz;
        v[4] = 0.5 * ((double)Pih + (double)Dc * dr + 0.5 * (double)G2);
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
        a.partials[(((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * 8 + tid] = s;
      }
    }
  } else {
    NodeSrc s;
    s.dr = 0.f;  // density deviation re-enters in apply_poly_h
    s.rho = rho;
    s.tb = a.isothermal ? 0.f : tb_m;
    s.u[0] = ux * inv_c0;
    s.u[1] = uy * inv_c0;
    s.u[2] = uz * inv_c0;
    s.F[0] = F0 * inv_c0;
    s.F[1] = F1 * inv_c0;
    s.F[2] = F2 * inv_c0;
    s.hG[0] = s.hG[1] = s.hG[2] = 0.f;
    s.sigma = 0.f;
    float K[20];
    poly3<L>(s, a.omega, a.beta, K);
    const float om1 = 1.f - a.omega;
    K[0] = fmaf(-om1, acc, K[0]);
    apply_poly_h<L, 20>(g, K, om1, dr);
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
cudaError_t launch_step3d_st(const StepArgs& a, int kind, bool mom, int rows, cudaStream_t s) {
  if (kind != KIND_LOCAL) return cudaErrorInvalidValue;
  const int by = (rows == 4) ? 4 : 8;
  const dim3 grid((a.nx + 31) / 32, (a.ny + by - 1) / by, a.nz);
  const dim3 block(32, by, 1);
  if (mom) step3d_kernel<ST, true, 8><<<dim3((a.nx + 31) / 32, (a.ny + 7) / 8, a.nz), dim3(32, 8), 0, s>>>(a);
  else if (by == 4) step3d_kernel<ST, false, 4><<<grid, block, 0, s>>>(a);
  else step3d_kernel<ST, false, 8><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hlbm
