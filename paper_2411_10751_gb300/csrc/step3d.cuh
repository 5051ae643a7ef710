// Fused pull-collide-source step on D3Q39 (Eq. 4.4 with the third-order
// equilibrium that the degree-7 quadrature supports), CTA tile 32 x BY x 1
// nodes, population planes [Q][nz][ny][nx], periodic.  Each thread gathers
// its nodes' pulled populations straight from global memory (wrapped
// indices) and runs NPT nodes (tile rows ty and ty + BY / NPT) on the paired
// FP32 lanes of float2 when NPT = 2.  Sources: body force F_i (Eq. 3.3) from
// a uniform, per-row or full acceleration field.
#pragma once

#include "step_common.cuh"

namespace hlbm {

template <bool MOM, int NPT>
constexpr int min_ctas3() {
  return MOM ? 2 : (NPT == 2 ? 3 : 2);
}

template <int ST, bool MOM, int BY, int NPT>
__global__ void __launch_bounds__(32 * BY / NPT, (min_ctas3<MOM, NPT>()))
    step3d_kernel(const __grid_constant__ StepArgs a) {
  using L = D3Q39;
  using C = Codec<ST>;
  using T = typename C::T;
  using V = typename std::conditional<NPT == 2, float2, float>::type;
  static_assert(!MOM || NPT == 1, "the moments readout runs one node per thread");
  constexpr int TR = BY / NPT;     // thread rows
  constexpr int NT = 32 * TR;
  constexpr float Dc = (float)(3.0 * L::cs2);
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  __shared__ double red[MOM ? (NT / 32) * 6 : 1];

  const T* __restrict__ fin = static_cast<const T*>(a.fin);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int gxp = blockIdx.x * 32 + tx, z = blockIdx.z;
  const int x = gxp < nx ? gxp : gxp % nx;
  int yk[NPT], nodek[NPT];
  bool activek[NPT];
  V g[L::Q];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int gyp = blockIdx.y * BY + ty + k * TR;
    activek[k] = gxp < nx && gyp < ny;
    yk[k] = gyp < ny ? gyp : gyp % ny;
    nodek[k] = (z * ny + yk[k]) * nx + x;
    float gk[L::Q];
    gather<L, C>(fin, a.N, nx, ny, nz, x, yk[k], z, gk);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) set_lane(g[i], k, gk[i]);
  }
  V dr, acc, J[3], Pih;
  moments_h<L>(g, dr, acc, J, Pih);
  const V rho = vadd(splat<V>(a.rho0), dr);
  V ga[3];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    float gk[3];
    accel<3>(a, nodek[k], yk[k], gk);
#pragma unroll
    for (int d = 0; d < 3; ++d) set_lane(ga[d], k, gk[d]);
  }
  const V F0 = vmul(rho, ga[0]), F1 = vmul(rho, ga[1]), F2 = vmul(rho, ga[2]);
  const V inv_rho = vmap(rho, [](float r) { return 1.f / r; });
  const V ux = vmul(vfma(splat<V>(0.5f), F0, J[0]), inv_rho);
  const V uy = vmul(vfma(splat<V>(0.5f), F1, J[1]), inv_rho);
  const V uz = vmul(vfma(splat<V>(0.5f), F2, J[2]), inv_rho);
  const V uu = vfma(ux, ux, vfma(uy, uy, vmul(uz, uz)));
  const V G2 = vmul(splat<V>(2.f), vfma(ux, F0, vfma(uy, F1, vmul(uz, F2))));
  const V tb_m = vmul(vmul(vfma(splat<V>(0.5f), G2, vsub(Pih, vmul(rho, uu))), inv_rho), splat<V>(1.f / Dc));

  if constexpr (MOM) {
    const float r = lane(rho, 0), vx = lane(ux, 0), vy = lane(uy, 0), vz = lane(uz, 0), tb = lane(tb_m, 0);
    const int node = nodek[0];
    if (activek[0]) {
      if (a.rho_out) a.rho_out[node] = r;
      if (a.u_out) {
        a.u_out[node] = vx;
        a.u_out[(size_t)a.N + node] = vy;
        a.u_out[2 * (size_t)a.N + node] = vz;
      }
      if (a.theta_out) a.theta_out[node] = 1.f + tb;
    }
    if (a.partials) {
      double v[6] = {0, 0, 0, 0, 0, 0};
      if (activek[0]) {
        const bool bad = !(isfinite(r) && r > 0.f && isfinite(vx) && isfinite(vy) && isfinite(vz) && isfinite(tb));
        v[0] = lane(dr, 0);
        v[1] = (double)r * vx;
        v[2] = (double)r * vy;
        v[3] = (double)r * vz;
        v[4] = 0.5 * ((double)lane(Pih, 0) + (double)Dc * lane(dr, 0) + 0.5 * (double)lane(G2, 0));
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
    NodeSrcT<V> s;
    s.dr = splat<V>(0.f);  // density deviation re-enters in apply_poly_h
    s.rho = rho;
    s.tb = a.isothermal ? splat<V>(0.f) : tb_m;
    s.u[0] = vmul(ux, splat<V>(inv_c0));
    s.u[1] = vmul(uy, splat<V>(inv_c0));
    s.u[2] = vmul(uz, splat<V>(inv_c0));
    s.F[0] = vmul(F0, splat<V>(inv_c0));
    s.F[1] = vmul(F1, splat<V>(inv_c0));
    s.F[2] = vmul(F2, splat<V>(inv_c0));
    s.hG[0] = s.hG[1] = s.hG[2] = splat<V>(0.f);
    s.sigma = splat<V>(0.f);
    V K[20];
    poly3<L>(s, a.omega, a.beta, K);
    const float om1 = 1.f - a.omega;
    K[0] = vfma(splat<V>(-om1), acc, K[0]);
    apply_poly_h<L, 20>(g, K, om1, dr);
    T* __restrict__ fout = static_cast<T*>(a.fout);
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (!activek[k]) continue;
      static_for<L::Q>([&](auto I) {
        constexpr int i = I;
        C::st(fout + (size_t)i * (size_t)a.N + nodek[k], lane(g[i], k));
      });
    }
  }
}

// rows: 4 or 8 tile rows; npt: nodes per thread (2 needs 8 rows).
template <int ST>
cudaError_t launch_step3d_st(const StepArgs& a, int kind, bool mom, int rows, int npt, cudaStream_t s) {
  if (kind != KIND_LOCAL) return cudaErrorInvalidValue;
  const int by = (rows == 4) ? 4 : 8;
  const dim3 grid((a.nx + 31) / 32, (a.ny + by - 1) / by, a.nz);
  if (mom) step3d_kernel<ST, true, 8, 1><<<dim3((a.nx + 31) / 32, (a.ny + 7) / 8, a.nz), dim3(32, 8), 0, s>>>(a);
  else if (by == 4) step3d_kernel<ST, false, 4, 1><<<grid, dim3(32, 4), 0, s>>>(a);
  else if (npt == 2) step3d_kernel<ST, false, 8, 2><<<grid, dim3(32, 4), 0, s>>>(a);
  else step3d_kernel<ST, false, 8, 1><<<grid, dim3(32, 8), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hlbm
