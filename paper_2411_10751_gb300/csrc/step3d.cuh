// Fused pull-collide-source step on D3Q39 (Eq. 4.4 with the third-order
// equilibrium that the degree-7 quadrature supports), CTA tile 32 x BY x 1
// nodes, population planes [Q][nz][ny][nx], periodic.  Each thread gathers
// its nodes' pulled populations straight from global memory (wrapped
// indices) and runs NPT nodes (tile rows ty and ty + BY / NPT) on the paired
// FP32 lanes of float2 when NPT = 2.  Sources: body force F_i (Eq. 3.3) from
// a uniform, per-row or full acceleration field.
#pragma once

#include <type_traits>

#include "step_common.cuh"
#include "tma.cuh"

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
  const V inv_rho = vmap(rho, [](float r) { return rcp_nr(r); });
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
      if (!activek[k] || !HLBM_IN(nodek[k], a.N, DBG_STORE)) continue;
      // 16-bit storage: stochastic rounding keyed by node and result (step_common.cuh)
      const uint32_t salt = std::is_same<T, float>::value ? 0u : node_salt(nodek[k], lane(g[0], k));
      static_for<L::Q>([&](auto I) {
        constexpr int i = I;
        fout[(size_t)i * (size_t)a.N + nodek[k]] = round_store<T>(lane(g[i], k), pop_bits(salt, i));
      });
    }
  }
}

// Persistent D3Q39 step on tiles of 256 nodes that span whole x-rows
// (nx = 32, 64, 128 or 256; a tile is 256 / nx rows of one z-plane).  Each
// population plane of a tile is one 4D tensor box at x = 0 shifted by
// (-c_y, -c_z), so the periodic wrap in x is an index mask in shared memory
// and the wrap in z a wrapped box coordinate; a plane whose rows cross the
// domain's y-edge is copied row by row with wrapped y.  With a force field
// the tile's three acceleration planes come on the same barrier, into one of
// two slots by tile parity.  Tiles come in order (y rows, then z planes; the
// order reversed on every other step) from the step's device counter; as soon
// as a tile's populations are in registers the CTA takes the next index and
// issues its copies, so the loads overlap the collision and the stores.  Two
// nodes per thread (tile nodes t and t + 128) on the paired FP32 lanes.
constexpr int kRows3Nodes = 256;

// population planes, then two slots (by tile parity) of the tile's
// acceleration (3 FP32 planes, used with a force field), then the mbarrier
template <int ST>
constexpr int rows3_smem() {
  return D3Q39::Q * kRows3Nodes * (int)sizeof(typename Codec<ST>::T) + 2 * 3 * kRows3Nodes * 4 + 16;
}

template <int ST>
__global__ void __launch_bounds__(128, 3)
    step3d_rows_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ CUtensorMap tm_box,
                       const __grid_constant__ CUtensorMap tm_row, const __grid_constant__ CUtensorMap tm_g) {
  using L = D3Q39;
  using C = Codec<ST>;
  using T = typename C::T;
  using V = float2;
  constexpr int NT = 128, TN = kRows3Nodes;
  constexpr uint32_t TX = (uint32_t)(L::Q * TN * (int)sizeof(T));
  constexpr float Dc = (float)(3.0 * L::cs2);
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_next[2];
  T* sp = reinterpret_cast<T*>(smem);
  float* sg = reinterpret_cast<float*>(smem + L::Q * TN * (int)sizeof(T));   // acceleration [2][3][TN]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::Q * TN * (int)sizeof(T) + 2 * 3 * TN * 4);
  // a.g_staged: the force field's planes come with the tile (threads Q .. Q + 2 copy them)
  const bool gs = a.g_staged != 0;
  const uint32_t tx = TX + (gs ? 3u * TN * 4u : 0u);
  const int issuers = L::Q + (gs ? 3 : 0);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int by = TN / nx;
  const int nty = (ny + by - 1) / by;
  const int ntiles = nty * nz;
  const unsigned long long period = (unsigned long long)ntiles + gridDim.x;
  const int tid = threadIdx.x, xm = nx - 1;
  if (!HLBM_IN(smem_u32(smem) & 127u, 1, DBG_SMEM)) return;   // TMA destinations need 128-byte alignment
  int xk[2], rk[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int j = tid + NT * k;
    xk[k] = j & xm;
    rk[k] = j / nx;
  }
  int pcy = 0, pcz = 0;   // this thread's plane (tid < Q) for issuing copies
  if (tid < L::Q) d3_cyz(tid, pcy, pcz, typename make_iseq<L::Q>::type{});
  // tile t's z-plane and first row; a.reverse (every other step) runs the
  // order backwards, so a step starts on the tiles the previous one wrote last
  auto tile_of = [&](int t, int& z, int& y0) {
    const int u = a.reverse ? ntiles - 1 - t : t;
    z = u / nty;
    y0 = (u - z * nty) * by;
  };
  // threads tid < Q: the copies of population plane tid of tile t; threads
  // Q .. Q + 2 (with a staged force field): acceleration plane tid - Q (the
  // barrier is armed)
  auto issue_plane = [&](int t, int slot) {
    int z, y0;
    tile_of(t, z, y0);
    if (tid >= L::Q) {   // acceleration plane tid - Q into slot `slot`; rows past the y-edge read zero
      fence_proxy_async_smem();
      tma_load_4d(sg + (slot * 3 + tid - L::Q) * TN, &tm_g, 0, y0, z, tid - L::Q, bar);
      return;
    }
    const int zz = wrap_near3(z - pcz, nz);
    const int ys = y0 - pcy;
    if (!HLBM_IN(zz, nz, DBG_BOX)) return;   // a dropped copy leaves the barrier short
    fence_proxy_async_smem();
    if (ys >= 0 && ys + by <= ny) {
      tma_load_4d(sp + tid * TN, &tm_box, 0, ys, zz, tid, bar);
    } else {
      for (int r = 0; r < by; ++r) {
        const int yy = ((ys + r) % ny + ny) % ny;   // rows may pass several periods when ny < by + 6
        tma_load_4d(sp + tid * TN + r * nx, &tm_row, 0, yy, zz, tid, bar);
      }
    }
  };
  // tid 0: takes the next tile index into slot `slot` and arms the barrier for it
  auto take = [&](int slot) {
    const int t = (int)(atomicAdd(a.tile_ctr, 1ull) % period);
    s_next[slot] = t;
    if (t < ntiles) mbar_arrive_expect_tx(bar, tx);
  };
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    take(0);
  }
  __syncthreads();
  int t = s_next[0];
  if (t < ntiles && tid < issuers && !a.debug_skip_tma) issue_plane(t, 0);
  uint32_t phase = 0;
  for (int it = 1; t < ntiles; ++it) {
    int z, y0;
    tile_of(t, z, y0);
    const bool ok = mbar_wait_bounded(bar, phase, a.wait_ns);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(a.status, (int)5 /* HLBM_ETIMEOUT */);
      mbar_wait_bounded(bar, phase, a.wait_ns);
      __syncthreads();
      return;
    }
    phase ^= 1u;
    if (tid == 0) take(it & 1);   // the barrier's next phase belongs to the next tile
    V g[L::Q];
    static_for<L::Q>([&](auto I) {
      constexpr int i = I;
      constexpr int cx = L::c(i, 0);
#pragma unroll
      for (int k = 0; k < 2; ++k) set_lane(g[i], k, to_float(sp[i * TN + HLBM_IDX(rk[k] * nx + ((xk[k] - cx) & xm), TN, DBG_STAGE)]));
    });
    __syncthreads();  // the staging buffer is free and the next index is published
    const int tn = s_next[it & 1];
    if (tn < ntiles && tid < issuers && !a.debug_skip_tma) issue_plane(tn, it & 1);

    int yk[2], nodek[2];
    bool activek[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int y = y0 + rk[k];
      activek[k] = y < ny;
      yk[k] = y < ny ? y : y - ny;
      nodek[k] = (z * ny + yk[k]) * nx + xk[k];
    }
    V dr, acc, J[3], Pih;
    moments_h<L>(g, dr, acc, J, Pih);
    const V rho = vadd(splat<V>(a.rho0), dr);
    V ga[3];
    if (gs) {   // this tile's slot; the next tile's copies go to the other one
      const float* sgc = sg + ((it - 1) & 1) * 3 * TN;
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 2; ++k) set_lane(ga[d], k, sgc[d * TN + rk[k] * nx + xk[k]]);
    } else {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        float gk[3];
        accel<3>(a, nodek[k], yk[k], gk);
#pragma unroll
        for (int d = 0; d < 3; ++d) set_lane(ga[d], k, gk[d]);
      }
    }
    const V F0 = vmul(rho, ga[0]), F1 = vmul(rho, ga[1]), F2 = vmul(rho, ga[2]);
    const V inv_rho = vmap(rho, [](float r) { return rcp_nr(r); });
    const V ux = vmul(vfma(splat<V>(0.5f), F0, J[0]), inv_rho);
    const V uy = vmul(vfma(splat<V>(0.5f), F1, J[1]), inv_rho);
    const V uz = vmul(vfma(splat<V>(0.5f), F2, J[2]), inv_rho);
    const V uu = vfma(ux, ux, vfma(uy, uy, vmul(uz, uz)));
    const V G2 = vmul(splat<V>(2.f), vfma(ux, F0, vfma(uy, F1, vmul(uz, F2))));
    const V tb_m =
        vmul(vmul(vfma(splat<V>(0.5f), G2, vsub(Pih, vmul(rho, uu))), inv_rho), splat<V>(1.f / Dc));
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
    for (int k = 0; k < 2; ++k) {
      if (!activek[k] || !HLBM_IN(nodek[k], a.N, DBG_STORE)) continue;
      const uint32_t salt = std::is_same<T, float>::value ? 0u : node_salt(nodek[k], lane(g[0], k));
      static_for<L::Q>([&](auto I) {
        constexpr int i = I;
        fout[(size_t)i * (size_t)a.N + nodek[k]] = round_store<T>(lane(g[i], k), pop_bits(salt, i));
      });
    }
    t = tn;
  }
}

// Whether the whole-row persistent kernel serves this domain: a row of the
// stored type must fill 128 bytes so that the single-row copies land on
// 128-byte aligned shared-memory addresses (16-bit storage from nx = 64).
template <int ST>
inline bool rows3_eligible(const StepArgs& a) {
  return a.tma && (a.nx == 32 || a.nx == 64 || a.nx == 128 || a.nx == 256) &&
         a.nx * (int)sizeof(typename Codec<ST>::T) >= 128;
}

template <int ST>
int rows3_ctas() {
  static std::atomic<int> cache[kMaxDevicesCached];
  return per_device_cached(cache, [](int dev) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step3d_rows_kernel<ST>, 128, rows3_smem<ST>());
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  });
}

// rows: 4 or 8 tile rows; npt: nodes per thread (2 needs 8 rows); tmaps: the
// whole-row box and single-row maps of the input buffer (persistent kernel),
// or null.
template <int ST>
cudaError_t launch_step3d_st(const StepArgs& a, int kind, bool mom, int rows, int npt, const CUtensorMap* tmaps,
                             cudaStream_t s) {
  if (kind != KIND_LOCAL) return cudaErrorInvalidValue;
  if (!mom && a.persistent && tmaps && rows3_eligible<ST>(a)) {
    const int by = kRows3Nodes / a.nx;
    const int tiles = ((a.ny + by - 1) / by) * a.nz;
    const int ctas = std::min(tiles, rows3_ctas<ST>());
    step3d_rows_kernel<ST><<<ctas, 128, rows3_smem<ST>(), s>>>(a, tmaps[0], tmaps[1], tmaps[2]);
    return cudaGetLastError();
  }
  const int by = (rows == 4) ? 4 : 8;
  const dim3 grid((a.nx + 31) / 32, (a.ny + by - 1) / by, a.nz);
  if (mom) step3d_kernel<ST, true, 8, 1><<<dim3((a.nx + 31) / 32, (a.ny + 7) / 8, a.nz), dim3(32, 8), 0, s>>>(a);
  else if (by == 4) step3d_kernel<ST, false, 4, 1><<<grid, dim3(32, 4), 0, s>>>(a);
  else if (npt == 2) step3d_kernel<ST, false, 8, 2><<<grid, dim3(32, 4), 0, s>>>(a);
  else step3d_kernel<ST, false, 8, 1><<<grid, dim3(32, 8), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hlbm
