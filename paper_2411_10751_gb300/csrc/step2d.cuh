// Fused pull-collide-source step on D2Q37 (Eq. 4.4), one node per thread,
// with the pulled populations staged in shared memory by TMA.
//
// CTA tile: 32 x BY nodes; population planes are [Q][ny][nx] in global
// memory (structure of arrays, periodic by index wrap, no halo cells).
// A node x pulls g_i from x - c_i.  For the tile and a frame of H nodes
// around it (the "region", (32 + 2H) x (BY + 2H) nodes), plane i is needed on
// the region shifted by -c_i; that rectangle, widened on the left to the
// 16-byte x alignment of tiled bulk copies and to a common width WB, is one
// TMA box.  One thread issues the Q boxes against an mbarrier; every gather is
// then a shared-memory load at a compile-time offset.  The left widening of
// plane i, rem_i = (-H - c_ix) mod A (A = 16 bytes / element), does not depend
// on the tile because tile x origins are multiples of 32.
// Tiles whose boxes would cross the periodic edge (or domains whose row pitch
// is not a multiple of 16 bytes) fill the same layout with wrapped loads.
//
// Neighbour fields of time t (no lag: all sources of Eq. 4.4 are taken at t):
//   KIND_THERMAL  grad theta for H_i: theta on the 4-neighbour ring (H = 1)
//   KIND_SC       F^SC (Eq. 3.8): psi(rho) on a three-node frame (H = 3)
// Both are computed from the staged populations of the region into a
// shared-memory tile, so the frame costs arithmetic but no extra HBM reads.
#pragma once

#include "step_common.cuh"
#include "tma.cuh"

#include <algorithm>
#include <type_traits>

namespace hlbm {

template <int ST, int KIND, bool MOM, int BY>
struct Cfg2 {
  using C = Codec<ST>;
  using T = typename C::T;
  using L = D2Q37;
  static constexpr int BX = 32;
  static constexpr int NT = BX * BY;
  static constexpr int H = (KIND == KIND_SC) ? 3 : ((KIND == KIND_THERMAL && !MOM) ? 1 : 0);
  static constexpr int A = 16 / (int)sizeof(T);
  static constexpr int RW = BX + 2 * H, RH = BY + 2 * H;
  static constexpr int WB = ((RW + A - 1 + A - 1) / A) * A;  // box width (elements)
  static constexpr int HB = RH;                             // box height
  static constexpr int PLANE_BYTES = ((WB * HB * (int)sizeof(T) + 127) / 128) * 128;
  static constexpr int PLANE = PLANE_BYTES / (int)sizeof(T);
  static constexpr int POP_BYTES = L::Q * PLANE_BYTES;
  static constexpr int AUX_BYTES = (H > 0) ? ((RW * RH * 4 + 127) / 128) * 128 : 0;
  static constexpr int RED_BYTES = MOM ? ((NT / 32) * 6 * 8 + 127) / 128 * 128 : 0;
  static constexpr int SMEM = POP_BYTES + AUX_BYTES + RED_BYTES + 128;  // + mbarrier
  static constexpr int OUT_BYTES = L::Q * BX * BY * (int)sizeof(T);        // separately staged results
  static constexpr uint32_t TX_BYTES = (uint32_t)L::Q * WB * HB * (uint32_t)sizeof(T);
  __host__ __device__ static constexpr int rem(int i) { return ((-H - L::c(i, 0)) % A + A) % A; }
};

template <int BX, int BY, int H>
struct Frame2 {
  static constexpr int SW = BX + 2 * H;
  static constexpr int SH = BY + 2 * H;
  // region nodes outside the tile: the 4-neighbour ring for H == 1 (no
  // corners), the full frame for H == 3
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

// Index of population i at in-box offset off in the staged planes, and of
// frame entry k (both checked against their extent in the debug build).
template <class Cf>
__device__ __forceinline__ int stg(int i, int off) {
  return i * Cf::PLANE + HLBM_IDX(off, Cf::WB * Cf::HB, DBG_STAGE);
}
template <class Fr>
__device__ __forceinline__ int frm(int k) {
  return HLBM_IDX(k, Fr::SW * Fr::SH, DBG_FRAME);
}

// the Q pulled populations of region node (rx, ry) from the staged planes
template <class Cf>
__device__ __forceinline__ void load_region(const typename Cf::T* sp, int rx, int ry, float (&g)[37]) {
  const int base = ry * Cf::WB + rx;
  static_for<37>([&](auto I) {
    constexpr int i = I;
    g[i] = to_float(sp[stg<Cf>(i, base + Cf::rem(i))]);
  });
}

// theta - 1 of a node from its pulled populations (Eq. 4.5), local force only
template <class L>
__device__ __forceinline__ float theta_bar_local(const StepArgs& a, float (&g)[L::Q], int node, int y) {
  float dr, acc, J[3], Pih;
  moments_h<L>(g, dr, acc, J, Pih);
  const float rho = a.rho0 + dr;
  float gacc[3];
  accel<2>(a, node, y, gacc);
  const float inv = rcp_nr(rho);
  const float ux = fmaf(0.5f * rho, gacc[0], J[0]) * inv;
  const float uy = fmaf(0.5f * rho, gacc[1], J[1]) * inv;
  const float G2 = 2.f * rho * (ux * gacc[0] + uy * gacc[1]);
  constexpr float Dc = (float)(2.0 * L::cs2);
  return (Pih - rho * (ux * ux + uy * uy) + 0.5f * G2) * inv * (1.f / Dc);
}

// CTAs per SM the register budget is sized for: as many as the staged tile's
// shared memory allows, at most 3 for 256 threads (80 registers), 2 for 512.
template <int ST, int KIND, bool MOM, int BY, int NPT>
constexpr int min_ctas2() {
  constexpr int threads = 32 * BY / NPT;
  constexpr int by_smem = (227 * 1024) / Cfg2<ST, KIND, MOM, BY>::SMEM;
  constexpr int cap = (threads >= 512) ? 2 : (threads <= 128 ? 4 : 3);
  return by_smem < 1 ? 1 : (by_smem < cap ? by_smem : cap);
}

// Issues the Q staging boxes of the tile at (x0, y0) against `bar`.
template <class Cf>
__device__ __forceinline__ void issue_tile(typename Cf::T* sp, const CUtensorMap* tmap, uint64_t* bar, int x0, int y0,
                                           int skip, int nx, int ny) {
  using L = D2Q37;
  constexpr int H = Cf::H;
  mbar_arrive_expect_tx(bar, Cf::TX_BYTES);
  if (!skip) {
    static_for<37>([&](auto I) {
      constexpr int i = I;
      const int bx = x0 - H - L::c(i, 0) - Cf::rem(i), by = y0 - H - L::c(i, 1);
#ifdef HLBM_DEBUG
      // the box must start on the 16-byte grid and lie inside the domain
      // (a dropped box leaves the barrier short: the bounded wait expires)
      if (!HLBM_IN(bx % Cf::A, 1, DBG_BOX) || !HLBM_IN(bx, nx - Cf::WB + 1, DBG_BOX) ||
          !HLBM_IN(by, ny - Cf::HB + 1, DBG_BOX))
        return;
#endif
      tma_load_3d(sp + i * Cf::PLANE, tmap, bx, by, i, bar);
    });
  }
}

// issue_tile with the Q boxes split over the CTA's warps: lane 0 of warp w
// issues the planes i = w (mod W), so that no warp spends the whole issue
// sequence while the others wait for it at the next barrier.  Every warp's
// lane 0 calls it (the plane parameters stay compile-time constants); warp 0
// arms the barrier (the order of arming and completion does not matter).
template <class Cf, int W>
__device__ __forceinline__ void issue_tile_split(typename Cf::T* sp, const CUtensorMap* tmap, uint64_t* bar, int x0,
                                                 int y0, int skip, int nx, int ny, int warp) {
  using L = D2Q37;
  constexpr int H = Cf::H;
  if (warp == 0) mbar_arrive_expect_tx(bar, Cf::TX_BYTES);
  if (skip) return;
  static_for<37>([&](auto I) {
    constexpr int i = I;
    if (i % W != warp) return;
    const int bx = x0 - H - L::c(i, 0) - Cf::rem(i), by = y0 - H - L::c(i, 1);
#ifdef HLBM_DEBUG
    if (!HLBM_IN(bx % Cf::A, 1, DBG_BOX) || !HLBM_IN(bx, nx - Cf::WB + 1, DBG_BOX) ||
        !HLBM_IN(by, ny - Cf::HB + 1, DBG_BOX))
      return;
#endif
    tma_load_3d(sp + i * Cf::PLANE, tmap, bx, by, i, bar);
  });
  (void)nx;
  (void)ny;
}

// Whether the tile's boxes lie inside the domain (no periodic wrap needed).
template <class Cf>
__device__ __forceinline__ bool tile_boxed(const StepArgs& a, int x0, int y0) {
  constexpr int H = Cf::H;
  return a.tma && (x0 - H - 3 - (Cf::A - 1) >= 0) && (x0 - H + 3 + Cf::WB <= a.nx) && (y0 - H - 3 >= 0) &&
         (y0 - H + 3 + Cf::HB <= a.ny);
}

// Edge tile: every region node gathers its Q pulled populations of `fin_v`
// with periodic wrap (independent loads through codec C) and writes them into
// the staged layout.
template <class Cf, int NT, class C = typename Cf::C>
__device__ __forceinline__ void fill_tile_wrapped(const StepArgs& a, const void* fin_v, typename Cf::T* sp, int x0,
                                                  int y0, int tid) {
  using L = D2Q37;
  using T = typename Cf::T;
  constexpr int H = Cf::H;
  const T* __restrict__ fin = static_cast<const T*>(fin_v);
  for (int k = tid; k < Cf::RW * Cf::RH; k += NT) {
    const int ry = k / Cf::RW, rx = k - ry * Cf::RW;
    const int X = wrapm(x0 - H + rx, a.nx), Y = wrapm(y0 - H + ry, a.ny);
    float gk[37];
    gather<L, C>(fin, a.N, a.nx, a.ny, 1, X, Y, 0, gk);
    const int base = ry * Cf::WB + rx;
    static_for<37>([&](auto I) {
      constexpr int i = I;
      sp[stg<Cf>(i, base + Cf::rem(i))] = from_float<T>(gk[i]);
    });
  }
}

// The work on one staged tile: moments, neighbour fields, sources, collision
// and stores (into fout_v).  `staged_done()` runs once every read of the
// staging buffer has finished (after a CTA barrier), so a caller may start
// refilling it then.  TMA_STORE: results leave through the staging buffer by
// bulk tensor stores.
// SEP_OUT: the results are staged for their bulk stores in a buffer of
// their own behind the tile's shared memory (Cfg2::OUT_BYTES at Cfg2::SMEM;
// planes of 32 x BY), so that the next tile may already be landing in the
// input planes.
template <int ST, int KIND, bool MOM, int BY, int NPT, bool TMA_STORE, bool SEP_OUT = false, class Done>
__device__ __forceinline__ void process_tile(const StepArgs& a, const CUtensorMap* tmap_out, unsigned char* smem,
                                             int x0, int y0, void* fout_v, Done&& staged_done) {
  using Cf = Cfg2<ST, KIND, MOM, BY>;
  using L = D2Q37;
  using T = typename Cf::T;
  using V = typename std::conditional<NPT == 2, float2, float>::type;
  constexpr int BX = Cf::BX, H = Cf::H;
  constexpr int TR = BY / NPT;     // thread rows
  constexpr int NT = BX * TR;      // threads
  using Fr = Frame2<BX, BY, (H > 0 ? H : 1)>;
  constexpr float Dc = (float)(2.0 * L::cs2);
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  T* sp = reinterpret_cast<T*>(smem);
  float* aux = reinterpret_cast<float*>(smem + Cf::POP_BYTES);
  double* red = reinterpret_cast<double*>(smem + Cf::POP_BYTES + Cf::AUX_BYTES);
  const int nx = a.nx, ny = a.ny;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;

  // ---- this thread's nodes (lane k: tile row ty + k * TR)
  const int x = (x0 + tx < nx) ? x0 + tx : (x0 + tx) % nx;
  int yk[NPT], nodek[NPT];
  bool activek[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int gyp = y0 + ty + k * TR;
    activek[k] = (x0 + tx < nx) && gyp < ny;
    yk[k] = gyp < ny ? gyp : gyp % ny;
    nodek[k] = yk[k] * nx + x;
  }

  V g[37];
  static_for<37>([&](auto I) {
    constexpr int i = I;
#pragma unroll
    for (int k = 0; k < NPT; ++k)
      set_lane(g[i], k, to_float(sp[stg<Cf>(i, (ty + k * TR + H) * Cf::WB + tx + H + Cf::rem(i))]));
  });
  V dr, dr_l, acc, J[3], Pih;
  moments_h<L>(g, dr, dr_l, acc, J, Pih);
  const V rho = vadd(splat<V>(a.rho0), dr);
  V gax = splat<V>(0.f), gay = splat<V>(0.f);
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    float ga[3];
    accel<2>(a, nodek[k], yk[k], ga);
    set_lane(gax, k, ga[0]);
    set_lane(gay, k, ga[1]);
  }
  V Fx = vmul(rho, gax), Fy = vmul(rho, gay);
  V sigma = splat<V>(0.f);

  if constexpr (KIND == KIND_SC) {
    V psi;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      set_lane(psi, k, psi_of<L>(a, lane(dr, k), lane(dr_l, k)));
      aux[frm<Fr>((ty + k * TR + H) * Fr::SW + tx + H)] = lane(psi, k);
    }
    for (int k = tid; k < Fr::count; k += NT) {
      int i, j;
      Fr::pos(k, i, j);
      float gh[37];
      static_for<37>([&](auto I) {
        constexpr int q = I;
        gh[q] = to_float(sp[stg<Cf>(q, j * Cf::WB + i + Cf::rem(q))]);
      });
      float hl;
      const float hd = density_h<L>(gh, hl);
      aux[frm<Fr>(j * Fr::SW + i)] = psi_of<L>(a, hd, hl);
    }
    __syncthreads();
    staged_done();
    // F^SC = -G psi(x) sum_i w_i psi(x + c_i) c_i with G = -1
    V sx = splat<V>(0.f), sy = splat<V>(0.f);
    static_for<L::NPAIR>([&](auto P) {
      constexpr int i = 2 * P + 1;
      constexpr int cx = L::c(i, 0), cy = L::c(i, 1);
      V dpsi;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int r = ty + k * TR + H;
        set_lane(dpsi, k, aux[frm<Fr>((r + cy) * Fr::SW + tx + H + cx)] - aux[frm<Fr>((r - cy) * Fr::SW + tx + H - cx)]);
      }
      if constexpr (cx != 0) sx = vfma(splat<V>((float)(L::w(i) * cx)), dpsi, sx);
      if constexpr (cy != 0) sy = vfma(splat<V>((float)(L::w(i) * cy)), dpsi, sy);
    });
    const V fsx = vmul(psi, sx), fsy = vmul(psi, sy);
    Fx = vadd(Fx, fsx);
    Fy = vadd(Fy, fsy);
    // P_i trace coefficient (Eq. 3.12): sigma = p_coef |F^SC|^2 / psi^2
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const float ps = lane(psi, k), fx = lane(fsx, k), fy = lane(fsy, k);
      set_lane(sigma, k, (ps > 0.f) ? a.p_coef * (fx * fx + fy * fy) * rcp_nr(ps * ps) : 0.f);
    }
  }

  const V inv_rho = vmap(rho, [](float r) { return rcp_nr(r); });
  const V ux = vmul(vfma(splat<V>(0.5f), Fx, J[0]), inv_rho);
  const V uy = vmul(vfma(splat<V>(0.5f), Fy, J[1]), inv_rho);
  const V uu = vfma(ux, ux, vmul(uy, uy));
  const V G2 = vfma(splat<V>(Dc), sigma, vmul(splat<V>(2.f), vfma(ux, Fx, vmul(uy, Fy))));
  const V tb_m = vmul(vmul(vfma(splat<V>(0.5f), G2, vsub(Pih, vmul(rho, uu))), inv_rho), splat<V>(1.f / Dc));

  if constexpr (MOM) {
    double v[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (!activek[k]) continue;
      const int node = nodek[k];
      const float r = lane(rho, k), vx = lane(ux, k), vy = lane(uy, k), tb = lane(tb_m, k);
      if (a.rho_out) a.rho_out[node] = r;
      if (a.u_out) {
        a.u_out[node] = vx;
        a.u_out[(size_t)a.N + node] = vy;
      }
      if (a.theta_out) a.theta_out[node] = 1.f + tb;
      // FP64 block sums: d rho, rho u, (Pi + G2/2)/2, non-finite count
      const bool bad = !(isfinite(r) && r > 0.f && isfinite(vx) && isfinite(vy) && isfinite(tb));
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
      if ((tid & 31) == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) red[(tid >> 5) * 6 + k] = v[k];
      __syncthreads();
      if (tid < 6) {
        double sum = 0.0;
        for (int w = 0; w < NT / 32; ++w) sum += red[w * 6 + tid];
        a.partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + tid] = sum;
      }
    }
  } else {
    NodeSrcT<V> s;
    s.hG[0] = s.hG[1] = s.hG[2] = splat<V>(0.f);
    if constexpr (KIND == KIND_LOCAL) {
      __syncthreads();
      staged_done();
    }
    if constexpr (KIND == KIND_THERMAL) {
      // theta - 1 on the tile and its 4-neighbour ring, then grad theta
#pragma unroll
      for (int k = 0; k < NPT; ++k) aux[frm<Fr>((ty + k * TR + 1) * Fr::SW + tx + 1)] = lane(tb_m, k);
      for (int k = tid; k < Fr::count; k += NT) {
        int i, j;
        Fr::pos(k, i, j);
        const int hx = wrapm(x0 - 1 + i, nx), hy = wrapm(y0 - 1 + j, ny);
        float gh[37];
        static_for<37>([&](auto I) {
          constexpr int q = I;
          gh[q] = to_float(sp[stg<Cf>(q, j * Cf::WB + i + Cf::rem(q))]);
        });
        aux[frm<Fr>(j * Fr::SW + i)] = theta_bar_local<L>(a, gh, hy * nx + hx, hy);
      }
      __syncthreads();
      staged_done();
      V gtx, gty;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int r = ty + k * TR + 1;
        set_lane(gtx, k, 0.5f * (aux[frm<Fr>(r * Fr::SW + tx + 2)] - aux[frm<Fr>(r * Fr::SW + tx)]));
        set_lane(gty, k, 0.5f * (aux[frm<Fr>((r + 1) * Fr::SW + tx + 1)] - aux[frm<Fr>((r - 1) * Fr::SW + tx + 1)]));
      }
      // s^(3) += rho theta (1 - 1/Pr) [delta grad_xi theta], grad_xi = c0 grad
      const V hc = vmul(vmul(rho, vadd(splat<V>(1.f), tb_m)), splat<V>(a.h_coef * (float)L::c0));
      s.hG[0] = vmul(hc, gtx);
      s.hG[1] = vmul(hc, gty);
    }
    s.dr = splat<V>(0.f);  // density deviation re-enters in apply_poly_h
    s.rho = rho;
    s.tb = a.isothermal ? splat<V>(0.f) : tb_m;
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
    // the density's rounding error matters where F^SC amplifies it
    if constexpr (KIND == KIND_SC) K[0] = vadd(K[0], dr_l);
    apply_poly_h<L, 15>(g, K, om1, dr);
    // 16-bit storage: stochastic rounding keyed by node and result (step_common.cuh)
    uint32_t salt[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) salt[k] = std::is_same<T, float>::value ? 0u : node_salt(nodek[k], lane(g[0], k));
    if (TMA_STORE && a.tma_store) {
      // stage the tile's results densely in the (now unused) input planes and
      // write each plane with one bulk tensor store; out-of-domain rows and
      // columns of a ragged tile are clipped by the copy
      constexpr int OP = SEP_OUT ? BX * BY : Cf::PLANE;   // plane stride of the staged results
      T* const so = SEP_OUT ? reinterpret_cast<T*>(smem + Cf::SMEM) : sp;
      __syncthreads();
      static_for<37>([&](auto I) {
        constexpr int i = I;
#pragma unroll
        for (int k = 0; k < NPT; ++k)
          so[i * OP + HLBM_IDX((ty + k * TR) * BX + tx, BX * BY, DBG_STAGE)] =
              round_store<T>(lane(g[i], k), pop_bits(salt[k], i));
      });
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        static_for<37>([&](auto I) {
          constexpr int i = I;
          tma_store_3d(tmap_out, so + i * OP, x0, y0, i);
        });
        bulk_commit();
        bulk_wait_read_all();   // the staging buffer has been read; the writes complete with the grid
      }
    } else {
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        if (!activek[k] || !HLBM_IN(nodek[k], a.N, DBG_STORE)) continue;
        T* __restrict__ fout = static_cast<T*>(fout_v) + nodek[k];
        static_for<37>([&](auto I) {
          constexpr int i = I;
          fout[(size_t)i * (size_t)a.N] = round_store<T>(lane(g[i], k), pop_bits(salt[k], i));
        });
      }
    }
  }
}

// One CTA per tile.
template <int ST, int KIND, bool MOM, int BY, int NPT>
__global__ void __launch_bounds__(32 * BY / NPT, (min_ctas2<ST, KIND, MOM, BY, NPT>()))
    step2d_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ CUtensorMap tmap,
                  const __grid_constant__ CUtensorMap tmap_out) {
  using Cf = Cfg2<ST, KIND, MOM, BY>;
  constexpr int NT = 32 * BY / NPT;
  extern __shared__ __align__(128) unsigned char smem[];
  typename Cf::T* sp = reinterpret_cast<typename Cf::T*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Cf::POP_BYTES + Cf::AUX_BYTES + Cf::RED_BYTES);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * BY;
  if (tile_boxed<Cf>(a, x0, y0) && ((smem_u32(smem) & 127u) == 0)) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) issue_tile<Cf>(sp, &tmap, bar, x0, y0, a.debug_skip_tma, a.nx, a.ny);
    const bool ok = mbar_wait_bounded(bar, 0, a.wait_ns);
    if (!__syncthreads_and(ok)) {
      // copies did not complete: report, give in-flight copies a second bounded
      // wait, and leave without touching the outputs
      if (tid == 0) atomicExch(a.status, (int)5 /* HLBM_ETIMEOUT */);
      mbar_wait_bounded(bar, 0, a.wait_ns);
      __syncthreads();
      return;
    }
  } else {
    fill_tile_wrapped<Cf, NT>(a, a.fin, sp, x0, y0, tid);
    __syncthreads();
  }
  process_tile<ST, KIND, MOM, BY, NPT, true>(a, &tmap_out, smem, x0, y0, a.fout, [] {});
}

// Tiles whose staging boxes lie inside the domain form a rectangle of tile
// indices [ix0, ix1) x [iy0, iy1) (tile_boxed is monotone in x0 and y0); the
// others, on the periodic edge, form a frame around it.
template <class Cf, int BY>
struct TileSplit {
  int ntx, nty, ix0, ix1, iy0, iy1, ni, ne;
  __device__ TileSplit(const StepArgs& a, bool tma) {
    constexpr int H = Cf::H;
    ntx = (a.nx + 31) / 32;
    nty = (a.ny + BY - 1) / BY;
    const int xl = H + 3 + (Cf::A - 1), xr = a.nx + H - 3 - Cf::WB;
    const int yl = H + 3, yr = a.ny + H - 3 - Cf::HB;
    ix0 = (xl + 31) / 32;
    ix1 = xr >= 0 ? min(ntx, xr / 32 + 1) : 0;
    iy0 = (yl + BY - 1) / BY;
    iy1 = yr >= 0 ? min(nty, yr / BY + 1) : 0;
    if (!tma || ix1 <= ix0 || iy1 <= iy0) ix0 = ix1 = iy0 = iy1 = 0;
    ni = (ix1 - ix0) * (iy1 - iy0);
    ne = ntx * nty - ni;
  }
  __device__ void interior(int j, int& tx, int& ty) const {
    const int w = ix1 - ix0;
    const int r = j / w;
    ty = iy0 + r;
    tx = ix0 + (j - r * w);
  }
  __device__ void edge(int e, int& tx, int& ty) const {
    const int top = iy0 * ntx;
    if (e < top) {
      ty = e / ntx;
      tx = e - ty * ntx;
      return;
    }
    e -= top;
    const int mw = ix0 + (ntx - ix1), mid = (iy1 - iy0) * mw;
    if (e < mid) {
      const int r = e / mw, cc = e - r * mw;
      ty = iy0 + r;
      tx = cc < ix0 ? cc : ix1 + (cc - ix0);
      return;
    }
    e -= mid;
    const int r = e / ntx;
    ty = iy1 + r;
    tx = e - r * ntx;
  }
};

// Persistent CTAs that take tiles in a global order from a device counter.
// Tiles on the periodic edge stage by per-node gathers, synchronously; when
// they are more than 5% of the tiles they come first (their stalls overlap
// one another at the start), otherwise all tiles go in row-major order (edge
// tiles then share L2-resident lines with their interior neighbours instead
// of reading them from DRAM a second time).  While a CTA works on a tile it already takes
// the next index and stages that tile by TMA as soon as the current tile's
// last staged read is done, so loads overlap the collision and stores; and
// since tiles are handed out in order, the tiles in flight stay a compact
// band of the domain (their frames are served by L2) however the CTAs' speeds
// differ.  The counter is never reset between launches: a launch of G CTAs
// over T tiles takes exactly T + G values (every CTA stops at its first index
// >= T), so the tile is the counter value mod (T + G).
// 16-bit storage: results leave by bulk tensor stores from a staging buffer
// of their own (the input planes hold the next tile by then); FP32 storage,
// whose 63 KB of staging leaves no room for it: coalesced global stores.
template <int ST>
constexpr bool persistent_sep_out() {
  return ST != ST_F32;
}
template <int ST, int KIND, int BY>
constexpr int persistent_smem() {
  return Cfg2<ST, KIND, false, BY>::SMEM + (persistent_sep_out<ST>() ? Cfg2<ST, KIND, false, BY>::OUT_BYTES : 0);
}

template <int ST, int KIND, int BY, int NPT>
constexpr int min_ctas_persistent() {
  constexpr int threads = 32 * BY / NPT;
  constexpr int by_smem = (227 * 1024) / persistent_smem<ST, KIND, BY>();
  constexpr int cap = (threads >= 512) ? 2 : (threads <= 128 ? 4 : 3);
  return by_smem < 1 ? 1 : (by_smem < cap ? by_smem : cap);
}

template <int ST, int KIND, int BY, int NPT>
__global__ void __launch_bounds__(32 * BY / NPT, (min_ctas_persistent<ST, KIND, BY, NPT>()))
    step2d_persistent_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ CUtensorMap tmap,
                             const __grid_constant__ CUtensorMap tmap_out) {
  using Cf = Cfg2<ST, KIND, false, BY>;
  constexpr int NT = 32 * BY / NPT;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_next;
  typename Cf::T* sp = reinterpret_cast<typename Cf::T*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Cf::POP_BYTES + Cf::AUX_BYTES + Cf::RED_BYTES);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const bool aligned = (smem_u32(smem) & 127u) == 0;
  const TileSplit<Cf, BY> ts(a, a.tma && aligned);
  const int ntiles = ts.ntx * ts.nty;
  const unsigned long long period = (unsigned long long)ntiles + gridDim.x;
  const bool edge_first = ts.ne * 20 > ntiles;
  // a.reverse (every other step): the row-major part of the order runs
  // backwards, so a step starts on the tiles the previous step wrote last,
  // which are still in L2
  auto origin = [&](int t, int& x0, int& y0) {
    int tx, ty;
    if (!edge_first) {
      const int u = a.reverse ? ntiles - 1 - t : t;
      ty = u / ts.ntx;
      tx = u - ty * ts.ntx;
    } else {
      // edge tiles first, except for the pseudopotential kind, where boxed
      // tiles open and close the step and the gathered edge tiles sit in the
      // middle (same-box: droplet 1024^2 12.07k -> 12.31k MLUPS; the thermal
      // step loses 4% that way)
      const int h = (KIND == KIND_SC) ? ts.ni / 2 : 0;
      if (t >= h && t < h + ts.ne) {
        ts.edge(t - h, tx, ty);
      } else {
        const int j = t < h ? t : t - ts.ne;
        ts.interior(a.reverse ? ts.ni - 1 - j : j, tx, ty);
      }
    }
    x0 = tx * 32;
    y0 = ty * BY;
  };
  // Tile indices come one tile ahead: during tile k the CTA stages tile k+1
  // (s_ahead, published at the end of tile k-1) at staged_done, its copies
  // split over the warps, and thread 0 takes the index of tile k+2 then; the
  // counter's raw value is reduced only at the end of tile k, so the atomic's
  // round trip overlaps the collision.  A CTA takes no index after its first
  // one >= T, so a launch still takes exactly T + G values.
  __shared__ int s_ahead;
  unsigned long long raw = 0;
  auto take = [&]() { return atomicAdd(a.tile_ctr, 1ull); };
  auto stage = [&](int tn) {   // lane 0 of every warp: stages tile tn if it is a boxed tile
    if (tn < ntiles) {
      int xn, yn;
      origin(tn, xn, yn);
      if (aligned && tile_boxed<Cf>(a, xn, yn)) {
        fence_proxy_async_smem();
        issue_tile_split<Cf, NT / 32>(sp, &tmap, bar, xn, yn, a.debug_skip_tma, a.nx, a.ny, tid >> 5);
      }
    }
  };
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    const int t0 = (int)(take() % period);
    s_next = t0;
    s_ahead = (t0 < ntiles) ? (int)(take() % period) : t0;
  }
  __syncthreads();
  if ((tid & 31) == 0) stage(s_next);
  uint32_t phase = 0;
  int t = s_next;
  while (t < ntiles) {
    const int tn = s_ahead;
    int x0, y0;
    origin(t, x0, y0);
    if (aligned && tile_boxed<Cf>(a, x0, y0)) {
      const bool ok = mbar_wait_bounded(bar, phase, a.wait_ns);
      if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(a.status, (int)5 /* HLBM_ETIMEOUT */);
        mbar_wait_bounded(bar, phase, a.wait_ns);
        __syncthreads();
        return;
      }
      phase ^= 1u;
    } else {
      fill_tile_wrapped<Cf, NT>(a, a.fin, sp, x0, y0, tid);
      __syncthreads();
    }
    constexpr bool SEP = persistent_sep_out<ST>();
    process_tile<ST, KIND, false, BY, NPT, SEP, SEP>(a, &tmap_out, smem, x0, y0, a.fout, [&] {
      if ((tid & 31) == 0) stage(tn);
      if (tid == 0 && tn < ntiles) raw = take();
    });
    if (tid == 0) s_ahead = (tn < ntiles) ? (int)(raw % period) : tn;
    __syncthreads();  // s_ahead is published; the shared aux tile is reused by the next tile
    t = tn;
  }
}

// Multi-step persistent D2Q37 step: one launch runs a.msteps steps of Eq. 4.4
// on a domain that the 32 x BY tiles cover exactly.  Tiles are taken in the
// order (step, tile row, tile column) from the launch's counter; the tile of
// step s reads the output of step s - 1 over its own region and the tiles
// around it (periodic), and overwrites the buffer that they read in step
// s - 1, so it starts once tile rows ty - 1, ty and ty + 1 have completed
// step s - 1.  Each tile row has a completion counter (tiles of that row
// finished, over all steps since the counters were zeroed): a row has
// completed step s - 1 when its counter reaches (gen0 + s) ntx, since no tile
// of a row can finish step s before the row has finished step s - 1.  Every
// wait points at tiles taken earlier, which running CTAs hold, so the launch
// needs no co-residency and no grid barrier: the ramp-up and tail of a launch
// per step are gone, and at a step boundary only the first tile row waits
// for the last one.
// Thread 0 keeps the synchronisation off the critical path: it takes tile
// indices one tile ahead and loads the three counters of a taken tile while
// the CTA works on the current one; at staged_done a single fence serves as
// the acquire for the next tile's counters and the release of the CTA's
// previous tile (its stores have drained by then), then the next tile's
// copies are issued.  A tile whose rows are not ready yet is waited for after
// the current tile's stores.  Waits are bounded by a.wait_ns; an expired wait
// or another CTA's error stops the CTA.
template <int ST, int KIND, int BY, int NPT>
__global__ void __launch_bounds__(32 * BY / NPT, (min_ctas2<ST, KIND, false, BY, NPT>()))
    step2d_multistep_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ CUtensorMap tm_even,
                            const __grid_constant__ CUtensorMap tm_odd) {
  using Cf = Cfg2<ST, KIND, false, BY>;
  constexpr int NT = 32 * BY / NPT;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_next, s_ready, s_ok;
  typename Cf::T* sp = reinterpret_cast<typename Cf::T*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Cf::POP_BYTES + Cf::AUX_BYTES + Cf::RED_BYTES);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const bool aligned = (smem_u32(smem) & 127u) == 0;
  const int ntx = a.nx / 32, nty = a.ny / BY;
  const int T = ntx * nty;
  const int total = T * a.msteps;
  unsigned* rowcnt = a.flags;
  auto decode = [&](int v, int& s, int& tx, int& ty) {
    s = v / T;
    const int t = v - s * T;
    ty = t / ntx;
    tx = t - ty * ntx;
  };
  // tid 0 state: the next tile and the counters of its rows (loaded when it
  // was taken), and the finished tile row whose completion is not released yet
  int nxt = -1, pend_row = -1;
  unsigned c0 = 0, c1 = 0, c2 = 0;
  auto load_rows = [&](int v) {
    int s, tx, ty;
    decode(v, s, tx, ty);
    if (s == 0) return;
    c0 = ld_relaxed_gpu(rowcnt + ((ty == 0) ? nty - 1 : ty - 1));
    c1 = ld_relaxed_gpu(rowcnt + ty);
    c2 = ld_relaxed_gpu(rowcnt + ((ty + 1 == nty) ? 0 : ty + 1));
  };
  auto rows_ready = [&](int v) -> bool {
    int s, tx, ty;
    decode(v, s, tx, ty);
    if (s == 0) return true;
    const unsigned need = (a.gen0 + (unsigned)s) * (unsigned)ntx;
    return (int)(c0 - need) >= 0 && (int)(c1 - need) >= 0 && (int)(c2 - need) >= 0;
  };
  auto release_pending = [&]() {   // after a fence
    if (pend_row >= 0) {
      red_relaxed_add_gpu(rowcnt + pend_row, 1u);
      pend_row = -1;
    }
  };
  // stages tile v (its rows are ready and acquired)
  auto issue = [&](int v) {
    int s, tx, ty;
    decode(v, s, tx, ty);
    if (aligned && tile_boxed<Cf>(a, tx * 32, ty * BY)) {
      fence_proxy_async_global();   // the acquired generic-proxy writes before these bulk reads
      fence_proxy_async_smem();
      issue_tile<Cf>(sp, (s & 1) ? &tm_odd : &tm_even, bar, tx * 32, ty * BY, a.debug_skip_tma, a.nx, a.ny);
    }
  };
  // tid 0 at staged_done: takes the tile after next, releases the previous
  // tile, and stages the next tile if its rows are ready
  auto advance = [&]() {
    const unsigned long long vv = atomicAdd(a.ms_ctr, 1ull);
    const int cur = nxt;
    const bool ok = cur >= 0 && rows_ready(cur);
    fence_acq_rel_gpu();
    release_pending();
    if (ok) issue(cur);
    s_next = cur;
    s_ready = ok ? 1 : 0;
    nxt = vv < (unsigned long long)total ? (int)vv : -1;
    if (nxt >= 0) load_rows(nxt);
  };
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    const unsigned long long v0 = atomicAdd(a.ms_ctr, 1ull);
    nxt = v0 < (unsigned long long)total ? (int)v0 : -1;
    if (nxt >= 0) load_rows(nxt);
    advance();
  }
  __syncthreads();
  uint32_t phase = 0;
  int v = s_next, ready = s_ready;
  while (v >= 0) {
    int s, tx, ty;
    decode(v, s, tx, ty);
    const int x0 = tx * 32, y0 = ty * BY;
    const bool boxed = aligned && tile_boxed<Cf>(a, x0, y0);
    if (!ready) {
      if (tid == 0) {
        fence_acq_rel_gpu();
        release_pending();   // the tile may wait for the one this CTA just finished
        const unsigned k0 = c0, k1 = c1, k2 = c2;   // the lookahead tile's counters
        bool ok = false;
        const uint64_t t0 = global_ns();
        for (uint32_t k = 0; k < (1u << 30); ++k) {
          load_rows(v);
          if (rows_ready(v)) {
            fence_acq_rel_gpu();
            ok = true;
            break;
          }
          if (*(volatile int*)a.status != 0 || global_ns() - t0 > a.wait_ns) break;
          __nanosleep(64);
        }
        c0 = k0;
        c1 = k1;
        c2 = k2;
        if (ok) issue(v);
        else atomicCAS(a.status, 0, (int)5 /* HLBM_ETIMEOUT */);
        s_ok = ok ? 1 : 0;
      }
      __syncthreads();
      if (!s_ok) return;   // nothing of this tile is in flight
    }
    if (boxed) {
      const bool ok = mbar_wait_bounded(bar, phase, a.wait_ns);
      if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(a.status, (int)5 /* HLBM_ETIMEOUT */);
        mbar_wait_bounded(bar, phase, a.wait_ns);
        __syncthreads();
        return;
      }
      phase ^= 1u;
    } else {
      fill_tile_wrapped<Cf, NT, CodecCG<ST>>(a, (s & 1) ? a.fout : a.fin, sp, x0, y0, tid);
      __syncthreads();
    }
    process_tile<ST, KIND, false, BY, NPT, false>(a, nullptr, smem, x0, y0, (s & 1) ? const_cast<void*>(a.fin) : a.fout,
                                                  [&] {
                                                    if (tid == 0) advance();
                                                  });
    __syncthreads();   // the tile's stores are issued; s_next and s_ready are published
    if (tid == 0) pend_row = ty;
    v = s_next;
    ready = s_ready;
  }
  if (tid == 0) {
    fence_acq_rel_gpu();
    release_pending();
  }
}

// Box geometry of the launch configuration (for the host's tensor maps).
template <int ST, int KIND, bool MOM, int BY>
void box_of(int& wb, int& hb) {
  wb = Cfg2<ST, KIND, MOM, BY>::WB;
  hb = Cfg2<ST, KIND, MOM, BY>::HB;
}
template <int ST, int KIND, bool MOM, int BY>
int rows_of() {
  return BY;
}

template <int ST, int KIND, bool MOM, int BY, int NPT = 1>
cudaError_t configure2() {
  cudaError_t e = cudaFuncSetAttribute(step2d_kernel<ST, KIND, MOM, BY, NPT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg2<ST, KIND, MOM, BY>::SMEM);
  if (e != cudaSuccess || MOM) return e;
  e = cudaFuncSetAttribute(step2d_persistent_kernel<ST, KIND, BY, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           persistent_smem<ST, KIND, BY>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(step2d_multistep_kernel<ST, KIND, BY, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Cfg2<ST, KIND, false, BY>::SMEM);
}

// CTAs of a persistent launch: the resident CTAs per SM times the SM count.
template <int ST, int KIND, int BY, int NPT>
int persistent_ctas() {
  static std::atomic<int> cache[kMaxDevicesCached];
  return per_device_cached(cache, [](int dev) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step2d_persistent_kernel<ST, KIND, BY, NPT>, 32 * BY / NPT,
                                                  persistent_smem<ST, KIND, BY>());
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  });
}

template <int ST, int KIND, int BY, int NPT>
int multistep_ctas() {
  static std::atomic<int> cache[kMaxDevicesCached];
  return per_device_cached(cache, [](int dev) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step2d_multistep_kernel<ST, KIND, BY, NPT>, 32 * BY / NPT,
                                                  Cfg2<ST, KIND, false, BY>::SMEM);
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  });
}

template <int ST, int KIND, bool MOM, int BY, int NPT = 1>
cudaError_t launch2(const StepArgs& a, const CUtensorMap* tmaps, cudaStream_t s) {
  using Cf = Cfg2<ST, KIND, MOM, BY>;
  if constexpr (!MOM) {
    if (a.msteps > 0) {
      // tmaps: the staging maps of fin and fout (same box)
      const int tiles = (a.nx / 32) * (a.ny / BY) * a.msteps;
      const int ctas = std::min(tiles, multistep_ctas<ST, KIND, BY, NPT>());
      CUtensorMap t0{}, t1{};
      if (tmaps) {
        t0 = tmaps[0];
        t1 = tmaps[1];
      }
      step2d_multistep_kernel<ST, KIND, BY, NPT><<<ctas, dim3(32, BY / NPT, 1), Cf::SMEM, s>>>(a, t0, t1);
      return cudaGetLastError();
    }
    if (a.persistent) {
      const int tiles = ((a.nx + 31) / 32) * ((a.ny + BY - 1) / BY);
      const int ctas = std::min(tiles, persistent_ctas<ST, KIND, BY, NPT>());
      CUtensorMap tm{}, tmo{};
      if (tmaps) {
        tm = tmaps[0];
        tmo = tmaps[1];
      }
      step2d_persistent_kernel<ST, KIND, BY, NPT>
          <<<ctas, dim3(32, BY / NPT, 1), persistent_smem<ST, KIND, BY>(), s>>>(a, tm, tmo);
      return cudaGetLastError();
    }
  }
  const dim3 grid((a.nx + 31) / 32, (a.ny + BY - 1) / BY, 1);
  const dim3 block(32, BY / NPT, 1);
  CUtensorMap tm{}, tmo{};
  if (tmaps) {
    tm = tmaps[0];
    tmo = tmaps[1];
  }
  step2d_kernel<ST, KIND, MOM, BY, NPT><<<grid, block, Cf::SMEM, s>>>(a, tm, tmo);
  return cudaGetLastError();
}

// Sets the shared-memory size attribute of every 2D kernel of this storage
// (done once, outside any stream capture).
template <int ST>
cudaError_t configure_step2d_st() {
  const cudaError_t es[] = {
      configure2<ST, KIND_LOCAL, false, 4>(),   configure2<ST, KIND_THERMAL, false, 4>(),
      configure2<ST, KIND_SC, false, 4>(),      configure2<ST, KIND_LOCAL, false, 8>(),
      configure2<ST, KIND_THERMAL, false, 8>(), configure2<ST, KIND_SC, false, 8>(),
      configure2<ST, KIND_LOCAL, false, 16>(),  configure2<ST, KIND_THERMAL, false, 16>(),
      configure2<ST, KIND_SC, false, 16>(),     configure2<ST, KIND_LOCAL, true, 8>(),
      configure2<ST, KIND_SC, true, 8>(),       configure2<ST, KIND_LOCAL, false, 8, 2>(),
      configure2<ST, KIND_THERMAL, false, 8, 2>(), configure2<ST, KIND_SC, false, 8, 2>(),
      configure2<ST, KIND_LOCAL, false, 16, 2>(), configure2<ST, KIND_THERMAL, false, 16, 2>(),
      configure2<ST, KIND_SC, false, 16, 2>()};
  for (cudaError_t e : es)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

// Dispatch: box geometry query (wb/hb/ob non-null: input box and output
// tile rows) or launch.  tm: {input map, output map} or null.
template <int ST>
cudaError_t launch_step2d_st(const StepArgs& a, int kind, bool mom, int rows, int npt, const CUtensorMap* tm,
                             cudaStream_t s, int* wb, int* hb, int* ob = nullptr) {
  const int by = (rows == 4 || rows == 16) ? rows : 8;
  const int np = (npt == 2 && by >= 8 && !mom) ? 2 : 1;
#define HLBM_CASE(K, M, R, NP)                    \
  do {                                            \
    if (wb) {                                     \
      box_of<ST, K, M, R>(*wb, *hb);              \
      if (ob) *ob = rows_of<ST, K, M, R>();       \
      return cudaSuccess;                         \
    }                                             \
    return launch2<ST, K, M, R, NP>(a, tm, s);    \
  } while (0)
#define HLBM_KINDS(R, NP)                                      \
  do {                                                         \
    if (kind == KIND_SC) HLBM_CASE(KIND_SC, false, R, NP);     \
    if (kind == KIND_THERMAL) HLBM_CASE(KIND_THERMAL, false, R, NP); \
    HLBM_CASE(KIND_LOCAL, false, R, NP);                       \
  } while (0)
  if (mom) {
    if (kind == KIND_SC) HLBM_CASE(KIND_SC, true, 8, 1);
    HLBM_CASE(KIND_LOCAL, true, 8, 1);
  }
  if (by == 4) HLBM_KINDS(4, 1);
  if (by == 8) {
    if (np == 2) HLBM_KINDS(8, 2);
    HLBM_KINDS(8, 1);
  }
  if (np == 2) HLBM_KINDS(16, 2);
  HLBM_KINDS(16, 1);
#undef HLBM_KINDS
#undef HLBM_CASE
}

}  // namespace hlbm
