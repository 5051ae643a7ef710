// Device building blocks of the fused lattice Boltzmann step: storage codecs,
// the pulled gather, the moments of Eq. 4.5 in deviation form, the
// equations of state, and the Hermite-space collision polynomial.
//
// Stored variable.  Populations are kept as Hermite-normalised deviations
//     g_i = (f^_i - w_i rho0) / w_i,
// so that f^eq_i and S_i, both of the form w_i sum_n A^(n) : H^(n)(xi_i) / n!
// (Eqs. 2.4-2.5), lose their weight factor, the stored numbers stay O(signal)
// (no cancellation against w_i rho0 in FP32, no FP16 subnormals for the small
// weights), and the update of Eq. 4.4 reads
//     g*_i = (1 - omega) g_i + sum_n B^(n) : H^(n)(xi_i) / n!,
//     B^(n) = omega a^(n,eq) + beta s^(n),  omega = 1/tau^, beta = 1 - 1/(2 tau^),
// with a^(0,eq) replaced by rho - rho0.
//
// Hermite coefficients (xi = c / c0, velocities and forces divided by c0).
// The Cartesian Hermite tensors factor per axis into probabilists' Hermite
// polynomials He_a, so a coefficient is indexed by its number of x, y (, z)
// indices (a, b (, c)) and the expansion is sum B_ab He_a(xi_x) He_b(xi_y) / (a! b!).
//  * Equilibrium (Eq. 2.6): the Hermite coefficients of the Maxwellian factor
//    into 1D Gaussian moments, a_ab = rho m_a(u_x) m_b(u_y) with
//    m_0 = 1, m_1 = u, m_2 = u^2 + tb, m_3 = u^3 + 3 u tb, m_4 = u^4 + 6 u^2 tb + 3 tb^2
//    (tb = theta - 1), truncated at order 4 (D2Q37) or 3 (D3Q39).
//  * Body force (Eq. 3.2): s^(1) = F, s^(2) = [F u], s^(3) = [F u u] + tb [F delta]
//    are exactly F . d/du of the equilibrium coefficients of orders 1-3 divided
//    by rho, so s_ab = F_x a m_{a-1}(u_x) m_b(u_y) + F_y b m_a(u_x) m_{b-1}(u_y).
//  * Thermal diffusion (Eq. 3.6): s^(3) += rho theta (1 - 1/Pr) [delta grad_xi theta].
//  * Pressure tensor (Eq. 3.12): s^(2) += sigma delta (trace only).
// The sum over n is then rewritten once per node as a polynomial in the
// integer velocity components, P(c) = sum_pq K_pq c_x^p c_y^q, whose monomials
// are compile-time constants per velocity; opposite velocities share the even
// part of P.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "lattice.cuh"

namespace hlbm {

// ------------------------------------------------------------- debug build
// Built with -DHLBM_DEBUG (a separate library), every gathered global index,
// staged shared-memory index, neighbour-frame index, population store, TMA box
// origin and TMA shared-memory destination is checked before the access.  An
// index outside its buffer is counted in the device record dbg_record
// ({count, site, index, bound} of the first; one record per translation unit,
// which registers a host reader for it) and the access is redirected to
// element 0 (loads) or dropped (stores and copies), so a faulty launch runs to
// its end without touching memory outside its buffers, and the host reads the
// records (hlbm_debug_record).  In the release build each check is the plain
// index.
enum DbgSite {
  DBG_GATHER = 1,   // wrapped global gather of the pulled populations
  DBG_STAGE = 2,    // staged populations in shared memory (reads and writes)
  DBG_FRAME = 3,    // neighbour-field frame in shared memory
  DBG_STORE = 4,    // global population store
  DBG_BOX = 5,      // TMA box origin outside the domain or off the 16-byte grid
  DBG_AUX = 6,      // neighbour fields and moments of the previous step (global)
  DBG_SMEM = 7,     // shared-memory base of a TMA destination not 128-byte aligned
};
#ifdef HLBM_DEBUG
static __device__ unsigned long long dbg_record[4];
namespace {
bool dbg_read_record(unsigned long long* out, bool clear) {
  if (cudaMemcpyFromSymbol(out, dbg_record, 4 * sizeof(unsigned long long)) != cudaSuccess) return false;
  const unsigned long long zero[4] = {0, 0, 0, 0};
  return !clear || cudaMemcpyToSymbol(dbg_record, zero, sizeof(zero)) == cudaSuccess;
}
const bool dbg_registered = dbg_register(&dbg_read_record);
}  // namespace
static __device__ __noinline__ void dbg_reject(long long i, long long n, int site) {
  if (atomicAdd(&dbg_record[0], 1ull) == 0ull) {
    dbg_record[1] = (unsigned long long)site;
    dbg_record[2] = (unsigned long long)i;
    dbg_record[3] = (unsigned long long)n;
  }
}
__device__ __forceinline__ bool dbg_ok(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  dbg_reject(i, n, site);
  return false;
}
#define HLBM_IDX(i, n, site) (::hlbm::dbg_ok((long long)(i), (long long)(n), (site)) ? (i) : 0)
#define HLBM_IN(i, n, site) ::hlbm::dbg_ok((long long)(i), (long long)(n), (site))
#else
#define HLBM_IDX(i, n, site) (i)
#define HLBM_IN(i, n, site) true
#endif

// ------------------------------------------------------------------ codecs
template <int S> struct Codec;
template <> struct Codec<ST_F32> {
  using T = float;
  __device__ static __forceinline__ float ld(const T* p) { return __ldg(p); }
  __device__ static __forceinline__ void st(T* p, float v) { *p = v; }
};
template <> struct Codec<ST_F16> {
  using T = __half;
  __device__ static __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)); }
  __device__ static __forceinline__ void st(T* p, float v) { *p = __float2half_rn(v); }
};
template <> struct Codec<ST_BF16> {
  using T = __nv_bfloat16;
  __device__ static __forceinline__ float ld(const T* p) { return __bfloat162float(__ldg(p)); }
  __device__ static __forceinline__ void st(T* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Loads through L2 only (no read-only or L1 path): for buffers that other
// CTAs of the same launch write (the multi-step kernel's edge tiles).
template <int S>
struct CodecCG {
  using T = typename Codec<S>::T;
  __device__ static __forceinline__ float ld(const T* p) {
    if constexpr (S == ST_F32) return __ldcg(p);
    else if constexpr (S == ST_F16) return __half2float(__ldcg(p));
    else return __bfloat162float(__ldcg(p));
  }
  __device__ static __forceinline__ void st(T* p, float v) { Codec<S>::st(p, v); }
};

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }

// c_y, c_z of D3Q39 velocity p for a runtime p (a fold over the compile-time
// table; each thread that issues a plane's copies does one lookup).
template <int... I>
__device__ __forceinline__ void d3_cyz(int p, int& cy, int& cz, iseq<I...>) {
  ((cy = (p == I) ? D3Q39::c(I, 1) : cy), ...);
  ((cz = (p == I) ? D3Q39::c(I, 2) : cz), ...);
}
// --------------------------------------------------- rounding of step results
// Results of a step are rounded to 16-bit storage stochastically: uniform
// random bits are added below the kept mantissa (13 bits for FP16, 16 for
// BF16) and the sum is truncated toward zero, so the stored value is the
// FP32 value on average.  Round-to-nearest gives equal values equal errors:
// a smooth field (neighbouring nodes, successive steps) then accumulates one
// coherent error that the viscosity does not damp, which at 1024^2 left FP16
// at twice its 256^2 error.  The random bits are a hash of the node index and
// of the bits of the node's post-collision rest population (so they change
// from step to step while the field changes, and a run is reproducible bit
// for bit whatever the schedule); the mixing function is the 32-bit
// finalizer of MurmurHash3 (Appleby).  Below the normal range (|v| < 2^-14
// for FP16) the truncation drops more than 13 bits and rounds toward zero
// more often; those values are a few FP16 subnormal steps from zero.
__host__ __device__ __forceinline__ constexpr uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint32_t node_salt(long long node, float g0) {
  return fmix32((uint32_t)node * 0x9E3779B1u ^ __float_as_uint(g0));
}
// random bits for population i of a node with salt h: one multiply by an odd
// constant of its own per population (the finalizer of i + 1, folded at
// compile time); round_store keeps the high bits of the product
__device__ __forceinline__ uint32_t pop_bits(uint32_t h, int i) { return h * (fmix32((uint32_t)i + 1u) | 1u); }
template <class T> __device__ __forceinline__ T round_store(float v, uint32_t bits);
template <> __device__ __forceinline__ float round_store<float>(float v, uint32_t) { return v; }
template <> __device__ __forceinline__ __half round_store<__half>(float v, uint32_t bits) {
  return __float2half_rz(__uint_as_float(__float_as_uint(v) + (bits >> 19)));
}
template <> __device__ __forceinline__ __nv_bfloat16 round_store<__nv_bfloat16>(float v, uint32_t bits) {
  return __float2bfloat16_rz(__uint_as_float(__float_as_uint(v) + (bits >> 16)));
}

// exact for values that came from to_float of the same type
template <class T> __device__ __forceinline__ T from_float(float v);
template <> __device__ __forceinline__ float from_float<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_float<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ------------------------------------------------------- lane arithmetic
// The node arithmetic is written once for V = float (one node per thread)
// and V = float2 (two nodes per thread, mapped onto Blackwell's paired FP32
// instructions FADD2 / FMUL2 / FFMA2, which halve the issue slots of the
// collision).  Every operation below rounds exactly like its scalar form.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <class V> __device__ __forceinline__ V splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 splat<float2>(float c) { return make_float2(c, c); }
template <class V> struct Lanes;
template <> struct Lanes<float> { static constexpr int n = 1; };
template <> struct Lanes<float2> { static constexpr int n = 2; };
__device__ __forceinline__ float lane(float v, int) { return v; }
__device__ __forceinline__ float lane(float2 v, int k) { return k ? v.y : v.x; }
__device__ __forceinline__ void set_lane(float& v, int, float x) { v = x; }
__device__ __forceinline__ void set_lane(float2& v, int k, float x) {
  if (k) v.y = x;
  else v.x = x;
}
template <class F> __device__ __forceinline__ float vmap(float a, F f) { return f(a); }
template <class F> __device__ __forceinline__ float2 vmap(float2 a, F f) { return make_float2(f(a.x), f(a.y)); }

// ----------------------------------------------------- compile-time helpers
__host__ __device__ constexpr int ipow_i(int x, int n) { return n == 0 ? 1 : x * ipow_i(x, n - 1); }
__host__ __device__ constexpr double ipow_d(double x, int n) { return n == 0 ? 1.0 : x * ipow_d(x, n - 1); }
__host__ __device__ constexpr double fact_d(int n) { return n <= 1 ? 1.0 : n * fact_d(n - 1); }
// coefficient of x^p in He_a(x) (a <= 4): He_2 = x^2 - 1, He_3 = x^3 - 3x, He_4 = x^4 - 6x^2 + 3
__host__ __device__ constexpr int he(int a, int p) {
  return a == 0   ? (p == 0 ? 1 : 0)
         : a == 1 ? (p == 1 ? 1 : 0)
         : a == 2 ? (p == 2 ? 1 : p == 0 ? -1 : 0)
         : a == 3 ? (p == 3 ? 1 : p == 1 ? -3 : 0)
                  : (p == 4 ? 1 : p == 2 ? -6 : p == 0 ? 3 : 0);
}

// 2D monomials c_x^p c_y^q, p + q <= 4
__host__ __device__ constexpr int mono2(int m, int axis) {
  constexpr int t[15][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}, {3, 0}, {2, 1},
                            {1, 2}, {0, 3}, {4, 0}, {3, 1}, {2, 2}, {1, 3}, {0, 4}};
  return t[m][axis];
}
// 3D monomials c_x^p c_y^q c_z^r, p + q + r <= 3
__host__ __device__ constexpr int mono3(int m, int axis) {
  constexpr int t[20][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
                            {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {3, 0, 0}, {0, 3, 0}, {0, 0, 3}, {2, 1, 0},
                            {2, 0, 1}, {1, 2, 0}, {0, 2, 1}, {1, 0, 2}, {0, 1, 2}, {1, 1, 1}};
  return t[m][axis];
}
__host__ __device__ constexpr int mono2_index(int p, int q) {
  for (int m = 0; m < 15; ++m)
    if (mono2(m, 0) == p && mono2(m, 1) == q) return m;
  return -1;
}
__host__ __device__ constexpr int mono3_index(int p, int q, int r) {
  for (int m = 0; m < 20; ++m)
    if (mono3(m, 0) == p && mono3(m, 1) == q && mono3(m, 2) == r) return m;
  return -1;
}

// ------------------------------------------------------------- index wrap
// v mod n for v in [-n, 2n) (no integer division)
__device__ __forceinline__ int wrap_near3(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int wrap1(int v, int n) {  // v in [-n, 2n)
  v += (v < 0) ? n : 0;
  v -= (v >= n) ? n : 0;
  return v;
}
__device__ __forceinline__ int wrapm(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// ------------------------------------------------------------------ gather
// g_i(x) = stored_i(x - c_i), periodic.  x in [0,nx), y in [0,ny), z in [0,nz).
template <class L, class C>
__device__ __forceinline__ void gather(const typename C::T* __restrict__ f, long long N, int nx, int ny,
                                       int nz, int x, int y, int z, float (&g)[L::Q]) {
  int xs[7], ys[7], zs[7];
#pragma unroll
  for (int d = -3; d <= 3; ++d) {
    xs[d + 3] = wrap1(x - d, nx);
    ys[d + 3] = wrap1(y - d, ny) * nx;
    if constexpr (L::D == 3) zs[d + 3] = wrap1(z - d, nz) * nx * ny;
  }
  static_for<L::Q>([&](auto I) {
    constexpr int i = I;
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    int off = ys[cy + 3] + xs[cx + 3];
    if constexpr (L::D == 3) off += zs[cz + 3];
    g[i] = C::ld(f + HLBM_IDX((size_t)i * (size_t)N + off, (long long)L::Q * N, DBG_GATHER));
  });
}

// ----------------------------------------------------------------- moments
// Moments of Eq. 4.5 in local-deviation form.  All g_i of a node are close to
// its density deviation dr = rho - rho0, which can be O(1) (liquid-gas), while
// velocity and temperature live in the differences.  So the sums run over
// differences of nearly equal numbers (exact in floating point):
//   d_i = g_i - g_0 (written back into g, d_0 = 0), acc = sum_{i>=1} w_i d_i,
//   dr = g_0 + acc,  J = sum_i w_i c_i d_i (= sum_i c_i f^_i),
//   Pih = sum_i w_i |c_i|^2 (g_i - dr) = sum_{i>=1} w_i |c_i|^2 d_i - D c0^2 acc
//       (= sum_i |c_i|^2 f^_i - rho D c0^2).
// Opposite pairs share the sum and difference of their d.
//
// dr_l is the rounding error of dr = g_0 + acc (Knuth's two-sum).  That error
// would reach all Q post-collision values of the node alike, i.e. act as a
// density error, which the pseudopotential force amplifies at a liquid-gas
// interface; with that force the collision adds dr_l back with the small
// terms and psi takes the density as rho0 + dr + dr_l.
template <class V>
__device__ __forceinline__ V two_sum_err(V a, V b, V s) {
  const V bb = vsub(s, a);
  return vadd(vsub(a, vsub(s, bb)), vsub(b, bb));
}

template <class L, class V>
__device__ __forceinline__ void moments_h(V (&g)[L::Q], V& dr, V& dr_l, V& acc, V (&J)[3], V& Pih) {
  const V g0 = g[0];
  V a = splat<V>(0.f), p = splat<V>(0.f);
  J[0] = J[1] = J[2] = splat<V>(0.f);
  static_for<L::NPAIR>([&](auto P) {
    constexpr int i = 2 * P + 1, j = 2 * P + 2;
    const V di = vsub(g[i], g0), dj = vsub(g[j], g0);
    g[i] = di;
    g[j] = dj;
    const V s = vadd(di, dj), d = vsub(di, dj);
    a = vfma(splat<V>((float)L::w(i)), s, a);
    p = vfma(splat<V>((float)(L::w(i) * L::norm2(i))), s, p);
    static_for<L::D>([&](auto A) {
      constexpr int ax = A;
      if constexpr (L::c(i, ax) != 0) J[ax] = vfma(splat<V>((float)(L::w(i) * L::c(i, ax))), d, J[ax]);
    });
  });
  g[0] = splat<V>(0.f);
  acc = a;
  dr = vadd(g0, a);
  dr_l = two_sum_err(g0, a, dr);
  Pih = vfma(splat<V>(-(float)(L::D * L::cs2)), a, p);
}

template <class L, class V>
__device__ __forceinline__ void moments_h(V (&g)[L::Q], V& dr, V& acc, V (&J)[3], V& Pih) {
  V dr_l;
  moments_h<L>(g, dr, dr_l, acc, J, Pih);
}

// dr and dr_l alone, same summation (g is not modified).
template <class L, class V>
__device__ __forceinline__ V density_h(const V (&g)[L::Q], V& dr_l) {
  const V g0 = g[0];
  V a = splat<V>(0.f);
  static_for<L::NPAIR>([&](auto P) {
    constexpr int i = 2 * P + 1, j = 2 * P + 2;
    a = vfma(splat<V>((float)L::w(i)), vadd(vsub(g[i], g0), vsub(g[j], g0)), a);
  });
  const V dr = vadd(g0, a);
  dr_l = two_sum_err(g0, a, dr);
  return dr;
}

// ---------------------------------------------------------- pseudopotential
// psi = sqrt(2 (p_EOS - rho c0^2) / (G c0^2)), G = -1, theta = 1 (Eq. 3.8).
// Written as psi^2 = 2 rho + k1 rho^2 - k2 rho Z(kb rho), the three terms
// cancel to a few times less than the largest (and p_EOS - rho c0^2 before
// them), and F^SC differences psi between neighbours, so a plain FP32
// evaluation leaves psi noise of several ulp that F^SC turns into force noise
// at the interface.  psi^2 is therefore formed in float-float arithmetic
// (Dekker/Knuth error-free sum and FMA product) from the FP32 density, and
// the square root takes one Newton correction against the float-float
// residual: psi is within about half an ulp of the value of the formula at
// the node's density.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff ff_norm(float h, float l) {
  const float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const float s = __fadd_rn(x.h, y.h);
  const float bb = __fsub_rn(s, x.h);
  const float e = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, bb)), __fsub_rn(y.h, bb));
  return ff_norm(s, __fadd_rn(e, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.h, -x.l}; }
__device__ __forceinline__ ff ff_mul_f(ff x, float y) {
  const float p = __fmul_rn(x.h, y);
  return ff_norm(p, fmaf(x.l, y, fmaf(x.h, y, -p)));
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.h, y.h);
  return ff_norm(p, fmaf(x.h, y.l, fmaf(x.l, y.h, fmaf(x.h, y.h, -p))));
}
// 1 / y: the hardware approximation refined by one Newton-Raphson step
// (e = 1 - y r0, r1 = r0 + r0 e); relative error about 2^-23 for normal y.
__device__ __forceinline__ float rcp_nr(float y) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(y));
  return fmaf(r0, fmaf(-y, r0, 1.f), r0);
}
// x / y: a quotient within a few ulp, its exact remainder r = x - q y (error-
// free product), and the correction r / y; the float-float result does not
// depend on q being correctly rounded.
__device__ __forceinline__ ff ff_div(ff x, ff y) {
  const float inv = rcp_nr(y.h);
  const float q = __fmul_rn(x.h, inv);
  const ff r = ff_add(x, ff_neg(ff_mul_f(y, q)));
  return ff_norm(q, __fmul_rn(r.h, inv));
}

// The density enters as rho0 + dr + dr_l, formed exactly as a float-float.
template <class L>
__device__ __forceinline__ float psi_of(const StepArgs& a, float dr, float dr_l) {
  const float rh = __fadd_rn(a.rho0, dr);
  const float bb = __fsub_rn(rh, a.rho0);
  const float rl = __fadd_rn(__fsub_rn(a.rho0, __fsub_rn(rh, bb)), __fsub_rn(dr, bb));
  const ff rho = ff_norm(rh, __fadd_rn(rl, dr_l));
  const ff k1{a.psi_k1[0], a.psi_k1[1]}, k2{a.psi_k2[0], a.psi_k2[1]};
  const ff e = ff_mul(ff{a.psi_kb[0], a.psi_kb[1]}, rho);
  const ff one{1.f, 0.f};
  const ff om = ff_add(one, ff_neg(e));
  ff z;
  if (a.eos == 0) {
    z = ff_div(rho, om);                                            // rho / (1 - e)
  } else {
    const ff e2 = ff_mul(e, e);
    const ff num = ff_add(ff_add(ff_add(one, e), e2), ff_neg(ff_mul(e2, e)));
    z = ff_div(ff_mul(num, rho), ff_mul(ff_mul(om, om), om));       // rho Z(e)
  }
  const ff quad = ff_mul(ff_add(ff{2.f, 0.f}, ff_mul(k1, rho)), rho);   // 2 rho + k1 rho^2
  const ff s = ff_add(quad, ff_neg(ff_mul(k2, z)));
  if (!(s.h > 0.f)) return 0.f;
  // square root of s.h + s.l: y ~ 1/sqrt(s.h) from the hardware, h = s.h y
  // (relative error about 2^-22), then one Newton step against the float-float
  // residual (Karp-Markstein): h + (s - h^2) y / 2
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(s.h));
  const float h = __fmul_rn(s.h, y);
  const float r = __fadd_rn(fmaf(-h, h, s.h), s.l);
  return fmaf(r, 0.5f * y, h);
}

// ---------------------------------------------------------- body acceleration
template <int D>
__device__ __forceinline__ void accel(const StepArgs& a, int node, int y, float (&g)[3]) {
  g[0] = g[1] = g[2] = 0.f;
  if (a.force_mode == FORCE_UNIFORM) {
#pragma unroll
    for (int d = 0; d < D; ++d) g[d] = a.g[d];
  } else if (a.force_mode == FORCE_FIELD) {
#pragma unroll
    for (int d = 0; d < D; ++d) g[d] = __ldg(a.gfield + (size_t)d * (size_t)a.N + node);
  } else if (a.force_mode == FORCE_PROFILE_Y) {
#pragma unroll
    for (int d = 0; d < D; ++d) g[d] = __ldg(a.gfield + (size_t)d * a.ny + y);
  }
}

// ------------------------------------------------------ collision polynomial
// Per-node inputs in xi units: u, F divided by c0; hG = rho theta (1 - 1/Pr)
// c0 grad theta; sigma the trace coefficient of P_i.
template <class V>
struct NodeSrcT {
  V dr, rho, tb;
  V u[3], F[3], hG[3];
  V sigma;
};
using NodeSrc = NodeSrcT<float>;

// Hermite moments of a unit-variance-plus-tb Gaussian, m_0..m_4.
template <class V>
__device__ __forceinline__ void gauss_moments(V u, V tb, V (&m)[5]) {
  const V u2 = vmul(u, u);
  m[0] = splat<V>(1.f);
  m[1] = u;
  m[2] = vadd(u2, tb);
  m[3] = vmul(u, vfma(splat<V>(3.f), tb, u2));
  m[4] = vfma(u2, vfma(splat<V>(6.f), tb, u2), vmul(splat<V>(3.f), vmul(tb, tb)));
}

// K[m] (monomial m of mono2) for D2Q37: 4th-order equilibrium + sources.
template <class L, class V>
__device__ __forceinline__ void poly2(const NodeSrcT<V>& s, float omega, float beta, V (&K)[15]) {
  V mx[5], my[5];
  gauss_moments(s.u[0], s.tb, mx);
  gauss_moments(s.u[1], s.tb, my);
#pragma unroll
  for (int m = 0; m < 15; ++m) K[m] = splat<V>(0.f);
  static_for<5>([&](auto A) {
    static_for<5>([&](auto Bq) {
      constexpr int a = A, b = Bq;
      if constexpr (a + b <= L::FEQ_ORDER) {
        const V eq = (a == 0 && b == 0) ? s.dr : vmul(s.rho, vmul(mx[a], my[b]));
        V src = splat<V>(0.f);
        if constexpr (a + b >= 1 && a + b <= 3) {
          if constexpr (a > 0)
            src = vfma(vmul(s.F[0], splat<V>((float)a)), vmul(mx[a > 0 ? a - 1 : 0], my[b]), src);
          if constexpr (b > 0)
            src = vfma(vmul(s.F[1], splat<V>((float)b)), vmul(mx[a], my[b > 0 ? b - 1 : 0]), src);
        }
        if constexpr ((a == 2 && b == 0) || (a == 0 && b == 2)) src = vadd(src, s.sigma);
        if constexpr (a == 3 && b == 0) src = vfma(splat<V>(3.f), s.hG[0], src);
        if constexpr (a == 2 && b == 1) src = vadd(src, s.hG[1]);
        if constexpr (a == 1 && b == 2) src = vadd(src, s.hG[0]);
        if constexpr (a == 0 && b == 3) src = vfma(splat<V>(3.f), s.hG[1], src);
        const V Bab = vfma(splat<V>(omega), eq, vmul(splat<V>(beta), src));
        // He_a(cx / c0) He_b(cy / c0) / (a! b!) -> monomials c_x^p c_y^q
        static_for<5>([&](auto Pp) {
          static_for<5>([&](auto Qq) {
            constexpr int p = Pp, q = Qq;
            if constexpr (p <= a && q <= b && he(a, p) != 0 && he(b, q) != 0) {
              constexpr float cf = (float)((double)(he(a, p) * he(b, q)) /
                                           (fact_d(a) * fact_d(b) * ipow_d(L::c0, p + q)));
              constexpr int m = mono2_index(p, q);
              K[m] = vfma(splat<V>(cf), Bab, K[m]);
            }
          });
        });
      }
    });
  });
}

// K[m] (monomial m of mono3) for D3Q39: 3rd-order equilibrium + body force.
template <class L, class V>
__device__ __forceinline__ void poly3(const NodeSrcT<V>& s, float omega, float beta, V (&K)[20]) {
  V mx[5], my[5], mz[5];
  gauss_moments(s.u[0], s.tb, mx);
  gauss_moments(s.u[1], s.tb, my);
  gauss_moments(s.u[2], s.tb, mz);
#pragma unroll
  for (int m = 0; m < 20; ++m) K[m] = splat<V>(0.f);
  static_for<4>([&](auto A) {
    static_for<4>([&](auto Bq) {
      static_for<4>([&](auto Cr) {
        constexpr int a = A, b = Bq, c = Cr;
        if constexpr (a + b + c <= L::FEQ_ORDER) {
          const V eq = (a == 0 && b == 0 && c == 0) ? s.dr : vmul(s.rho, vmul(mx[a], vmul(my[b], mz[c])));
          V src = splat<V>(0.f);
          if constexpr (a + b + c >= 1) {
            if constexpr (a > 0)
              src = vfma(vmul(s.F[0], splat<V>((float)a)), vmul(mx[a > 0 ? a - 1 : 0], vmul(my[b], mz[c])), src);
            if constexpr (b > 0)
              src = vfma(vmul(s.F[1], splat<V>((float)b)), vmul(mx[a], vmul(my[b > 0 ? b - 1 : 0], mz[c])), src);
            if constexpr (c > 0)
              src = vfma(vmul(s.F[2], splat<V>((float)c)), vmul(mx[a], vmul(my[b], mz[c > 0 ? c - 1 : 0])), src);
          }
          if constexpr ((a == 2 && b == 0 && c == 0) || (a == 0 && b == 2 && c == 0) ||
                        (a == 0 && b == 0 && c == 2))
            src = vadd(src, s.sigma);
          // [delta hG] components: (3,0,0) -> 3 hGx, (2,1,0) -> hGy, (1,2,0) -> hGx, ...
          if constexpr (a + b + c == 3) {
            if constexpr (a == 3) src = vfma(splat<V>(3.f), s.hG[0], src);
            if constexpr (b == 3) src = vfma(splat<V>(3.f), s.hG[1], src);
            if constexpr (c == 3) src = vfma(splat<V>(3.f), s.hG[2], src);
            if constexpr (a == 2 && b == 1) src = vadd(src, s.hG[1]);
            if constexpr (a == 2 && c == 1) src = vadd(src, s.hG[2]);
            if constexpr (b == 2 && a == 1) src = vadd(src, s.hG[0]);
            if constexpr (b == 2 && c == 1) src = vadd(src, s.hG[2]);
            if constexpr (c == 2 && a == 1) src = vadd(src, s.hG[0]);
            if constexpr (c == 2 && b == 1) src = vadd(src, s.hG[1]);
          }
          const V Babc = vfma(splat<V>(omega), eq, vmul(splat<V>(beta), src));
          static_for<4>([&](auto Pp) {
            static_for<4>([&](auto Qq) {
              static_for<4>([&](auto Rr) {
                constexpr int p = Pp, q = Qq, r = Rr;
                if constexpr (p <= a && q <= b && r <= c && he(a, p) != 0 && he(b, q) != 0 && he(c, r) != 0) {
                  constexpr float cf = (float)((double)(he(a, p) * he(b, q) * he(c, r)) /
                                               (fact_d(a) * fact_d(b) * fact_d(c) * ipow_d(L::c0, p + q + r)));
                  constexpr int m = mono3_index(p, q, r);
                  K[m] = vfma(splat<V>(cf), Babc, K[m]);
                }
              });
            });
          });
        }
      });
    });
  });
}

// Evaluates P(c_i) for all velocities and applies g*_i = (1 - omega) g_i + P(c_i)
// in place; the even part of P is shared by each opposite pair.
template <class L, int NM>
__device__ __forceinline__ void apply_poly(float (&g)[L::Q], const float (&K)[NM], float om1) {
  g[0] = fmaf(om1, g[0], K[0]);
  static_for<L::NPAIR>([&](auto P) {
    constexpr int i = 2 * P + 1, j = 2 * P + 2;
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    float E = K[0], O = 0.f;
    static_for<NM>([&](auto M) {
      constexpr int m = M;
      if constexpr (m > 0) {
        constexpr int px = (NM == 15) ? mono2(m, 0) : mono3(m, 0);
        constexpr int py = (NM == 15) ? mono2(m, 1) : mono3(m, 1);
        constexpr int pz = (NM == 15) ? 0 : mono3(m, 2);
        constexpr int mv = ipow_i(cx, px) * ipow_i(cy, py) * ipow_i(cz, pz);
        if constexpr (mv != 0) {
          if constexpr ((px + py + pz) % 2 == 0) {
            if constexpr (mv == 1) E += K[m];
            else E = fmaf((float)mv, K[m], E);
          } else {
            if constexpr (mv == 1) O += K[m];
            else if constexpr (mv == -1) O -= K[m];
            else O = fmaf((float)mv, K[m], O);
          }
        }
      }
    });
    g[i] = fmaf(om1, g[i], E + O);
    g[j] = fmaf(om1, g[j], E - O);
  });
}


// Collision in local-deviation form.  With d_i = g_i - g_0 and dr, acc from
// moments_h, and K computed with B_00 = 0 and K_00 reduced by (1 - omega) acc
// (and increased by dr_l with the pseudopotential force),
//   g*_i = dr + [(1 - omega) d_i + P(c_i)]
// equals (1 - omega) g_i + P_full(c_i) (P_full with B_00 = omega (dr + dr_l)),
// but only small numbers pass through the arithmetic before the final add of dr.
//
// On D2Q37 the polynomial is evaluated per symmetry class: for a = |c_x|,
// b = |c_y| and signs s_x, s_y,
//   P(c) = S(a, b) + s_x s_y T(a, b) + s_x OA(a, b) + s_y OB(a, b),
//   S  = K00 + a^2 K20 + b^2 K02 + a^4 K40 + a^2 b^2 K22 + b^4 K04,
//   T  = a b K11 + a^3 b K31 + a b^3 K13,
//   OA = a K10 + a^3 K30 + a b^2 K12,   OB = b K01 + a^2 b K21 + b^3 K03,
// so S, T, OA, OB are formed once for the (up to) four velocities of a class
// and each opposite pair shares its even part.
template <class V>
__device__ __forceinline__ V vfma_c(float c, V x, V acc) {
  if (c == 1.f) return vadd(acc, x);
  return vfma(splat<V>(c), x, acc);
}

template <class L, class V>
__device__ __forceinline__ void apply_poly_h2(V (&g)[L::Q], const V (&K)[15], V o1, V dr) {
  constexpr int M00 = mono2_index(0, 0), M10 = mono2_index(1, 0), M01 = mono2_index(0, 1);
  constexpr int M20 = mono2_index(2, 0), M11 = mono2_index(1, 1), M02 = mono2_index(0, 2);
  constexpr int M30 = mono2_index(3, 0), M21 = mono2_index(2, 1), M12 = mono2_index(1, 2), M03 = mono2_index(0, 3);
  constexpr int M40 = mono2_index(4, 0), M31 = mono2_index(3, 1), M22 = mono2_index(2, 2), M13 = mono2_index(1, 3);
  constexpr int M04 = mono2_index(0, 4);
  g[0] = vadd(dr, K[M00]);
  // classes (a, b) = (|c_x|, |c_y|) of the pair representatives
  static_for<4>([&](auto Aa) {
    static_for<4>([&](auto Bb) {
      constexpr int a = Aa, b = Bb;
      constexpr bool used = [] {
        for (int p = 0; p < L::NPAIR; ++p) {
          const int cx = L::c(2 * p + 1, 0), cy = L::c(2 * p + 1, 1);
          if ((cx < 0 ? -cx : cx) == a && (cy < 0 ? -cy : cy) == b) return true;
        }
        return false;
      }();
      if constexpr (used && (a + b) > 0) {
        constexpr float a2 = (float)(a * a), b2 = (float)(b * b), ab = (float)(a * b);
        V S = K[M00];
        if constexpr (a > 0) S = vfma_c(a2 * a2, K[M40], vfma_c(a2, K[M20], S));
        if constexpr (b > 0) S = vfma_c(b2 * b2, K[M04], vfma_c(b2, K[M02], S));
        if constexpr (a > 0 && b > 0) S = vfma_c(a2 * b2, K[M22], S);
        V T = splat<V>(0.f), OA = splat<V>(0.f), OB = splat<V>(0.f);
        if constexpr (a > 0 && b > 0)
          T = vmul(splat<V>(ab), vfma_c(b2, K[M13], vfma_c(a2, K[M31], K[M11])));
        if constexpr (a > 0) {
          V t = vfma_c(a2, K[M30], K[M10]);
          if constexpr (b > 0) t = vfma_c(b2, K[M12], t);
          OA = (a == 1) ? t : vmul(splat<V>((float)a), t);
        }
        if constexpr (b > 0) {
          V t = vfma_c(b2, K[M03], K[M01]);
          if constexpr (a > 0) t = vfma_c(a2, K[M21], t);
          OB = (b == 1) ? t : vmul(splat<V>((float)b), t);
        }
        static_for<L::NPAIR>([&](auto P) {
          constexpr int i = 2 * P + 1, j = 2 * P + 2;
          constexpr int cx = L::c(i, 0), cy = L::c(i, 1);
          if constexpr ((cx < 0 ? -cx : cx) == a && (cy < 0 ? -cy : cy) == b) {
            constexpr int sx = cx > 0 ? 1 : (cx < 0 ? -1 : 0), sy = cy > 0 ? 1 : (cy < 0 ? -1 : 0);
            V E, O;   // even part, odd part at c_i
            if constexpr (sx * sy > 0) E = vadd(S, T);
            else if constexpr (sx * sy < 0) E = vsub(S, T);
            else E = S;
            if constexpr (sy == 0) O = OA;
            else if constexpr (sx == 0) O = OB;
            else if constexpr (sx == sy) O = vadd(OA, OB);
            else O = vsub(OA, OB);
            constexpr bool flip = (sx < 0) || (sx == 0 && sy < 0);   // O above is -(odd part at c_i)
            if constexpr (!flip) {
              g[i] = vadd(dr, vfma(o1, g[i], vadd(E, O)));
              g[j] = vadd(dr, vfma(o1, g[j], vsub(E, O)));
            } else {
              g[i] = vadd(dr, vfma(o1, g[i], vsub(E, O)));
              g[j] = vadd(dr, vfma(o1, g[j], vadd(E, O)));
            }
          }
        });
      }
    });
  });
}

template <class L, int NM, class V>
__device__ __forceinline__ void apply_poly_h(V (&g)[L::Q], const V (&K)[NM], float om1, V dr) {
  const V o1 = splat<V>(om1);
  if constexpr (NM == 15 && L::D == 2) {
    apply_poly_h2<L>(g, K, o1, dr);
  } else {
  g[0] = vadd(dr, K[0]);
  static_for<L::NPAIR>([&](auto P) {
    constexpr int i = 2 * P + 1, j = 2 * P + 2;
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    V E = K[0], O = splat<V>(0.f);
    bool have_o = false;
    static_for<NM>([&](auto M) {
      constexpr int m = M;
      if constexpr (m > 0) {
        constexpr int px = (NM == 15) ? mono2(m, 0) : mono3(m, 0);
        constexpr int py = (NM == 15) ? mono2(m, 1) : mono3(m, 1);
        constexpr int pz = (NM == 15) ? 0 : mono3(m, 2);
        constexpr int mv = ipow_i(cx, px) * ipow_i(cy, py) * ipow_i(cz, pz);
        if constexpr (mv != 0) {
          if constexpr ((px + py + pz) % 2 == 0) {
            if constexpr (mv == 1) E = vadd(E, K[m]);
            else E = vfma(splat<V>((float)mv), K[m], E);
          } else {
            if (!have_o) {
              O = (mv == 1) ? K[m] : vmul(splat<V>((float)mv), K[m]);
              have_o = true;
            } else if constexpr (mv == 1) {
              O = vadd(O, K[m]);
            } else if constexpr (mv == -1) {
              O = vsub(O, K[m]);
            } else {
              O = vfma(splat<V>((float)mv), K[m], O);
            }
          }
        }
      }
    });
    g[i] = vadd(dr, vfma(o1, g[i], vadd(E, O)));
    g[j] = vadd(dr, vfma(o1, g[j], vsub(E, O)));
  });
  }
}

}  // namespace hlbm
