// hlbm_population_sums_noalloc: FP64 domain totals of a population buffer
// without any device allocation.
//
// Who needs it: callers that must not allocate device memory once they are
// running -- for instance a host application whose device memory is handed
// out up front by another framework's allocator under a fixed budget, or an
// embedded service that forbids allocation after initialisation.  hlbm_diag
// keeps its block partials in the context's workspace; this entry point
// keeps them in a statically sized device array owned by the library, so the
// caller only passes the population buffer and a host output array.
//
// Scratch: kSumMaxBlocks x 8 doubles of block partials plus 8 result slots
// (1 MiB + 64 bytes), held by every GPU that loads the library until the
// process exits.  One CTA reduces kSumNodesPerBlock nodes, so a call accepts
// at most kSumMaxBlocks * kSumNodesPerBlock = 33,554,432 nodes.  Each call
// overwrites the partials and result slots it uses (nothing has to start at
// zero); all calls share the array, so calls whose kernels overlap on the GPU
// (different streams, or different host threads) race and must be avoided.
#include <atomic>
#include <cstdio>

#include "hlbm.h"
#include "step_common.cuh"

namespace hlbm {
namespace {

constexpr int kSumThreads = 256;
constexpr int kSumNodesPerThread = 8;
constexpr int kSumNodesPerBlock = kSumThreads * kSumNodesPerThread;
constexpr int kSumMaxBlocks = 16384;
constexpr long long kSumMaxNodes = (long long)kSumMaxBlocks * kSumNodesPerBlock;

static __device__ __align__(256) double g_sum_scratch[kSumMaxBlocks * 8 + 8];

// host-side copies of the scratch's device address, one per device
constexpr int kMaxDevices = 64;
std::atomic<double*> g_scratch_ptr[kMaxDevices];   // per-device address of g_sum_scratch (looked up once)

// Block b sums nodes [b * 2048, (b + 1) * 2048): per node the FP32 moments of
// the stored deviations g_i = (f_i - w_i rho0) / w_i, accumulated in FP64.
template <class L, int ST>
__global__ void __launch_bounds__(kSumThreads) sums_partial_kernel(const void* __restrict__ pop, long long N,
                                                                   double* __restrict__ scratch) {
  using C = Codec<ST>;
  using T = typename C::T;
  const T* __restrict__ f = static_cast<const T*>(pop);
  double v[5] = {0, 0, 0, 0, 0};
  const long long base = (long long)blockIdx.x * kSumNodesPerBlock + threadIdx.x;
#pragma unroll 1
  for (int k = 0; k < kSumNodesPerThread; ++k) {
    const long long n = base + (long long)k * kSumThreads;
    if (n >= N) break;
    float dr = 0.f, j[3] = {0.f, 0.f, 0.f}, pi = 0.f;
    static_for<L::Q>([&](auto I) {
      constexpr int i = I;
      const float gi = C::ld(f + (size_t)i * (size_t)N + n);
      dr = fmaf((float)L::w(i), gi, dr);
      pi = fmaf((float)(L::w(i) * L::norm2(i)), gi, pi);
      static_for<L::D>([&](auto A) {
        constexpr int a = A;
        if constexpr (L::c(i, a) != 0) j[a] = fmaf((float)(L::w(i) * L::c(i, a)), gi, j[a]);
      });
    });
    v[0] += dr;
    v[1] += j[0];
    v[2] += j[1];
    v[3] += j[2];
    v[4] += pi;
  }
  __shared__ double red[kSumThreads / 32][5];
#pragma unroll
  for (int k = 0; k < 5; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 5; ++k) red[threadIdx.x >> 5][k] = v[k];
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < kSumThreads / 32; ++w) s += red[w][threadIdx.x];
    scratch[(size_t)blockIdx.x * 8 + threadIdx.x] = s;
  }
}

// One CTA: result slots scratch[kSumMaxBlocks * 8 + k] = sum over blocks.
__global__ void __launch_bounds__(kSumThreads) sums_final_kernel(double* __restrict__ scratch, int blocks) {
  __shared__ double red[kSumThreads / 32][5];
  double v[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < blocks; b += kSumThreads)
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += scratch[(size_t)b * 8 + k];
#pragma unroll
  for (int k = 0; k < 5; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 5; ++k) red[threadIdx.x >> 5][k] = v[k];
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < kSumThreads / 32; ++w) s += red[w][threadIdx.x];
    scratch[(size_t)kSumMaxBlocks * 8 + threadIdx.x] = s;
  }
}

template <class L>
cudaError_t launch_partial(int storage, const void* pop, long long N, int blocks, double* scratch, cudaStream_t s) {
  switch (storage) {
    case ST_F32: sums_partial_kernel<L, ST_F32><<<blocks, kSumThreads, 0, s>>>(pop, N, scratch); break;
    case ST_F16: sums_partial_kernel<L, ST_F16><<<blocks, kSumThreads, 0, s>>>(pop, N, scratch); break;
    default: sums_partial_kernel<L, ST_BF16><<<blocks, kSumThreads, 0, s>>>(pop, N, scratch); break;
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace hlbm

using namespace hlbm;

extern "C" hlbm_status hlbm_population_sums_noalloc(int lattice, long long nodes, int storage, double rho0,
                                                    const void* populations, void* cuda_stream, double* out) {
  if (lattice != HLBM_D2Q37 && lattice != HLBM_D3Q39) return HLBM_EINVAL;
  if (storage < HLBM_F32 || storage > HLBM_BF16 || !populations || !out || !(rho0 > 0.0)) return HLBM_EINVAL;
  if (nodes <= 0 || nodes > kSumMaxNodes) {
    std::fprintf(stderr,
                 "hlbm_population_sums_noalloc: %lld nodes; this entry point uses a fixed device scratch "
                 "array and accepts 1 to %lld nodes\n",
                 nodes, kSumMaxNodes);
    return HLBM_EINVAL;
  }
  // per-device set-up: the host-side address of the static scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HLBM_ECUDA;
  double* scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sum_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HLBM_ECUDA;
    }
    scratch = static_cast<double*>(p);
    g_scratch_ptr[dev].store(scratch, std::memory_order_release);   // concurrent first calls store the same address
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int blocks = (int)((nodes + kSumNodesPerBlock - 1) / kSumNodesPerBlock);
  cudaError_t e = lattice == HLBM_D2Q37 ? launch_partial<D2Q37>(storage, populations, nodes, blocks, scratch, s)
                                        : launch_partial<D3Q39>(storage, populations, nodes, blocks, scratch, s);
  if (e == cudaSuccess) {
    sums_final_kernel<<<1, kSumThreads, 0, s>>>(scratch, blocks);
    e = cudaGetLastError();
  }
  double r[5];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r, scratch + (size_t)kSumMaxBlocks * 8, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return HLBM_ECUDA;
  const int D = lattice == HLBM_D2Q37 ? 2 : 3;
  const double cs2 = lattice == HLBM_D2Q37 ? D2Q37::cs2 : D3Q39::cs2;
  const double Nn = (double)nodes;
  out[0] = Nn * rho0 + r[0];
  for (int a = 0; a < D; ++a) out[1 + a] = r[1 + a];
  out[1 + D] = 0.5 * (Nn * rho0 * D * cs2 + r[4]);
  return HLBM_OK;
}
