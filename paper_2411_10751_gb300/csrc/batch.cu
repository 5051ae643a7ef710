// Batched step: many independent periodic D2Q37 domains (any sizes, sources
// and parameters) advanced by ONE persistent launch per time step, replayed
// from a CUDA graph.  Resident CTAs (all of the same shape: 128 threads,
// shared memory for the largest tile) take (domain, tile) items from a global
// work list in order through a device counter, dispatch on the domain's
// source kind and run exactly the single-domain kernel's tile code
// (process_tile): 32 x 8 tiles with two nodes per thread for the body-force
// and thermal kinds, 32 x 4 tiles with one node per thread for the
// pseudopotential kind (its frame of psi values is three nodes wide; a 4-row
// tile keeps its staging at 67 KB FP32, so three CTAs fit on an SM whatever
// kind they run).  The pseudopotential tiles, the slowest, come first in the
// work list, so the launch ends on short tiles.  Each domain's step arguments
// (for both buffer parities) and its TMA tensor maps are read from device
// memory.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "hlbm.h"
#include "internal.h"
#include "step2d.cuh"

namespace hlbm {
namespace {

// tile rows and nodes per thread of a kind (256 threads for every kind)
template <int KIND>
constexpr int kind_rows() {
  return 8;
}
template <int KIND>
constexpr int kind_npt() {
  return 1;
}
constexpr int kThreads = 256;
int kind_rows_rt(int) { return 8; }

template <int ST>
constexpr int batch_smem() {
  constexpr int a = Cfg2<ST, KIND_LOCAL, false, 8>::SMEM, b = Cfg2<ST, KIND_THERMAL, false, 8>::SMEM,
                c = Cfg2<ST, KIND_SC, false, 8>::SMEM;
  return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

struct alignas(64) BatchDomain {
  CUtensorMap tmap[2];    // input maps of buffer 0 / 1 (box of the domain's kind)
  StepArgs args[2];       // args[p]: reads buffer p, writes buffer p ^ 1
  int kind;
  int tiles_x;
  int cur;                // buffer holding the state at the start of the batch call
  int has_map;
};

template <int ST, int KIND>
__device__ __forceinline__ bool batch_tile(const BatchDomain& dom, const StepArgs& a, unsigned char* smem, int x0,
                                           int y0, int par, uint32_t& phase) {
  constexpr int BY = kind_rows<KIND>();
  using Cf = Cfg2<ST, KIND, false, BY>;
  typename Cf::T* sp = reinterpret_cast<typename Cf::T*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + batch_smem<ST>() - 128);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (dom.has_map && tile_boxed<Cf>(a, x0, y0) && ((smem_u32(smem) & 127u) == 0)) {
    if (tid == 0) {
      fence_proxy_async_smem();   // the previous tile's generic accesses of the buffer come first
      issue_tile<Cf>(sp, &dom.tmap[par], bar, x0, y0, a.debug_skip_tma, a.nx, a.ny);
    }
    const bool ok = mbar_wait_bounded(bar, phase, a.wait_ns);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      // copies did not complete: report, give in-flight copies a second
      // bounded wait, and stop this CTA (the batch is then in an error state)
      if (tid == 0) atomicExch(a.status, (int)5 /* HLBM_ETIMEOUT */);
      mbar_wait_bounded(bar, phase ^ 1u, a.wait_ns);
      __syncthreads();
      return false;
    }
  } else {
    fill_tile_wrapped<Cf, kThreads>(a, a.fin, sp, x0, y0, tid);
    __syncthreads();
  }
  process_tile<ST, KIND, false, BY, kind_npt<KIND>(), false>(a, nullptr, smem, x0, y0, a.fout, [] {});
  return true;
}

// One step of every domain: CTAs take work-list items (T = nitems) through
// the counter; a launch of G CTAs takes exactly T + G values (each CTA ends
// on one value past the list), so the counter is never reset and the item is
// the value modulo T + G.
template <int ST>
__global__ void __launch_bounds__(kThreads, 2)
    batch_step_kernel(const BatchDomain* __restrict__ doms, const int2* __restrict__ items, int nitems, int flip,
                      unsigned long long* ctr) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + batch_smem<ST>() - 128);
  // thread 0 takes the counter one item ahead and keeps the raw value until
  // the next item starts, so the atomic's round trip overlaps a whole tile
  unsigned long long nxt_raw = 0;
  const unsigned long long period = (unsigned long long)nitems + gridDim.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    nxt_raw = atomicAdd(ctr, 1ull);
  }
  uint32_t phase = 0;
  for (;;) {
    if (tid == 0) {
      const int gi = (int)(nxt_raw % period);
      s_item = gi;
      if (gi < nitems) nxt_raw = atomicAdd(ctr, 1ull);
    }
    __syncthreads();
    const int gi = s_item;
    if (gi >= nitems) break;
    const int2 it = items[gi];                   // (domain, tile)
    const BatchDomain& dom = doms[it.x];
    const int par = dom.cur ^ flip;
    const StepArgs& a = dom.args[par];
    const int t = it.y;
    const int ty = t / dom.tiles_x;
    const int x0 = (t - ty * dom.tiles_x) * 32;
    bool ok;
    if (dom.kind == KIND_SC) ok = batch_tile<ST, KIND_SC>(dom, a, smem, x0, ty * kind_rows<KIND_SC>(), par, phase);
    else if (dom.kind == KIND_THERMAL) ok = batch_tile<ST, KIND_THERMAL>(dom, a, smem, x0, ty * 8, par, phase);
    else ok = batch_tile<ST, KIND_LOCAL>(dom, a, smem, x0, ty * 8, par, phase);
    if (!ok) return;
    __syncthreads();   // the staging buffer and s_item are reused
  }
}

template <int ST>
int batch_grid(int nitems) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step_kernel<ST>, kThreads, batch_smem<ST>());
  if (per_sm < 1) per_sm = 1;
  return std::max(1, std::min(nitems, sms * per_sm));
}

template <int ST>
cudaError_t launch_batch(const BatchDomain* doms, const int2* items, int nitems, int grid, int flip,
                         unsigned long long* ctr, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  batch_step_kernel<ST><<<grid, dim3(32, kThreads / 32, 1), batch_smem<ST>(), s>>>(doms, items, nitems, flip, ctr);
  return cudaGetLastError();
}

template <int ST>
cudaError_t configure_batch() {
  return cudaFuncSetAttribute(batch_step_kernel<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem<ST>());
}

template <int ST>
void box_for_kind(int kind, int& wb, int& hb) {
  if (kind == KIND_SC) box_of<ST, KIND_SC, false, 8>(wb, hb);
  else if (kind == KIND_THERMAL) box_of<ST, KIND_THERMAL, false, 8>(wb, hb);
  else box_of<ST, KIND_LOCAL, false, 8>(wb, hb);
}

}  // namespace

// Host-side helpers the C ABI (api.cu) uses; the batch owns the device arrays.
struct BatchDevice {
  BatchDomain* doms = nullptr;
  int2* items = nullptr;
  unsigned long long* ctr = nullptr;   // the persistent launch's item counter (zeroed once)
  int nitems = 0;
};

cudaError_t batch_upload(const std::vector<BatchDomain>& host, const std::vector<int2>& items, BatchDevice& dev,
                         cudaStream_t s) {
  if (!dev.doms) {
    cudaError_t e = cudaMalloc(&dev.doms, host.size() * sizeof(BatchDomain));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&dev.items, items.size() * sizeof(int2));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&dev.ctr, sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(dev.ctr, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemcpyAsync(dev.doms, host.data(), host.size() * sizeof(BatchDomain), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev.items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
  dev.nitems = (int)items.size();
  return e;
}

}  // namespace hlbm

// ----------------------------------------------------------------- C ABI
using namespace hlbm;

struct hlbm_batch {
  std::vector<hlbm_ctx*> ctxs;
  int storage = 0;
  cudaStream_t stream = nullptr;
  std::vector<BatchDomain> host;
  std::vector<int2> items;        // (domain, tile), the pseudopotential kind's tiles first
  int grid = 0;                   // resident CTAs of the persistent launch
  BatchDevice dev;
  cudaGraphExec_t graph = nullptr;
  std::string msg;
};

// accessors of hlbm_ctx implemented in api.cu
namespace hlbm {
bool ctx_batchable(const hlbm_ctx* c, int* storage, int* kind, int* nx, int* ny);
StepArgs ctx_step_args(hlbm_ctx* c, int parity);
const CUtensorMap* ctx_tensor_map(hlbm_ctx* c, int buf, int wb, int hb);
int ctx_cur(const hlbm_ctx* c);
void ctx_advance(hlbm_ctx* c, int steps);
}  // namespace hlbm

extern "C" {

hlbm_status hlbm_batch_create(int n, hlbm_ctx* const* ctxs, hlbm_batch** out) {
  if (!out || n < 1 || !ctxs) return HLBM_EINVAL;
  *out = nullptr;
  int storage = -1;
  for (int k = 0; k < n; ++k) {
    int st, kind, nx, ny;
    if (!ctxs[k] || !ctx_batchable(ctxs[k], &st, &kind, &nx, &ny)) {
      std::fprintf(stderr, "hlbm_batch_create: context %d is not an initialised periodic D2Q37 context\n", k);
      return HLBM_EINVAL;
    }
    if (storage >= 0 && st != storage) {
      std::fprintf(stderr, "hlbm_batch_create: all contexts must share one storage type\n");
      return HLBM_EINVAL;
    }
    storage = st;
  }
  hlbm_batch* b = new (std::nothrow) hlbm_batch();
  if (!b) return HLBM_ENOMEM;
  b->ctxs.assign(ctxs, ctxs + n);
  b->storage = storage;
  if (cudaStreamCreate(&b->stream) != cudaSuccess) {
    delete b;
    return HLBM_ECUDA;
  }
  for (hlbm_ctx* c : b->ctxs) {
    hlbm_synchronize(c);
    hlbm_set_stream(c, b->stream);
  }
  cudaError_t e = storage == ST_F32 ? configure_batch<ST_F32>()
                  : storage == ST_F16 ? configure_batch<ST_F16>()
                                      : configure_batch<ST_BF16>();
  if (e != cudaSuccess) {
    hlbm_batch_destroy(b);
    return HLBM_ECUDA;
  }
  *out = b;
  return HLBM_OK;
}

static hlbm_status batch_refresh(hlbm_batch* b) {
  b->host.assign(b->ctxs.size(), BatchDomain{});
  b->items.clear();
  std::vector<int2> heavy, light;   // pseudopotential tiles (compute-bound) and the others (HBM-bound)
  for (int kind : {(int)KIND_SC, (int)KIND_THERMAL, (int)KIND_LOCAL}) {
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
      hlbm_ctx* c = b->ctxs[k];
      int st, dkind, nx, ny;
      ctx_batchable(c, &st, &dkind, &nx, &ny);
      if (dkind != kind) continue;
      BatchDomain& d = b->host[k];
      std::memset(&d, 0, sizeof(d));
      d.kind = dkind;
      d.tiles_x = (nx + 31) / 32;
      d.cur = ctx_cur(c);
      d.args[0] = ctx_step_args(c, 0);
      d.args[1] = ctx_step_args(c, 1);
      int wb = 0, hb = 0;
      if (st == ST_F32) box_for_kind<ST_F32>(dkind, wb, hb);
      else if (st == ST_F16) box_for_kind<ST_F16>(dkind, wb, hb);
      else box_for_kind<ST_BF16>(dkind, wb, hb);
      const CUtensorMap* m0 = d.args[0].tma ? ctx_tensor_map(c, 0, wb, hb) : nullptr;
      const CUtensorMap* m1 = d.args[0].tma ? ctx_tensor_map(c, 1, wb, hb) : nullptr;
      d.has_map = (m0 && m1) ? 1 : 0;
      if (d.has_map) {
        d.tmap[0] = *m0;
        d.tmap[1] = *m1;
      }
      const int rows = kind_rows_rt(dkind);
      const int tiles = d.tiles_x * ((ny + rows - 1) / rows);
      for (int t = 0; t < tiles; ++t) (dkind == KIND_SC ? heavy : light).push_back(make_int2((int)k, t));
    }
  }
  // the slow tiles first, so the launch ends on short ones (measured against
  // spreading them evenly among the others: 8.30k vs 8.22k MLUPS)
  b->items = heavy;
  b->items.insert(b->items.end(), light.begin(), light.end());
  if (b->grid == 0)
    b->grid = b->storage == ST_F32 ? batch_grid<ST_F32>((int)b->items.size())
              : b->storage == ST_F16 ? batch_grid<ST_F16>((int)b->items.size())
                                     : batch_grid<ST_BF16>((int)b->items.size());
  cudaError_t e = batch_upload(b->host, b->items, b->dev, b->stream);
  if (e != cudaSuccess) {
    b->msg = std::string("batch upload: ") + cudaGetErrorString(e);
    return HLBM_ECUDA;
  }
  return HLBM_OK;
}

static cudaError_t batch_launch(hlbm_batch* b, int flip) {
  const int n = b->dev.nitems;
  switch (b->storage) {
    case ST_F32: return launch_batch<ST_F32>(b->dev.doms, b->dev.items, n, b->grid, flip, b->dev.ctr, b->stream);
    case ST_F16: return launch_batch<ST_F16>(b->dev.doms, b->dev.items, n, b->grid, flip, b->dev.ctr, b->stream);
    default: return launch_batch<ST_BF16>(b->dev.doms, b->dev.items, n, b->grid, flip, b->dev.ctr, b->stream);
  }
}

hlbm_status hlbm_batch_step(hlbm_batch* b, int n) {
  NvtxRange range("hlbm_batch_step");
  if (!b || n < 0) return HLBM_EINVAL;
  if (n == 0) return HLBM_OK;
  hlbm_status st = batch_refresh(b);
  if (st != HLBM_OK) return st;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  // graph of two steps (buffer parity returns); odd remainder launched directly
  if (n >= 2) {
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HLBM_ECUDA;
    cudaError_t le = batch_launch(b, 0);
    if (le == cudaSuccess) le = batch_launch(b, 1);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
      b->msg = std::string("batch capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ce);
      if (g) cudaGraphDestroy(g);
      return HLBM_ECUDA;
    }
    cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      b->graph = nullptr;
      return HLBM_ECUDA;
    }
    for (int k = 0; k < n / 2; ++k)
      if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return HLBM_ECUDA;
  }
  if (n % 2)
    if (batch_launch(b, 0) != cudaSuccess) return HLBM_ECUDA;
  for (hlbm_ctx* c : b->ctxs) ctx_advance(c, n);
  return HLBM_OK;
}

hlbm_status hlbm_batch_synchronize(hlbm_batch* b) {
  if (!b) return HLBM_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HLBM_ECUDA;
  for (hlbm_ctx* c : b->ctxs) {
    hlbm_status st = hlbm_synchronize(c);
    if (st != HLBM_OK) return st;
  }
  return HLBM_OK;
}

void* hlbm_batch_get_stream(hlbm_batch* b) { return b ? b->stream : nullptr; }

hlbm_status hlbm_batch_destroy(hlbm_batch* b) {
  if (!b) return HLBM_EINVAL;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (hlbm_ctx* c : b->ctxs) hlbm_set_stream(c, nullptr);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->dev.doms) cudaFree(b->dev.doms);
  if (b->dev.items) cudaFree(b->dev.items);
  if (b->dev.ctr) cudaFree(b->dev.ctr);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return HLBM_OK;
}

}  // extern "C"
