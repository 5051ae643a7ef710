// Batched step: many independent periodic D2Q37 domains (any sizes, sources
// and parameters) advanced by one launch per source kind and time step,
// replayed from a CUDA graph.  Each CTA takes one 32 x 8 tile of one domain
// from a tile -> domain work list (grouped by kind, so each kind's kernel gets
// its own shared-memory size and register budget); the domain's step
// arguments (for both buffer parities) and its TMA tensor maps are read from
// device memory, so the tile work is exactly the single-domain kernel's
// (process_tile).
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

constexpr int kRows = 8;
// nodes per thread: the pseudopotential kind runs one (its frame of psi values
// then spreads over 256 threads; about 10% faster on droplets), the others two
template <int KIND>
constexpr int kind_npt() {
  return KIND == KIND_SC ? 1 : 2;
}

struct alignas(64) BatchDomain {
  CUtensorMap tmap[2];    // input maps of buffer 0 / 1 (box of the domain's kind)
  StepArgs args[2];       // args[p]: reads buffer p, writes buffer p ^ 1
  int kind;
  int tiles_x;
  int tile0;
  int cur;                // buffer holding the state at the start of the batch call
  int has_map;
};

template <int ST, int KIND>
__device__ __forceinline__ void batch_tile(const BatchDomain& dom, const StepArgs& a, unsigned char* smem, int x0,
                                           int y0, int par) {
  using Cf = Cfg2<ST, KIND, false, kRows>;
  constexpr int NT = 32 * kRows / kind_npt<KIND>();
  typename Cf::T* sp = reinterpret_cast<typename Cf::T*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Cf::POP_BYTES + Cf::AUX_BYTES + Cf::RED_BYTES);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (dom.has_map && tile_boxed<Cf>(a, x0, y0) && ((smem_u32(smem) & 127u) == 0)) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) issue_tile<Cf>(sp, &dom.tmap[par], bar, x0, y0, a.debug_skip_tma);
    const bool ok = mbar_wait_bounded(bar, 0, a.wait_ns);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(a.status, (int)5 /* HLBM_ETIMEOUT */);
      mbar_wait_bounded(bar, 0, a.wait_ns);
      __syncthreads();
      return;
    }
  } else {
    fill_tile_wrapped<Cf, NT>(a, a.fin, sp, x0, y0, tid);
    __syncthreads();
  }
  process_tile<ST, KIND, false, kRows, kind_npt<KIND>(), false>(a, nullptr, smem, x0, y0, a.fout, [] {});
}

// Tiles base .. base + gridDim.x - 1 of the work list, all of kind KIND.
template <int ST, int KIND>
__global__ void __launch_bounds__(32 * kRows / kind_npt<KIND>(),
                                  (min_ctas2<ST, KIND, false, kRows, kind_npt<KIND>()>()))
    batch_step_kernel(const BatchDomain* __restrict__ doms, const int* __restrict__ item_dom, int base, int flip) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int gi = base + blockIdx.x;
  const int d = item_dom[gi];
  const BatchDomain& dom = doms[d];
  const int par = dom.cur ^ flip;
  const StepArgs& a = dom.args[par];
  const int t = gi - dom.tile0;
  const int ty = t / dom.tiles_x;
  const int x0 = (t - ty * dom.tiles_x) * 32, y0 = ty * kRows;
  batch_tile<ST, KIND>(dom, a, smem, x0, y0, par);
}

template <int ST, int KIND>
cudaError_t launch_batch_kind(const BatchDomain* doms, const int* items, int base, int count, int flip,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  batch_step_kernel<ST, KIND><<<count, dim3(32, kRows / kind_npt<KIND>(), 1), Cfg2<ST, KIND, false, kRows>::SMEM, s>>>(
      doms, items, base, flip);
  return cudaGetLastError();
}

// off[k], cnt[k]: the work-list segment of kind k (KIND_LOCAL, KIND_THERMAL, KIND_SC)
template <int ST>
cudaError_t launch_batch(const BatchDomain* doms, const int* items, const int* off, const int* cnt, int flip,
                         cudaStream_t s) {
  cudaError_t e = launch_batch_kind<ST, KIND_LOCAL>(doms, items, off[KIND_LOCAL], cnt[KIND_LOCAL], flip, s);
  if (e == cudaSuccess) e = launch_batch_kind<ST, KIND_THERMAL>(doms, items, off[KIND_THERMAL], cnt[KIND_THERMAL], flip, s);
  if (e == cudaSuccess) e = launch_batch_kind<ST, KIND_SC>(doms, items, off[KIND_SC], cnt[KIND_SC], flip, s);
  return e;
}

template <int ST>
cudaError_t configure_batch() {
  cudaError_t e = cudaFuncSetAttribute(batch_step_kernel<ST, KIND_LOCAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg2<ST, KIND_LOCAL, false, kRows>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_step_kernel<ST, KIND_THERMAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg2<ST, KIND_THERMAL, false, kRows>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_step_kernel<ST, KIND_SC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg2<ST, KIND_SC, false, kRows>::SMEM);
  return e;
}

template <int ST>
void box_for_kind(int kind, int& wb, int& hb) {
  if (kind == KIND_SC) box_of<ST, KIND_SC, false, kRows>(wb, hb);
  else if (kind == KIND_THERMAL) box_of<ST, KIND_THERMAL, false, kRows>(wb, hb);
  else box_of<ST, KIND_LOCAL, false, kRows>(wb, hb);
}

}  // namespace

// Host-side helpers the C ABI (api.cu) uses; the batch owns the device arrays.
struct BatchDevice {
  BatchDomain* doms = nullptr;
  int* items = nullptr;
  int nitems = 0;
};

cudaError_t batch_upload(const std::vector<BatchDomain>& host, const std::vector<int>& items, BatchDevice& dev,
                         cudaStream_t s) {
  if (!dev.doms) {
    cudaError_t e = cudaMalloc(&dev.doms, host.size() * sizeof(BatchDomain));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&dev.items, items.size() * sizeof(int));
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemcpyAsync(dev.doms, host.data(), host.size() * sizeof(BatchDomain), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev.items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice, s);
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
  std::vector<int> items;         // tile -> domain, grouped by kind
  int off[3] = {0, 0, 0}, cnt[3] = {0, 0, 0};   // each kind's segment of `items`
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
  for (int kind : {(int)KIND_LOCAL, (int)KIND_THERMAL, (int)KIND_SC}) {
    b->off[kind] = (int)b->items.size();
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
      hlbm_ctx* c = b->ctxs[k];
      int st, dkind, nx, ny;
      ctx_batchable(c, &st, &dkind, &nx, &ny);
      if (dkind != kind) continue;
      BatchDomain& d = b->host[k];
      std::memset(&d, 0, sizeof(d));
      d.kind = dkind;
      d.tiles_x = (nx + 31) / 32;
      d.tile0 = (int)b->items.size();
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
      const int tiles = d.tiles_x * ((ny + kRows - 1) / kRows);
      for (int t = 0; t < tiles; ++t) b->items.push_back((int)k);
    }
    b->cnt[kind] = (int)b->items.size() - b->off[kind];
  }
  cudaError_t e = batch_upload(b->host, b->items, b->dev, b->stream);
  if (e != cudaSuccess) {
    b->msg = std::string("batch upload: ") + cudaGetErrorString(e);
    return HLBM_ECUDA;
  }
  return HLBM_OK;
}

static cudaError_t batch_launch(hlbm_batch* b, int flip) {
  switch (b->storage) {
    case ST_F32: return launch_batch<ST_F32>(b->dev.doms, b->dev.items, b->off, b->cnt, flip, b->stream);
    case ST_F16: return launch_batch<ST_F16>(b->dev.doms, b->dev.items, b->off, b->cnt, flip, b->stream);
    default: return launch_batch<ST_BF16>(b->dev.doms, b->dev.items, b->off, b->cnt, flip, b->stream);
  }
}

hlbm_status hlbm_batch_step(hlbm_batch* b, int n) {
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
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return HLBM_OK;
}

}  // extern "C"
