// Host implementation of the hlbm C ABI (include/hlbm.h): validation,
// device memory (own allocation or a caller-bound arena), stream ordering,
// CUDA-graph replay of the step loop, diagnostics and checkpoints.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <deque>
#include <vector>

#include "hlbm.h"
#include "internal.h"
#include "lattice.cuh"

using namespace hlbm;

struct hlbm_ctx {
  int lattice = 0, D = 2, Q = 37;
  int nx = 0, ny = 0, nz = 1;
  long long N = 0;
  double tau_hat = 1.0;
  hlbm_source_params p{};
  int kind = KIND_LOCAL;
  int storage = ST_F32;
  size_t elem = 4;
  int rows = 8;
  int npt = 2;
  int persistent = 0;
  bool multistep = false;         // D2Q37: one persistent launch for many steps (tile-row counters)
  unsigned gen = 0;               // multi-step kernel: steps run since the counters were zeroed

  cudaStream_t stream = nullptr;
  bool own_stream = false;

  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  void* pop[2] = {nullptr, nullptr};
  float* gfield = nullptr;
  double* partials = nullptr;
  double* red = nullptr;
  int cur = 0;
  bool initialised = false;

  int force_mode = FORCE_NONE;
  long long steps = 0;

  // walls (HLBM_WALLS): [4][N] moments rho, u_x, u_y, theta - 1 of the
  // previous step (mom[cur]) and of the step being taken (mom[cur ^ 1])
  bool walls = false;
  float* mom[2] = {nullptr, nullptr};

  // in-place step (HLBM_AA): one population buffer (pop[0]; pop[1] is then a
  // staging area of 4 N floats), the step parity in `cur`, and two neighbour
  // fields: aux[cur ^ 1] is read by the next step, aux[cur] written
  bool aa = false;
  float* aux[2] = {nullptr, nullptr};
  float* comp = nullptr;          // walls: completed unknowns of the six wall rows

  bool failed = false;
  std::string msg;

  // graphs replaying kGraphSteps steps from buffer parity 0 / 1
  cudaGraphExec_t graph[2] = {nullptr, nullptr};

  // TMA staging: tensor maps per (population buffer address, box); the
  // buffers are the context's two and, during hlbm_adjoint_run, its
  // workspace's recomputed states
  bool tma_ok = false;
  bool tma_store_ok = false;
  struct TMap {
    const void* base;
    int wb, hb;
    bool f32;    // viewed as FP32 (the adjoint's lambda) instead of the storage type
    int planes;  // outermost extent: Q, or D for a per-node vector field
    CUtensorMap map;
  };
  std::deque<TMap> tmaps;         // deque: pointers to entries stay valid as maps are added
  int* status = nullptr;          // device status word (bounded waits)
  unsigned long long* tile_ctr = nullptr;  // persistent step's tile counter
  unsigned long long* adj_ctr = nullptr;   // whole-row reverse step's tile counter
  unsigned long long* ms_ctr = nullptr;    // multi-step kernel's tile counter (zeroed per launch)
  unsigned* flags = nullptr;               // multi-step kernel: per-tile-row completion counters
  size_t nflags = 0;
  bool ctr_reset = true;          // the counter must be zeroed before the next step
  unsigned long long wait_ns = 2000000000ull;
  int debug_skip_tma = 0;
};

static const int kGraphSteps = 32;  // even: a replay returns to the same buffer parity

namespace {

struct Layout {
  size_t pop_bytes, off_pop1, off_g, off_part, off_red, off_flags, nflags, off_mom, mom_bytes, off_aux, aux_bytes,
      off_comp, comp_bytes, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout layout(int lattice, int nx, int ny, int nz, const hlbm_source_params* p) {
  Layout L{};
  const long long N = (long long)nx * ny * nz;
  const int Q = lattice == 0 ? 37 : 39, D = lattice == 0 ? 2 : 3;
  const size_t elem = (p->storage == HLBM_F32) ? 4 : 2;
  L.pop_bytes = align256((size_t)Q * (size_t)N * elem);
  L.off_pop1 = L.pop_bytes;
  // in place: the second buffer is only a staging area for host fields
  const size_t second = (p->flags & HLBM_AA) ? align256((size_t)(2 + D) * (size_t)N * 4) : L.pop_bytes;
  L.off_g = L.off_pop1 + second;
  const size_t gbytes = (p->flags & HLBM_SRC_FORCE) ? align256((size_t)D * (size_t)N * 4) : 0;
  L.off_part = L.off_g + gbytes;
  L.off_red = L.off_part + align256((size_t)moment_blocks(lattice, nx, ny, nz) * 8 * sizeof(double));
  L.off_flags = L.off_red + 256;
  // D2Q37: one completion counter per tile row of the smallest tiles (4 rows)
  L.nflags = (lattice == 0) ? (size_t)((ny + 3) / 4) : 0;
  L.off_mom = L.off_flags + align256(L.nflags * 4);
  // walls: two [4][N] FP32 moment fields (previous step, this step)
  L.mom_bytes = (p->flags & HLBM_WALLS) ? align256((size_t)4 * (size_t)N * 4) : 0;
  L.off_aux = L.off_mom + 2 * L.mom_bytes;
  L.aux_bytes = (p->flags & HLBM_AA) ? align256((size_t)N * 4) : 0;
  // walls: the completed unknowns of the six wall rows, [6][37][nx] FP32
  L.off_comp = L.off_aux + 2 * L.aux_bytes;
  L.comp_bytes = (p->flags & HLBM_WALLS) ? align256((size_t)6 * 37 * (size_t)nx * 4) : 0;
  L.total = L.off_comp + L.comp_bytes;
  return L;
}

// v = hi + lo with hi = fl32(v), lo = fl32(v - hi)
void split_ff(double v, float (&out)[2]) {
  out[0] = (float)v;
  out[1] = (float)(v - (double)out[0]);
}

hlbm_status fail(hlbm_ctx* c, hlbm_status st, const std::string& m, bool sticky = false) {
  if (c) {
    c->msg = m;
    if (sticky) c->failed = true;
  }
  return st;
}

hlbm_status cuda_fail(hlbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, HLBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e), true);
}

#define HLBM_CUDA(c, call, where)                 \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

bool finite(double v) { return std::isfinite(v); }

hlbm_status validate(int lattice, int nx, int ny, int nz, double tau_hat, const hlbm_source_params* p,
                     std::string& why) {
  if (!p) { why = "params is NULL"; return HLBM_EINVAL; }
  if (lattice != HLBM_D2Q37 && lattice != HLBM_D3Q39) { why = "unknown lattice"; return HLBM_EINVAL; }
  if (nx < 7 || ny < 7) { why = "nx and ny must be >= 7 (reach-3 velocities)"; return HLBM_EINVAL; }
  if (lattice == HLBM_D2Q37 && nz != 1) { why = "nz must be 1 on D2Q37"; return HLBM_EINVAL; }
  if (lattice == HLBM_D3Q39 && nz < 7) { why = "nz must be >= 7 on D3Q39"; return HLBM_EINVAL; }
  if ((long long)nx * ny * nz >= (1LL << 31)) { why = "nx*ny*nz must be < 2^31"; return HLBM_EINVAL; }
  if (!finite(tau_hat) || !(tau_hat > 0.5)) { why = "tau_hat must be finite and > 1/2"; return HLBM_EINVAL; }
  if (p->storage < HLBM_F32 || p->storage > HLBM_BF16) { why = "unknown storage"; return HLBM_EINVAL; }
  if (!finite(p->rho0) || !(p->rho0 > 0)) { why = "rho0 must be finite and > 0"; return HLBM_EINVAL; }
  const uint32_t known =
      HLBM_SRC_FORCE | HLBM_SRC_H | HLBM_SRC_SC | HLBM_SRC_P | HLBM_ISOTHERMAL | HLBM_WALLS | HLBM_AA;
  if (p->flags & ~known) { why = "unknown flag bits"; return HLBM_EINVAL; }
  for (int d = 0; d < 3; ++d)
    if (!finite(p->force[d])) { why = "force must be finite"; return HLBM_EINVAL; }
  if ((p->flags & HLBM_SRC_H) && (!finite(p->Pr) || !(p->Pr > 0))) { why = "Pr must be > 0"; return HLBM_EINVAL; }
  if ((p->flags & HLBM_SRC_H) && (p->flags & HLBM_ISOTHERMAL)) {
    why = "the thermal diffusion source needs the thermal mode"; return HLBM_EINVAL;
  }
  if ((p->flags & HLBM_SRC_SC) && !(p->flags & HLBM_ISOTHERMAL)) {
    why = "the pseudopotential force needs the isothermal mode (theta == 1)"; return HLBM_EINVAL;
  }
  if ((p->flags & HLBM_SRC_P) && !(p->flags & HLBM_SRC_SC)) {
    why = "the pressure-tensor source needs the pseudopotential force"; return HLBM_EINVAL;
  }
  if (p->flags & HLBM_SRC_SC) {
    if (p->eos != 0 && p->eos != 1) { why = "eos must be 0 (vdW) or 1 (C-S)"; return HLBM_EINVAL; }
    if (!finite(p->eos_a) || !finite(p->eos_b) || !finite(p->eos_T) || !finite(p->k) || !(p->eos_b > 0) ||
        !(p->eos_T > 0)) {
      why = "EOS parameters must be finite with b, T > 0"; return HLBM_EINVAL;
    }
  }
  if (lattice == HLBM_D3Q39 && (p->flags & (HLBM_SRC_H | HLBM_SRC_SC))) {
    why = "D3Q39 supports the body-force source only"; return HLBM_EUNSUPPORTED;
  }
  if (p->flags & HLBM_AA) {
    if (lattice != HLBM_D2Q37) { why = "the in-place step is built for D2Q37"; return HLBM_EUNSUPPORTED; }
    if (p->flags & HLBM_WALLS) { why = "the in-place step is built for periodic domains"; return HLBM_EUNSUPPORTED; }
  }
  if (p->flags & HLBM_WALLS) {
    if (lattice != HLBM_D2Q37) { why = "walls are built for D2Q37"; return HLBM_EUNSUPPORTED; }
    if (p->flags & (HLBM_SRC_SC | HLBM_ISOTHERMAL)) {
      why = "walls are built for the thermal mode without the pseudopotential force"; return HLBM_EUNSUPPORTED;
    }
    for (int k = 0; k < 2; ++k) {
      if (!finite(p->wall_theta[k]) || !(p->wall_theta[k] > 0)) { why = "wall temperatures must be > 0"; return HLBM_EINVAL; }
      for (int d = 0; d < 3; ++d)
        if (!finite(p->wall_u[k][d])) { why = "wall velocities must be finite"; return HLBM_EINVAL; }
      if (p->wall_u[k][1] != 0.0) { why = "walls move along x only (no normal velocity)"; return HLBM_EINVAL; }
    }
  }
  return HLBM_OK;
}

hlbm_status ensure_memory(hlbm_ctx* c) {
  if (c->arena) return HLBM_OK;
  const char* inj = std::getenv("HLBM_FAULT_ALLOC");
  if (inj && inj[0] == '1') return fail(c, HLBM_ENOMEM, "device allocation failed (injected by HLBM_FAULT_ALLOC)");
  const Layout L = layout(c->lattice, c->nx, c->ny, c->nz, &c->p);
  void* m = nullptr;
  cudaError_t e = cudaMalloc(&m, L.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HLBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->arena = static_cast<char*>(m);
  c->arena_bytes = L.total;
  c->own_arena = true;
  return HLBM_OK;
}

void carve(hlbm_ctx* c) {
  const Layout L = layout(c->lattice, c->nx, c->ny, c->nz, &c->p);
  c->pop[0] = c->arena;
  c->pop[1] = c->arena + L.off_pop1;
  c->gfield = (c->p.flags & HLBM_SRC_FORCE) ? reinterpret_cast<float*>(c->arena + L.off_g) : nullptr;
  c->partials = reinterpret_cast<double*>(c->arena + L.off_part);
  c->red = reinterpret_cast<double*>(c->arena + L.off_red);
  c->status = reinterpret_cast<int*>(c->arena + L.off_red + 64);
  c->tile_ctr = reinterpret_cast<unsigned long long*>(c->arena + L.off_red + 128);
  c->adj_ctr = reinterpret_cast<unsigned long long*>(c->arena + L.off_red + 192);
  c->ms_ctr = reinterpret_cast<unsigned long long*>(c->arena + L.off_red + 224);
  c->flags = L.nflags ? reinterpret_cast<unsigned*>(c->arena + L.off_flags) : nullptr;
  c->nflags = L.nflags;
  c->mom[0] = L.mom_bytes ? reinterpret_cast<float*>(c->arena + L.off_mom) : nullptr;
  c->mom[1] = L.mom_bytes ? reinterpret_cast<float*>(c->arena + L.off_mom + L.mom_bytes) : nullptr;
  c->aux[0] = L.aux_bytes ? reinterpret_cast<float*>(c->arena + L.off_aux) : nullptr;
  c->aux[1] = L.aux_bytes ? reinterpret_cast<float*>(c->arena + L.off_aux + L.aux_bytes) : nullptr;
  c->comp = L.comp_bytes ? reinterpret_cast<float*>(c->arena + L.off_comp) : nullptr;
}

hlbm_status ensure_stream(hlbm_ctx* c) {
  if (c->stream) return HLBM_OK;
  HLBM_CUDA(c, cudaStreamCreate(&c->stream), "cudaStreamCreate");
  c->own_stream = true;
  return HLBM_OK;
}

void drop_graphs(hlbm_ctx* c) {
  for (int k = 0; k < 2; ++k)
    if (c->graph[k]) {
      cudaGraphExecDestroy(c->graph[k]);
      c->graph[k] = nullptr;
    }
}

StepArgs make_args(const hlbm_ctx* c) {
  StepArgs a{};
  a.N = c->N;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  a.force_mode = c->force_mode;
  a.gfield = c->gfield;
  a.isothermal = (c->p.flags & HLBM_ISOTHERMAL) ? 1 : 0;
  a.rho0 = (float)c->p.rho0;
  a.omega = (float)(1.0 / c->tau_hat);
  a.beta = (float)(1.0 - 0.5 / c->tau_hat);
  for (int d = 0; d < 3; ++d) a.g[d] = (float)c->p.force[d];
  a.h_coef = (c->p.flags & HLBM_SRC_H) ? (float)(1.0 - 1.0 / c->p.Pr) : 0.f;
  a.eos = c->p.eos;
  const double cs2 = c->lattice == 0 ? D2Q37::cs2 : D3Q39::cs2;
  split_ff(2.0 * c->p.eos_a / cs2, a.psi_k1);
  split_ff(2.0 * c->p.eos_T / cs2, a.psi_k2);
  split_ff(c->p.eos == 0 ? c->p.eos_b : 0.25 * c->p.eos_b, a.psi_kb);
  a.status = c->status;
  a.tma = c->tma_ok ? 1 : 0;
  a.persistent = c->persistent;
  a.tile_ctr = c->tile_ctr;
  a.wait_ns = c->wait_ns;
  a.debug_skip_tma = c->debug_skip_tma;
  // sigma = -k c0^2 |F^SC|^2 / (D tau G psi^2), tau = tau^ - 1/2, G = -1 (Eq. 3.12, Table 2)
  a.p_coef = (c->p.flags & HLBM_SRC_P) ? (float)(c->p.k * cs2 / (c->D * (c->tau_hat - 0.5))) : 0.f;
  return a;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Tensor map of population buffer `buf` viewed as [Q][ny][nx] with a
// wb x hb x 1 box (D2Q37), or as [Q][nz][ny][nx] with a wb x hb x 1 x 1 box
// (D3Q39), in the storage type or (f32) in FP32, with `planes` instead of Q
// outermost when given (a [D][N] FP32 field); null if it cannot be encoded
// (the kernels then stage every tile with plain loads).
const CUtensorMap* tensor_map_at(hlbm_ctx* c, const void* base, int wb, int hb, bool f32 = false, int planes = 0) {
  if (planes <= 0) planes = c->Q;
  for (auto& t : c->tmaps)
    if (t.base == base && t.wb == wb && t.hb == hb && t.f32 == f32 && t.planes == planes) return &t.map;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return nullptr;
  hlbm_ctx::TMap t{};
  t.base = base;
  t.wb = wb;
  t.hb = hb;
  t.f32 = f32;
  t.planes = planes;
  const CUtensorMapDataType dt = (f32 || c->storage == ST_F32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : c->storage == ST_F16        ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const bool d3 = c->lattice == HLBM_D3Q39;
  const cuuint64_t e = f32 ? 4 : (cuuint64_t)c->elem;
  const cuuint64_t dims2[3] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)planes};
  const cuuint64_t strides2[2] = {(cuuint64_t)c->nx * e, (cuuint64_t)c->N * e};
  const cuuint64_t dims3[4] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)c->nz, (cuuint64_t)planes};
  const cuuint64_t strides3[3] = {(cuuint64_t)c->nx * e, (cuuint64_t)c->nx * c->ny * e, (cuuint64_t)c->N * e};
  const cuuint32_t box[4] = {(cuuint32_t)wb, (cuuint32_t)hb, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&t.map, dt, d3 ? 4 : 3, const_cast<void*>(base), d3 ? dims3 : dims2, d3 ? strides3 : strides2,
                   box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return nullptr;
  c->tmaps.push_back(t);
  return &c->tmaps.back().map;
}

const CUtensorMap* tensor_map(hlbm_ctx* c, int buf, int wb, int hb) { return tensor_map_at(c, c->pop[buf], wb, hb); }

cudaError_t launch_step(hlbm_ctx* c, StepArgs a, bool moments) {
  if (c->lattice != 0) {
    // persistent whole-row kernel: box of 256 / nx rows, and single rows
    // and, with a force field, a box of its three planes
    CUtensorMap maps3[3];
    std::memset(maps3, 0, sizeof(maps3));
    const CUtensorMap* tm = nullptr;
    a.g_staged = 0;
    if (!moments && a.persistent && a.tma && (c->nx == 32 || c->nx == 64 || c->nx == 128 || c->nx == 256)) {
      const CUtensorMap* mb = tensor_map_at(c, a.fin, c->nx, 256 / c->nx);
      const CUtensorMap* mr = tensor_map_at(c, a.fin, c->nx, 1);
      if (mb && mr) {
        maps3[0] = *mb;
        maps3[1] = *mr;
        tm = maps3;
        if (a.force_mode == FORCE_FIELD && c->gfield) {
          const CUtensorMap* mg = tensor_map_at(c, c->gfield, c->nx, 256 / c->nx, true, 3);
          if (mg) {
            maps3[2] = *mg;
            a.g_staged = 1;
          }
        }
      }
    }
    return launch_step_d3q39(a, c->kind, c->storage, moments, c->rows, c->npt, tm, c->stream);
  }
  CUtensorMap maps[2];
  std::memset(maps, 0, sizeof(maps));
  a.tma_store = 0;
  if (a.tma) {
    int wb = 0, hb = 0, ob = 0;
    step_box_d2q37(c->kind, c->storage, moments, c->rows, &wb, &hb, &ob);
    const CUtensorMap* in = tensor_map_at(c, a.fin, wb, hb);
    const CUtensorMap* out = moments ? nullptr : tensor_map_at(c, a.fout, 32, ob);
    if (in) maps[0] = *in;
    else a.tma = 0;
    if (out && c->tma_store_ok) {
      maps[1] = *out;
      a.tma_store = 1;
    }
  }
  return launch_step_d2q37(a, c->kind, c->storage, moments, c->rows, c->npt, maps, c->stream);
}

// HLBM_ETIMEOUT if a kernel reported an expired bounded wait (synchronises).
hlbm_status check_status(hlbm_ctx* c) {
  int st = 0;
  HLBM_CUDA(c, cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  HLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st == HLBM_ETIMEOUT) return fail(c, HLBM_ETIMEOUT, "a bounded device wait expired (TMA staging)", true);
  return HLBM_OK;
}

WallArgs make_wall_args(const hlbm_ctx* c) {
  WallArgs w{};
  w.N = c->N;
  w.nx = c->nx;
  w.ny = c->ny;
  w.gfield = c->gfield;
  w.force_mode = c->force_mode;
  for (int d = 0; d < 3; ++d) w.g[d] = (float)c->p.force[d];
  w.rho0 = (float)c->p.rho0;
  w.omega = (float)(1.0 / c->tau_hat);
  w.beta = (float)(1.0 - 0.5 / c->tau_hat);
  w.h_coef = (c->p.flags & HLBM_SRC_H) ? (float)(1.0 - 1.0 / c->p.Pr) : 0.f;
  for (int k = 0; k < 2; ++k) {
    w.wall_u[k][0] = (float)c->p.wall_u[k][0];
    w.wall_u[k][1] = (float)c->p.wall_u[k][1];
    w.wall_tb[k] = (float)(c->p.wall_theta[k] - 1.0);
  }
  // stored deviations are taken from the rest equilibrium at the mean wall temperature
  const double tbr = 0.5 * (c->p.wall_theta[0] + c->p.wall_theta[1]) - 1.0;
  w.tb_ref = (float)tbr;
  w.e_ref = (float)(c->p.rho0 * 2.0 * D2Q37::cs2 * tbr);
  w.mprev = c->mom[c->cur];
  w.fin = c->pop[c->cur];
  w.comp = c->comp;
  return w;
}

// One wall-bounded step: the moments launch (completed moments of time t into
// mom[cur ^ 1]), then the collide launch.
cudaError_t wall_step(hlbm_ctx* c) {
  WallArgs w = make_wall_args(c);
  w.mcur = c->mom[c->cur ^ 1];
  cudaError_t e = launch_walls(w, c->storage, 2, false, c->stream);
  if (e != cudaSuccess) return e;
  e = launch_walls(w, c->storage, 0, false, c->stream);
  if (e != cudaSuccess) return e;
  w.fout = c->pop[c->cur ^ 1];
  e = launch_walls(w, c->storage, 1, c->kind == KIND_THERMAL, c->stream);
  c->cur ^= 1;
  return e;
}

// One in-place step of parity cur: reads aux[cur ^ 1], writes aux[cur].
cudaError_t aa_step(hlbm_ctx* c, bool mom, StepArgs* margs = nullptr) {
  StepArgs a = margs ? *margs : make_args(c);
  a.fin = c->pop[0];
  a.fout = c->pop[0];
  a.aux_rd = c->aux[c->cur ^ 1];
  a.aux_wr = c->aux[c->cur];
  cudaError_t e = launch_aa(a, c->kind, c->storage, c->cur == 1, mom, c->stream);
  if (!mom) c->cur ^= 1;
  return e;
}

cudaError_t one_step(hlbm_ctx* c) {
  if (c->walls) return wall_step(c);
  if (c->aa) return aa_step(c, false);
  StepArgs a = make_args(c);
  a.fin = c->pop[c->cur];
  a.fout = c->pop[c->cur ^ 1];
  a.reverse = c->cur;   // alternate the tile order: each step starts where the previous one ended
  cudaError_t e = launch_step(c, a, false);
  c->cur ^= 1;
  return e;
}

// Whether hlbm_step runs the multi-step kernel: D2Q37, tiles that cover the
// domain exactly, and a read region (pull 3 + neighbour frame H) within one
// tile row of the tile.
bool multistep_ok(const hlbm_ctx* c) {
  if (!c->multistep || c->lattice != HLBM_D2Q37 || !c->flags || c->walls || c->aa) return false;
  const int H = c->kind == KIND_SC ? 3 : (c->kind == KIND_THERMAL ? 1 : 0);
  return c->nx % 32 == 0 && c->ny % c->rows == 0 && H + 3 <= c->rows;
}

// Steps of one multi-step launch (tile indices stay below 2^31).
int multistep_max(const hlbm_ctx* c) {
  const long long T = (long long)(c->nx / 32) * (c->ny / c->rows);
  return (int)std::max(1LL, std::min(1024LL, 0x7fffffffLL / T));
}

// One multi-step launch of S steps from the current buffer.
cudaError_t launch_multistep(hlbm_ctx* c, int S) {
  StepArgs a = make_args(c);
  a.fin = c->pop[c->cur];
  a.fout = c->pop[c->cur ^ 1];
  a.msteps = S;
  a.gen0 = c->gen;
  a.flags = c->flags;
  a.ms_ctr = c->ms_ctr;
  a.tma_store = 0;
  CUtensorMap maps[2];
  std::memset(maps, 0, sizeof(maps));
  if (a.tma) {
    int wb = 0, hb = 0, ob = 0;
    step_box_d2q37(c->kind, c->storage, false, c->rows, &wb, &hb, &ob);
    const CUtensorMap* m0 = tensor_map_at(c, a.fin, wb, hb);
    const CUtensorMap* m1 = tensor_map_at(c, a.fout, wb, hb);
    if (m0 && m1) {
      maps[0] = *m0;
      maps[1] = *m1;
    } else {
      a.tma = 0;
    }
  }
  cudaError_t e = cudaMemsetAsync(c->ms_ctr, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = launch_step_d2q37(a, c->kind, c->storage, false, c->rows, c->npt, maps, c->stream);
  if (e != cudaSuccess) return e;
  c->gen += (unsigned)S;
  c->cur ^= (S & 1);
  c->steps += S;
  return cudaSuccess;
}

hlbm_status usable(hlbm_ctx* c) {
  if (!c) return HLBM_EINVAL;
  if (c->failed) return HLBM_ESTATE;
  return HLBM_OK;
}

}  // namespace

namespace hlbm {
// accessors used by the batched step (batch.cu)
bool ctx_batchable(const hlbm_ctx* c, int* storage, int* kind, int* nx, int* ny) {
  if (!c || c->lattice != HLBM_D2Q37 || !c->initialised || c->failed || c->walls || c->aa) return false;
  *storage = c->storage;
  *kind = c->kind;
  *nx = c->nx;
  *ny = c->ny;
  return true;
}
StepArgs ctx_step_args(hlbm_ctx* c, int parity) {
  StepArgs a = make_args(c);
  a.fin = c->pop[parity];
  a.fout = c->pop[parity ^ 1];
  a.tma_store = 0;
  a.persistent = 0;
  return a;
}
const CUtensorMap* ctx_tensor_map(hlbm_ctx* c, int buf, int wb, int hb) { return tensor_map(c, buf, wb, hb); }
int ctx_cur(const hlbm_ctx* c) { return c->cur; }
void ctx_advance(hlbm_ctx* c, int steps) {
  c->cur ^= (steps & 1);
  c->steps += steps;
}
}  // namespace hlbm

extern "C" {

size_t hlbm_workspace_bytes(int lattice, int nx, int ny, int nz, const hlbm_source_params* p) {
  std::string why;
  if (validate(lattice, nx, ny, nz, 1.0, p, why) != HLBM_OK) return 0;
  return layout(lattice, nx, ny, nz, p).total;
}

hlbm_status hlbm_create(int lattice, int nx, int ny, int nz, double tau_hat, const hlbm_source_params* p,
                        hlbm_ctx** out) {
  NvtxRange range("hlbm_create");
  if (!out) return HLBM_EINVAL;
  *out = nullptr;
  std::string why;
  hlbm_status st = validate(lattice, nx, ny, nz, tau_hat, p, why);
  if (st != HLBM_OK) {
    std::fprintf(stderr, "hlbm_create: %s\n", why.c_str());
    return st;
  }
  hlbm_ctx* c = new (std::nothrow) hlbm_ctx();
  if (!c) return HLBM_ENOMEM;
  c->lattice = lattice;
  c->D = lattice == 0 ? 2 : 3;
  c->Q = lattice == 0 ? 37 : 39;
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->N = (long long)nx * ny * nz;
  c->tau_hat = tau_hat;
  c->p = *p;
  c->storage = p->storage;
  c->elem = p->storage == HLBM_F32 ? 4 : 2;
  c->kind = (p->flags & HLBM_SRC_SC) ? KIND_SC : (p->flags & HLBM_SRC_H) ? KIND_THERMAL : KIND_LOCAL;
  c->force_mode = (p->flags & HLBM_SRC_FORCE) ? FORCE_UNIFORM : FORCE_NONE;
  c->walls = (p->flags & HLBM_WALLS) != 0;
  c->aa = (p->flags & HLBM_AA) != 0;
  c->rows = 8;
  // TMA needs a row pitch that is a multiple of 16 bytes
  const char* no_tma = std::getenv("HLBM_NO_TMA");
  c->tma_ok = ((size_t)nx * c->elem) % 16 == 0 && !(no_tma && no_tma[0] == '1');
  const char* no_tma_st = std::getenv("HLBM_NO_TMA_STORE");
  c->tma_store_ok = c->tma_ok && !(no_tma_st && no_tma_st[0] == '1');
  const char* skip = std::getenv("HLBM_TEST_SKIP_TMA");
  c->debug_skip_tma = (skip && skip[0] == '1') ? 1 : 0;
  *out = c;
  return HLBM_OK;
}

hlbm_status hlbm_bind_memory(hlbm_ctx* c, void* dev_ptr, size_t bytes) {
  if (!c || !dev_ptr) return HLBM_EINVAL;
  if (c->arena) return fail(c, HLBM_ESTATE, "memory already allocated or bound");
  if ((reinterpret_cast<uintptr_t>(dev_ptr) & 255) != 0) return fail(c, HLBM_EINVAL, "memory must be 256-byte aligned");
  const Layout L = layout(c->lattice, c->nx, c->ny, c->nz, &c->p);
  if (bytes < L.total) return fail(c, HLBM_ENOMEM, "bound memory smaller than hlbm_workspace_bytes()");
  c->arena = static_cast<char*>(dev_ptr);
  c->arena_bytes = bytes;
  c->own_arena = false;
  return HLBM_OK;
}

hlbm_status hlbm_set_stream(hlbm_ctx* c, void* s) {
  if (!c) return HLBM_EINVAL;
  drop_graphs(c);
  if (c->own_stream && c->stream) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
  }
  c->own_stream = false;
  c->stream = static_cast<cudaStream_t>(s);
  return HLBM_OK;
}

void* hlbm_get_stream(hlbm_ctx* c) {
  if (!c || ensure_stream(c) != HLBM_OK) return nullptr;
  return c->stream;
}

hlbm_status hlbm_init(hlbm_ctx* c, const float* rho, const float* u, const float* theta, int on_device) {
  NvtxRange range("hlbm_init");
  if (!c || !rho || !u || !theta) return HLBM_EINVAL;
  hlbm_status st = ensure_memory(c);
  if (st != HLBM_OK) return st;
  if ((st = ensure_stream(c)) != HLBM_OK) return st;
  carve(c);
  if (c->lattice == 0) HLBM_CUDA(c, configure_step_d2q37(c->storage), "cudaFuncSetAttribute");
  InitArgs a{};
  a.N = c->N;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  a.rho0 = (float)c->p.rho0;
  a.fout = c->pop[0];
  if (on_device) {
    a.rho = rho;
    a.u = u;
    a.theta = theta;
  } else {
    // stage the host fields in the second population buffer (the init
    // kernel writes only the first); (D + 2) N floats always fit in Q N elements
    const size_t n = (size_t)c->N;
    float* stage = static_cast<float*>(c->pop[1]);
    HLBM_CUDA(c, cudaMemcpyAsync(stage, rho, n * 4, cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
    HLBM_CUDA(c, cudaMemcpyAsync(stage + n, u, c->D * n * 4, cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
    HLBM_CUDA(c, cudaMemcpyAsync(stage + (1 + c->D) * n, theta, n * 4, cudaMemcpyHostToDevice, c->stream),
              "cudaMemcpyAsync");
    a.rho = stage;
    a.u = stage + n;
    a.theta = stage + (1 + c->D) * n;
  }
  cudaError_t e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->tile_ctr, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess && c->flags) e = cudaMemsetAsync(c->flags, 0, c->nflags * 4, c->stream);
  if (e == cudaSuccess && c->aa) {
    StepArgs s = make_args(c);
    s.fout = c->pop[0];
    s.aux_wr = c->aux[1];               // read by the first step (parity 0)
    e = launch_aa_init(s, c->kind, c->storage, a.rho, a.u, a.theta, c->stream);
  }
  if (e == cudaSuccess && !c->walls && !c->aa) e = launch_init(c->lattice, a, c->storage, c->stream);
  if (e == cudaSuccess && c->walls) {
    WallArgs w = make_wall_args(c);
    w.fout = c->pop[0];
    e = launch_wall_init(w, c->storage, a.rho, a.u, a.theta, c->mom[0], c->stream);
  }
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->stream);  // host buffers are borrowed
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  c->cur = 0;
  c->steps = 0;
  c->gen = 0;
  c->initialised = true;
  c->failed = false;
  return HLBM_OK;
}

hlbm_status hlbm_set_force_field(hlbm_ctx* c, const float* g, int kind, int on_device) {
  hlbm_status st = usable(c);
  if (st != HLBM_OK) return st;
  if (!(c->p.flags & HLBM_SRC_FORCE)) return fail(c, HLBM_EINVAL, "context was created without HLBM_SRC_FORCE");
  if (kind == 0) {
    c->force_mode = FORCE_UNIFORM;
    drop_graphs(c);
    return HLBM_OK;
  }
  if ((kind != 1 && kind != 2) || !g) return fail(c, HLBM_EINVAL, "kind must be 0, 1 or 2 with a field pointer");
  if ((st = ensure_memory(c)) != HLBM_OK) return st;
  if ((st = ensure_stream(c)) != HLBM_OK) return st;
  carve(c);
  const size_t n = (kind == 1) ? (size_t)c->D * (size_t)c->N : (size_t)c->D * (size_t)c->ny;
  HLBM_CUDA(c, cudaMemcpyAsync(c->gfield, g, n * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               c->stream), "cudaMemcpyAsync");
  if (!on_device) HLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  c->force_mode = (kind == 1) ? FORCE_FIELD : FORCE_PROFILE_Y;
  drop_graphs(c);
  return HLBM_OK;
}

hlbm_status hlbm_step(hlbm_ctx* c, int n) {
  NvtxRange range("hlbm_step");
  hlbm_status st = usable(c);
  if (st != HLBM_OK) return st;
  if (n < 0) return fail(c, HLBM_EINVAL, "n must be >= 0");
  if (!c->initialised) return fail(c, HLBM_ESTATE, "hlbm_init has not been called");
  if (c->ctr_reset) {
    // the persistent launch's CTA count may have changed: restart the counter
    HLBM_CUDA(c, cudaMemsetAsync(c->tile_ctr, 0, sizeof(unsigned long long), c->stream), "cudaMemsetAsync");
    c->ctr_reset = false;
  }
  if (multistep_ok(c)) {
    while (n > 0) {
      NvtxRange chunk("hlbm_step: multi-step launch");
      const int S = std::min(n, multistep_max(c));
      HLBM_CUDA(c, launch_multistep(c, S), "multi-step kernel");
      n -= S;
    }
    return HLBM_OK;
  }
  while (n >= kGraphSteps) {
    NvtxRange chunk("hlbm_step: graph of 32 steps");
    cudaGraphExec_t& ge = c->graph[c->cur];
    if (!ge) {
      NvtxRange capture("hlbm_step: capture and instantiate");
      const int cur0 = c->cur;
      HLBM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
      cudaError_t le = cudaSuccess;
      for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k) le = one_step(c);
      cudaGraph_t gr = nullptr;
      cudaError_t ce = cudaStreamEndCapture(c->stream, &gr);
      c->cur = cur0;
      if (le != cudaSuccess) return cuda_fail(c, le, "step kernel (capture)");
      if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
      cudaError_t ie = cudaGraphInstantiate(&ge, gr, 0);
      cudaGraphDestroy(gr);
      if (ie != cudaSuccess) {
        ge = nullptr;
        return cuda_fail(c, ie, "cudaGraphInstantiate");
      }
    }
    HLBM_CUDA(c, cudaGraphLaunch(ge, c->stream), "cudaGraphLaunch");
    n -= kGraphSteps;
    c->steps += kGraphSteps;
  }
  if (n > 0) {
    NvtxRange chunk("hlbm_step: single launches");
    for (int k = 0; k < n; ++k) {
      cudaError_t e = one_step(c);
      if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
      c->steps += 1;
    }
  }
  return HLBM_OK;
}

hlbm_status hlbm_moments(hlbm_ctx* c, float* rho, float* u, float* theta, int on_device) {
  NvtxRange range("hlbm_moments");
  hlbm_status st = usable(c);
  if (st != HLBM_OK) return st;
  if (!c->initialised) return fail(c, HLBM_ESTATE, "hlbm_init has not been called");
  StepArgs a = make_args(c);
  a.fin = c->pop[c->cur];
  const size_t n = (size_t)c->N;
  float* stage = nullptr;
  if (on_device) {
    a.rho_out = rho;
    a.u_out = u;
    a.theta_out = theta;
  } else {
    // stage in the population buffer that does not hold the current state
    // (in place: the staging area)
    stage = static_cast<float*>(c->pop[c->aa ? 1 : (c->cur ^ 1)]);
    a.rho_out = stage;
    a.u_out = stage + n;
    a.theta_out = stage + (1 + c->D) * n;
  }
  cudaError_t e;
  if (c->walls) {
    WallArgs w = make_wall_args(c);
    w.rho_out = a.rho_out;
    w.u_out = a.u_out;
    w.theta_out = a.theta_out;
    e = launch_walls(w, c->storage, 2, false, c->stream);
    if (e == cudaSuccess) e = launch_walls(w, c->storage, 0, false, c->stream);
  } else if (c->aa) {
    e = aa_step(c, true, &a);
  } else {
    e = launch_step(c, a, true);
  }
  if (e == cudaSuccess && !on_device) {
    if (rho) e = cudaMemcpyAsync(rho, stage, n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, stage + n, c->D * n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && theta)
      e = cudaMemcpyAsync(theta, stage + (1 + c->D) * n, n * 4, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "moments");
  return on_device ? HLBM_OK : check_status(c);
}

hlbm_status hlbm_diag(hlbm_ctx* c, double* out) {
  NvtxRange range("hlbm_diag");
  hlbm_status st = usable(c);
  if (st != HLBM_OK) return st;
  if (!out) return HLBM_EINVAL;
  if (!c->initialised) return fail(c, HLBM_ESTATE, "hlbm_init has not been called");
  StepArgs a = make_args(c);
  a.fin = c->pop[c->cur];
  a.partials = c->partials;
  if (c->walls) {
    WallArgs w = make_wall_args(c);
    w.partials = c->partials;
    HLBM_CUDA(c, launch_walls(w, c->storage, 2, false, c->stream), "wall completion kernel");
    HLBM_CUDA(c, launch_walls(w, c->storage, 0, false, c->stream), "moments kernel");
  } else if (c->aa) {
    HLBM_CUDA(c, aa_step(c, true, &a), "moments kernel");
  } else {
    HLBM_CUDA(c, launch_step(c, a, true), "moments kernel");
  }
  const int nb = moment_blocks(c->lattice, c->nx, c->ny, c->nz);
  HLBM_CUDA(c, launch_reduce_partials(c->partials, nb, c->red, c->stream), "reduce kernel");
  double s[8];
  HLBM_CUDA(c, cudaMemcpyAsync(s, c->red, sizeof(s), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if ((st = check_status(c)) != HLBM_OK) return st;
  const double cs2 = c->lattice == 0 ? D2Q37::cs2 : D3Q39::cs2;
  const double Nn = (double)c->N;
  out[0] = Nn * c->p.rho0 + s[0];
  for (int d = 0; d < c->D; ++d) out[1 + d] = s[1 + d];
  out[1 + c->D] = 0.5 * Nn * c->p.rho0 * c->D * cs2 + s[4];
  if (s[5] > 0.0) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "diverged: %.0f nodes with non-finite moments or rho <= 0", s[5]);
    return fail(c, HLBM_EDIVERGED, buf, true);
  }
  return HLBM_OK;
}

size_t hlbm_state_bytes(const hlbm_ctx* c) {
  if (!c) return 0;
  return 64 + (size_t)c->Q * (size_t)c->N * c->elem + (c->walls ? (size_t)16 * (size_t)c->N : 0) +
         (c->aa ? (size_t)4 * (size_t)c->N : 0);
}

hlbm_status hlbm_save(hlbm_ctx* c, void* host_buf, size_t bytes) {
  NvtxRange range("hlbm_save");
  hlbm_status st = usable(c);
  if (st != HLBM_OK) return st;
  if (!host_buf || bytes < hlbm_state_bytes(c)) return fail(c, HLBM_EINVAL, "buffer too small");
  if (!c->initialised) return fail(c, HLBM_ESTATE, "hlbm_init has not been called");
  long long hdr[8] = {0x484c424d31LL, c->lattice, c->nx, c->ny, c->nz, c->storage, c->steps, 0};
  std::memcpy(host_buf, hdr, sizeof(hdr));
  const size_t pbytes = (size_t)c->Q * c->N * c->elem;
  HLBM_CUDA(c, cudaMemcpyAsync(static_cast<char*>(host_buf) + 64, c->pop[c->aa ? 0 : c->cur], pbytes,
                               cudaMemcpyDeviceToHost,
                               c->stream), "cudaMemcpyAsync");
  if (c->walls)   // the wall targets: the previous step's moments
    HLBM_CUDA(c, cudaMemcpyAsync(static_cast<char*>(host_buf) + 64 + pbytes, c->mom[c->cur], (size_t)16 * c->N,
                                 cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if (c->aa)      // the neighbour field the next step reads (the step parity is in the step count)
    HLBM_CUDA(c, cudaMemcpyAsync(static_cast<char*>(host_buf) + 64 + pbytes, c->aux[c->cur ^ 1], (size_t)4 * c->N,
                                 cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  HLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return HLBM_OK;
}

hlbm_status hlbm_load(hlbm_ctx* c, const void* host_buf, size_t bytes) {
  NvtxRange range("hlbm_load");
  if (!c || !host_buf) return HLBM_EINVAL;
  if (bytes < hlbm_state_bytes(c)) return fail(c, HLBM_EINVAL, "buffer too small");
  long long hdr[8];
  std::memcpy(hdr, host_buf, sizeof(hdr));
  if (hdr[0] != 0x484c424d31LL || hdr[1] != c->lattice || hdr[2] != c->nx || hdr[3] != c->ny || hdr[4] != c->nz ||
      hdr[5] != c->storage)
    return fail(c, HLBM_EINVAL, "checkpoint does not match this context");
  c->failed = false;
  hlbm_status st = ensure_memory(c);
  if (st != HLBM_OK) return st;
  if ((st = ensure_stream(c)) != HLBM_OK) return st;
  carve(c);
  if (c->lattice == 0) HLBM_CUDA(c, configure_step_d2q37(c->storage), "cudaFuncSetAttribute");
  const size_t pbytes = (size_t)c->Q * c->N * c->elem;
  HLBM_CUDA(c, cudaMemcpyAsync(c->pop[0], static_cast<const char*>(host_buf) + 64, pbytes, cudaMemcpyHostToDevice,
                               c->stream), "cudaMemcpyAsync");
  if (c->walls)
    HLBM_CUDA(c, cudaMemcpyAsync(c->mom[0], static_cast<const char*>(host_buf) + 64 + pbytes, (size_t)16 * c->N,
                                 cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
  const int par = c->aa ? (int)(hdr[6] & 1) : 0;   // in place: the layout of the saved step's parity
  if (c->aa)
    HLBM_CUDA(c, cudaMemcpyAsync(c->aux[par ^ 1], static_cast<const char*>(host_buf) + 64 + pbytes, (size_t)4 * c->N,
                                 cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
  HLBM_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "cudaMemsetAsync");
  HLBM_CUDA(c, cudaMemsetAsync(c->tile_ctr, 0, sizeof(unsigned long long), c->stream), "cudaMemsetAsync");
  if (c->flags) HLBM_CUDA(c, cudaMemsetAsync(c->flags, 0, c->nflags * 4, c->stream), "cudaMemsetAsync");
  HLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  c->cur = par;
  c->gen = 0;
  c->steps = hdr[6];
  drop_graphs(c);
  c->initialised = true;
  return HLBM_OK;
}

long long hlbm_step_count(const hlbm_ctx* c) { return c ? c->steps : -1; }

hlbm_status hlbm_set_tile(hlbm_ctx* c, int rows, int nodes_per_thread, int persistent) {
  if (!c) return HLBM_EINVAL;
  if (persistent < 0 || persistent > 3)
    return fail(c, HLBM_EINVAL, "persistent must be 0 (default off), 1 (off), 2 (on) or 3 (multi-step)");
  if (rows == 0) rows = 8;
  if (nodes_per_thread == 0) nodes_per_thread = 2;
  if (rows != 4 && rows != 8 && rows != 16) return fail(c, HLBM_EINVAL, "rows must be 4, 8 or 16");
  if (nodes_per_thread != 1 && nodes_per_thread != 2) return fail(c, HLBM_EINVAL, "nodes_per_thread must be 1 or 2");
  if (nodes_per_thread == 2 && rows == 4) return fail(c, HLBM_EINVAL, "two nodes per thread need 8 or 16 rows");
  if (c->lattice == 1 && rows == 16) return fail(c, HLBM_EINVAL, "D3Q39 tiles have 4 or 8 rows");
  c->rows = rows;
  c->npt = nodes_per_thread;
  c->persistent = (persistent >= 2) ? 1 : 0;
  c->multistep = persistent == 3 && c->lattice == HLBM_D2Q37;
  c->ctr_reset = true;
  drop_graphs(c);
  return HLBM_OK;
}

hlbm_status hlbm_synchronize(hlbm_ctx* c) {
  if (!c) return HLBM_EINVAL;
  if (!c->stream) return HLBM_OK;
  HLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (c->status && c->initialised) return check_status(c);
  return HLBM_OK;
}

hlbm_status hlbm_set_wait_timeout(hlbm_ctx* c, double seconds) {
  if (!c || !std::isfinite(seconds) || !(seconds > 0) || seconds > 60) return HLBM_EINVAL;
  c->wait_ns = (unsigned long long)(seconds * 1e9);
  drop_graphs(c);
  return HLBM_OK;
}

const char* hlbm_last_error(const hlbm_ctx* c) { return c ? c->msg.c_str() : "null context"; }

hlbm_status hlbm_destroy(hlbm_ctx* c) {
  if (!c) return HLBM_EINVAL;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->own_arena && c->arena) cudaFree(c->arena);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return HLBM_OK;
}

namespace {
struct AdjLayout {
  size_t state, nseg, nstates, off_lam0, off_lam1, off_part, total;
};
AdjLayout adj_layout(const hlbm_ctx* c, int steps, int K) {
  AdjLayout L{};
  L.state = align256((size_t)c->Q * (size_t)c->N * c->elem);
  L.nseg = (size_t)((steps + K - 1) / K);
  L.nstates = L.nseg + (size_t)(K - 1);  // checkpoints + recomputed states of one segment
  const size_t lam = align256((size_t)c->Q * (size_t)c->N * 4);
  L.off_lam0 = L.nstates * L.state;
  L.off_lam1 = L.off_lam0 + lam;
  L.off_part = L.off_lam1 + lam;
  L.total = L.off_part + align256(((size_t)adjoint_seed_blocks(c->N) + 1) * 8 * sizeof(double));
  return L;
}
}  // namespace

size_t hlbm_adjoint_workspace_bytes(const hlbm_ctx* c, int steps, int ckpt_every) {
  if (!c || steps < 1 || ckpt_every < 1) return 0;
  return adj_layout(c, steps, std::min(ckpt_every, steps)).total;
}

hlbm_status hlbm_adjoint_run(hlbm_ctx* c, int steps, int ckpt_every, void* workspace, size_t bytes, float* dLdg,
                             double* loss) {
  NvtxRange range("hlbm_adjoint_run");
  hlbm_status st = usable(c);
  if (st != HLBM_OK) return st;
  if (!c->initialised) return fail(c, HLBM_ESTATE, "hlbm_init has not been called");
  if (steps < 1 || ckpt_every < 1 || !workspace || !dLdg || !loss) return fail(c, HLBM_EINVAL, "bad adjoint arguments");
  if (c->force_mode != FORCE_FIELD)
    return fail(c, HLBM_EINVAL, "the gradient is taken with respect to a force field: call hlbm_set_force_field(kind 1)");
  if (c->p.flags & (HLBM_SRC_H | HLBM_SRC_SC | HLBM_WALLS | HLBM_AA))
    return fail(c, HLBM_EUNSUPPORTED, "the adjoint covers the periodic body-force step on two buffers");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return fail(c, HLBM_EINVAL, "workspace must be 256-byte aligned");
  const int K = std::min(ckpt_every, steps);
  const AdjLayout L = adj_layout(c, steps, K);
  if (bytes < L.total) return fail(c, HLBM_ENOMEM, "adjoint workspace smaller than hlbm_adjoint_workspace_bytes()");
  // a map depends only on (address, box, type, extent), so maps of an earlier
  // run's workspace stay valid for a workspace at the same address; the cache
  // is only trimmed back to the context's own buffers when it grows large
  if (c->tmaps.size() > 8192) {
    std::deque<hlbm_ctx::TMap> keep;
    for (const auto& t : c->tmaps)
      if (t.base == c->pop[0] || t.base == c->pop[1]) keep.push_back(t);
    c->tmaps.swap(keep);
  }
  char* ws = static_cast<char*>(workspace);
  auto state = [&](size_t k) { return static_cast<void*>(ws + k * L.state); };
  float* lam[2] = {reinterpret_cast<float*>(ws + L.off_lam0), reinterpret_cast<float*>(ws + L.off_lam1)};
  double* part = reinterpret_cast<double*>(ws + L.off_part);
  const size_t sbytes = (size_t)c->Q * (size_t)c->N * c->elem;
  const int thermal = (c->p.flags & HLBM_ISOTHERMAL) ? 0 : 1;
  const float rho0 = (float)c->p.rho0, omega = (float)(1.0 / c->tau_hat), beta = (float)(1.0 - 0.5 / c->tau_hat);
  // forward: checkpoint k is the state before step k K (its gather is f_{kK})
  const int nseg = (int)L.nseg;
  // K = 1 keeps every state: step k reads slot k and writes slot k + 1, slot 0
  // being the current buffer and slot T the other one (the final state, as
  // after hlbm_step), so there is neither a checkpoint copy nor a recompute
  const int cur0 = c->cur;
  auto slot = [&](int k) -> void* { return k == 0 ? c->pop[cur0] : (k == steps ? c->pop[cur0 ^ 1] : state(k)); };
  {
    NvtxRange fwd("adjoint: forward sweep with checkpoints");
    if (K == 1) {
      for (int k = 0; k < steps; ++k) {
        StepArgs a = make_args(c);
        a.fin = slot(k);
        a.fout = slot(k + 1);
        a.reverse = k & 1;
        HLBM_CUDA(c, launch_step(c, a, false), "forward step");
      }
      c->cur = cur0 ^ 1;
      c->steps += steps;
    } else {
      for (int k = 0; k < nseg; ++k) {
        HLBM_CUDA(c, cudaMemcpyAsync(state(k), c->pop[c->cur], sbytes, cudaMemcpyDeviceToDevice, c->stream),
                  "checkpoint");
        const int len = std::min(K, steps - k * K);
        for (int j = 0; j < len; ++j) HLBM_CUDA(c, one_step(c), "forward step");
        c->steps += len;
      }
    }
  }
  // seed from the final state: lambda_T, dL/dg at T, kinetic energy
  const AdjRows gather_only{nullptr, c->status, c->wait_ns, nullptr};
  HLBM_CUDA(c, launch_adjoint(c->lattice, c->storage, true, c->pop[c->cur], nullptr, lam[0], c->gfield, dLdg, part,
                              c->N, c->nx, c->ny, c->nz, rho0, omega, beta, thermal, gather_only, c->stream),
            "adjoint seed");
  // D3Q39 whole-row reverse kernel: tiles of 256 / nx rows; maps of the
  // forward state (box, row), of lambda_{n+1} (box, row), of the acceleration
  // and of dL/dg (boxes) per launch
  const bool rows = c->lattice == HLBM_D3Q39 && c->tma_ok &&
                    (c->nx == 32 || c->nx == 64 || c->nx == 128 || c->nx == 256) &&
                    (reinterpret_cast<uintptr_t>(dLdg) & 15) == 0;
  if (rows) HLBM_CUDA(c, cudaMemsetAsync(c->adj_ctr, 0, sizeof(unsigned long long), c->stream), "cudaMemsetAsync");
  auto rows_of = [&](const void* fwd, const float* lin, CUtensorMap (&m)[6]) {
    AdjRows r{nullptr, c->status, c->wait_ns, c->adj_ctr};
    if (!rows) return r;
    const int hb = 256 / c->nx;
    const CUtensorMap* p[6] = {tensor_map_at(c, fwd, c->nx, hb), tensor_map_at(c, fwd, c->nx, 1),
                               tensor_map_at(c, lin, c->nx, hb, true), tensor_map_at(c, lin, c->nx, 1, true),
                               tensor_map_at(c, c->gfield, c->nx, hb, true, 3),
                               tensor_map_at(c, dLdg, c->nx, hb, true, 3)};
    for (int i = 0; i < 6; ++i) {
      if (!p[i]) return r;
      m[i] = *p[i];
    }
    r.tmaps = m;
    return r;
  };
  const int nb = adjoint_seed_blocks(c->N);
  HLBM_CUDA(c, launch_reduce_partials(part, nb, part + (size_t)nb * 8, c->stream), "reduce");
  int cur = 0;
  // backward over segments: recompute the segment's states, then reverse steps
  for (int k = nseg - 1; k >= 0; --k) {
    NvtxRange segment("adjoint: segment (recompute, reverse steps)");
    const int len = std::min(K, steps - k * K);
    // states of the segment: j = 0 is checkpoint k, j >= 1 are recomputed into slots nseg + j - 1
    auto seg = [&](int j) { return j == 0 ? (K == 1 ? slot(k) : state(k)) : state((size_t)nseg + j - 1); };
    for (int j = 1; j < len; ++j) {
      StepArgs a = make_args(c);   // staged by tensor maps of the workspace slots
      a.fin = seg(j - 1);
      a.fout = seg(j);
      HLBM_CUDA(c, launch_step(c, a, false), "recompute step");
    }
    for (int j = len - 1; j >= 0; --j) {
      CUtensorMap m[6];
      const AdjRows r = rows_of(seg(j), lam[cur], m);
      HLBM_CUDA(c, launch_adjoint(c->lattice, c->storage, false, seg(j), lam[cur], lam[cur ^ 1], c->gfield, dLdg,
                                  nullptr, c->N, c->nx, c->ny, c->nz, rho0, omega, beta, thermal, r, c->stream),
                "adjoint step");
      cur ^= 1;
    }
  }
  HLBM_CUDA(c, cudaMemcpyAsync(loss, part + (size_t)nb * 8, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
            "cudaMemcpyAsync");
  return check_status(c);
}

int hlbm_lattice_info(int lattice, int* cvec, double* w, double* cs2) {
  if (lattice == HLBM_D2Q37) {
    for (int i = 0; i < 37; ++i) {
      if (cvec)
        for (int a = 0; a < 3; ++a) cvec[3 * i + a] = D2Q37::c(i, a);
      if (w) w[i] = D2Q37::w(i);
    }
    if (cs2) *cs2 = D2Q37::cs2;
    return 37;
  }
  if (lattice == HLBM_D3Q39) {
    for (int i = 0; i < 39; ++i) {
      if (cvec)
        for (int a = 0; a < 3; ++a) cvec[3 * i + a] = D3Q39::c(i, a);
      if (w) w[i] = D3Q39::w(i);
    }
    if (cs2) *cs2 = D3Q39::cs2;
    return 39;
  }
  return 0;
}

hlbm_status hlbm_debug_record(unsigned long long* out, int clear) {
#ifdef HLBM_DEBUG
  if (!out) return HLBM_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return HLBM_ECUDA;
  return debug_record(out, clear != 0) ? HLBM_OK : HLBM_ECUDA;
#else
  (void)out;
  (void)clear;
  return HLBM_EUNSUPPORTED;
#endif
}

}  // extern "C"
