// Initialisation (f^_i = f^eq_i, written pre-streamed for the pull scheme),
// the FP64 reduction of per-block diagnostics, and launch dispatch by
// lattice and storage.
#include "step_common.cuh"

#include <mutex>
#include <vector>

namespace hlbm {

cudaError_t launch_step2d_f32(const StepArgs&, int, bool, int, int, const CUtensorMap*, cudaStream_t);
cudaError_t launch_step2d_f16(const StepArgs&, int, bool, int, int, const CUtensorMap*, cudaStream_t);
cudaError_t launch_step2d_bf16(const StepArgs&, int, bool, int, int, const CUtensorMap*, cudaStream_t);
cudaError_t configure_step2d_f32();
cudaError_t configure_step2d_f16();
cudaError_t configure_step2d_bf16();
void box_step2d_f32(int, bool, int, int*, int*, int*);
void box_step2d_f16(int, bool, int, int*, int*, int*);
void box_step2d_bf16(int, bool, int, int*, int*, int*);
cudaError_t launch_step3d_f32(const StepArgs&, int, bool, int, int, const CUtensorMap*, cudaStream_t);
cudaError_t launch_step3d_f16(const StepArgs&, int, bool, int, int, const CUtensorMap*, cudaStream_t);
cudaError_t launch_step3d_bf16(const StepArgs&, int, bool, int, int, const CUtensorMap*, cudaStream_t);

cudaError_t launch_step_d2q37(const StepArgs& a, int kind, int storage, bool mom, int rows, int npt,
                              const CUtensorMap* tm, cudaStream_t s) {
  switch (storage) {
    case ST_F32: return launch_step2d_f32(a, kind, mom, rows, npt, tm, s);
    case ST_F16: return launch_step2d_f16(a, kind, mom, rows, npt, tm, s);
    case ST_BF16: return launch_step2d_bf16(a, kind, mom, rows, npt, tm, s);
  }
  return cudaErrorInvalidValue;
}

// Kernel attributes (dynamic shared memory) belong to the device's context:
// set once per device and storage (concurrent first calls set them twice,
// which is harmless).
cudaError_t configure_step_d2q37(int storage) {
  static std::atomic<int> done[3][kMaxDevicesCached];
  if (storage < 0 || storage > 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  per_device_cached(done[storage], [&](int) {
    e = storage == ST_F32   ? configure_step2d_f32()
        : storage == ST_F16 ? configure_step2d_f16()
                            : configure_step2d_bf16();
    return e == cudaSuccess ? 1 : 0;
  });
  return e;
}

namespace {
std::vector<bool (*)(unsigned long long*, bool)>& dbg_readers() {
  static std::vector<bool (*)(unsigned long long*, bool)> r;
  return r;
}
std::mutex& dbg_mutex() {
  static std::mutex m;
  return m;
}
}  // namespace

bool dbg_register(bool (*reader)(unsigned long long*, bool)) {
  std::lock_guard<std::mutex> lock(dbg_mutex());
  dbg_readers().push_back(reader);
  return true;
}

// The debug build's records of rejected indices (step_common.cuh): summed
// count and the first non-empty record, optionally cleared; false in the
// release build (no unit registers a reader there).
bool debug_record(unsigned long long* out, bool clear) {
  std::lock_guard<std::mutex> lock(dbg_mutex());
  if (dbg_readers().empty()) return false;
  out[0] = out[1] = out[2] = out[3] = 0;
  for (auto* rd : dbg_readers()) {
    unsigned long long r[4];
    if (!rd(r, clear)) return false;
    if (r[0] && !out[0]) {
      out[1] = r[1];
      out[2] = r[2];
      out[3] = r[3];
    }
    out[0] += r[0];
  }
  return true;
}

void step_box_d2q37(int kind, int storage, bool mom, int rows, int* wb, int* hb, int* ob) {
  switch (storage) {
    case ST_F32: box_step2d_f32(kind, mom, rows, wb, hb, ob); return;
    case ST_F16: box_step2d_f16(kind, mom, rows, wb, hb, ob); return;
    default: box_step2d_bf16(kind, mom, rows, wb, hb, ob); return;
  }
}

cudaError_t launch_step_d3q39(const StepArgs& a, int kind, int storage, bool mom, int rows, int npt,
                              const CUtensorMap* tm, cudaStream_t s) {
  switch (storage) {
    case ST_F32: return launch_step3d_f32(a, kind, mom, rows, npt, tm, s);
    case ST_F16: return launch_step3d_f16(a, kind, mom, rows, npt, tm, s);
    case ST_BF16: return launch_step3d_bf16(a, kind, mom, rows, npt, tm, s);
  }
  return cudaErrorInvalidValue;
}

int moment_blocks(int lattice, int nx, int ny, int nz) {
  return ((nx + 31) / 32) * ((ny + 7) / 8) * (lattice == 1 ? nz : 1);
}

// The pull step reads stored_i(x - c_i); so that the first step sees
// f^eq(x), node x writes its equilibrium to stored_i(x - c_i).
template <class L, int ST>
__global__ void __launch_bounds__(256) init_kernel(const __grid_constant__ InitArgs a) {
  using C = Codec<ST>;
  using T = typename C::T;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
  NodeSrc s;
  const float rho = a.rho[n];
  s.dr = rho - a.rho0;
  s.rho = rho;
  s.tb = a.theta[n] - 1.f;
  constexpr float inv_c0 = (float)(1.0 / L::c0);
  for (int d = 0; d < 3; ++d) {
    s.u[d] = (d < L::D) ? a.u[(size_t)d * a.N + n] * inv_c0 : 0.f;
    s.F[d] = 0.f;
    s.hG[d] = 0.f;
  }
  s.sigma = 0.f;
  float g[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) g[i] = 0.f;
  if constexpr (L::D == 2) {
    float K[15];
    poly2<L>(s, 1.f, 0.f, K);
    apply_poly<L, 15>(g, K, 0.f);
  } else {
    float K[20];
    poly3<L>(s, 1.f, 0.f, K);
    apply_poly<L, 20>(g, K, 0.f);
  }
  T* __restrict__ fout = static_cast<T*>(a.fout);
  static_for<L::Q>([&](auto I) {
    constexpr int i = I;
    const int xs = wrap1(x - L::c(i, 0), nx), ys = wrap1(y - L::c(i, 1), ny);
    const int zs = (L::D == 3) ? wrap1(z - L::c(i, 2), nz) : 0;
    C::st(fout + (size_t)i * (size_t)a.N + ((size_t)zs * ny + ys) * nx + xs, g[i]);
  });
}

template <class L>
static cudaError_t launch_init_l(const InitArgs& a, int storage, cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.N + 255) / 256);
  switch (storage) {
    case ST_F32: init_kernel<L, ST_F32><<<blocks, 256, 0, s>>>(a); break;
    case ST_F16: init_kernel<L, ST_F16><<<blocks, 256, 0, s>>>(a); break;
    case ST_BF16: init_kernel<L, ST_BF16><<<blocks, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_init(int lattice, const InitArgs& a, int storage, cudaStream_t s) {
  return lattice == 0 ? launch_init_l<D2Q37>(a, storage, s) : launch_init_l<D3Q39>(a, storage, s);
}

// out[k] = sum over blocks of partials[b][k], k < 8, in FP64 (one CTA).
__global__ void __launch_bounds__(256) reduce_partials_kernel(const double* __restrict__ partials, int blocks,
                                                              double* __restrict__ out) {
  __shared__ double red[8][8];
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < blocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] += partials[(size_t)b * 8 + k];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 8; ++k) red[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x < 8) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

cudaError_t launch_reduce_partials(const double* partials, int blocks, double* out, cudaStream_t s) {
  reduce_partials_kernel<<<1, 256, 0, s>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace hlbm
