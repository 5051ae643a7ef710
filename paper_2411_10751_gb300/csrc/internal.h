// Kernel argument blocks and launcher declarations shared by the CUDA
// translation units of libhlbm (not part of the public C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <atomic>
#include <cstdint>

namespace hlbm {

// NVTX range over a host scope (entry points, step chunks, adjoint sweeps and
// segments), shown on the timeline by Nsight Systems and usable as an ncu
// range filter; without an attached tool a push or pop is one test of an
// unset function pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// A per-device value (a kernel's resident-CTA count) computed once per device:
// compute(dev) runs on the first call with that device current; concurrent
// first calls compute the same value, and the atomic keeps the store free of
// data races.
constexpr int kMaxDevicesCached = 64;
template <class F>
int per_device_cached(std::atomic<int> (&cache)[kMaxDevicesCached], F&& compute) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDevicesCached) return compute(dev);
  int n = cache[dev].load(std::memory_order_relaxed);
  if (!n) {
    n = compute(dev);
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

enum Kind : int {
  KIND_LOCAL = 0,    // sources need only the node itself (F_i)
  KIND_THERMAL = 1,  // + H_i: theta of the 2D / 3D nearest neighbours
  KIND_SC = 2        // + F^SC (and P_i): psi of the reach-3 neighbourhood
};
enum Storage : int { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };
enum ForceMode : int { FORCE_NONE = 0, FORCE_UNIFORM = 1, FORCE_FIELD = 2, FORCE_PROFILE_Y = 3 };

// Arguments of the fused step / moments kernels (passed as a grid constant).
struct StepArgs {
  const void* fin;        // populations at time t (post-collision state of t-1), [Q][N]
  void* fout;             // populations written by this step, [Q][N]
  const float* gfield;    // FORCE_FIELD: [D][N]; FORCE_PROFILE_Y: [D][ny]
  float* rho_out;         // moments mode outputs (may be null)
  float* u_out;
  float* theta_out;
  double* partials;       // moments mode: per-block FP64 sums [blocks][8] (may be null)
  long long N;            // nodes
  int nx, ny, nz;
  int force_mode;
  int isothermal;
  float rho0;
  float omega;            // 1 / tau^
  float beta;             // 1 - 1 / (2 tau^)
  float g[3];             // uniform acceleration
  float h_coef;           // 1 - 1/Pr (H_i)
  int eos;                // 0 van der Waals, 1 Carnahan-Starling
  // psi^2 = 2 rho + k1 rho^2 - k2 rho Z(e), e = kb rho (float-float pairs hi, lo):
  // k1 = 2 a / c0^2, k2 = 2 T / c0^2; vdW Z = 1 / (1 - e), kb = b;
  // Carnahan-Starling Z = (1 + e + e^2 - e^3) / (1 - e)^3, kb = b / 4
  float psi_k1[2], psi_k2[2], psi_kb[2];
  float p_coef;           // trace coefficient of P_i: sigma = p_coef |F^SC|^2 / psi^2
  int* status;            // device status word: set to HLBM_ETIMEOUT when a bounded wait expires
  int tma;                // 1: interior tiles are staged by TMA (input tensor map valid)
  int tma_store;          // 1: results are written by TMA (output tensor map valid)
  int persistent;         // 1: persistent CTAs that prefetch their next tile (2D step)
  unsigned long long* tile_ctr;  // persistent step: tile counter; each launch takes exactly tiles + CTAs values
  unsigned long long wait_ns;  // wall-time limit of a bounded mbarrier wait
  int debug_skip_tma;     // test hook: arm the barrier but issue no copy (the wait must expire)
  int reverse;            // persistent step: take the tiles in reverse order (set on every other step)
  int g_staged;           // D3Q39 whole-row step: the force field is staged with the tiles (third tensor map)
  // multi-step persistent 2D kernel: steps of this launch (step s reads fin
  // for even s, fout for odd s), steps run before it since the counters were
  // zeroed, per-tile-row completion counters and the launch's tile counter
  // (zeroed)
  int msteps;
  unsigned gen0;
  unsigned* flags;
  unsigned long long* ms_ctr;
  // in-place (AA) step: the previous step's neighbour field (theta - 1 or psi)
  // read on the tile's frame, and this step's written per node
  const float* aux_rd;
  float* aux_wr;
};

// Arguments of the wall-bounded D2Q37 step (walls.cu): moments and collide
// launches of one step.
struct WallArgs {
  const void* fin;        // post-collision state of step t - 1, [Q][N]
  void* fout;             // collide: state written by this step
  const float* mprev;     // [4][N] rho, u_x, u_y, theta - 1 of the previous step (completed)
  float* mcur;            // moments: this step's [4][N] (may be null); collide: read for grad theta
  float* rho_out;         // moments readout (may be null)
  float* u_out;
  float* theta_out;
  double* partials;       // moments: per-block FP64 sums [blocks][8] (may be null)
  const float* gfield;
  int force_mode;
  float g[3];
  long long N;
  int nx, ny;
  float rho0;
  float omega, beta;
  float h_coef;           // 1 - 1/Pr (H_i)
  float wall_u[2][2];     // velocity of the bottom (0) and top (1) wall
  float wall_tb[2];       // their temperature minus 1
  float tb_ref;           // reference temperature of the stored deviations minus 1
  float e_ref;            // rho0 D c0^2 tb_ref: energy moment of the reference offset
  float* comp;            // completed unknowns of the six wall rows, [6][37][nx] (slot 3 side + r)
};

// Arguments of the initialisation kernel.
struct InitArgs {
  const float* rho;
  const float* u;
  const float* theta;
  void* fout;
  long long N;
  int nx, ny, nz;
  float rho0;
};

// Launchers (return the launch error).  rows: tile rows per CTA (4, 8, 16);
// tmap: {input map, output map} of the population buffers with the boxes of
// step_box_d2q37 (may be null when a.tma == 0 and a.tma_store == 0).
// npt: nodes per thread (1, or 2 on float2 lanes; 8- and 16-row tiles).
cudaError_t launch_step_d2q37(const StepArgs& a, int kind, int storage, bool moments, int rows, int npt,
                              const CUtensorMap* tmap, cudaStream_t s);
// tmap: {whole-row box, single-row} maps of the input buffer for the persistent
// whole-row kernel (nx = 32, 64, 128, 256), or null.
cudaError_t launch_step_d3q39(const StepArgs& a, int kind, int storage, bool moments, int rows, int npt,
                              const CUtensorMap* tmap, cudaStream_t s);
// Sets the dynamic shared-memory limit of every D2Q37 kernel of a storage type
// (call before the first launch, outside stream capture).
cudaError_t configure_step_d2q37(int storage);
// TMA boxes that launch_step_d2q37 expects: input box wb x hb, output tile
// 32 x ob.
void step_box_d2q37(int kind, int storage, bool moments, int rows, int* wb, int* hb, int* ob);
cudaError_t launch_init(int lattice, const InitArgs& a, int storage, cudaStream_t s);
// Sums per-block partials into out[0..7] (FP64) and the non-finite counter.
cudaError_t launch_reduce_partials(const double* partials, int blocks, double* out, cudaStream_t s);
// Number of CTAs a moments-mode launch with these sizes uses (size of the partials).
int moment_blocks(int lattice, int nx, int ny, int nz);

// In-place D2Q37 step (aa.cu): odd = the step's parity (fin == fout, the one
// population buffer); mom = moments readout (rho_out / u_out / theta_out,
// partials) of the state before that step.  aa_init writes the even layout
// and the first step's neighbour field (a.aux_wr).
cudaError_t launch_aa(const StepArgs& a, int kind, int storage, bool odd, bool mom, cudaStream_t s);
cudaError_t launch_aa_init(const StepArgs& a, int kind, int storage, const float* rho, const float* u,
                           const float* theta, cudaStream_t s);

// Wall-bounded D2Q37 step (walls.cu), in launch order: mode 2 = the FP64
// completion of the wall rows' unknowns into a.comp, mode 0 = the moments
// launch (moments into mcur / the readout pointers, partials), mode 1 = the
// collide launch (thermal: with H_i).  Modes 0 and 1 read a.comp.
cudaError_t launch_walls(const WallArgs& a, int storage, int mode, bool thermal, cudaStream_t s);
// Initial state of a wall-bounded context into a.fout and m [4][N] = rho,
// u_x, u_y, theta - 1 of the initial fields.
cudaError_t launch_wall_init(const WallArgs& a, int storage, const float* rho, const float* u, const float* theta,
                             float* m, cudaStream_t s);

// Adjoint of the body-force step (adjoint.cu).  seed: lambda_T, dL/dg and
// per-block kinetic-energy sums (adjoint_seed_blocks(N) blocks, stride 8) from
// the state `fwd`; otherwise one reverse step lam_in -> lam_out with the
// forward state `fwd` whose gather is f_n, accumulating dL/dg.
// rows: the D3Q39 whole-row reverse kernel's tensor maps (forward state box
// and row, lambda_{n+1} box and row, acceleration box, dL/dg box; null: the
// gather kernel), status word,
// wait bound and tile counter (zero before the first reverse step of a run).
struct AdjRows {
  const CUtensorMap* tmaps;
  int* status;
  unsigned long long wait_ns;
  unsigned long long* ctr;
};
cudaError_t launch_adjoint(int lattice, int storage, bool seed, const void* fwd, const float* lam_in, float* lam_out,
                           const float* gfield, float* dLdg, double* partials, long long N, int nx, int ny, int nz,
                           float rho0, float omega, float beta, int thermal, const AdjRows& rows, cudaStream_t s);
int adjoint_seed_blocks(long long N);

// debug build only (kernels_misc.cu): the records of rejected indices of all
// translation units, summed (count) and the first non-empty one's site,
// index and bound; each unit registers the reader of its own record
bool debug_record(unsigned long long* out, bool clear);
bool dbg_register(bool (*reader)(unsigned long long*, bool));

}  // namespace hlbm
