/*
 * hlbm: one fused time step of the high-order (multi-speed) BGK lattice
 * Boltzmann method with Hermite-polynomial body sources, after
 * S. Li et al., "Constructing the body source for high-order lattice
 * Boltzmann method", on one NVIDIA GB300 (sm_103a).
 *
 * The step (Eq. 4.4 with the shift of Eq. 4.3) on D2Q37 (Sec. 4.1, Table 1)
 * or D3Q39 is
 *     f^_i(x + c_i, t + 1) = f^_i - (f^_i - f^eq_i) / tau^ + (1 - 1 / (2 tau^)) S_i
 * with the 4th-order Hermite equilibrium (Eq. 2.2, 3rd order on D3Q39), the
 * moments of Eq. 4.5 (half-source shift), and S_i = F_i + H_i + P_i:
 *   F_i  body force (Eqs. 3.1-3.3), force density F = rho g + F^SC
 *   H_i  thermal diffusion source setting the Prandtl number (Eqs. 3.4-3.7),
 *        grad theta by second-order central differences
 *   F^SC pseudopotential force (Eq. 3.8) over the lattice's reach-3 stencil
 *   P_i  pressure-tensor source (Eqs. 3.10-3.12)
 * All sources at time t use fields of time t at every node (no time lag).
 * Domains are periodic in every direction, or (D2Q37, HLBM_WALLS) periodic in
 * x between two Tamm-Mott-Smith walls below and above (Sec. 4.3).
 *
 * Conventions
 *   Units: lattice units (dx = dt = 1), integer velocities c_i, lattice
 *     temperature c0^2 theta; tau_hat is the shifted relaxation time tau^,
 *     so the kinematic viscosity is c0^2 theta (tau_hat - 1/2).
 *   Field layout (row-major, x fastest): scalar fields [nz][ny][nx];
 *     vector fields [D][nz][ny][nx] (nz = 1 in 2D).
 *   Memory: "on_device" = 1 means the pointer is CUDA device memory, 0 means
 *     host memory (the call then copies and synchronises its stream).
 *     Input pointers are borrowed for the duration of the call only.
 *   Streams: every call is ordered on the context's stream
 *     (hlbm_set_stream); calls that return host data synchronise it.
 *   Errors: every call returns an hlbm_status; hlbm_last_error gives the
 *     message.  After a CUDA error or a detected divergence the context is
 *     in an error state and further calls return HLBM_ESTATE until it is
 *     destroyed or reloaded with hlbm_load.
 *   Threading: a context must not be used from two threads at once.
 */
#ifndef HLBM_H
#define HLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { HLBM_D2Q37 = 0, HLBM_D3Q39 = 1 } hlbm_lattice;

/* Storage of the populations.  The stored quantity is always the
 * Hermite-normalised deviation g_i = (f^_i - w_i rho0) / w_i; arithmetic is
 * FP32 in every case. */
typedef enum { HLBM_F32 = 0, HLBM_F16 = 1, HLBM_BF16 = 2 } hlbm_storage;

typedef enum {
  HLBM_OK = 0,
  HLBM_EINVAL = 1,       /* invalid argument */
  HLBM_ENOMEM = 2,       /* allocation failed or bound memory too small */
  HLBM_ECUDA = 3,        /* a CUDA call failed */
  HLBM_EDIVERGED = 4,    /* non-finite or non-positive density found */
  HLBM_ETIMEOUT = 5,     /* a bounded device wait expired */
  HLBM_ESTATE = 6,       /* context is in an error state */
  HLBM_EUNSUPPORTED = 7  /* valid request this build does not implement */
} hlbm_status;

/* source flags */
#define HLBM_SRC_FORCE 1u      /* body force F_i (Eq. 3.3), F = rho g */
#define HLBM_SRC_H 2u          /* thermal diffusion source H_i (Eq. 3.7) */
#define HLBM_SRC_SC 4u         /* pseudopotential force F^SC (Eq. 3.8) */
#define HLBM_SRC_P 8u          /* pressure-tensor source P_i (Eq. 3.12), needs SC */
#define HLBM_ISOTHERMAL 16u    /* theta == 1 in f^eq and F_i (Sec. 5.4); required by SC */
/* Walls (Sec. 4.3, Eqs. 4.7-4.8; the cases of Sec. 5.1-5.3), D2Q37 in the
 * thermal mode without F^SC: rows 0 and ny - 1 are wall nodes and the
 * solid-liquid interfaces lie half a cell inside them (y = 1/2, ny - 3/2), so
 * the fluid layer is ny - 2 high; x stays periodic.  After streaming, the
 * populations that come from beyond a wall are replaced, at a node r rows
 * from its wall node, by
 *     f_i = f*_ibar(x) + s f^eq_i(rho_p, u_i, theta_i) - f^eq_ibar(rho_p, u_p, theta_p)
 * (Eq. 4.7): f*_ibar(x) is the population that left x in the opposite
 * direction at the last streaming, (rho_p, u_p, theta_p) the node's moments
 * of the previous step, (u_i, theta_i) the wall's velocity and temperature
 * (params->wall_u, wall_theta) extrapolated linearly from the interface,
 * through the first fluid row's previous moments, to the point where the
 * population turned back (r - |c_iy| / 2 rows from the wall node), and s
 * keeps the mass that left equal to the mass returned (impermeable wall).
 * grad theta for H_i is one-sided into the fluid at the wall rows.  Each step
 * is three launches (the completion of the six wall rows, in FP64; moments;
 * collision); the context keeps the previous step's moments (4 N floats, part
 * of the state that hlbm_save writes) and a 6 x 37 x nx float buffer of
 * completed populations (workspace, rebuilt every step). */
#define HLBM_WALLS 32u
/* In-place step (D2Q37, periodic): one population buffer instead of two (the
 * AA pattern: even steps collide in place and store each result in the
 * opposite velocity's slot of the same node; odd steps read those from the
 * neighbours and store into them), with the single-pass variant of the
 * neighbour fields: grad theta (H_i) and the pseudopotential of F^SC and P_i
 * are taken from the previous step's temperature and density (the fields of
 * time t would need neighbour populations that other threads overwrite in
 * place).  Results differ from the two-pass step by that lag (not with the
 * body force alone, where the two are identical).  Workspace: one buffer, a
 * staging area of 4 N floats and two N-float neighbour fields (1024^2 FP32:
 * 179 MB instead of 310 MB).  hlbm_population_sums_noalloc reads its totals
 * only after an even number of steps (odd steps leave each population in its
 * opposite's slot).  Not with HLBM_WALLS, the adjoint or the batched step. */
#define HLBM_AA 64u

typedef struct {
  uint32_t flags;     /* HLBM_SRC_* | HLBM_ISOTHERMAL | HLBM_WALLS | HLBM_AA */
  double force[3];    /* uniform acceleration g when no force field is set */
  double Pr;          /* Prandtl number for H_i (Sec. 3.2), > 0 */
  int eos;            /* 0: van der Waals p = rho T/(1 - b rho) - a rho^2;
                         1: Carnahan-Starling (Eq. 5.9), R = 1 */
  double eos_a, eos_b, eos_T;  /* EOS parameters a, b and temperature T */
  double k;           /* free parameter k of Eq. 3.12 */
  double rho0;        /* reference density of the stored deviations, > 0 */
  int storage;        /* hlbm_storage */
  double wall_u[2][3];    /* HLBM_WALLS: velocity of the bottom (0) and top (1) wall, x only */
  double wall_theta[2];   /* HLBM_WALLS: their temperature theta, > 0 */
} hlbm_source_params;

typedef struct hlbm_ctx hlbm_ctx;

/* Bytes of device memory a context needs (two population buffers, the force
 * field when HLBM_SRC_FORCE is set, diagnostics scratch).  0 on bad input. */
size_t hlbm_workspace_bytes(int lattice, int nx, int ny, int nz, const hlbm_source_params* p);

/* Creates a context.  nx, ny (and nz for D3Q39) >= 7 so that the reach-3
 * velocities do not alias on the periodic grid; nz must be 1 for D2Q37;
 * nx*ny*nz < 2^31; tau_hat > 1/2.  HLBM_SRC_SC requires HLBM_ISOTHERMAL,
 * HLBM_SRC_H forbids it.  No device memory is allocated until the first call
 * that needs it (or hlbm_bind_memory). */
hlbm_status hlbm_create(int lattice, int nx, int ny, int nz, double tau_hat,
                        const hlbm_source_params* params, hlbm_ctx** out);

/* Uses caller-owned device memory of at least hlbm_workspace_bytes() bytes,
 * 256-byte aligned, instead of allocating.  The caller keeps it alive until
 * hlbm_destroy.  Must precede hlbm_init. */
hlbm_status hlbm_bind_memory(hlbm_ctx* ctx, void* dev_ptr, size_t bytes);

/* Orders all work of the context on this cudaStream_t (0: a private stream
 * that synchronises with the legacy default stream). */
hlbm_status hlbm_set_stream(hlbm_ctx* ctx, void* cuda_stream);

/* The cudaStream_t the context orders its work on (its private stream is
 * created here if none was set); NULL on error.  Lets callers time or
 * order their own work against the context's. */
void* hlbm_get_stream(hlbm_ctx* ctx);

/* Initial state f^_i = f^eq_i(rho, u, theta) with no non-equilibrium part.
 * rho, theta: [nz][ny][nx]; u: [D][nz][ny][nx]; FP32. Resets the step count. */
hlbm_status hlbm_init(hlbm_ctx* ctx, const float* rho, const float* u, const float* theta,
                      int on_device);

/* Body-force acceleration field (F = rho g).  kind 0: none (the uniform
 * params->force is used); kind 1: full field [D][nz][ny][nx]; kind 2: a
 * profile along y, [D][ny] (the same at every x and z).  The data are copied. */
hlbm_status hlbm_set_force_field(hlbm_ctx* ctx, const float* g, int kind, int on_device);

/* Advances n >= 0 time steps, asynchronously on the context's stream. */
hlbm_status hlbm_step(hlbm_ctx* ctx, int n);

/* rho, u, theta at the current time (Eq. 4.5, theta from the moments even in
 * isothermal mode).  Any output pointer may be NULL. */
hlbm_status hlbm_moments(hlbm_ctx* ctx, float* rho, float* u, float* theta, int on_device);

/* FP64 sums over the domain: out[0] mass sum rho, out[1..D] momentum
 * sum rho u, out[D+1] energy sum rho (|u|^2 + D c0^2 theta) / 2 (Eq. 2.3
 * invariants).  Synchronises.  Returns HLBM_EDIVERGED (and enters the error
 * state) if any node has a non-finite moment or rho <= 0. */
hlbm_status hlbm_diag(hlbm_ctx* ctx, double* out);

/* Checkpoint: size in bytes, then a copy of the populations and step count
 * into / out of host memory.  save/load synchronise; load clears the error
 * state.  A run of a + b steps equals a steps, save, load, b steps, bit for bit. */
size_t hlbm_state_bytes(const hlbm_ctx* ctx);
hlbm_status hlbm_save(hlbm_ctx* ctx, void* host_buf, size_t bytes);
hlbm_status hlbm_load(hlbm_ctx* ctx, const void* host_buf, size_t bytes);

/* Steps taken since hlbm_init / hlbm_load. */
long long hlbm_step_count(const hlbm_ctx* ctx);

/* Schedule of the fused periodic step (wall-bounded contexts accept and
 * ignore it: they have one schedule): tile rows per CTA (2D: 4, 8 or 16; D3Q39: 4
 * or 8; 0 = default 8), nodes per thread (1, or 2 on paired FP32 lanes
 * with 8 or 16 rows; 0 = default 2; D2Q37 only) and persistent CTAs that
 * prefetch their next tile (0 = default off, 1 = off, 2 = on, 3 = on and, on
 * D2Q37 domains that the 32 x rows tiles cover exactly, one launch for up to
 * 1024 steps of hlbm_step: a tile of step s starts as soon as the tile rows
 * around it have completed step s - 1, tracked by per-tile-row counters in
 * the workspace; where a read region exceeds one tile row, 3 runs as 2).
 * Chosen by the autotuner among 1 and 2 (3, measured slower on GB300, is
 * opt-in); results agree to rounding across schedules, and 3 agrees with 2
 * bit for bit. */
hlbm_status hlbm_set_tile(hlbm_ctx* ctx, int rows, int nodes_per_thread, int persistent);

/* Waits for all work on the context's stream.  Returns HLBM_ETIMEOUT (and
 * enters the error state) if a kernel reported an expired bounded wait. */
hlbm_status hlbm_synchronize(hlbm_ctx* ctx);

/* Wall-time limit of each bounded device-side wait (the mbarrier wait of
 * the TMA staging), in seconds, 0 < seconds <= 60; default 2.  A kernel
 * whose wait expires skips its tile, sets a status word, and the next
 * hlbm_synchronize / hlbm_moments / hlbm_diag returns HLBM_ETIMEOUT.  The
 * state is then undefined (the skipped tiles were not written, and copies
 * that were still in flight may land after the kernel ended) until
 * hlbm_init or hlbm_load replaces it. */
hlbm_status hlbm_set_wait_timeout(hlbm_ctx* ctx, double seconds);

/* Message of the last failing call on this context (never NULL). */
const char* hlbm_last_error(const hlbm_ctx* ctx);

hlbm_status hlbm_destroy(hlbm_ctx* ctx);

/* Gradient of the kinetic energy L = sum_x rho |u|^2 / 2 after `steps` steps
 * from the current state, with respect to the body-force acceleration field
 * set by hlbm_set_force_field (kind 1), by the discrete adjoint of the step
 * (reverse streaming and the transposed Jacobian of the collision, Eqs. 2.2,
 * 3.3, 4.4, 4.5) with checkpoint-and-recompute: a checkpoint every
 * `ckpt_every` steps and one segment of recomputed states.  ckpt_every = 1
 * keeps every state (the forward steps write straight into the workspace:
 * no checkpoint copies, no recompute; 128^3 D3Q39 FP32 over 400 steps takes
 * about 131 GB).  Body-force contexts only (HLBM_EUNSUPPORTED with H_i or F^SC).
 *   workspace  caller-owned device memory, 256-byte aligned, of at least
 *              hlbm_adjoint_workspace_bytes(ctx, steps, ckpt_every) bytes
 *              (ceil(steps / ckpt_every) + ckpt_every - 1 states, two FP32
 *              adjoint fields, reduction scratch)
 *   dLdg       device [D][nz][ny][nx] FP32 output
 *   loss       host output, L in FP64
 * The context's state advances by `steps` (as hlbm_step would).  Synchronises. */
size_t hlbm_adjoint_workspace_bytes(const hlbm_ctx* ctx, int steps, int ckpt_every);
hlbm_status hlbm_adjoint_run(hlbm_ctx* ctx, int steps, int ckpt_every, void* workspace, size_t bytes, float* dLdg,
                             double* loss);

/* Batched step (D2Q37): advances many independent periodic contexts -- any
 * sizes, sources and parameters, one storage type -- together, with ONE
 * persistent kernel launch per time step (replayed from a CUDA graph of two
 * steps): resident CTAs take (domain, tile) items of every domain from a work
 * list through a device counter and run the single-domain tile code (32 x 8
 * tiles, two nodes per thread; 32 x 4 tiles, one node per thread, for the
 * pseudopotential kind), so each context's state equals that of hlbm_step
 * with those schedules bit for bit.  The contexts must be initialised;
 * hlbm_batch_create moves them onto the batch's stream, so their own calls
 * stay ordered with batch steps.  Each context's state and step count advance
 * as if hlbm_step had been called; hlbm_moments / hlbm_diag / hlbm_save work
 * on them as usual.  A context must not be destroyed before the batch.
 * Wall-bounded contexts (HLBM_WALLS) cannot be batched (HLBM_EINVAL).  After
 * hlbm_batch_synchronize reports HLBM_ETIMEOUT the batch is unusable: destroy
 * it and reload the contexts. */
typedef struct hlbm_batch hlbm_batch;
hlbm_status hlbm_batch_create(int n, hlbm_ctx* const* ctxs, hlbm_batch** out);
hlbm_status hlbm_batch_step(hlbm_batch* batch, int n);
hlbm_status hlbm_batch_synchronize(hlbm_batch* batch);
void* hlbm_batch_get_stream(hlbm_batch* batch);
hlbm_status hlbm_batch_destroy(hlbm_batch* batch);

/* Quadrature of a lattice as compiled into the library: c[Q*3] (int),
 * w[Q], *cs2 = c0^2, returns Q (0 on bad lattice).  Any pointer may be NULL. */
int hlbm_lattice_info(int lattice, int* c, double* w, double* cs2);

/* Domain totals of a population buffer without allocating any device memory.
 * The paper has no counterpart: this serves callers that must not allocate
 * device memory while they run (device memory handed out up front by another
 * framework under a fixed budget, or an environment that forbids allocation
 * after start-up); hlbm_diag needs the context's workspace for its scratch.
 *   populations  device pointer to Q * nodes stored values laid out as a
 *                context's state ([Q][nz][ny][nx], storage type `storage`,
 *                g_i = (f_i - w_i rho0) / w_i), e.g. the first population
 *                buffer of memory bound with hlbm_bind_memory after an even
 *                number of steps
 *   out          host array of D + 2 doubles: sum f (mass), sum c f
 *                (momentum), sum |c|^2 f / 2 (energy) over all nodes and
 *                velocities.  Streaming does not change these totals; without
 *                a body force they equal hlbm_diag's mass, momentum and energy
 *   cuda_stream  stream to run on (0: legacy default stream); the call
 *                synchronises it
 * Scratch is a 1 MiB static device array inside the library, held by every
 * GPU that loads it until the process exits; it limits a call to 1 ..
 * 33,554,432 nodes (HLBM_EINVAL beyond, with a message on stderr).  All calls
 * share it and overwrite what they use: calls that overlap on the GPU race.
 * The call copies the totals to the host and synchronises the stream, so it
 * must not be made while the stream is being captured into a graph.  The
 * first call on a device looks up the array's device address with that
 * device current; with CUDA's lazy module loading that first call (and the
 * first call for each lattice and storage pair, whose kernels load then) may
 * place the array and the kernels' code in device memory: a caller that must
 * not allocate after start-up makes one warm-up call per device, lattice and
 * storage during its initialisation.  The stored values of wall-bounded
 * contexts (HLBM_WALLS) are deviations from another reference state; their
 * energy total is not this one. */
hlbm_status hlbm_population_sums_noalloc(int lattice, long long nodes, int storage, double rho0,
                                         const void* populations, void* cuda_stream, double* out);

/* Bounds record of the debug build.  The library built with HLBM_DEBUG
 * (libhlbm_debug.so) checks, before each access, every index of a wrapped
 * global gather, of the shared-memory staging planes and neighbour frames,
 * of every population store, every TMA box origin (inside the domain, on
 * the 16-byte grid) and TMA shared-memory base (128-byte aligned) against
 * its buffer; an index outside it is counted and the access goes to element
 * 0 (loads) or is dropped (stores, copies: a dropped copy makes the bounded
 * wait expire, HLBM_ETIMEOUT; a misaligned base ends the CTA).  No kernel
 * reads or writes outside its buffers then, and no fault is raised.
 *   out    host array of 4: number of rejected accesses since the last clear,
 *          then site, index and bound of the first (site 1 gather, 2 staging
 *          plane, 3 neighbour frame, 4 population store, 5 TMA box origin,
 *          6 previous-step field, 7 TMA shared-memory base)
 *   clear  nonzero: zero the record after reading it
 * There is one record per device, shared by all contexts on it; the call
 * reads the current device's record and synchronises the device first.  The
 * release build returns HLBM_EUNSUPPORTED. */
hlbm_status hlbm_debug_record(unsigned long long* out, int clear);

#ifdef __cplusplus
}
#endif

#endif /* HLBM_H */
