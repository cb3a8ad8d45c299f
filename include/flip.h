/*
 * flip.h — C ABI of the GB300 FLIP step library (libflip_gb300.so).
 *
 * One simulation step of the FLuid-Implicit-Particle method as described by
 * Centeno & Pereira, "Fluid Implicit Particle Simulation for CPU and GPU"
 * (arXiv 2404.01931), Section 3:
 *
 *   bin particles by cell (Sec. 3.1.5, 3.2.2)
 *   -> particle-to-grid transfer onto the MAC grid (Sec. 3.1.6, Eq. 4)
 *   -> gravity and solid-wall conditions (Eq. 1, Sec. 2.1.3 splitting)
 *   -> pressure projection: b = -div u* (Eq. 6), A p = b by matrix-free
 *      preconditioned conjugate gradient (Sec. 3.1.7), u_new = u* - dt/rho grad p (Eq. 5)
 *   -> grid-to-particle PIC/FLIP blend (Sec. 2.1.4, 3.1.8)
 *   -> forward-Euler advection and wall clamp (Sec. 3.1.3).
 *
 * Everything runs as CUDA kernels for sm_103a on the stream given at creation.
 * Pointers are plain host or device addresses; sizes are in elements unless a
 * name says bytes.  No function throws; every function that can fail returns
 * a status code (FLIP_OK = 0) and flip_last_error() gives a message for the
 * calling thread's last failure.
 *
 * Grid conventions (Sec. 3.1.1, Figs. 1-2): nx*ny*nz cells of edge dx, domain
 * [0, n*dx) per axis, y up.  Cell (i,j,k) has index i + nx*(j + ny*k).  The
 * u, v, w face arrays have (nx+1)*ny*nz, nx*(ny+1)*nz and nx*ny*(nz+1)
 * entries; u[i,j,k] (at x = i*dx) has index i + (nx+1)*(j + ny*k), v[i,j,k]
 * index i + nx*(j + (ny+1)*k), w[i,j,k] index i + nx*(j + ny*k).  The six
 * domain planes are solid walls.
 */
#ifndef FLIP_GB300_H
#define FLIP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLIP_ABI_VERSION 5

/* ------------------------------------------------------------ status codes */
enum {
  FLIP_OK = 0,
  FLIP_E_ARG = 1,            /* bad argument, or a state the method cannot solve
                                (every cell fluid: A is singular, Sec. 3.1.7) */
  FLIP_E_OOM = 2,            /* device allocation failed */
  FLIP_E_CUDA = 3,           /* a CUDA call failed (message in flip_last_error) */
  FLIP_E_NOT_CONVERGED = 4,  /* warning: PCG hit its iteration cap; the step was
                                still taken with the last iterate */
  FLIP_E_TIMEOUT = 5,        /* a device-side wait gave up; the step's results are
                                not valid, the handle stays usable */
  FLIP_E_SIZE = 6,           /* a buffer size does not match the field */
  FLIP_E_NOGPU = 7,          /* no CUDA device, or not an sm_103 device */
  FLIP_E_CAPACITY = 8        /* warning: reseeding wanted more particles than
                                max_particles holds; the step was committed with
                                the particles that fit */
};

/* ------------------------------------------------------------ parameters */
enum {
  FLIP_PREC_FP32 = 0,     /* FP32 vectors and SpMV.  Dot products: each thread
                             accumulates exact FP32 products as a float pair
                             (hi + lo, error-free transforms, ~48 significant
                             bits), warps and CTAs add the pairs, and the CTAs'
                             pairs are added in FP64 (flip_dot_f32 runs it) */
  FLIP_PREC_MIXED_IR = 1  /* FP32 CG on a correction d inside; the solution x and
                             the outer residual r = b - A x are carried as float
                             pairs (~48 bits, not FP64) with the operator's scale
                             as a pair too (flip_residual_pairs runs that
                             residual), refined without restarting the Krylov
                             direction (reliable updates).  The right-hand side
                             enters as FP64 and the result leaves as FP64
                             (FLIP_FIELD_PRESSURE_F64). */
};

enum {
  FLIP_ADVECT_PARTICLE = 0, /* x += dt * (blended particle velocity) */
  FLIP_ADVECT_GRID = 1      /* x += dt * (interpolated projected grid velocity) */
};

enum {
  FLIP_PRECOND_JACOBI = 0, /* diagonal preconditioner */
  FLIP_PRECOND_MG = 1,     /* one multigrid V-cycle per iteration: levels coarsened 2x
                              per axis to an extent <= 4, red-black Gauss-Seidel
                              smoothing (Sec. 3.2.3), restriction (1/16) x sum of
                              the fluid children's residuals, correction 2x the
                              parent's value; symmetric positive definite */
  FLIP_PRECOND_RBGS = 2    /* no CG: red-black Gauss-Seidel sweeps from p = 0 (the
                              paper's GPU solver, Sec. 3.2.3) until
                              ||b - A p|| <= cg_tol ||b||, checked every 8 sweep pairs;
                              cg_max_iter caps the sweep pairs; FP32 precision only */
};

typedef struct {
  int32_t n[3];          /* cells per axis, each in [2, 2048] */
  double dx;             /* cell edge; 1/dx must be an integer <= 2^24 so that
                            the cell of a float32 position is exact */
  double dt;             /* time step (s) */
  double gravity[3];     /* body acceleration (m/s^2), e.g. {0, -9.81, 0} */
  double rho;            /* density (> 0) */
  double flip_ratio;     /* FLIP share r of the blend r*FLIP + (1-r)*PIC, [0,1] */
  double skin;           /* wall clamp distance (> 0, < dx) */
  double cg_tol;         /* FP32 mode: PCG stops at ||r|| <= cg_tol*||b||.
                            Mixed mode: refinement trigger in (0,1): the FP32
                            correction is folded into the float-pair (~48-bit)
                            solution and the residual recomputed in float pairs
                            whenever the recursive residual has dropped by this
                            factor (e.g. 1e-3). */
  double ir_tol;         /* mixed mode: outer stop at ||b - A x|| <= ir_tol*||b|| */
  int32_t cg_max_iter;   /* PCG iteration cap (per solve; per inner solve in mixed) */
  int32_t ir_max_iter;   /* mixed mode: cap on the refinements per solve */
  int32_t precision;     /* FLIP_PREC_* */
  int32_t advect_source; /* FLIP_ADVECT_* */
  int32_t preconditioner; /* FLIP_PRECOND_* (flip_step; flip_solve_pressure and
                             its no-alloc variant always use Jacobi) */
  int32_t mg_smooth;     /* multigrid: red-black sweep pairs before and after the
                            coarse correction, in [1, 8] */
  int32_t warm_start;    /* 0: every solve starts from p = 0 (the pinned reading).
                            1 (multigrid only): it starts from the pressure of the
                            last solve on this handle (values of cells that were not
                            fluid then are whatever the storage holds); the stopping
                            rule ||r|| <= tol*||b|| is unchanged, so the result is the
                            same solution to the same tolerance, usually in fewer
                            iterations.  Not in the paper (a standard device). */
  double cfl;            /* CFL number alpha of Sec. 3.1.4 (the paper takes 3).  0:
                            every step takes dt.  > 0: step n takes
                            dt_n = min(dt, alpha * dx / v_max), v_max the largest
                            particle speed at the start of the step (dt when all
                            particles rest); the pressure solve then runs on
                            q = dt_n p / (rho dx^2), and reads give p. */
  /* Reseeding (Sec. 3.1.2: a fluid cell should hold between three and twelve
   * particles, and a cell that falls short is reseeded).  Off when both are 0.
   *   ppc_min in [1, 64]: after every step, each cell holding 1..ppc_min-1
   *     particles gets new ones up to ppc_min, placed uniformly in the cell by
   *     SplitMix64 (reseed_seed, counter ((step * n_cells + cell) * 64 + slot) * 3
   *     + axis; top 53 bits as a double in [0,1), x = (i + U) dx rounded to
   *     float and clamped like the advection), with the projected grid
   *     velocity interpolated at their position (Eq. 4 weights), and new ids
   *     from the running count.  "step" counts this handle's steps from 0.
   *   ppc_max (0 or >= max(ppc_min, 1)): at the start of every step, a cell
   *     holding more particles keeps ppc_max of them (which ones is unspecified).
   * The particle count then varies; it is bounded by max_particles. */
  int32_t ppc_min;
  int32_t ppc_max;
  int64_t max_particles;   /* particle capacity, >= np (0: np without reseeding,
                              else max(2 np, np + ppc_min * min(np, n_cells),
                              1024)) */
  uint64_t reseed_seed;
} flip_params;

/* Fills p with the defaults of the 32^3 dam break: dx = 1/n, dt = 1/240,
 * g = (0, -9.81, 0), rho = 1, r = 0.95, skin = 1e-3*dx, cg_tol = 1e-6,
 * ir_tol = 1e-8, cg_max_iter = 20*max(n), ir_max_iter = 100, FP32, particle
 * advection, multigrid preconditioner with 2 sweep pairs, no warm start,
 * fixed time step (cfl = 0). */
void flip_default_params(flip_params* p, int32_t nx, int32_t ny, int32_t nz);

/* Optional allocator: when given to flip_create, every device allocation of
 * the handle goes through it (one arena per handle, freed at flip_destroy).
 * alloc returns NULL on failure.  stream is the handle's cudaStream_t. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
} flip_alloc;

/* Per-call statistics of flip_step (all times in ms, summed over the steps of
 * the call, measured with CUDA events on the handle's stream). */
typedef struct {
  int64_t steps;              /* steps taken by this call */
  int64_t n_particles;
  int64_t n_fluid_cells;      /* fluid cells of the last step */
  int64_t n_active_bricks;    /* 8x8x8 cell bricks holding fluid, last step */
  int64_t cg_iterations;      /* PCG iterations, summed over the steps */
  int32_t ir_iterations;      /* outer refinements, summed over the steps */
  int32_t kernel_launches;    /* kernels this library launched in the call */
  double cg_rel_residual;     /* last step: ||r||/||b|| the solver stopped at
                                 (mixed: the FP64 outer residual) */
  double rel_divergence;      /* last step: ||div u_new||_2 / ||div u*||_2 over
                                 fluid cells, FP64 from the stored fields */
  double max_speed;           /* last step: max particle speed after the blend */
  double ms_bin, ms_p2g, ms_divergence, ms_pcg, ms_g2p, ms_total;
  double dt_last;             /* time step of the last step (dt, or the adaptive one) */
  int64_t particles_added;    /* reseeding: particles created by this call */
  int64_t particles_removed;  /* reseeding: particles dropped by this call */
} flip_stats;

typedef struct flip_handle flip_handle;

/* Particle and grid fields for flip_read / flip_write. */
typedef enum {
  FLIP_FIELD_PX = 0, FLIP_FIELD_PY, FLIP_FIELD_PZ, /* float32[np] positions */
  FLIP_FIELD_PU, FLIP_FIELD_PV, FLIP_FIELD_PW,     /* float32[np] velocities */
  FLIP_FIELD_PID,       /* int32[np]: creation index of each particle */
  FLIP_FIELD_U_OLD, FLIP_FIELD_V_OLD, FLIP_FIELD_W_OLD, /* float32 faces: P2G
                           result of the last step, before gravity and walls */
  FLIP_FIELD_U_NEW, FLIP_FIELD_V_NEW, FLIP_FIELD_W_NEW, /* float32 faces: the
                           projected velocity of the last step (Eq. 5) */
  FLIP_FIELD_PRESSURE,  /* float32[n_cells], 0 in air */
  FLIP_FIELD_PRESSURE_F64, /* float64[n_cells] */
  FLIP_FIELD_RHS,       /* float32[n_cells]: b = -div u* (Eq. 6), 0 off fluid */
  FLIP_FIELD_CELL_TYPE, /* uint8[n_cells]: 1 fluid, 0 air */
  FLIP_FIELD_COUNT_
} flip_field;

int flip_abi_version(void);

/* Creates a scene from np particles (float32 SoA, Sec. 3.2.1).  The arrays are
 * copied (host memory when src_is_device == 0, device memory otherwise); the
 * caller keeps ownership.  np must be in [0, 2^31-1].  Device memory is owned
 * by the handle: taken through *alloc when non-NULL, else with cudaMallocAsync
 * on the stream.  stream is a cudaStream_t (NULL: the handle creates its own).
 * Particle i gets id i (FLIP_FIELD_PID).  On success *out is set and the
 * particles are already binned for the first step. */
int flip_create(const flip_params* params, const float* x, const float* y, const float* z,
                const float* u, const float* v, const float* w, int64_t np,
                int32_t src_is_device, const flip_alloc* alloc, void* stream,
                flip_handle** out);

/* Advances the scene by nsteps FLIP steps, stream-ordered and asynchronous.
 * When stats is non-NULL the call waits for the stream and fills *stats, and
 * the return value carries device-side conditions of the steps
 * (FLIP_E_NOT_CONVERGED, FLIP_E_TIMEOUT, FLIP_E_ARG for a singular system);
 * without stats those conditions are reported by the next flip_sync. */
int flip_step(flip_handle* h, int32_t nsteps, flip_stats* stats);

/* Waits for the handle's stream; returns the device-side condition of the steps
 * since the last report (FLIP_OK when none). */
int flip_sync(flip_handle* h);

/* Copies a field into caller memory (dst_is_device: device pointer).  bytes must
 * equal the field's size (FLIP_E_SIZE otherwise).  Particle fields come in the
 * handle's current (cell-sorted) order, with FLIP_FIELD_PID telling which
 * particle each entry is.  Synchronous. */
int flip_read(flip_handle* h, flip_field which, void* dst, size_t bytes, int32_t dst_is_device);

/* Overwrites a particle field (PX..PW or PID) in the handle's current order and
 * re-bins the particles.  Synchronous with respect to the source buffer. */
int flip_write(flip_handle* h, flip_field which, const void* src, size_t bytes,
               int32_t src_is_device);

/* All six particle arrays (float32[n] each) at once, in the handle's current
 * order; id (int32[n], nullable) receives the creation index of each entry.
 * n is the current particle count, flip_field_bytes(h, FLIP_FIELD_PX) / 4
 * (np unless reseeding changed it); the caller's arrays must hold n entries.
 * Synchronous. */
int flip_read_particles(flip_handle* h, float* x, float* y, float* z, float* u, float* v,
                        float* w, int32_t* id, int32_t dst_is_device);

/* Overwrites all six particle arrays (float32[n] each, n the current count as
 * above; the handle's current order, ids unchanged) and re-bins once.
 * Synchronous with respect to the sources. */
int flip_write_particles(flip_handle* h, const float* x, const float* y, const float* z,
                         const float* u, const float* v, const float* w, int32_t src_is_device);

/* Device time (ms) of each step of the last flip_step call that took stats, from
 * the step's first kernel to its last (CUDA events on the handle's stream, read
 * once after the call's steps were all enqueued).  Writes min(n, count) entries
 * to ms (nullable) and returns count, the number of steps of that call (0 when
 * no timed call was made), or -FLIP_E_ARG for a NULL handle. */
int32_t flip_step_times(const flip_handle* h, double* ms, int32_t n);

/* Limit (ns) of every bounded device-side wait of this handle's kernels: the grid
 * barriers of the persistent solve and G2P's waits for its bulk copies of
 * particles.  A wait that runs out sets the step's status to FLIP_E_TIMEOUT (the
 * step's results are then not valid: rewrite the particles, flip_write_particles,
 * before stepping again); G2P then waits for its copies in flight, up to 1 s, before
 * its CTA leaves.  0 restores the defaults (5 s for a barrier, 1 s for a copy).
 * FLIP_E_ARG for a NULL handle. */
int flip_set_wait_timeout(flip_handle* h, uint64_t timeout_ns);

/* CTAs of the scene's persistent solve kernel, in [1, the co-resident maximum]
 * (0, the default: one per SM).  Fewer CTAs mean fewer arrivals at each grid
 * barrier, which pays on small grids; the solution is the same up to the order
 * of floating-point sums.  FLIP_E_ARG outside the range. */
int flip_set_solver_blocks(flip_handle* h, int32_t nblocks);

/* Autotuner of that count: for each of m, m/2, m/4, m/8 CTAs (m the maximum) it
 * takes steps_per_candidate real steps through flip_step, timing the solves with
 * CUDA events, and keeps the fastest (written to *nblocks, nullable).  The scene
 * advances by 4 * steps_per_candidate steps.  Returns the first error, else the
 * first warning, else FLIP_OK. */
int flip_autotune_solver(flip_handle* h, int32_t steps_per_candidate, int32_t* nblocks);

/* Launch shapes of the scene's particle transfers (Sec. 3.1.6, 3.1.8): the grids
 * of the P2G and G2P kernels are p2g_per_sm and g2p_per_sm CTAs per SM (0: the
 * defaults, 8 for P2G and G2P's co-resident count).  Both kernels loop over the
 * active bricks, so any count gives the same step (up to the order of P2G's
 * floating-point sums); more CTAs than fit at once let the scheduler balance
 * bricks of uneven particle counts.  The best count depends on the scene.
 * FLIP_E_ARG for a NULL handle or a count outside [0, 64]. */
int flip_set_transfer_ctas(flip_handle* h, int32_t p2g_per_sm, int32_t g2p_per_sm);

/* The CTAs per SM in use (defaults resolved); either pointer may be NULL. */
int flip_get_transfer_ctas(const flip_handle* h, int32_t* p2g_per_sm, int32_t* g2p_per_sm);

/* Autotuner of those shapes: for the pairs (P2G, G2P) = (4, c), (8, 2c), (16, 4c)
 * CTAs per SM (c: G2P's co-resident count) it takes steps_per_candidate real
 * steps through flip_step, in that order and then in reverse (the scene evolves
 * while it is timed), adds each stage's CUDA-event times, and keeps for each
 * stage the count that took least time (written to the nullable outputs).  The
 * scene advances by 6 * steps_per_candidate steps.  Returns the first error, else
 * the first warning, else FLIP_OK. */
int flip_autotune_transfers(flip_handle* h, int32_t steps_per_candidate, int32_t* p2g_per_sm,
                            int32_t* g2p_per_sm);

/* Total mechanical energy of the particles, the quantity the paper follows over
 * a run to compare its CPU and GPU versions (Sec. 4, Fig. 10).  With particle
 * mass m = particle_mass and the handle's gravity g:
 *   out[0] kinetic   = m/2 * sum_p |v_p|^2
 *   out[1] potential = -m * sum_p g . x_p      (zero at the origin)
 *   out[2] total     = out[0] + out[1]
 * The sums are accurate to FP64 rounding (float pairs per thread, FP64 across
 * threads); their order follows the particle buffer, so the last bits may vary
 * from run to run.  Synchronous.  FLIP_E_ARG for a NULL handle or out, or a
 * negative or non-finite mass. */
int flip_energy(flip_handle* h, double particle_mass, double out[3]);

/* Device bytes a scene with these parameters and np particles holds (its arena;
 * what flip_create allocates, particle arrays at the capacity max_particles
 * implies).  0 when the parameters are invalid or no device is usable.
 * Allocates nothing. */
size_t flip_footprint_bytes(const flip_params* params, int64_t np);

/* Size in bytes of a field of this handle. */
size_t flip_field_bytes(const flip_handle* h, flip_field which);

void flip_destroy(flip_handle* h);

const char* flip_strerror(int status);
const char* flip_last_error(void);

/* ---------------------------------------------------------------- batches
 * Many independent scenes advanced together.  The pressure solves of all scenes
 * run in one cooperative launch per (precision, preconditioner) group, each scene
 * on its own team of CTAs sized by its particle count, with per-scene barriers,
 * reductions and convergence.  The other step kernels take one of two forms:
 *   per-scene (the default): every scene's binning, P2G and right-hand side run on
 *     the scene's own stream before the solves, and its G2P on its own stream
 *     after them, so the stages of different scenes overlap on the device;
 *   fused (flip_batch_set_fused(b, 1), when no scene of the call uses an adaptive
 *     time step or reseeding): each step kernel runs once for all scenes -- the two
 *     binning scans, the scatter, P2G (over one flat list of every scene's active
 *     bricks), its normalisation and the right-hand side, each one launch over a
 *     table of the scenes -- and G2P once per precision group: about 9 launches
 *     per step whatever the number of scenes, all on the batch's stream.
 * flip_batch_autotune times both (and their graph replays) and keeps the faster.
 * A scene's results are those of flip_step up to the order of floating-point sums. */
typedef struct flip_batch flip_batch;

/* A batch runner for up to capacity scenes (capacity <= 4096).  It owns small
 * device buffers for the per-scene solver arguments and the stream the batched
 * solves run on (stream: a cudaStream_t, NULL to create one); it owns no
 * scene. */
int flip_batch_create(int32_t capacity, void* stream, flip_batch** out);

/* Advances the n distinct scenes hs[0..n-1] (n <= capacity, all on the current
 * device) by nsteps steps each.  Stream-ordered with respect to each scene's
 * stream.  stats (nullable) receives n entries, as flip_step's per scene, with
 * ms_total the wall time of the whole call and ms_pcg the time of the batched
 * solves (in the fused form ms_bin, ms_p2g, ms_divergence and ms_g2p are the
 * batch-wide stage times, every scene's stage being one launch); when stats is
 * given the call waits and returns the first device-side condition of any scene. */
int flip_batch_step(flip_batch* b, flip_handle* const* hs, int32_t n, int32_t nsteps,
                    flip_stats* stats);

/* With enable = 1, untimed flip_batch_step calls of two or more steps run their
 * steps in pairs as one captured CUDA graph (scenes without reseeding, whose
 * step index the graph would freeze), cached for the same scenes and CTA split;
 * the remaining step, and any call the capture cannot serve, runs as usual.
 * Default 0: on GB300 the replays measured slower than stream-ordered launches
 * (64 dam breaks: 12.2 against 11.5 ms per step). */
int flip_batch_set_graphs(flip_batch* b, int32_t enable);

/* enable = 1: the fused form above where every scene allows it; 0 (default):
 * per-scene launches on the scenes' streams. */
int flip_batch_set_fused(flip_batch* b, int32_t enable);

/* 1 when a captured graph is cached (the last graph-eligible call used it). */
int flip_batch_graph_active(const flip_batch* b);

/* How the batched solves split their CTAs: each scene's team is proportional to
 * its particle count raised to `exponent` (default 1; in [0, 3]). */
int flip_batch_set_team_exponent(flip_batch* b, double exponent);

/* Autotuner of that split and of the step's form.  For each exponent in {0.5,
 * 0.75, 1, 1.25, 1.5, 2, 2.5} it advances the scenes by steps_per_candidate real
 * steps through flip_batch_step, timing the batched solves with CUDA events, and
 * keeps the exponent whose solves took least time (written to *exponent,
 * nullable).  Then, with that split, it times the four forms of the step -- fused
 * or per-scene launches, each stream-ordered or replayed as CUDA graphs -- over
 * 2 * steps_per_candidate steps each (after a 2-step call that warms the form) and
 * keeps the fastest (flip_batch_get_form tells which).  Last, with that form, it
 * times the transfers' launch shapes (the candidate pairs of
 * flip_autotune_transfers, set on every scene) over steps_per_candidate steps
 * each: in the fused form each stage keeps its fastest count by the batch-wide
 * stage times, in the per-scene form the pair with the least wall time is kept.
 * Since the scenes evolve while they are timed, every candidate is timed twice,
 * in forward then reverse order, and the two times added.  The scenes advance by
 * 20 * steps_per_candidate + 8 * (2 + 2 * steps_per_candidate) steps in all.
 * Returns the first error, else the first warning, else FLIP_OK. */
int flip_batch_autotune(flip_batch* b, flip_handle* const* hs, int32_t n,
                        int32_t steps_per_candidate, double* exponent);

/* The form the batch's steps take: *fused (flip_batch_set_fused) and *graphs
 * (flip_batch_set_graphs), each 0 or 1; either pointer may be NULL. */
int flip_batch_get_form(const flip_batch* b, int32_t* fused, int32_t* graphs);

void flip_batch_destroy(flip_batch* b);

/* Standalone pressure solve (Sec. 3.1.7): A p = b for the cell types in type.
 * type: device uint8[n_cells] (1 fluid, anything else air); b: device
 * float32[n_cells] (read on fluid cells only); p: device float32[n_cells],
 * written on every cell (0 off fluid).  Uses params->n, dx, dt, rho, cg_tol,
 * cg_max_iter (FP32 mode; precision must be FLIP_PREC_FP32; Jacobi preconditioner
 * whatever params->preconditioner says).  Scratch memory is
 * allocated and freed with cudaMallocAsync/cudaFreeAsync on stream.  Waits for
 * the stream before returning; *iterations (nullable) gets the iteration count
 * and *rel_residual (nullable) the final ||r||/||b||. */
int flip_solve_pressure(const flip_params* params, const uint8_t* type, const float* b,
                        float* p, void* stream, int32_t* iterations, double* rel_residual);

/* The two extended-precision steps of the mixed-precision solve, run on caller
 * data so that their rounding can be checked against exact sums.  The paper runs
 * its CG in one precision (Sec. 3.1.7); the GB300 build keeps the dot products
 * and the refinement residual in float pairs instead of FP64 (FP32's rate, about
 * 48 significant bits).
 *
 * flip_dot_f32: out = sum_i a[i] b[i] over n float32 entries (device arrays), as
 * every CG dot product of this library is formed: the solver's CTA count splits
 * [0, n) into contiguous slices (multiples of 32 long), each thread accumulates
 * exact FP32 products in a float pair (TwoProduct by FMA, TwoSum), warps and the
 * CTA add pairs, and one warp adds the CTAs' pairs in CTA order; the pair is
 * returned as the FP64 value hi + lo.  Its error is at most about
 * (m^2 + 3 L) u^2 sum_i |a[i] b[i]| with u = 2^-24, m the longest per-thread run
 * and L the levels of the pair additions above it.  n in [0, 2^31-1]; scratch is
 * allocated and freed on stream (cudaMallocAsync); waits for the stream.
 *
 * flip_residual_pairs: r = b - A x over the grid of params (natural layout,
 * n_cells entries per array, device memory), with A the 7-point operator of
 * Sec. 3.1.7 (scale s = dt/(rho dx^2), p = 0 in air, walls dropped), x, b, r as
 * float pairs (hi, lo arrays) and s as a float pair: the per-cell function the
 * mixed-mode multigrid solve applies in each refinement.  type[c] == 1 marks a
 * fluid cell; r is 0 on the others.  Allocates nothing; waits for the stream. */
int flip_dot_f32(const float* a, const float* b, int64_t n, double* out, void* stream);
int flip_residual_pairs(const flip_params* params, const uint8_t* type, const float* x_hi,
                        const float* x_lo, const float* b_hi, const float* b_lo, float* r_hi,
                        float* r_lo, void* stream);

/* Allocation-free variant of flip_solve_pressure, for callers that cannot
 * allocate device memory while they run: a plug-in whose device memory belongs
 * to its host application's allocator under a fixed budget, or a latency-critical
 * loop in which cudaMalloc/cudaFree are not allowed because they can synchronise
 * the whole device.  The paper has no counterpart; this is a deployment aid.
 *
 * Same arguments, results and status codes as flip_solve_pressure, but the
 * scratch (CG vectors, brick list, reduction slots, barrier, statistics) lives in
 * one fixed-size array in device memory owned by the library, so the call
 * allocates and frees nothing.  Limits: at most FLIP_NOALLOC_MAX_CELLS cells and
 * FLIP_NOALLOC_MAX_BRICKS 8x8x8 bricks; larger grids return FLIP_E_SIZE before
 * any device work (flip_last_error names the limit).  The array (about 4.3 MB) is
 * reserved on every GPU that loads the library and held until the process exits.
 * The first call on a device looks up the array's device address with that
 * device current (a one-time set-up per device); make that first call before any
 * stream capture.  Every call shares the one array per device and leaves its
 * contents behind (each call clears what it needs at the start), so calls that
 * overlap on the GPU race: serialise them, e.g. on one stream.  Waits for the
 * stream before returning. */
#define FLIP_NOALLOC_MAX_CELLS 262144
#define FLIP_NOALLOC_MAX_BRICKS 4096
int flip_solve_pressure_noalloc(const flip_params* params, const uint8_t* type, const float* b,
                                float* p, void* stream, int32_t* iterations,
                                double* rel_residual);

#ifdef __cplusplus
}
#endif
#endif
