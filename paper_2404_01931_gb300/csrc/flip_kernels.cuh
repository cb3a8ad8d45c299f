// flip_kernels.cuh — argument structs and host-side launchers of the FLIP kernels.
#pragma once

#include <cuda.h>

#include "flip_internal.cuh"

namespace flipk {

struct PartView {
  float* x;
  float* y;
  float* z;
  float* u;
  float* v;
  float* w;
  int* id;
};

struct BinView {
  unsigned int* cell_count;   // [nkeys] histogram, all zero between steps
  unsigned int* local_start;  // [nkeys] exclusive scan of the counts inside each brick
  unsigned int* brick_count;  // [nbricks]
  unsigned int* brick_fluid;  // [nbricks] fluid cells per brick
  unsigned int* brick_start;  // [nbricks + 1]
  unsigned int* active;       // [nbricks] bricks that hold particles, ascending
  unsigned int* key;          // [np] cell key of each particle (current buffer order)
  unsigned int* rank;         // [np] rank of the particle inside its cell
};

struct StepConsts {
  float gdt[3];      // gravity * dt
  float pscale;      // dt / (rho dx): pressure-difference to velocity (Eq. 5)
  double pscale64;   // the same in FP64, for the FP64 divergence diagnostic
  float flip_ratio;
  int advect_grid;   // 1: advect with the grid velocity
  float dt;
  const float* dyn;  // adaptive time step (Sec. 3.1.4): device words {g*dt, dt}
                     // written by the step's first kernel, which replace gdt and
                     // dt; nullptr for a fixed step.  The solve then runs on the
                     // dt-free unknown q = dt p / (rho dx^2) (pscale = dx).
  unsigned long long wait_ns;  // limit of G2P's bounded waits for its bulk copies
};

// The step constants a kernel uses: the host values, with g*dt and dt taken
// from device memory when the time step is adaptive.
__device__ __forceinline__ StepConsts step_consts(const StepConsts& K) {
  StepConsts k = K;
  if (K.dyn) {
    k.gdt[0] = K.dyn[0];
    k.gdt[1] = K.dyn[1];
    k.gdt[2] = K.dyn[2];
    k.dt = K.dyn[3];
  }
  return k;
}

// One scene of a batched launch (several scenes' step kernels in one launch): what
// the step kernels read, for one step (src is the particle buffer the binning
// scatters from, dst the one it scatters into, which P2G and G2P then use).
struct SceneDev {
  Grid g;
  StepConsts K;
  PartView src, dst;
  BinView B;
  uint8_t* type;
  float2* acc[3];
  float* uo[3];
  float* b32;
  double* b64;
  float* x32;
  double* x64;
  float2* pff;
  unsigned int* bar;
  DevStats* st;
  long long np;
  unsigned int nbricks;
};

// CTAs of a batched launch: scene s (of n) owns CTAs first[s] .. first[s+1]-1.
struct BatchLaunch {
  const SceneDev* scenes;
  const unsigned int* first;
  int n;
};

// The scene a CTA of a batched launch works on (binary search of first).
__device__ __forceinline__ int batch_scene(const BatchLaunch& L, unsigned int cta) {
  int lo = 0, hi = L.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.first[mid] <= cta) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int PCG_SLOTS = 7;
constexpr int PRECOND_RBGS = 2;   // FLIP_PRECOND_RBGS: red-black Gauss-Seidel as the solver

// Multigrid V-cycle preconditioner (levels coarsened 2x per axis until the
// largest extent is <= 4; red-black Gauss-Seidel smoothing).
constexpr int MG_MAX_LEVELS = 12;
constexpr int MG_COARSE_SWEEPS = 2;   // red-black pairs each way on the coarsest level
constexpr int MG_CTA_CELLS = 4800;    // the coarsest levels, up to this many cells in
                                      // total, run inside one CTA in shared memory
constexpr float MG_OMEGA = 2.0f;      // over-correction of the coarse correction

// One level of the hierarchy.  The grid-wide levels (l < lgrid) are stored
// colour-split: cell (i, j, k) of colour c = (i+j+k) & 1 sits at
//     c * half + margin + hx * (j + ny * k) + (i >> 1),
// hx = ceil(nx / 2) rounded up to even, so the cells of one colour form
// contiguous runs along x, the six neighbours of a cell are contiguous runs of
// the other colour at fixed offsets, and every even slot starts an 8-byte pair.
// margin = hx * ny + 2 slots before and after each colour's half keep every
// neighbour address inside the array.  The CTA-local levels (l >= lgrid) use the
// natural x-fastest layout.
struct MgLevel {
  int lvl;            // this level's index
  int nx, ny, nz, ncells;
  float inv_scnt[8];  // 1 / (s_l * count), s_l = dt / (rho (2^l dx)^2)
  float s;
  float* x;           // level solution (level 0: the preconditioned residual z)
  float* b;           // level right-hand side (level 0: the CG residual r)
  uint8_t* t;         // fluid flags, natural layout (level 0: the cell types)
  uint8_t* code;      // CTA-local levels: per cell, bit q (0..5 = -x,+x,-y,+y,-z,+z)
                      // set when that neighbour is in the grid and fluid, bit 6
                      // when the cell is fluid; built at the start of every solve
  // colour-split levels
  int split;          // 1 for the grid-wide levels
  int hx;             // slots per row and colour (even)
  int half;           // one colour's slots: hx * ny * nz + 2 * margin
  int margin;         // hx * ny + 2
  int nw;             // segments per row: ceil(hx / 32); a segment is 32 slots
                      // of each colour, i.e. 64 cells of a row
  int nbx, nby, nbz;  // 8x8x8 blocks of this level's cells
  uint16_t* code16;   // per slot: the code bits above plus the count of
                      // neighbours inside the grid in bits 8..10
  int4* seg;          // active segments {row j + ny k, segment in row, j, k}
  unsigned int* nseg; // their number (device)
  uint8_t* bflag;     // levels >= 1: block holds a fluid cell (level 0 reads the
                      // brick fluid counts of the binning)
};

struct MgArgs {
  int nlev;           // levels, >= 1
  int lgrid;          // levels [lgrid, nlev) run inside CTA 0
  int nu;             // red-black pairs before and after the coarse correction
  float omega;
  float inv_cnt[8];   // 1 / count
  float* pa0;         // level-0 CG vectors, colour-split like level 0: search
  float* pb0;         // direction (double-buffered), A p, and the solution /
  float* q0;          // mixed-mode correction d
  float* d0;
  float2* x2;         // mixed mode: the solution as a float pair (hi, lo), and
  float2* b2;         // the right-hand side as a float pair, colour-split like level 0
  unsigned int* segcount;  // [MG_MAX_LEVELS * max_blocks] per-CTA segment counts
  MgLevel lv[MG_MAX_LEVELS];
};

struct PcgArgs {
  Grid g;
  float diag_tab[8];   // dt/(rho dx^2) * count
  float minv_tab[8];   // 1 / diag
  float s;             // dt/(rho dx^2) rounded to FP32
  float s_lo;          // s64 - s rounded to FP32: (s, s_lo) is the scale as a float pair
  double s64;
  const uint8_t* type;
  const unsigned int* active;
  const unsigned int* n_active;
  const unsigned int* brick_fluid;  // fluid cells per brick, from the binning
  const float* b32;     // FP32 mode right-hand side
  const double* b64;    // mixed mode right-hand side
  float* x32;           // FP32 mode solution / mixed inner correction
  double* x64;          // mixed mode solution
  float2* pff;          // mixed mode: solution as a float pair (hi, lo) for G2P
  float* r;
  float* pa;
  float* pb;
  float* q;
  double* partials;     // [PCG_SLOTS * max_blocks]: one slot per reduced value
                        // of each phase, so no slot is rewritten before all
                        // CTAs have read it
  unsigned int* bar;    // [BAR_WORDS] grid barrier
  int* status;          // DevStats::status
  DevStats* stats;
  double tol;           // FP32 stop / mixed inner stop
  double ir_tol;
  int max_iter;
  int ir_max_iter;
  int check_singular;   // compare n_fluid with the cell count
  unsigned long long timeout_ns;
  int precond;          // 0 Jacobi, 1 multigrid
  int warm_start;       // multigrid: start from the last solve's solution
  MgArgs mg;
};

// Several scenes' solves in one cooperative launch: args[s] is scene s's
// argument block (device memory), CTA b works on scene block_scene[b] in the
// team of CTAs team_first[s] .. team_first[s+1]-1.
struct PcgBatch {
  const PcgArgs* args;
  const int* block_scene;
  const int* team_first;
  int nscenes;
};

// Level shapes of the multigrid hierarchy for an (nx, ny, nz) grid; returns the
// number of levels (dims[l] = ceil(dims[l-1] / 2) until max extent <= 4).
int mg_level_dims(int nx, int ny, int nz, int dims[MG_MAX_LEVELS][3]);

// Projected velocity on face node (a,b,c) of component D (Eq. 5 with gravity
// and the wall condition): 0 on the domain planes, otherwise
//   u_new = u_old + g_D dt - dt/(rho dx) (p(+) - p(-))
// with p = 0 in air cells.  The pressure difference is taken in FP32 from the
// FP32 pressure, or from the float-pair pressure of mixed mode as
// (hi+ - hi-) + (lo+ - lo-).  G2P and the read-back of U_NEW share this
// function, so both give the same bits.
template <int D, bool PAIR>
__device__ __forceinline__ float face_unew(const Grid& g, const StepConsts& k, float uo, int a,
                                           int b, int c, const float* p32, const float2* pff) {
  const int nd = (D == 0) ? a : (D == 1) ? b : c;
  const int nmax = (D == 0) ? g.nx : (D == 1) ? g.ny : g.nz;
  if (nd == 0 || nd == nmax) return 0.0f;
  const int cp = a + g.nx * (b + g.ny * c);
  const int cm = cp - ((D == 0) ? 1 : (D == 1) ? g.nx : g.nx * g.ny);
  float dp;
  if constexpr (PAIR) {
    const float2 hp = pff[cp], hm = pff[cm];
    dp = __fadd_rn(__fsub_rn(hp.x, hm.x), __fsub_rn(hp.y, hm.y));
  } else {
    dp = __fsub_rn(p32[cp], p32[cm]);
  }
  return __fsub_rn(__fadd_rn(uo, k.gdt[D]), __fmul_rn(k.pscale, dp));
}

// k_bin.cu
// Histogram and ranks of the particles' cells; also the largest particle speed
// (atomic max into *st_speed, float bits, which the caller clears).
void launch_rebin(const Grid& g, const PartView& p, const BinView& b, long long np,
                  unsigned int* st_speed,
                  cudaStream_t s);
// cmax: reseeding's per-cell upper bound (~0u: none).
void launch_bin(const Grid& g, const BinView& b, uint8_t* type, DevStats* st, cudaStream_t s,
                unsigned int cmax = ~0u);
// np: source particles (with np_dev non-null: at most np, bounded by *np_dev);
// particles of rank >= rank_max in their cell are dropped.
void launch_scatter(const PartView& src, const PartView& dst, const BinView& b, long long np,
                    cudaStream_t s, const long long* np_dev = nullptr,
                    unsigned int rank_max = ~0u);
void launch_iota(int* id, long long np, cudaStream_t s);

// Batched forms: every scene of the table in one launch per kernel (no
// reseeding, fixed time step).  first[] per launch as above; `ctas` its total.
// Per-scene CTA counts: cell_local_scan ceil(nbricks / 8); brick_scan one; scatter
// ceil(np / 512); finalize ceil(faces / 1024); divergence ny * nz.
void launch_bin_batch(const BatchLaunch& L_scan, unsigned int ctas_scan, const BatchLaunch& L_one,
                      cudaStream_t s);
void launch_scatter_batch(const BatchLaunch& L, unsigned int ctas, cudaStream_t s);
// P2G and G2P take L.first from launch_active_prefix (device-computed running sum
// of the scenes' active bricks; entries first[0] .. first[n] of the scenes given)
// and share all those bricks over `ctas` CTAs.
void launch_active_prefix(const SceneDev* scenes, int n, unsigned int* out, cudaStream_t s);
void launch_p2g_batch(const BatchLaunch& L, unsigned int ctas, cudaStream_t s);
void launch_finalize_batch(const BatchLaunch& L, unsigned int ctas, cudaStream_t s);
void launch_divergence_batch(const BatchLaunch& L, unsigned int ctas, cudaStream_t s);
void launch_g2p_batch(const BatchLaunch& L, unsigned int ctas, bool pair, cudaStream_t s);

// k_p2g.cu
void launch_p2g(const Grid& g, const PartView& p, const BinView& b, float2* const acc[3],
                const DevStats* st, int nblocks, cudaStream_t s);
void launch_finalize(const Grid& g, float2* const acc[3], float* const uo[3], cudaStream_t s);
void launch_divergence(const Grid& g, const StepConsts& k, const uint8_t* type,
                       const float* const uo[3], float* b32, double* b64, float* x32,
                       double* x64, float2* pff, unsigned int* bar, DevStats* st,
                       cudaStream_t s);
// finalize and divergence over the bricks within one brick of an active brick,
// this step's or last step's (full: the whole-grid kernels, after which the marks
// are current again), walked as whole x-rows of the brick-rows holding such a
// brick.  launch_finalize_near marks the bricks (hmark: [nbricks], kept across
// steps), lists the brick-rows (rowflag: [ceil(by bz / 32)] words; list: [by bz];
// list_n: one word), resets the step words and finalizes: two kernels;
// launch_divergence_near: one.
cudaError_t launch_finalize_near(const Grid& g, const unsigned int* brick_count, uint8_t* hmark,
                                 unsigned int* rowflag, unsigned int* list, unsigned int* list_n,
                                 float2* const acc[3], float* const uo[3], unsigned int* bar,
                                 DevStats* st, int sm_count, bool full, cudaStream_t s);
void launch_divergence_near(const Grid& g, const StepConsts& k, const uint8_t* type,
                            const float* const uo[3], float* b32, double* b64, float* x32,
                            double* x64, float2* pff, unsigned int* bar, DevStats* st,
                            const unsigned int* list, const unsigned int* list_n, int sm_count,
                            bool full, cudaStream_t s);
void launch_u_new(const Grid& g, const StepConsts& k, int d, const float* uo, const float* p32,
                  const float2* pff, float* out, cudaStream_t s);
void launch_div_norms(const Grid& g, const StepConsts& k, const uint8_t* type,
                      const float* const uo[3], const float* p32, const double* p64,
                      double* out2, cudaStream_t s);
void launch_f64_to_f32(const double* src, float* dst, long long n, cudaStream_t s);
void launch_f32_to_f64(const float* src, double* dst, long long n, cudaStream_t s);

// k_pcg.cu
int pcg_block_size();
cudaError_t pcg_max_blocks(int* max_blocks, int* sm_count);
cudaError_t launch_pcg(const PcgArgs& a, bool mixed, int nblocks, cudaStream_t s);

cudaError_t launch_pcg_batch(const PcgBatch& b, bool mixed, int nblocks, cudaStream_t s);

// k_mg.cu
cudaError_t launch_pcg_mg(const PcgArgs& a, bool mixed, int nblocks, cudaStream_t s);
cudaError_t launch_pcg_mg_batch(const PcgBatch& b, bool mixed, int nblocks, cudaStream_t s);
cudaError_t pcg_mg_check_occupancy();
void launch_mark_bricks(const Grid& g, const uint8_t* type, unsigned int* brick_fluid,
                        cudaStream_t s);
void launch_compact_bricks(const Grid& g, const unsigned int* brick_fluid,
                           unsigned int* active, DevStats* st, cudaStream_t s);
void launch_zero_off_fluid(const Grid& g, const uint8_t* type, float* p, unsigned int* bar,
                           cudaStream_t s);

// k_reseed.cu (Sec. 3.1.2 reseeding)
struct ReseedArgs {
  int ppc_min;
  unsigned long long seed;
  long long step;          // the handle's step index
  long long capacity;
  double dx;               // cell edge in FP64 (the parameter, not 1/inv_dx)
};
// After G2P: cells holding 1..ppc_min-1 particles (the next step's histogram)
// get new particles appended to p up to ppc_min, with their keys and ranks.
void launch_spawn(const Grid& g, const StepConsts& k, const PartView& p, const BinView& b,
                  const float* const uo[3], const float* p32, const float2* pff, DevStats* st,
                  const ReseedArgs& r, long long nkeys, cudaStream_t s);

// k_g2p.cu
int g2p_blocks(int sm_count);
// pmap (nullable): tensor map of the pressure (encode_pressure_map) for the TMA
// staging of the pressure slab; plain loads when NULL.
void launch_g2p(const Grid& g, const StepConsts& k, const PartView& p, const BinView& b,
                const float* const uo[3], const float* p32, const float2* pff, DevStats* st,
                long long np, int nblocks, const CUtensorMap* pmap, cudaStream_t s);
// Tensor map of a pressure field (float pairs when pair, else FP32; natural
// layout) for G2P's slab staging; false when the grid's pitches do not allow one.
bool encode_pressure_map(const Grid& g, void* base, bool pair, CUtensorMap* out);

// k_diag.cu
// Adaptive time step (Sec. 3.1.4): dt = min(dt_max, alpha dx / v_max), v_max the
// largest particle speed (DevStats::max_speed_bits); writes st->dt_cur and st->dyn.
void launch_cfl_dt(DevStats* st, const double g[3], double dt_max, double alpha_dx,
                   cudaStream_t s);
// out[i] *= f for i < n (device arrays).
void launch_scale(float* out, long long n, double f, cudaStream_t s);
void launch_scale(double* out, long long n, double f, cudaStream_t s);
// Sums over the particles (FP64): out[0] = sum |v|^2, out[1..3] = sum x, y, z.
// partials holds 4 * nblocks doubles.
int energy_blocks(int sm_count);
void launch_energy(const PartView& p, long long np, double* partials, int nblocks, double* out,
                   cudaStream_t s);

}  // namespace flipk
