// flip_internal.cuh — device-side types and helpers shared by the FLIP kernels.
//
// Data layout in device memory (one scene):
//   particles   SoA float32 x,y,z,u,v,w + int32 id, double-buffered for the
//               counting-sort scatter (Sec. 3.2.1 / 3.2.2 double buffering)
//   keys        per particle: cell key (brick-major, see below) and its rank
//               inside the cell (the value its histogram atomic returned)
//   cell grid   x-fastest dense arrays (Sec. 3.1.1, Fig. 2): type (u8),
//               pressure, right-hand side, CG vectors
//   face grid   u, v, w face arrays (MAC layout), P2G accumulators (num, den)
//   key space   cells grouped in 8x8x8 bricks: key = brick*512 + local, with
//               brick = bi + bx*(bj + by*bk) and local = li + 8*(lj + 8*lk).
//               Sorting particles by this key makes each brick's particles one
//               contiguous range, which the P2G tile kernel reads at once.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace flipk {

constexpr int BRICK = 8;
constexpr int BRICK_CELLS = 512;

// Sticky device-side condition bits (DevStats::status).
enum : int { DEV_TIMEOUT = 1, DEV_NOT_CONVERGED = 2, DEV_SINGULAR = 4, DEV_CAPACITY = 8 };

struct DevStats {
  int status;                 // DEV_* bits, cleared by the host when reported
  int cg_iters;               // last solve
  int ir_iters;               // last solve
  unsigned int n_fluid;       // fluid cells, last binning
  unsigned int n_active;      // active bricks, last binning
  unsigned int max_speed_bits;  // float bits of the last step's max speed
  long long cg_iters_total;   // running sums
  long long ir_iters_total;
  long long cg_iters_mark;    // the running sums at the start of the last call
  long long ir_iters_mark;    // that asked for statistics (copied on the stream)
  double rel_res;             // last solve's stopping residual ||r||/||b||
  double bnorm;               // last solve's ||b||
  double dt_cur;              // adaptive time step: dt of the current / last step
  float dyn[4];               // adaptive time step: g * dt (3 components) and dt,
                              // rounded to float, for the step's kernels
  // particle counts when reseeding makes them vary (otherwise np throughout)
  long long np_layout;        // particles in the binned layout of the current step
  long long np_buffer;        // particles in the current buffer: the layout plus
                              // the ones the last spawn appended
  unsigned long long spawn_req;  // spawn requests of the running step
  long long next_id;          // id of the next created particle
  long long added_total, removed_total;  // running sums
  long long added_mark, removed_mark;    // the sums at the start of a stats call
};

struct Grid {
  int nx, ny, nz;     // cells
  int bx, by, bz;     // bricks per axis
  float inv_dx;       // 1/dx, integer-valued
  float dx;
  float hi[3];        // n*dx - skin, upper clamp per axis
  float skin;
};

__host__ __device__ __forceinline__ long long n_faces(const Grid& g, int d) {
  return (long long)(g.nx + (d == 0)) * (g.ny + (d == 1)) * (g.nz + (d == 2));
}

// Exact floor(x * inv) for a float32 x and an integer-valued inv: the rounded
// product plus its FMA residual decide the integer part, so the cell of a
// particle equals the one an exact (FP64) evaluation gives.  Clamped to [0, n-1];
// NaN maps to 0.
__device__ __forceinline__ int cell_of(float x, float inv, int n) {
  const float p = __fmul_rn(x, inv);
  const float e = __fmaf_rn(x, inv, -p);
  float f = floorf(p);
  if (p == f && e < 0.0f) f -= 1.0f;
  f = fmaxf(f, 0.0f);
  f = fminf(f, (float)(n - 1));
  return (int)f;
}

__device__ __forceinline__ unsigned int brick_key(const Grid& g, int i, int j, int k) {
  const unsigned int b = (unsigned)(i >> 3) + (unsigned)g.bx * ((unsigned)(j >> 3) + (unsigned)g.by * (unsigned)(k >> 3));
  return b * BRICK_CELLS + (unsigned)((i & 7) + 8 * ((j & 7) + 8 * (k & 7)));
}

// Per-axis transfer weights (Eq. 4 on the clamped sample coordinate).  For the
// component's own axis the nodes are the cell's two faces, c and c+1; for the
// other two axes the nodes sit at half-cell offsets and are base, base+1 with
// base in {c-1, c}.  'off' is base relative to c-1 for those axes (0 or 1) and
// 0 for the own axis; w0, w1 weight nodes base and base+1.
struct AxisW {
  int off;
  float w0, w1;
};

__device__ __forceinline__ AxisW axis_weights_normal(float x, float inv, int c) {
  const float g = __fmul_rn(x, inv);
  float f = g - (float)c;
  f = fminf(fmaxf(f, 0.0f), 1.0f);
  return AxisW{0, 1.0f - f, f};
}

__device__ __forceinline__ AxisW axis_weights_stag(float x, float inv, int c, int n) {
  float g = __fmul_rn(x, inv) - 0.5f;
  g = fminf(fmaxf(g, 0.0f), (float)(n - 1));
  const int base = min((int)floorf(g), n - 2);
  const float f = g - (float)base;
  return AxisW{base - (c - 1), 1.0f - f, f};
}

template <int D, int AX>
__device__ __forceinline__ AxisW axis_weights(float x, float inv, int c, int n) {
  if constexpr (D == AX) return axis_weights_normal(x, inv, c);
  else return axis_weights_stag(x, inv, c, n);
}

// Per-thread accumulator of a float32 dot product in a float pair (hi + lo):
// each product is split exactly by an FMA and added with Knuth's TwoSum, so the
// pair carries ~48 significant bits.  Threads' pairs are summed in FP64.
struct FF {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(hi, p);
    const float bv = __fsub_rn(t, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(p, bv));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ void add(float t) {
    const float s = __fadd_rn(hi, t);
    const float bv = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(t, bv));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of K doubles in a fixed order; the result is valid in every
// thread.  scratch must hold 32*K doubles.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) scratch[q * 32 + warp] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double s = (lane < nw) ? scratch[q * 32 + lane] : 0.0;
    v[q] = warp_sum(s);
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  bar[0]
// counts arrivals and is never reset inside a launch: the k-th barrier of a CTA
// ends when the counter reaches k * nblocks, k counted per CTA in s_bar_gen
// (zeroed at kernel entry by team_enter).  Arrival is a release reduction (no
// value comes back, so the CTA starts polling at once) and the wait an acquire
// load, so every write before the barrier (ordered by __syncthreads before
// thread 0's release) is visible to every thread after it.  The caller resets
// bar[0] to 0 before the launch; the rest of the BAR_WORDS-word block is spare.
// Every wait is bounded: after timeout_ns without progress the CTA sets
// DEV_TIMEOUT in *status and returns false; a CTA that sees another one's failure
// returns false too.  Callers stop their loop on false, so no CTA is left waiting.
constexpr unsigned int BAR_WORDS = 64;

__shared__ unsigned int s_bar_gen;

__device__ __forceinline__ void red_add_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* status, unsigned int nblocks,
                                             unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int target = (s_bar_gen + 1u) * nblocks;
    s_bar_gen += 1u;
    red_add_release_gpu(bar, 1u);
    const unsigned long long t0 = global_timer_ns();
    while ((int)(ld_acquire_gpu(bar) - target) < 0) {
      if (*(volatile int*)status & DEV_TIMEOUT) { ok = 0; break; }
      if (global_timer_ns() - t0 > timeout_ns) {
        atomicOr(status, DEV_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Number of a cell's neighbours that are not solid walls (the domain planes
// are the only solids), i.e. the diagonal of the 7-point Laplacian in units of
// dt/(rho dx^2) (Sec. 3.1.7).
__device__ __forceinline__ int nonsolid_count(const Grid& g, int i, int j, int k) {
  return (i > 0) + (i < g.nx - 1) + (j > 0) + (j < g.ny - 1) + (k > 0) + (k < g.nz - 1);
}

}  // namespace flipk
