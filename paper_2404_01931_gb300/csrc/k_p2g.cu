// k_p2g.cu — particle-to-grid transfer (Sec. 3.1.6, Eq. 4), forces and walls,
// divergence (Eq. 6), and read-back / diagnostic kernels of the grid fields.
//
// P2G computes, for every face node of each component,
//     u_node = sum_P u_P k(x_P - x_node) / sum_P k(x_P - x_node)     (0 if no P)
// The paper gathers per grid point; here the sum is split by particle bricks.
// One CTA takes one active 8x8x8 brick (its particles are one contiguous range
// after binning).  A thread owns a cell: it sums the weighted velocities and
// weights of that cell's particles into registers over the 2x3x3 face nodes
// they can reach, then adds them to a shared-memory tile of the brick plus its
// halo (9x10x10 nodes per component), and the CTA adds the tile to the global
// (num, den) accumulators with vector float2 atomics.  The normalisation
// num/den happens in k_finalize_rows (over the rows near the liquid; k_finalize
// sweeps the whole grid), which also clears the accumulators.
// A warp takes 8 x-cells by 4 z-planes of one y-row, and the tile's planes are
// TILE_PLANE = 104 nodes apart (8 mod 32 banks): the 32 lanes of every atomic
// then fall on 32 different banks.
#include <algorithm>

#include "flip_kernels.cuh"

namespace flipk {

constexpr int P2G_THREADS = 256;

template <int D>
struct Tile {
  static constexpr int X = (D == 0) ? 9 : 10;
  static constexpr int Y = (D == 1) ? 9 : 10;
  static constexpr int Z = (D == 2) ? 9 : 10;
  static constexpr int N = X * Y * Z;
};
constexpr int TILE_PLANE = 104;              // >= X * Y of every component; 8 mod 32
constexpr int TILE_PAD = 10 * TILE_PLANE;     // up to 10 planes
static_assert(TILE_PLANE % 32 == 8, "lanes 8 apart in z must take the next 8 banks");
static_assert(Tile<0>::X * Tile<0>::Y <= TILE_PLANE && Tile<1>::X * Tile<1>::Y <= TILE_PLANE &&
                  Tile<2>::X * Tile<2>::Y <= TILE_PLANE, "a plane of the tile fits");

// Weights of one axis over the node window of a cell: the component's own axis
// has 2 nodes (c, c+1); the other axes 3 nodes (c-1, c, c+1).
template <int NN>
__device__ __forceinline__ void expand(const AxisW& a, float (&w)[NN]) {
  if constexpr (NN == 2) {
    w[0] = a.w0;
    w[1] = a.w1;
  } else {
    const bool lo = (a.off == 0);
    w[0] = lo ? a.w0 : 0.0f;
    w[1] = lo ? a.w1 : a.w0;
    w[2] = lo ? 0.0f : a.w1;
  }
}

template <int D>
__device__ __forceinline__ void p2g_cell(const Grid& g, const PartView& P, unsigned int beg,
                                         unsigned int end, int ci, int cj, int ck, int li,
                                         int lj, int lk, float* tnum, float* tden) {
  constexpr int NX = (D == 0) ? 2 : 3, NY = (D == 1) ? 2 : 3, NZ = (D == 2) ? 2 : 3;
  constexpr int TX = Tile<D>::X;
  // (num, den) of a node accumulate together: one packed two-lane FMA per node,
  // each lane rounded like __fmaf_rn
  float2 acc[NZ][NY][NX];
#pragma unroll
  for (int z = 0; z < NZ; ++z)
#pragma unroll
    for (int y = 0; y < NY; ++y)
#pragma unroll
      for (int x = 0; x < NX; ++x) acc[z][y][x] = make_float2(0.0f, 0.0f);
  const float* vel = (D == 0) ? P.u : (D == 1) ? P.v : P.w;
  for (unsigned int q = beg; q < end; ++q) {
    const float px = P.x[q], py = P.y[q], pz = P.z[q], pv = vel[q];
    float wx[NX], wy[NY], wz[NZ];
    expand<NX>(axis_weights<D, 0>(px, g.inv_dx, ci, g.nx), wx);
    expand<NY>(axis_weights<D, 1>(py, g.inv_dx, cj, g.ny), wy);
    expand<NZ>(axis_weights<D, 2>(pz, g.inv_dx, ck, g.nz), wz);
#pragma unroll
    for (int z = 0; z < NZ; ++z)
#pragma unroll
      for (int y = 0; y < NY; ++y) {
        const float wyz = __fmul_rn(wy[y], wz[z]);
        const float2 tw = make_float2(__fmul_rn(wyz, pv), wyz);
#pragma unroll
        for (int x = 0; x < NX; ++x)
          acc[z][y][x] = __ffma2_rn(make_float2(wx[x], wx[x]), tw, acc[z][y][x]);
      }
  }
#pragma unroll
  for (int z = 0; z < NZ; ++z)
#pragma unroll
    for (int y = 0; y < NY; ++y)
#pragma unroll
      for (int x = 0; x < NX; ++x)
        if (acc[z][y][x].y != 0.0f) {
          const int t = (li + x) + TX * (lj + y) + TILE_PLANE * (lk + z);
          atomicAdd(tnum + t, acc[z][y][x].x);
          atomicAdd(tden + t, acc[z][y][x].y);
        }
}

template <int D>
__device__ __forceinline__ void flush_tile(const Grid& g, int b0, int b1, int b2,
                                           const float* tnum, const float* tden, float2* acc) {
  constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, N = Tile<D>::N;
  const int o0 = (D == 0) ? b0 : b0 - 1, o1 = (D == 1) ? b1 : b1 - 1, o2 = (D == 2) ? b2 : b2 - 1;
  const int FX = g.nx + (D == 0), FY = g.ny + (D == 1), FZ = g.nz + (D == 2);
  for (int t = threadIdx.x; t < N; t += P2G_THREADS) {
    const int ta = t % TX, tb = (t / TX) % TY, tc = t / (TX * TY);
    const int ts = ta + TX * tb + TILE_PLANE * tc;
    const float dn = tden[ts];
    if (dn == 0.0f) continue;
    const int a = o0 + ta, b = o1 + tb, c = o2 + tc;
    if (a < 0 || b < 0 || c < 0 || a >= FX || b >= FY || c >= FZ) continue;
    atomicAdd(acc + (a + FX * (b + FY * c)), make_float2(tnum[ts], dn));
  }
}

// One brick: zero the tiles, splat its cells' particles, add the tiles to the
// global accumulators.  CTA-uniform; ends with a __syncthreads.
__device__ __forceinline__ void p2g_brick(const Grid& g, const PartView& P, const BinView& B,
                                          float2* acc0, float2* acc1, float2* acc2,
                                          unsigned int brick, float (*tnum)[TILE_PAD],
                                          float (*tden)[TILE_PAD]) {
  const int b0 = (int)(brick % (unsigned)g.bx) * BRICK;
  const int b1 = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK;
  const int b2 = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK;
  for (int t = threadIdx.x; t < 3 * TILE_PAD; t += P2G_THREADS) {
    (&tnum[0][0])[t] = 0.0f;
    (&tden[0][0])[t] = 0.0f;
  }
  __syncthreads();
  const unsigned int bstart = B.brick_start[brick], bend = B.brick_start[brick + 1];
  static_assert(BRICK_CELLS == 2 * P2G_THREADS, "two passes of 8 x 8 x 4 cells");
  for (int pass = 0; pass < 2; ++pass) {
    const int li = threadIdx.x & 7, lk = ((threadIdx.x >> 3) & 3) + 4 * pass,
              lj = threadIdx.x >> 5;
    const int l = li + BRICK * (lj + BRICK * lk);
    const unsigned int key = brick * BRICK_CELLS + (unsigned)l;
    const unsigned int beg = bstart + B.local_start[key];
    const unsigned int end = (l < BRICK_CELLS - 1) ? bstart + B.local_start[key + 1] : bend;
    if (beg == end) continue;
    const int ci = b0 + li, cj = b1 + lj, ck = b2 + lk;
    p2g_cell<0>(g, P, beg, end, ci, cj, ck, li, lj, lk, tnum[0], tden[0]);
    p2g_cell<1>(g, P, beg, end, ci, cj, ck, li, lj, lk, tnum[1], tden[1]);
    p2g_cell<2>(g, P, beg, end, ci, cj, ck, li, lj, lk, tnum[2], tden[2]);
  }
  __syncthreads();
  flush_tile<0>(g, b0, b1, b2, tnum[0], tden[0], acc0);
  flush_tile<1>(g, b0, b1, b2, tnum[1], tden[1], acc1);
  flush_tile<2>(g, b0, b1, b2, tnum[2], tden[2], acc2);
  __syncthreads();
}

__global__ void __launch_bounds__(P2G_THREADS, 4) k_p2g(const Grid g, const PartView P,
                                                     const BinView B, float2* acc0, float2* acc1,
                                                     float2* acc2, const DevStats* st) {
  __shared__ float tnum[3][TILE_PAD];
  __shared__ float tden[3][TILE_PAD];
  const unsigned int nact = st->n_active;
  for (unsigned int bi = blockIdx.x; bi < nact; bi += gridDim.x)
    p2g_brick(g, P, B, acc0, acc1, acc2, B.active[bi], tnum, tden);
}

// All scenes' active bricks as one list: L.first holds the running sum of the
// scenes' active-brick counts (k_active_prefix), so the CTAs share the bricks of
// every scene evenly whatever their sizes.
__global__ void __launch_bounds__(P2G_THREADS, 4) k_p2g_batch(const BatchLaunch L) {
  __shared__ float tnum[3][TILE_PAD];
  __shared__ float tden[3][TILE_PAD];
  const unsigned int g0 = L.first[0], g1 = L.first[L.n];
  for (unsigned int gb = g0 + blockIdx.x; gb < g1; gb += gridDim.x) {
    const int s = batch_scene(L, gb);
    const SceneDev& S = L.scenes[s];
    p2g_brick(S.g, S.dst, S.B, S.acc[0], S.acc[1], S.acc[2], S.B.active[gb - L.first[s]], tnum,
              tden);
  }
}

// The running sum of the scenes' active-brick counts (their binning's result):
// out[0] = 0, out[s + 1] = out[s] + n_active of scene s.  One thread.
__global__ void k_active_prefix(const SceneDev* scenes, int n, unsigned int* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned int run = 0;
  out[0] = 0;
  for (int s = 0; s < n; ++s) {
    run += scenes[s].st->n_active;
    out[s + 1] = run;
  }
}

// u_old = num / den (0 where no particle reached the node); clears the
// accumulator for the next step.
__device__ __forceinline__ void finalize_face(float2* acc, float* uo, long long idx) {
  const float2 v = acc[idx];
  uo[idx] = (v.y != 0.0f) ? __fdiv_rn(v.x, v.y) : 0.0f;
  if (v.x != 0.0f || v.y != 0.0f) acc[idx] = make_float2(0.0f, 0.0f);  // empty faces stay clear
}

// Every face of the grid.
__device__ __forceinline__ void finalize(const Grid& g, float2* acc0, float2* acc1, float2* acc2,
                                         float* uo0, float* uo1, float* uo2, unsigned int blk,
                                         unsigned int nblk) {
  const long long n0 = n_faces(g, 0), n1 = n_faces(g, 1), n2 = n_faces(g, 2);
  const long long tot = n0 + n1 + n2;
  for (long long f = blk * (long long)blockDim.x + threadIdx.x; f < tot;
       f += (long long)nblk * blockDim.x) {
    float2* acc;
    float* uo;
    long long idx;
    if (f < n0) { acc = acc0; uo = uo0; idx = f; }
    else if (f < n0 + n1) { acc = acc1; uo = uo1; idx = f - n0; }
    else { acc = acc2; uo = uo2; idx = f - n0 - n1; }
    finalize_face(acc, uo, idx);
  }
}

__global__ void k_finalize(const Grid g, float2* acc0, float2* acc1, float2* acc2, float* uo0,
                           float* uo1, float* uo2) {
  finalize(g, acc0, acc1, acc2, uo0, uo1, uo2, blockIdx.x, gridDim.x);
}

__global__ void k_finalize_batch(const BatchLaunch L) {
  const int s = batch_scene(L, blockIdx.x);
  const SceneDev& S = L.scenes[s];
  finalize(S.g, S.acc[0], S.acc[1], S.acc[2], S.uo[0], S.uo[1], S.uo[2], blockIdx.x - L.first[s],
           L.first[s + 1] - L.first[s]);
}

// The rounding error of s = fl(a + b) (Knuth's TwoSum): a + b = s + err exactly.
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bv = __fsub_rn(s, a);
  return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// Gravity + walls give u* on the fly; b = -div u* (Eq. 6) in fluid cells (0
// elsewhere), and the solve's start p = 0 (every cell, so air cells hold p = 0).
__device__ __forceinline__ void divergence_cell(const Grid& g, const StepConsts& K,
                                                const uint8_t* __restrict__ type,
                                                const float* __restrict__ uo0,
                                                const float* __restrict__ uo1,
                                                const float* __restrict__ uo2, float* b32,
                                                double* b64, float* x32, double* x64,
                                                float2* pff, int i, int j, int k) {
  const int c = i + g.nx * (j + g.ny * k);
  if (x32) x32[c] = 0.0f;
  if (x64) x64[c] = 0.0;
  if (pff) pff[c] = make_float2(0.0f, 0.0f);
  const bool fluid = (type[c] == 1);
  const int fu = i + (g.nx + 1) * (j + g.ny * k);
  const int fv = i + g.nx * (j + (g.ny + 1) * k);
  const int fw = c;
  const float uL = (i == 0) ? 0.0f : __fadd_rn(uo0[fu], K.gdt[0]);
  const float uR = (i + 1 == g.nx) ? 0.0f : __fadd_rn(uo0[fu + 1], K.gdt[0]);
  const float vB = (j == 0) ? 0.0f : __fadd_rn(uo1[fv], K.gdt[1]);
  const float vT = (j + 1 == g.ny) ? 0.0f : __fadd_rn(uo1[fv + g.nx], K.gdt[1]);
  const float wK = (k == 0) ? 0.0f : __fadd_rn(uo2[fw], K.gdt[2]);
  const float wF = (k + 1 == g.nz) ? 0.0f : __fadd_rn(uo2[fw + g.nx * g.ny], K.gdt[2]);
  if (b32) {
    const float d = __fadd_rn(__fadd_rn(__fsub_rn(uR, uL), __fsub_rn(vT, vB)), __fsub_rn(wF, wK));
    b32[c] = fluid ? -__fmul_rn(d, g.inv_dx) : 0.0f;
  }
  if (b64) {
    // the FP64 pipe is narrow: warps without a fluid cell skip the FP64 work, and a
    // difference of two floats whose FP32 result is exact (Knuth's TwoSum error is
    // 0) is the FP64 difference too, so one conversion stands for two conversions
    // and a subtraction (the same bits)
    double v = 0.0;
    const unsigned int am = __activemask();
    if (__ballot_sync(am, fluid)) {
      const float su = __fsub_rn(uR, uL), sv = __fsub_rn(vT, vB), sw = __fsub_rn(wF, wK);
      const bool exact = two_sum_err(uR, -uL, su) == 0.0f && two_sum_err(vT, -vB, sv) == 0.0f &&
                         two_sum_err(wF, -wK, sw) == 0.0f;
      double d;
      if (__all_sync(am, exact)) {
        d = ((double)su + (double)sv) + (double)sw;
      } else {
        d = ((double)uR - (double)uL) + ((double)vT - (double)vB) + ((double)wF - (double)wK);
      }
      v = fluid ? -d * (double)g.inv_dx : 0.0;
    }
    b64[c] = v;
  }
}

// The grid barrier's arrival counter and spare words, and the per-step max-speed
// word, reset before the solve (a block may have 32 threads).
__device__ __forceinline__ void reset_step_words(unsigned int* bar, DevStats* st) {
  for (unsigned int t = threadIdx.x; t < BAR_WORDS; t += blockDim.x) bar[t] = 0u;
  if (threadIdx.x == 0) st->max_speed_bits = 0u;
}

// Every cell: block (j, k) of a scene walks the x-row of cells (i, j, k), no
// index divisions; the first block also resets the step words.
__device__ __forceinline__ void divergence(const Grid& g, const StepConsts& K0,
                                           const uint8_t* __restrict__ type,
                                           const float* __restrict__ uo0,
                                           const float* __restrict__ uo1,
                                           const float* __restrict__ uo2, float* b32, double* b64,
                                           float* x32, double* x64, float2* pff,
                                           unsigned int* bar, DevStats* st, int j, int k) {
  const StepConsts K = step_consts(K0);
  if (j == 0 && k == 0) reset_step_words(bar, st);
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x)
    divergence_cell(g, K, type, uo0, uo1, uo2, b32, b64, x32, x64, pff, i, j, k);
}

__global__ void k_divergence(const Grid g, const StepConsts K0, const uint8_t* __restrict__ type,
                             const float* __restrict__ uo0, const float* __restrict__ uo1,
                             const float* __restrict__ uo2, float* b32, double* b64, float* x32,
                             double* x64, float2* pff, unsigned int* bar, DevStats* st) {
  divergence(g, K0, type, uo0, uo1, uo2, b32, b64, x32, x64, pff, bar, st, (int)blockIdx.x,
             (int)blockIdx.y);
}

// CTA r of scene s takes row (j, k) = (r % ny, r / ny).
__global__ void k_divergence_batch(const BatchLaunch L) {
  const int s = batch_scene(L, blockIdx.x);
  const SceneDev& S = L.scenes[s];
  const int r = (int)(blockIdx.x - L.first[s]);
  divergence(S.g, S.K, S.type, S.uo[0], S.uo[1], S.uo[2], S.b32, S.b64, S.x32, S.x64, S.pff, S.bar,
             S.st, r % S.g.ny, r / S.g.ny);
}

// ---------------------------------------------------------------- bricks near the liquid
//
// After P2G only the faces of the active bricks' tiles (the brick and a one-node
// halo) can hold a sum, and only fluid cells (in active bricks) get a nonzero b or
// p.  So finalize and divergence need only visit the bricks within one brick of
// an active brick (this step's set S), plus last step's set, whose faces and cells
// they return to zero: outside S of the last step every face and cell is zero
// already (the arena starts zeroed, and each step re-zeroes what leaves S).  A
// face belongs to the cell at its node index (the last node along an axis to the
// last cell), and the passes walk whole x-rows of cells: every row of a brick-row
// (bricks (*, J, K)) that holds a brick to visit, so that their loads and stores
// stream along x as in the full sweep.  Each face and cell visited gets the full
// sweep's arithmetic: the fields come out the same.
//
// hmark[b]: bit 1 = b in S this step, bit 0 = b in S last step.

// S, and the list of brick-rows to visit (rowflag: zero on entry, one bit per
// brick-row; list_n: zero on entry); block 0 also resets the step words (the full
// divergence's job).
__global__ void k_halo_bricks(const Grid g, const unsigned int* __restrict__ brick_count,
                              uint8_t* hmark, unsigned int* rowflag, unsigned int* list,
                              unsigned int* list_n, unsigned int* bar, DevStats* st) {
  if (blockIdx.x == 0) reset_step_words(bar, st);
  const int nb = g.bx * g.by * g.bz;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    const int I = b % g.bx, J = (b / g.bx) % g.by, K = b / (g.bx * g.by);
    bool near = false;
    for (int dk = -1; dk <= 1 && !near; ++dk)
      for (int dj = -1; dj <= 1 && !near; ++dj)
        for (int di = -1; di <= 1 && !near; ++di) {
          const int i = I + di, j = J + dj, k = K + dk;
          if (i < 0 || j < 0 || k < 0 || i >= g.bx || j >= g.by || k >= g.bz) continue;
          near = brick_count[i + g.bx * (j + g.by * k)] > 0u;
        }
    const unsigned int m = ((near ? 1u : 0u) << 1) | ((unsigned)hmark[b] >> 1);
    hmark[b] = (uint8_t)m;
    if (m != 0u) {
      const unsigned int row = (unsigned)(J + g.by * K);
      const unsigned int bit = 1u << (row & 31u);
      // the first to flag a brick-row lists it
      if (!(atomicOr(rowflag + (row >> 5), bit) & bit)) list[atomicAdd(list_n, 1u)] = row;
    }
  }
}

// Cell row u of the listed brick-rows (64 per brick-row): (j, k), or false past
// the grid.
__device__ __forceinline__ bool listed_row(const Grid& g, const unsigned int* list,
                                           unsigned int u, int& j, int& k) {
  const unsigned int row = list[u >> 6];
  const int J = (int)(row % (unsigned)g.by), K = (int)(row / (unsigned)g.by);
  j = J * BRICK + (int)(u & 7u);
  k = K * BRICK + (int)((u >> 3) & 7u);
  return j < g.ny && k < g.nz;
}

// The faces of cell row (j, k): u at nodes (0 .. nx, j, k); v at (0 .. nx-1, j, k)
// and, on the last row, (.., ny, k); w at (.., j, k) and, on the last plane,
// (.., j, nz).
__device__ __forceinline__ void finalize_row(const Grid& g, int j, int k, float2* acc0,
                                             float2* acc1, float2* acc2, float* uo0, float* uo1,
                                             float* uo2) {
  const long long ru = (long long)(g.nx + 1) * (j + (long long)g.ny * k);
  for (int i = threadIdx.x; i <= g.nx; i += blockDim.x) finalize_face(acc0, uo0, ru + i);
  const int nv = (j + 1 == g.ny) ? 2 : 1, nw = (k + 1 == g.nz) ? 2 : 1;
  for (int q = 0; q < nv; ++q) {
    const long long rv = (long long)g.nx * ((j + q) + (long long)(g.ny + 1) * k);
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) finalize_face(acc1, uo1, rv + i);
  }
  for (int q = 0; q < nw; ++q) {
    const long long rw = (long long)g.nx * (j + (long long)g.ny * (k + q));
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) finalize_face(acc2, uo2, rw + i);
  }
}

__global__ void k_finalize_rows(const Grid g, float2* acc0, float2* acc1, float2* acc2,
                                float* uo0, float* uo1, float* uo2,
                                const unsigned int* __restrict__ list,
                                const unsigned int* __restrict__ list_n) {
  const unsigned int n = *list_n * 64u;
  for (unsigned int u = blockIdx.x; u < n; u += gridDim.x) {
    int j, k;
    if (listed_row(g, list, u, j, k)) finalize_row(g, j, k, acc0, acc1, acc2, uo0, uo1, uo2);
  }
}

__global__ void k_divergence_rows(const Grid g, const StepConsts K0,
                                  const uint8_t* __restrict__ type,
                                  const float* __restrict__ uo0, const float* __restrict__ uo1,
                                  const float* __restrict__ uo2, float* b32, double* b64,
                                  float* x32, double* x64, float2* pff,
                                  const unsigned int* __restrict__ list,
                                  const unsigned int* __restrict__ list_n) {
  const StepConsts K = step_consts(K0);
  const unsigned int n = *list_n * 64u;
  for (unsigned int u = blockIdx.x; u < n; u += gridDim.x) {
    int j, k;
    if (!listed_row(g, list, u, j, k)) continue;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x)
      divergence_cell(g, K, type, uo0, uo1, uo2, b32, b64, x32, x64, pff, i, j, k);
  }
}

template <int D, bool PAIR>
__global__ void k_u_new(const Grid g, const StepConsts K0, const float* __restrict__ uo,
                        const float* __restrict__ p32, const float2* __restrict__ pff,
                        float* __restrict__ out) {
  const StepConsts K = step_consts(K0);
  const int FX = g.nx + (D == 0), FY = g.ny + (D == 1);
  const long long nf = n_faces(g, D);
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(f % FX), b = (int)((f / FX) % FY), c = (int)(f / ((long long)FX * FY));
    out[f] = face_unew<D, PAIR>(g, K, uo[f], a, b, c, p32, pff);
  }
}

// ||div u*||^2 and ||div u_new||^2 over fluid cells in FP64, u_new from the
// stored pressure (FP32 or FP64) by Eq. 5 evaluated in FP64.
__global__ void k_div_norms(const Grid g, const StepConsts K0, const uint8_t* __restrict__ type,
                            const float* __restrict__ uo0, const float* __restrict__ uo1,
                            const float* __restrict__ uo2, const float* __restrict__ p32,
                            const double* __restrict__ p64, double* out2) {
  const StepConsts K = step_consts(K0);
  const long long nc = (long long)g.nx * g.ny * g.nz;
  const double ps = K.pscale64;
  double s_star = 0.0, s_new = 0.0;
  for (long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x; cl < nc;
       cl += (long long)gridDim.x * blockDim.x) {
    const int c = (int)cl;
    if (type[c] != 1) continue;
    const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    const int sxy = g.nx * g.ny;
    auto P = [&](int cc) -> double { return p64 ? p64[cc] : (double)p32[cc]; };
    const int fu = i + (g.nx + 1) * (j + g.ny * k);
    const int fv = i + g.nx * (j + (g.ny + 1) * k);
    const int fw = c;
    // star and projected values of the six faces (0 on walls)
    double us[6], un[6];
    const bool wall[6] = {i == 0, i + 1 == g.nx, j == 0, j + 1 == g.ny, k == 0, k + 1 == g.nz};
    const float uov[6] = {uo0[fu], uo0[fu + 1], uo1[fv], uo1[fv + g.nx], uo2[fw], uo2[fw + sxy]};
    const int dm[6] = {c - 1, c, c - g.nx, c, c - sxy, c};
    const int dp[6] = {c, c + 1, c, c + g.nx, c, c + sxy};
    for (int f = 0; f < 6; ++f) {
      if (wall[f]) { us[f] = un[f] = 0.0; continue; }
      us[f] = (double)__fadd_rn(uov[f], K.gdt[f >> 1]);
      un[f] = us[f] - ps * (P(dp[f]) - P(dm[f]));
    }
    const double d0 = ((us[1] - us[0]) + (us[3] - us[2]) + (us[5] - us[4])) * (double)g.inv_dx;
    const double d1 = ((un[1] - un[0]) + (un[3] - un[2]) + (un[5] - un[4])) * (double)g.inv_dx;
    s_star += d0 * d0;
    s_new += d1 * d1;
  }
  s_star = warp_sum(s_star);
  s_new = warp_sum(s_new);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out2, s_star);
    atomicAdd(out2 + 1, s_new);
  }
}

__global__ void k_f64_to_f32(const double* s, float* d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = (float)s[i];
}

__global__ void k_f32_to_f64(const float* s, double* d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = (double)s[i];
}

static unsigned int grid_for(long long n, int threads, int cap = 1 << 16) {
  long long b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  return (unsigned int)(b < 1 ? 1 : b);
}

void launch_p2g(const Grid& g, const PartView& p, const BinView& b, float2* const acc[3],
                const DevStats* st, int nblocks, cudaStream_t s) {
  k_p2g<<<nblocks, P2G_THREADS, 0, s>>>(g, p, b, acc[0], acc[1], acc[2], st);
}

void launch_finalize(const Grid& g, float2* const acc[3], float* const uo[3], cudaStream_t s) {
  const long long tot = n_faces(g, 0) + n_faces(g, 1) + n_faces(g, 2);
  k_finalize<<<grid_for(tot, 256), 256, 0, s>>>(g, acc[0], acc[1], acc[2], uo[0], uo[1], uo[2]);
}

void launch_divergence(const Grid& g, const StepConsts& k, const uint8_t* type,
                       const float* const uo[3], float* b32, double* b64, float* x32,
                       double* x64, float2* pff, unsigned int* bar, DevStats* st,
                       cudaStream_t s) {
  // one block per x-row, threads along x (nx <= 2048, rows ny x nz <= 2048 x 2048)
  const int threads = std::min(256, (g.nx + 31) / 32 * 32);
  k_divergence<<<dim3((unsigned)g.ny, (unsigned)g.nz), threads, 0, s>>>(
      g, k, type, uo[0], uo[1], uo[2], b32, b64, x32, x64, pff, bar, st);
}

cudaError_t launch_finalize_near(const Grid& g, const unsigned int* brick_count, uint8_t* hmark,
                                 unsigned int* rowflag, unsigned int* list, unsigned int* list_n,
                                 float2* const acc[3], float* const uo[3], unsigned int* bar,
                                 DevStats* st, int sm_count, bool full, cudaStream_t s) {
  const long long nb = (long long)g.bx * g.by * g.bz;
  const size_t rows = (size_t)g.by * g.bz;
  cudaError_t e = cudaMemsetAsync(rowflag, 0, sizeof(unsigned int) * ((rows + 31) / 32), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(list_n, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  k_halo_bricks<<<(unsigned)std::min<long long>((nb + 255) / 256, 4LL * sm_count), 256, 0, s>>>(
      g, brick_count, hmark, rowflag, list, list_n, bar, st);
  if (full) {
    launch_finalize(g, acc, uo, s);
  } else {
    k_finalize_rows<<<(unsigned)(16 * sm_count), 256, 0, s>>>(g, acc[0], acc[1], acc[2], uo[0],
                                                            uo[1], uo[2], list, list_n);
  }
  return cudaSuccess;
}

void launch_divergence_near(const Grid& g, const StepConsts& k, const uint8_t* type,
                            const float* const uo[3], float* b32, double* b64, float* x32,
                            double* x64, float2* pff, unsigned int* bar, DevStats* st,
                            const unsigned int* list, const unsigned int* list_n, int sm_count,
                            bool full, cudaStream_t s) {
  if (full) {
    launch_divergence(g, k, type, uo, b32, b64, x32, x64, pff, bar, st, s);
    return;
  }
  const int threads = std::min(256, (g.nx + 31) / 32 * 32);
  k_divergence_rows<<<(unsigned)(16 * sm_count), threads, 0, s>>>(
      g, k, type, uo[0], uo[1], uo[2], b32, b64, x32, x64, pff, list, list_n);
}

void launch_active_prefix(const SceneDev* scenes, int n, unsigned int* out, cudaStream_t s) {
  if (n > 0) k_active_prefix<<<1, 32, 0, s>>>(scenes, n, out);
}

void launch_p2g_batch(const BatchLaunch& L, unsigned int ctas, cudaStream_t s) {
  if (ctas) k_p2g_batch<<<ctas, P2G_THREADS, 0, s>>>(L);
}

void launch_finalize_batch(const BatchLaunch& L, unsigned int ctas, cudaStream_t s) {
  if (ctas) k_finalize_batch<<<ctas, 256, 0, s>>>(L);
}

void launch_divergence_batch(const BatchLaunch& L, unsigned int ctas, cudaStream_t s) {
  if (ctas) k_divergence_batch<<<ctas, 128, 0, s>>>(L);
}

void launch_u_new(const Grid& g, const StepConsts& k, int d, const float* uo, const float* p32,
                  const float2* pff, float* out, cudaStream_t s) {
  const bool pair = (pff != nullptr);
  const unsigned int gb = grid_for(n_faces(g, d), 256);
  if (d == 0) {
    if (pair) k_u_new<0, true><<<gb, 256, 0, s>>>(g, k, uo, p32, pff, out);
    else k_u_new<0, false><<<gb, 256, 0, s>>>(g, k, uo, p32, pff, out);
  } else if (d == 1) {
    if (pair) k_u_new<1, true><<<gb, 256, 0, s>>>(g, k, uo, p32, pff, out);
    else k_u_new<1, false><<<gb, 256, 0, s>>>(g, k, uo, p32, pff, out);
  } else {
    if (pair) k_u_new<2, true><<<gb, 256, 0, s>>>(g, k, uo, p32, pff, out);
    else k_u_new<2, false><<<gb, 256, 0, s>>>(g, k, uo, p32, pff, out);
  }
}

void launch_div_norms(const Grid& g, const StepConsts& k, const uint8_t* type,
                      const float* const uo[3], const float* p32, const double* p64,
                      double* out2, cudaStream_t s) {
  const long long nc = (long long)g.nx * g.ny * g.nz;
  k_div_norms<<<grid_for(nc, 256, 4096), 256, 0, s>>>(g, k, type, uo[0], uo[1], uo[2], p32, p64,
                                                      out2);
}

void launch_f64_to_f32(const double* src, float* dst, long long n, cudaStream_t s) {
  k_f64_to_f32<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
}

void launch_f32_to_f64(const float* src, double* dst, long long n, cudaStream_t s) {
  k_f32_to_f64<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
}

}  // namespace flipk
