// k_mg.cu — conjugate gradient on A p = b (Sec. 3.1.7) preconditioned by one
// multigrid V-cycle per iteration, whose smoother is the red-black Gauss-Seidel
// the paper runs on the GPU (Sec. 3.2.3).  One persistent cooperative kernel
// per solve, like the Jacobi version in k_pcg.cu.
//
// Hierarchy: level 0 is the cell grid; level l+1 has ceil(n_l/2) cells per axis
// and a coarse cell is fluid when any of its children is; coarsening stops when
// the largest extent is <= 4.  Level l carries the 7-point operator with scale
// dt/(rho (2^l dx)^2).  V-cycle from a zero guess at every level: nu
// (red, black) half-sweep pairs, restriction of the residual b_{l+1} =
// (1/16) sum over fluid children (Galerkin scaling for piecewise-constant
// prolongation), the coarse cycle, correction x += omega x_{l+1}(parent), nu
// (black, red) pairs; the coarsest level does MG_COARSE_SWEEPS pairs each way.
// The cycle is a symmetric positive-definite operator, as CG requires.
//
// Levels with more than MG_CTA_CELLS cells are processed by all CTAs with grid
// barriers between half-sweeps; the small levels run inside CTA 0 with
// __syncthreads.  The correction is never written: the first post-smoothing
// half-sweep (black) reads its red neighbours plus omega times their parents'
// values, and the red half-sweep that follows overwrites the red cells anyway.
// The first red half-sweep from zero only needs the residual, so at level 0 it
// is fused into the phase that produces the residual.
//
// Memory-level parallelism: the passes are latency-bound (a thread owns many
// cells and each cell needs ~8 independent loads), so every pass handles U
// cells per thread at a time: it issues the loads of all U cells, then does the
// arithmetic and the stores.  The neighbour structure comes from one code byte
// per cell (built at the start of the solve), so the value loads never wait on
// neighbour flags.  The arithmetic and the per-thread order of the reductions
// are those of one cell at a time.
#include "pcg_common.cuh"

namespace flipk {

namespace {

constexpr unsigned int CODE_SELF = 64u;

// Runs slots first, first + stride, ... < end in batches of U: pre(e, ok)
// returns a state with the slot's first loads, load(state) adds the loads that
// depend on them, apply(state) computes and stores.  All loads of a batch come
// before its first store.  Slots past the end are handed to pre() as 'first'
// with ok = false (valid addresses; apply must skip them).
template <int U, class Pre, class Load, class Apply>
__device__ __forceinline__ void run_batched(unsigned int first, unsigned int end,
                                            unsigned int stride, Pre&& pre, Load&& load,
                                            Apply&& apply) {
  using S = decltype(pre(0u, false));
  for (unsigned int e0 = first; e0 < end; e0 += (unsigned)U * stride) {
    S s[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned int e = e0 + (unsigned)u * stride;
      const bool ok = e < end;
      s[u] = pre(ok ? e : e0, ok);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) load(s[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) apply(s[u]);
  }
}

// ---------------------------------------------------------------- cells

struct Cell {
  int i, j, k, c;
  bool ok;
};

// Slot e of level 0's active-cell index space (512 slots per active brick).
__device__ __forceinline__ Cell slot_dense0(const PcgArgs& A, unsigned int e) {
  const Grid& g = A.g;
  const unsigned int brick = A.active[e >> 9];
  const int l = (int)(e & 511u);
  int i = (int)(brick % (unsigned)g.bx) * BRICK + (l & 7);
  int j = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK + ((l >> 3) & 7);
  int k = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK + (l >> 6);
  const bool ok = i < g.nx && j < g.ny && k < g.nz;
  i = min(i, g.nx - 1);
  j = min(j, g.ny - 1);
  k = min(k, g.nz - 1);
  return Cell{i, j, k, i + g.nx * (j + g.ny * k), ok};
}

// Slot e of one colour's index space of level 0 (256 slots per active brick):
// brick e/256, row m/4 of the brick (y fastest within z), x position
// 2(m%4) + parity, so no lane idles on a cell of the other colour.
__device__ __forceinline__ Cell slot_colour0(const PcgArgs& A, unsigned int e, int colour) {
  const Grid& g = A.g;
  const unsigned int brick = A.active[e >> 8];
  const int m = (int)(e & 255u);
  const int lj = (m >> 2) & 7, lk = m >> 5;
  const int li = 2 * (m & 3) + ((colour + lj + lk) & 1);
  int i = (int)(brick % (unsigned)g.bx) * BRICK + li;
  int j = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK + lj;
  int k = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK + lk;
  const bool ok = i < g.nx && j < g.ny && k < g.nz;
  i = min(i, g.nx - 1);
  j = min(j, g.ny - 1);
  k = min(k, g.nz - 1);
  return Cell{i, j, k, i + g.nx * (j + g.ny * k), ok};
}

// Slot e of one colour's index space of a dense level: each x-row has
// ceil(nx/2) slots, slot q of row (j, k) is x = 2q + parity.
__device__ __forceinline__ Cell slot_colour(const MgLevel& L, int e, int colour) {
  const int hx = (L.nx + 1) >> 1;
  const int row = e / hx, q = e - row * hx;
  const int j = row % L.ny, k = row / L.ny;
  int i = 2 * q + ((colour + j + k) & 1);
  const bool ok = i < L.nx;
  i = min(i, L.nx - 1);
  return Cell{i, j, k, i + L.nx * row, ok};
}

__device__ __forceinline__ Cell cell_at(const MgLevel& L, int c) {
  return Cell{c % L.nx, (c / L.nx) % L.ny, c / (L.nx * L.ny), c, true};
}

// ---------------------------------------------------------------- partitions

struct Part {
  int begin, end, stride;
};

// Slots of a level owned by this thread: a contiguous slice per CTA (grid-wide
// levels) or all slots by CTA 0's threads (CTA-local levels).
__device__ __forceinline__ Part level_part(int n, bool cta_local) {
  if (cta_local) return Part{(int)threadIdx.x, n, PCG_THREADS};
  int per = (n + (int)team_size() - 1) / (int)team_size();
  per = (per + 31) & ~31;
  const int b = min(n, (int)team_rank() * per);
  return Part{b + (int)threadIdx.x, min(n, b + per), PCG_THREADS};
}

// This thread's slots of level 0's colour index space: [first, end) step
// PCG_THREADS, a contiguous slice per CTA.
__device__ __forceinline__ Part colour_part0(const PcgArgs& A) {
  const unsigned int total = *A.n_active * (BRICK_CELLS / 2);
  unsigned int per = (total + team_size() - 1) / team_size();
  per = (per + 31u) & ~31u;
  const unsigned int b = min(total, team_rank() * per);
  return Part{(int)(b + threadIdx.x), (int)min(total, b + per), PCG_THREADS};
}

__device__ __forceinline__ int lcount(const MgLevel& L, int i, int j, int k) {
  return (i > 0) + (i < L.nx - 1) + (j > 0) + (j < L.ny - 1) + (k > 0) + (k < L.nz - 1);
}

// Indices of the six neighbours (-x, +x, -y, +y, -z, +z); the cell itself
// where a neighbour is off the grid.
__device__ __forceinline__ void nbr_index(const MgLevel& L, const Cell& cl, int (&idx)[6]) {
  const int sy = L.nx, sz = L.nx * L.ny;
  idx[0] = cl.i > 0 ? cl.c - 1 : cl.c;
  idx[1] = cl.i < L.nx - 1 ? cl.c + 1 : cl.c;
  idx[2] = cl.j > 0 ? cl.c - sy : cl.c;
  idx[3] = cl.j < L.ny - 1 ? cl.c + sy : cl.c;
  idx[4] = cl.k > 0 ? cl.c - sz : cl.c;
  idx[5] = cl.k < L.nz - 1 ? cl.c + sz : cl.c;
}

__device__ __forceinline__ uint8_t make_code(const MgLevel& L, const uint8_t* fl, const Cell& cl) {
  const bool in[6] = {cl.i > 0, cl.i < L.nx - 1, cl.j > 0, cl.j < L.ny - 1, cl.k > 0,
                      cl.k < L.nz - 1};
  int idx[6];
  nbr_index(L, cl, idx);
  unsigned int code = (fl[cl.c] == 1) ? CODE_SELF : 0u;
#pragma unroll
  for (int q = 0; q < 6; ++q)
    if (in[q] && fl[idx[q]] == 1) code |= 1u << q;
  return (uint8_t)code;
}

// Index of the parent (level l+1 cell) of the level-l cell (i, j, k).
__device__ __forceinline__ int parent_index(const MgLevel& C, int i, int j, int k) {
  return (i >> 1) + C.nx * ((j >> 1) + C.ny * (k >> 1));
}

// ---------------------------------------------------------------- arithmetic

enum SweepMode { FIRST = 0, NORMAL = 1, CORRECT = 2 };

// One Gauss-Seidel update of a cell: x_c = b_c / (s n_c) + (sum of fluid
// neighbours' x) / n_c, with n_c the count of neighbours inside the grid.
__device__ __forceinline__ float gs_first(const MgLevel& L, int cnt, float bc) {
  return __fmul_rn(bc, L.inv_scnt[cnt]);
}

__device__ __forceinline__ float gs_sum(const MgArgs& M, const MgLevel& L, int cnt,
                                        unsigned int code, float bc, const float (&xv)[6]) {
  const float base = __fmul_rn(bc, L.inv_scnt[cnt]);
  float sum = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) sum += ((code >> q) & 1u) ? xv[q] : 0.0f;
  return __fmaf_rn(sum, M.inv_cnt[cnt], base);
}

// Residual b - A x of a fluid cell, A x in difference form
// s (sum_fluid (x_c - x_n) + n_air x_c).
__device__ __forceinline__ float resid(const MgLevel& L, int cnt, unsigned int code, float bc,
                                       float xc, const float (&xv)[6]) {
  float d = 0.0f;
  int nfl = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const bool f = (code >> q) & 1u;
    d += f ? __fsub_rn(xc, xv[q]) : 0.0f;
    nfl += f;
  }
  return __fsub_rn(bc, __fmul_rn(L.s, __fmaf_rn((float)(cnt - nfl), xc, d)));
}

// ---------------------------------------------------------------- sweeps

struct GsIn {
  Cell cl;
  unsigned int code;
  float b;
  float xv[6];
  float pv[6];  // CORRECT: the neighbours' parents on the next coarser level
};

// Loads of a Gauss-Seidel update on level L (b from bsrc; C is the next coarser
// level, read in CORRECT mode).  COND: skip the value loads of cells that are
// not fluid (worth it where many slots are air).
template <int MODE, bool COND>
__device__ __forceinline__ void gs_load(const MgLevel& L, const MgLevel& C, const float* bsrc,
                                        GsIn& s) {
  if (COND && !(s.code & CODE_SELF)) return;
  s.b = bsrc[s.cl.c];
  if constexpr (MODE != FIRST) {
    int idx[6];
    nbr_index(L, s.cl, idx);
#pragma unroll
    for (int q = 0; q < 6; ++q) s.xv[q] = L.x[idx[q]];
  }
  if constexpr (MODE == CORRECT) {
    const int i = s.cl.i, j = s.cl.j, k = s.cl.k;
    const int pi[6] = {max(i - 1, 0), min(i + 1, L.nx - 1), i, i, i, i};
    const int pj[6] = {j, j, max(j - 1, 0), min(j + 1, L.ny - 1), j, j};
    const int pk[6] = {k, k, k, k, max(k - 1, 0), min(k + 1, L.nz - 1)};
#pragma unroll
    for (int q = 0; q < 6; ++q) s.pv[q] = C.x[parent_index(C, pi[q], pj[q], pk[q])];
  }
}

// The update of a loaded cell; returns false for slots that are not fluid cells.
template <int MODE>
__device__ __forceinline__ bool gs_apply(const MgArgs& M, const MgLevel& L, GsIn& s, float& v) {
  if (!s.cl.ok || !(s.code & CODE_SELF)) return false;
  const int cnt = lcount(L, s.cl.i, s.cl.j, s.cl.k);
  if constexpr (MODE == FIRST) {
    v = gs_first(L, cnt, s.b);
  } else {
    if constexpr (MODE == CORRECT) {
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if ((s.code >> q) & 1u) s.xv[q] = __fmaf_rn(M.omega, s.pv[q], s.xv[q]);
    }
    v = gs_sum(M, L, cnt, s.code, s.b, s.xv);
  }
  L.x[s.cl.c] = v;
  return true;
}

// Half-sweep of one colour over level 0; the right-hand side is the CG residual.
// With rz, also accumulates r z over the updated cells (the last half-sweep of
// each colour gives the final z of that colour).
template <int MODE>
__device__ __noinline__ void sweep_level0(const PcgArgs& A, int colour, FF* rz) {
  constexpr int U = (MODE == CORRECT) ? 2 : 4;
  const MgArgs& M = A.mg;
  const MgLevel& L0 = M.lv[0];
  const MgLevel& L1 = M.lv[M.nlev > 1 ? 1 : 0];
  const Part p = colour_part0(A);
  FF acc;
  run_batched<U>(
      (unsigned)p.begin, (unsigned)p.end, (unsigned)p.stride,
      [&](unsigned int e, bool ok) {
        GsIn s;
        s.cl = slot_colour0(A, e, colour);
        s.cl.ok &= ok;
        s.code = L0.code[s.cl.c];
        return s;
      },
      [&](GsIn& s) { gs_load<MODE, false>(L0, L1, A.r, s); },
      [&](GsIn& s) {
        float v;
        if (gs_apply<MODE>(M, L0, s, v) && rz) acc.add_prod(s.b, v);
      });
  if (rz) {
    // fold this pass's pair into the caller's accumulator
    rz->add_prod(acc.hi, 1.0f);
    rz->add_prod(acc.lo, 1.0f);
  }
}

// Half-sweep of one colour over a coarse level L (next coarser level C).
template <int MODE>
__device__ __noinline__ void sweep_level(const MgArgs& M, const MgLevel& L, const MgLevel& C,
                                         int colour, bool cta_local) {
  constexpr int U = (MODE == CORRECT) ? 2 : 4;
  const Part p = level_part(((L.nx + 1) >> 1) * L.ny * L.nz, cta_local);
  run_batched<U>(
      (unsigned)p.begin, (unsigned)p.end, (unsigned)p.stride,
      [&](unsigned int e, bool ok) {
        GsIn s;
        s.cl = slot_colour(L, (int)e, colour);
        s.cl.ok &= ok;
        s.code = L.code[s.cl.c];
        return s;
      },
      [&](GsIn& s) { gs_load<MODE, true>(L, C, L.b, s); },
      [&](GsIn& s) {
        float v;
        gs_apply<MODE>(M, L, s, v);
      });
}

// ---------------------------------------------------------------- restriction

// Residual of the red child (dy, dz) of coarse cell (I, J, K): the x offset
// makes 2I+dx + 2J+dy + 2K+dz even.
struct ChildIn {
  Cell cl;
  unsigned int code;
  float b, xc;
  float xv[6];
};

__device__ __forceinline__ void child_load(const MgLevel& F, const float* fb, const Cell& p,
                                           int dy, int dz, ChildIn& s) {
  const int dx = (dy + dz) & 1;
  int i = 2 * p.i + dx, j = 2 * p.j + dy, k = 2 * p.k + dz;
  s.cl.ok = i < F.nx && j < F.ny && k < F.nz;
  i = min(i, F.nx - 1);
  j = min(j, F.ny - 1);
  k = min(k, F.nz - 1);
  s.cl.i = i;
  s.cl.j = j;
  s.cl.k = k;
  s.cl.c = i + F.nx * (j + F.ny * k);
  s.code = F.code[s.cl.c];
  s.b = fb[s.cl.c];
  s.xc = F.x[s.cl.c];
  int idx[6];
  nbr_index(F, s.cl, idx);
#pragma unroll
  for (int q = 0; q < 6; ++q) s.xv[q] = F.x[idx[q]];
}

// b_{l+1} = (1/16) sum over fluid children of the level-l residual.  The
// restriction follows the pre-smoothing, whose last half-sweep is black: a black
// cell's update solves its own equation against the red neighbours it read, so
// its residual is exactly zero and only the red children contribute.  The four
// red children are loaded two at a time and summed in the order (dy, dz) =
// (0,0), (1,0), (0,1), (1,1).
__device__ __forceinline__ void restrict_cell(const MgLevel& F, const MgLevel& C, const float* fb,
                                              const Cell& p) {
  float sum = 0.0f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    ChildIn ch[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) child_load(F, fb, p, q, h, ch[q]);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const ChildIn& c = ch[q];
      if (!c.cl.ok || !(c.code & CODE_SELF)) continue;
      sum = __fadd_rn(sum, resid(F, lcount(F, c.cl.i, c.cl.j, c.cl.k), c.code, c.b, c.xc, c.xv));
    }
  }
  C.b[p.c] = __fmul_rn(sum, 0.0625f);
}

// Level 0 -> 1.  Coarse cells are taken per active fine brick (a 4x4x4 block of
// level 1 whose children all lie in that brick), so no slot falls in the air
// outside the active bricks.
__device__ __noinline__ void restrict_level0(const PcgArgs& A) {
  const MgArgs& M = A.mg;
  const MgLevel& F = M.lv[0];
  const MgLevel& C = M.lv[1];
  const Grid& g = A.g;
  const unsigned int total = *A.n_active * 64u;
  unsigned int per = (total + team_size() - 1) / team_size();
  per = (per + 31u) & ~31u;
  const unsigned int b = min(total, team_rank() * per), end = min(total, b + per);
  for (unsigned int e = b + threadIdx.x; e < end; e += PCG_THREADS) {
    const unsigned int brick = A.active[e >> 6];
    const int m = (int)(e & 63u);
    const int i = (int)(brick % (unsigned)g.bx) * (BRICK / 2) + (m & 3);
    const int j = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * (BRICK / 2) + ((m >> 2) & 3);
    const int k = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * (BRICK / 2) + (m >> 4);
    if (i >= C.nx || j >= C.ny || k >= C.nz) continue;
    const Cell p{i, j, k, i + C.nx * (j + C.ny * k), true};
    if (!(C.code[p.c] & CODE_SELF)) continue;
    restrict_cell(F, C, A.r, p);
  }
}

// Coarse level F -> C, over C's cells.
__device__ __noinline__ void restrict_level(const MgLevel& F, const MgLevel& C, bool cta_local) {
  const Part p = level_part(C.ncells, cta_local);
  for (int c = p.begin; c < p.end; c += p.stride) {
    if (!(C.code[c] & CODE_SELF)) continue;
    restrict_cell(F, C, F.b, cell_at(C, c));
  }
}

// ---------------------------------------------------------------- cycle pieces

struct Sync {
  const PcgArgs* A;
  bool cta_local;
  __device__ __forceinline__ bool operator()() const {
    if (cta_local) {
      __syncthreads();
      return true;
    }
    return grid_barrier(A->bar, A->status, team_size(), A->timeout_ns);
  }
};

// Pre-smoothing of coarse level L from zero, then restriction to C.
__device__ __forceinline__ bool down_level(const PcgArgs& A, const MgLevel& L, const MgLevel& C,
                                           bool cta_local) {
  const MgArgs& M = A.mg;
  const Sync sync{&A, cta_local};
  sweep_level<FIRST>(M, L, C, 0, cta_local);
  if (!sync()) return false;
  sweep_level<NORMAL>(M, L, C, 1, cta_local);
  if (!sync()) return false;
  for (int s = 1; s < M.nu; ++s) {
    sweep_level<NORMAL>(M, L, C, 0, cta_local);
    if (!sync()) return false;
    sweep_level<NORMAL>(M, L, C, 1, cta_local);
    if (!sync()) return false;
  }
  restrict_level(L, C, cta_local);
  return sync();
}

// Coarse correction from C + post-smoothing of coarse level L.
__device__ __forceinline__ bool up_level(const PcgArgs& A, const MgLevel& L, const MgLevel& C,
                                         bool cta_local) {
  const MgArgs& M = A.mg;
  const Sync sync{&A, cta_local};
  sweep_level<CORRECT>(M, L, C, 1, cta_local);
  if (!sync()) return false;
  sweep_level<NORMAL>(M, L, C, 0, cta_local);
  if (!sync()) return false;
  for (int s = 1; s < M.nu; ++s) {
    sweep_level<NORMAL>(M, L, C, 1, cta_local);
    if (!sync()) return false;
    sweep_level<NORMAL>(M, L, C, 0, cta_local);
    if (!sync()) return false;
  }
  return true;
}

// The coarsest level: MG_COARSE_SWEEPS (red, black) pairs from zero, then as many
// (black, red) pairs.
__device__ __forceinline__ bool coarsest_level(const PcgArgs& A, const MgLevel& L, bool cta_local) {
  const MgArgs& M = A.mg;
  const Sync sync{&A, cta_local};
  sweep_level<FIRST>(M, L, L, 0, cta_local);
  if (!sync()) return false;
  sweep_level<NORMAL>(M, L, L, 1, cta_local);
  if (!sync()) return false;
  for (int s = 1; s < MG_COARSE_SWEEPS; ++s) {
    sweep_level<NORMAL>(M, L, L, 0, cta_local);
    if (!sync()) return false;
    sweep_level<NORMAL>(M, L, L, 1, cta_local);
    if (!sync()) return false;
  }
  for (int s = 0; s < MG_COARSE_SWEEPS; ++s) {
    sweep_level<NORMAL>(M, L, L, 1, cta_local);
    if (!sync()) return false;
    sweep_level<NORMAL>(M, L, L, 0, cta_local);
    if (!sync()) return false;
  }
  return true;
}

// The CTA-local levels [lgrid, nlev) live in shared memory of CTA 0: x, b and
// the codes of every such level (MG_CTA_CELLS cells in total at most).
struct CtaMg {
  float x[MG_CTA_CELLS];
  float b[MG_CTA_CELLS];
  uint8_t code[MG_CTA_CELLS];
  MgLevel lv[MG_MAX_LEVELS];  // level descriptions pointing into the arrays above
};

// Points the shared level descriptions at the shared arrays and loads the codes
// (once per solve, after build_levels).  CTA 0 only.
__device__ __noinline__ void cta_levels_init(const MgArgs& M, CtaMg& sm) {
  if (threadIdx.x == 0) {
    int off = 0;
    for (int l = M.lgrid; l < M.nlev; ++l) {
      sm.lv[l] = M.lv[l];
      sm.lv[l].x = sm.x + off;
      sm.lv[l].b = sm.b + off;
      sm.lv[l].code = sm.code + off;
      sm.lv[l].t = nullptr;
      off += M.lv[l].ncells;
    }
  }
  __syncthreads();
  for (int l = M.lgrid; l < M.nlev; ++l)
    for (int c = threadIdx.x; c < M.lv[l].ncells; c += PCG_THREADS) sm.lv[l].code[c] = M.lv[l].code[c];
  __syncthreads();
}

// Levels [lgrid, nlev) inside CTA 0, from the right-hand side that the grid-wide
// restriction left in level lgrid's global b; leaves level lgrid's x in global
// memory for the correction of level lgrid - 1.
__device__ __noinline__ void cta_cycle(const PcgArgs& A, CtaMg& sm) {
  const MgArgs& M = A.mg;
  const int lg = M.lgrid;
  for (int c = threadIdx.x; c < M.lv[lg].ncells; c += PCG_THREADS) sm.lv[lg].b[c] = M.lv[lg].b[c];
  __syncthreads();
  for (int l = lg; l < M.nlev - 1; ++l) down_level(A, sm.lv[l], sm.lv[l + 1], true);
  coarsest_level(A, sm.lv[M.nlev - 1], true);
  for (int l = M.nlev - 2; l >= lg; --l) up_level(A, sm.lv[l], sm.lv[l + 1], true);
  for (int c = threadIdx.x; c < M.lv[lg].ncells; c += PCG_THREADS) M.lv[lg].x[c] = sm.lv[lg].x[c];
}

// z = V(r), given that the first red half-sweep of level 0 (from zero) has been
// done in the phase that produced r, and that a grid barrier has passed since.
// The last black and the last red half-sweeps of level 0 accumulate r.z over
// their cells into rz.  The caller publishes rz and meets the next barrier.
// Returns false if a barrier failed.
__device__ bool vcycle_rest(const PcgArgs& A, CtaMg& sm, FF& rz) {
  const MgArgs& M = A.mg;
  const Sync gsync{&A, false};
  if (M.nlev == 1) {  // level 0 is the coarsest level
    // rest of the pre pairs (red, black) after the fused first red half-sweep
    for (int s = 0; s < MG_COARSE_SWEEPS; ++s) {
      sweep_level0<NORMAL>(A, 1, nullptr);
      if (!gsync()) return false;
      if (s + 1 < MG_COARSE_SWEEPS) {
        sweep_level0<NORMAL>(A, 0, nullptr);
        if (!gsync()) return false;
      }
    }
    // post pairs (black, red); the last black and the last red give r.z
    for (int s = 0; s < MG_COARSE_SWEEPS; ++s) {
      sweep_level0<NORMAL>(A, 1, s + 1 == MG_COARSE_SWEEPS ? &rz : nullptr);
      if (!gsync()) return false;
      if (s + 1 < MG_COARSE_SWEEPS) {
        sweep_level0<NORMAL>(A, 0, nullptr);
        if (!gsync()) return false;
      }
    }
    sweep_level0<NORMAL>(A, 0, &rz);
    return true;
  }
  sweep_level0<NORMAL>(A, 1, nullptr);
  if (!gsync()) return false;
  for (int s = 1; s < M.nu; ++s) {
    sweep_level0<NORMAL>(A, 0, nullptr);
    if (!gsync()) return false;
    sweep_level0<NORMAL>(A, 1, nullptr);
    if (!gsync()) return false;
  }
  restrict_level0(A);
  if (!gsync()) return false;
  for (int l = 1; l < M.lgrid; ++l)
    if (!down_level(A, M.lv[l], M.lv[l + 1], false)) return false;
  if (team_rank() == 0) cta_cycle(A, sm);
  if (!gsync()) return false;
  for (int l = M.lgrid - 1; l >= 1; --l)
    if (!up_level(A, M.lv[l], M.lv[l + 1], false)) return false;
  sweep_level0<CORRECT>(A, 1, M.nu == 1 ? &rz : nullptr);
  if (!gsync()) return false;
  for (int s = 1; s < M.nu; ++s) {
    sweep_level0<NORMAL>(A, 0, nullptr);
    if (!gsync()) return false;
    sweep_level0<NORMAL>(A, 1, s + 1 == M.nu ? &rz : nullptr);
    if (!gsync()) return false;
  }
  sweep_level0<NORMAL>(A, 0, &rz);  // the last red half-sweep
  return true;
}

// ---------------------------------------------------------------- level-0 passes

// This thread's slots of level 0's active-cell index space.
__device__ __forceinline__ Part dense_part0(const Chunk& ch) {
  return Part{(int)(ch.begin + threadIdx.x), (int)ch.end, PCG_THREADS};
}

// Phase A with z from the V-cycle: p_new = z + beta p_old (recomputed for the
// neighbours), q = A p_new in difference form, partial p.q.
__device__ __noinline__ void phase_a(const PcgArgs& A, const Chunk& ch, const float* z,
                                        const float* pold, float* pnew, float beta, FF& pq) {
  const MgLevel& L0 = A.mg.lv[0];
  const Part p = dense_part0(ch);
  struct S {
    Cell cl;
    unsigned int code;
    float zc, pc;
    float zv[6], pv[6];
  };
  run_batched<2>(
      (unsigned)p.begin, (unsigned)p.end, (unsigned)p.stride,
      [&](unsigned int e, bool ok) {
        S s;
        s.cl = slot_dense0(A, e);
        s.cl.ok &= ok;
        s.code = L0.code[s.cl.c];
        s.zc = z[s.cl.c];
        s.pc = pold[s.cl.c];
        int idx[6];
        nbr_index(L0, s.cl, idx);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          s.zv[q] = z[idx[q]];
          s.pv[q] = pold[idx[q]];
        }
        return s;
      },
      [&](S&) {},
      [&](S& s) {
        if (!s.cl.ok || !(s.code & CODE_SELF)) return;
        const int cnt = lcount(L0, s.cl.i, s.cl.j, s.cl.k);
        const float pc = __fmaf_rn(beta, s.pc, s.zc);
        float d = 0.0f;
        int nfl = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const bool f = (s.code >> q) & 1u;
          d += f ? __fsub_rn(pc, __fmaf_rn(beta, s.pv[q], s.zv[q])) : 0.0f;
          nfl += f;
        }
        const float qc = __fmul_rn(A.s, __fmaf_rn((float)(cnt - nfl), pc, d));
        pnew[s.cl.c] = pc;
        A.q[s.cl.c] = qc;
        pq.add_prod(pc, qc);
      });
}

// Phase B: x += alpha p, r -= alpha q, partial r.r, and the next V-cycle's first
// red half-sweep (from zero) z = r / (s n) on red cells.
__device__ __noinline__ void phase_b(const PcgArgs& A, const Chunk& ch, float* x, float* z,
                                        const float* pnew, float alpha, FF& rr) {
  const MgLevel& L0 = A.mg.lv[0];
  const Part p = dense_part0(ch);
  struct S {
    Cell cl;
    unsigned int code;
    float x, p, q, r;
  };
  run_batched<4>(
      (unsigned)p.begin, (unsigned)p.end, (unsigned)p.stride,
      [&](unsigned int e, bool ok) {
        S s;
        s.cl = slot_dense0(A, e);
        s.cl.ok &= ok;
        s.code = L0.code[s.cl.c];
        s.x = x[s.cl.c];
        s.p = pnew[s.cl.c];
        s.q = A.q[s.cl.c];
        s.r = A.r[s.cl.c];
        return s;
      },
      [&](S&) {},
      [&](S& s) {
        if (!s.cl.ok || !(s.code & CODE_SELF)) return;
        const int c = s.cl.c;
        x[c] = __fmaf_rn(alpha, s.p, s.x);
        const float rc = __fmaf_rn(-alpha, s.q, s.r);
        A.r[c] = rc;
        if (((s.cl.i + s.cl.j + s.cl.k) & 1) == 0)
          z[c] = gs_first(L0, lcount(L0, s.cl.i, s.cl.j, s.cl.k), rc);
        rr.add_prod(rc, rc);
      });
}

// One pass over this thread's fluid cells of level 0 (start of the solve and the
// rare refinement passes; not batched).
template <class F>
__device__ __forceinline__ void for_fluid0(const PcgArgs& A, const Chunk& ch, F&& f) {
  const MgLevel& L0 = A.mg.lv[0];
  for (unsigned int e = ch.begin + threadIdx.x; e < ch.end; e += PCG_THREADS) {
    const Cell cl = slot_dense0(A, e);
    if (!cl.ok || !(L0.code[cl.c] & CODE_SELF)) continue;
    f(cl);
  }
}

// FP64 residual of one cell for the refinement: b - A x with x in FP64.
__device__ __forceinline__ double residual64(const PcgArgs& A, const Cell& cl) {
  const MgLevel& L0 = A.mg.lv[0];
  const unsigned int code = L0.code[cl.c];
  int idx[6];
  nbr_index(L0, cl, idx);
  const double xc = A.x64[cl.c];
  double xv[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) xv[q] = A.x64[idx[q]];
  double d = 0.0;
  int nfl = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const bool f = (code >> q) & 1u;
    d += f ? xc - xv[q] : 0.0;
    nfl += f;
  }
  const int cnt = lcount(L0, cl.i, cl.j, cl.k);
  return A.b64[cl.c] - A.s64 * ((double)(cnt - nfl) * xc + d);
}

// Builds the neighbour codes of level 0 (cells of active bricks), the fluid flags
// of levels 1.. (a coarse cell is fluid when any child is) and their codes.
// Ends with a grid barrier.
__device__ __noinline__ bool build_levels(const PcgArgs& A, const Chunk& ch) {
  const MgArgs& M = A.mg;
  const MgLevel& L0 = M.lv[0];
  for (unsigned int e = ch.begin + threadIdx.x; e < ch.end; e += PCG_THREADS) {
    const Cell cl = slot_dense0(A, e);
    if (cl.ok) L0.code[cl.c] = make_code(L0, A.type, cl);
  }
  for (int l = 1; l < M.nlev; ++l) {
    const MgLevel& F = M.lv[l - 1];
    const MgLevel& C = M.lv[l];
    const Part p = level_part(C.ncells, false);
    for (int c = p.begin; c < p.end; c += p.stride) {
      const int i = c % C.nx, j = (c / C.nx) % C.ny, k = c / (C.nx * C.ny);
      uint8_t f = 0;
      for (int d = 0; d < 8; ++d) {
        const int fi = 2 * i + (d & 1), fj = 2 * j + ((d >> 1) & 1), fk = 2 * k + (d >> 2);
        if (fi < F.nx && fj < F.ny && fk < F.nz && F.t[fi + F.nx * (fj + F.ny * fk)] == 1) f = 1;
      }
      C.t[c] = f;
    }
    if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) return false;
  }
  for (int l = 1; l < M.nlev; ++l) {
    const MgLevel& C = M.lv[l];
    const Part p = level_part(C.ncells, false);
    for (int c = p.begin; c < p.end; c += p.stride) C.code[c] = make_code(C, C.t, cell_at(C, c));
  }
  return grid_barrier(A.bar, A.status, team_size(), A.timeout_ns);
}

struct SolveState {
  int iters = 0;
  int refinements = 0;
  bool conv = false;
  bool ok = true;
  double rel = 0.0;
  double bnorm = 0.0;
};

// Partial-sum slots (float pairs): 0 = p.q (phase A), 1 = r.r (phase B),
// 3 = r.z (end of the V-cycle), 4 = ||b||^2 (start), 5 = FP64 residual norm
// (refinement).  A slot's readers always pass another barrier before the slot
// is written again.
template <bool MIXED>
__device__ void solve_mg(const PcgArgs& A, const Chunk& ch, Shared& sh, CtaMg& sm,
                         SolveState& S) {
  float* x = A.x32;
  float* z = A.mg.lv[0].x;
  const MgLevel& L0 = A.mg.lv[0];
  if (!build_levels(A, ch)) { S.ok = false; return; }
  if (A.mg.nlev > 1 && team_rank() == 0) cta_levels_init(A.mg, sm);
  // ---- start: r = b, x = 0, p_old = 0, first red half-sweep of the V-cycle
  {
    FF bb;
    for_fluid0(A, ch, [&](const Cell& cl) {
      const float bc = MIXED ? (float)A.b64[cl.c] : A.b32[cl.c];
      A.r[cl.c] = bc;
      x[cl.c] = 0.0f;
      A.pa[cl.c] = 0.0f;
      if (((cl.i + cl.j + cl.k) & 1) == 0) z[cl.c] = gs_first(L0, lcount(L0, cl.i, cl.j, cl.k), bc);
      bb.add_prod(bc, bc);
    });
    F2 v[1] = {f2_of(bb)};
    publish<1>(A, 4, v, sh);
  }
  if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
  double rz = 0.0, bnorm = 0.0, rnorm = 0.0, rmax = 0.0;
  const double target = MIXED ? A.ir_tol : A.tol;
  {
    double s0[1];
    gather<1>(A, 4, s0, sh);
    if (threadIdx.x == 0) {
      bnorm = sqrt(fmax(s0[0], 0.0));
      rnorm = rmax = bnorm;
      sh.flag = (bnorm == 0.0) ? 1 : 0;
    }
  }
  __syncthreads();
  int it = 0, refinements = 0;
  bool conv = sh.flag == 1, first = true;
  float* pold = A.pa;
  float* pnew = A.pb;
  while (!conv) {
    FF rzp;
    if (!vcycle_rest(A, sm, rzp)) { S.ok = false; return; }
    {
      F2 v[1] = {f2_of(rzp)};
      publish<1>(A, 3, v, sh);
    }
    if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
    {
      double s[1];
      gather<1>(A, 3, s, sh);
      if (threadIdx.x == 0) {
        sh.beta = first ? 0.0f : (float)(s[0] / rz);
        rz = s[0];
        if (sh.flag == 0 && it >= A.max_iter) sh.flag = 3;
      }
    }
    __syncthreads();
    if (sh.flag == 1) { conv = true; break; }
    if (sh.flag == 3) break;
    first = false;
    ++it;
    const float beta = sh.beta;
    // ---- phase A
    FF pq;
    phase_a(A, ch, z, pold, pnew, beta, pq);
    {
      F2 v[1] = {f2_of(pq)};
      publish<1>(A, 0, v, sh);
    }
    if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
    {
      double s[1];
      gather<1>(A, 0, s, sh);
      if (threadIdx.x == 0) sh.alpha = (float)(rz / s[0]);
    }
    __syncthreads();
    const float alpha = sh.alpha;
    // ---- phase B (+ the next V-cycle's first red half-sweep)
    FF rr;
    phase_b(A, ch, x, z, pnew, alpha, rr);
    {
      F2 v[1] = {f2_of(rr)};
      publish<1>(A, 1, v, sh);
    }
    if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
    {
      double s[1];
      gather<1>(A, 1, s, sh);
      if (threadIdx.x == 0) {
        rnorm = sqrt(fmax(s[0], 0.0));
        int f = 0;  // 0 continue, 1 converged, 2 refine
        if (rnorm <= target * bnorm) f = MIXED ? 2 : 1;
        else if (MIXED && rnorm <= A.tol * rmax) f = 2;
        sh.flag = f;
      }
    }
    __syncthreads();
    float* t = pold; pold = pnew; pnew = t;
    if constexpr (MIXED) {
      if (sh.flag == 2) {
        // ---- refinement: x64 += d, d = 0; r = b - A x64 in FP64 (+ first red half-sweep)
        for_fluid0(A, ch, [&](const Cell& cl) {
          A.x64[cl.c] += (double)x[cl.c];
          x[cl.c] = 0.0f;
        });
        if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
        FF rr64;
        for_fluid0(A, ch, [&](const Cell& cl) {
          const float r32 = (float)residual64(A, cl);
          A.r[cl.c] = r32;
          if (((cl.i + cl.j + cl.k) & 1) == 0)
            z[cl.c] = gs_first(L0, lcount(L0, cl.i, cl.j, cl.k), r32);
          rr64.add_prod(r32, r32);
        });
        F2 v[1] = {f2_of(rr64)};
        publish<1>(A, 5, v, sh);
        if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
        double s[1];
        gather<1>(A, 5, s, sh);
        ++refinements;
        if (threadIdx.x == 0) {
          rnorm = sqrt(fmax(s[0], 0.0));
          rmax = rnorm;
          if (rnorm <= target * bnorm) sh.flag = 1;
          else if (refinements >= A.ir_max_iter) sh.flag = 3;
          else sh.flag = 0;
        }
        __syncthreads();
        if (sh.flag == 1) { conv = true; break; }
        if (sh.flag == 3) break;
        continue;  // the refinement's barrier has made the fused red half-sweep visible
      }
    }
    if (sh.flag == 1) { conv = true; break; }
  }
  if constexpr (MIXED) {
    if (!conv) {
      for_fluid0(A, ch, [&](const Cell& cl) {
        A.x64[cl.c] += (double)x[cl.c];
        x[cl.c] = 0.0f;
      });
    }
    for_fluid0(A, ch, [&](const Cell& cl) {
      const double xv = A.x64[cl.c];
      const float hi = __double2float_rn(xv);
      const float lo = __double2float_rn(xv - (double)hi);
      A.pff[cl.c] = make_float2(hi, lo);
    });
  }
  S.iters = it;
  S.refinements = refinements;
  S.conv = conv;
  S.rel = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  S.bnorm = bnorm;
}

template <bool MIXED>
__device__ void solve_scene_mg(const PcgArgs& A, Shared& sh, CtaMg& sm) {
  const unsigned int nact = *A.n_active;
  const long long ncells = (long long)A.g.nx * A.g.ny * A.g.nz;
  const bool singular = A.check_singular && ((long long)A.stats->n_fluid == ncells);
  SolveState S;
  if (!singular) solve_mg<MIXED>(A, my_chunk(nact), sh, sm, S);
  if (team_rank() == 0 && threadIdx.x == 0) {
    int st = 0;
    if (singular) st |= DEV_SINGULAR;
    else if (S.ok && !S.conv) st |= DEV_NOT_CONVERGED;
    if (st) atomicOr(A.status, st);
    A.stats->cg_iters = S.iters;
    A.stats->ir_iters = S.refinements;
    A.stats->cg_iters_total += S.iters;
    A.stats->ir_iters_total += S.refinements;
    A.stats->rel_res = S.rel;
    A.stats->bnorm = S.bnorm;
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg_mg(const __grid_constant__ PcgArgs A) {
  __shared__ Shared sh;
  __shared__ CtaMg sm;
  team_enter(blockIdx.x, gridDim.x);
  solve_scene_mg<MIXED>(A, sh, sm);
}

// Several scenes in one launch: CTA b works on scene block_scene[b], in the team
// of CTAs team_first[s] .. team_first[s+1]-1.
template <bool MIXED>
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg_mg_batch(const __grid_constant__ PcgBatch B) {
  __shared__ Shared sh;
  __shared__ CtaMg sm;
  const int s = B.block_scene[blockIdx.x];
  team_enter(blockIdx.x - B.team_first[s], B.team_first[s + 1] - B.team_first[s]);
  solve_scene_mg<MIXED>(B.args[s], sh, sm);
}

}  // namespace

int mg_level_dims(int nx, int ny, int nz, int dims[MG_MAX_LEVELS][3]) {
  int n[3] = {nx, ny, nz};
  int L = 0;
  for (;;) {
    for (int a = 0; a < 3; ++a) dims[L][a] = n[a];
    ++L;
    const int m = n[0] > n[1] ? (n[0] > n[2] ? n[0] : n[2]) : (n[1] > n[2] ? n[1] : n[2]);
    if (m <= 4 || L == MG_MAX_LEVELS) break;
    for (int a = 0; a < 3; ++a) n[a] = (n[a] + 1) / 2;
  }
  return L;
}

cudaError_t launch_pcg_mg(const PcgArgs& a, bool mixed, int nblocks, cudaStream_t s) {
  void* args[] = {const_cast<PcgArgs*>(&a)};
  if (mixed)
    return cudaLaunchCooperativeKernel((const void*)k_pcg_mg<true>, dim3(nblocks),
                                       dim3(PCG_THREADS), args, 0, s);
  return cudaLaunchCooperativeKernel((const void*)k_pcg_mg<false>, dim3(nblocks),
                                     dim3(PCG_THREADS), args, 0, s);
}

cudaError_t launch_pcg_mg_batch(const PcgBatch& b, bool mixed, int nblocks, cudaStream_t s) {
  void* args[] = {const_cast<PcgBatch*>(&b)};
  if (mixed)
    return cudaLaunchCooperativeKernel((const void*)k_pcg_mg_batch<true>, dim3(nblocks),
                                       dim3(PCG_THREADS), args, 0, s);
  return cudaLaunchCooperativeKernel((const void*)k_pcg_mg_batch<false>, dim3(nblocks),
                                     dim3(PCG_THREADS), args, 0, s);
}

cudaError_t pcg_mg_check_occupancy() {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg_mg<false>, PCG_THREADS, 0);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg_mg<true>, PCG_THREADS, 0);
  if (e != cudaSuccess) return e;
  return (a >= 1 && b >= 1) ? cudaSuccess : cudaErrorInvalidConfiguration;
}

}  // namespace flipk
