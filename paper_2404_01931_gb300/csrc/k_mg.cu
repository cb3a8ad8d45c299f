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
// Layout and work split.  The grid-wide levels (l < lgrid) are stored
// colour-split (see MgLevel): a half-sweep reads and writes contiguous runs of
// one colour and its six neighbour runs of the other colour, so it moves half
// the bytes of a natural-layout sweep, every access coalesced.  Work is a list
// of active segments per level (64 cells of a row that meet a block holding
// fluid), built at the start of every solve; a warp takes one segment, a lane
// one slot, and each CTA a contiguous slice of the list.  Per cell one 16-bit
// code carries the fluid neighbours and the neighbour count, so value loads
// never wait on flags, and each warp loads several segments before it computes
// (memory-level parallelism).  The small coarsest levels (at most MG_CTA_CELLS
// cells together) run inside CTA 0 from shared memory with __syncthreads; the
// others use grid barriers between half-sweeps.
//
// The correction is never written: the first post-smoothing half-sweep (black)
// reads its red neighbours plus omega times their parents' values, and the red
// half-sweep that follows overwrites the red cells anyway.  The first red
// half-sweep from zero only needs the residual, so it is fused into the pass
// that produces it: at level 0 the CG phase that updates r, at a grid-wide
// coarse level the restriction.  The last black and the last red half-sweeps of
// level 0 also accumulate r.z.
#include "pcg_common.cuh"

namespace flipk {

// Solve trace, in builds with -DFLIP_SOLVE_TRACE only (compiled out otherwise):
// thread 0 of the team's first CTA stamps the global timer after each phase of
// a solve into flip_trace_ns[slot] (slots below), each stamp taken after the grid
// barrier that ends its phase; flip_solve_trace copies them to the host.
#ifdef FLIP_SOLVE_TRACE
__device__ unsigned long long flip_trace_ns[64];
#define SOLVE_TRACE(slot) trace_stamp(slot)
#else
#define SOLVE_TRACE(slot) ((void)0)
#endif

enum TraceSlot {
  TR_ENTRY = 0,       // kernel entry
  TR_TABLES = 1,      // shared tables loaded
  TR_BFLAG = 2,       // block flags cleared
  TR_FLAGS = 2,       // + l: fluid flags of level l (l = 1 .. 11) built
  TR_SEG_COUNT = 14,  // active segments counted
  TR_SEG_WRITE = 15,  // active-segment lists written
  TR_CODES = 16,      // neighbour codes built
  TR_SEG_CACHE = 17,  // segment slices cached
  TR_CTA_LISTS = 18,  // CTA-local lists built (CTA 0)
  TR_START = 19,      // start pass (r, z, b) done
  TR_ITER = 20,       // + 3 i, + 1, + 2: V-cycle, phase A, phase B of iteration i (i < 3)
  TR_LOOP_END = 29,   // CG loop left
  TR_END = 30,        // solution written
  TR_EXIT = 31,       // kernel exit
  TR_V_PRE1 = 32,     // the V-cycle's pieces (the last V-cycle of the solve):
  TR_V_PRE = 33,      //   level-0 pre-smoothing (first black, the rest),
  TR_V_RESTRICT = 34, //   restriction 0 -> 1,
  TR_V_DOWN = 34,     //   + l: level l's pre-smoothing and restriction (l = 1 .. 11),
  TR_V_CTA = 46,      //   the CTA-local levels,
  TR_V_UP = 46,       //   + l: level l's correction and post-smoothing (l = 1 .. 11),
  TR_V_CORRECT = 58,  //   level-0 correction and first black half-sweep,
  TR_V_POST = 59,     //   the rest of level 0's post-smoothing but the last red
  TR_REFINE = 60      // + 0, 1, 2: the first refinement's start, x += d, residual
};

namespace {

#ifdef FLIP_SOLVE_TRACE
__device__ __forceinline__ void trace_stamp(int slot) {
  if (team_rank() == 0 && threadIdx.x == 0) flip_trace_ns[slot] = global_timer_ns();
}
#endif

constexpr unsigned int CODE_SELF = 64u;
constexpr unsigned int CODE_FULL = 0x67fu;  // fluid, six fluid neighbours, count 6
// Both cells of a slot pair's codes (16 bits each) are CODE_FULL.
__device__ __forceinline__ bool pair_full(unsigned int code2) {
  return code2 == (CODE_FULL | (CODE_FULL << 16));
}
constexpr int SEG_SLOTS = 32;  // slots of one colour per segment (a warp)

// Gauss-Seidel coefficients per level, copied to shared memory at kernel start:
// s_inv_scnt[l][n] = 1 / (s_l n), s_inv_cnt[n] = 1 / n.
__shared__ float s_inv_scnt[MG_MAX_LEVELS][8];
__shared__ float s_inv_cnt[8];

__device__ __forceinline__ void load_tables(const MgArgs& M) {
  if (threadIdx.x < MG_MAX_LEVELS * 8) {
    const int l = threadIdx.x >> 3, n = threadIdx.x & 7;
    s_inv_scnt[l][n] = l < M.nlev ? M.lv[l].inv_scnt[n] : 0.0f;
  }
  if (threadIdx.x < 8) s_inv_cnt[threadIdx.x] = M.inv_cnt[threadIdx.x];
  __syncthreads();
}

// Each CTA's slice of a level's active segments is the same in every pass of a
// solve, so after the lists are built the CTA copies its slices into shared
// memory (as many levels as SEG_CACHE holds, level 0 first): the first load of
// every item of a pass, the segment, is then a shared-memory read.  s_segc[l] is
// the copy of level l's slice (nullptr: read the list in global memory) and
// s_segb[l] the index of its first segment.
constexpr int SEG_CACHE = 1024;
__shared__ const int4* s_segc[MG_MAX_LEVELS];
__shared__ int s_segb[MG_MAX_LEVELS];

// The fields of a colour-split level a pass uses, read once into registers at
// the start of the pass (the level descriptions live in parameter or shared
// memory and would otherwise be re-read through generic pointers per cell).
// Segment t of the level is seg[t - seg_base].
struct SV {
  float* x;
  float* b;
  uint16_t* code;
  const int4* seg;
  int seg_base;
  int nx, ny, hx, half, margin, pl;
  float s;
};

__device__ __forceinline__ SV sview(const MgLevel& L) {
  const int4* c = s_segc[L.lvl];
  return SV{L.x, L.b, L.code16, c ? c : L.seg, c ? s_segb[L.lvl] : 0, L.nx, L.ny, L.hx,
            L.half, L.margin, L.hx * L.ny, L.s};
}

// The same for the level whose x a correction reads (colour-split or natural).
struct PV {
  const float* x;
  int split, nx, ny, nz, hx, half, margin;
};

__device__ __forceinline__ PV pview(const MgLevel& C) {
  return PV{C.x, C.split, C.nx, C.ny, C.nz, C.hx, C.half, C.margin};
}

// Runs items first, first + stride, ... < end in batches of U: pre(e, ok)
// returns a state with the item's first loads, load(state) adds the loads that
// depend on them, apply(state) computes and stores.  All loads of a batch come
// before its first store.  Items past the end are handed to pre() as 'first'
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

// ---------------------------------------------------------------- indexing

// Index of cell (i, j, k) of a level in its storage (colour-split or natural).
__device__ __forceinline__ int level_index(const PV& C, int i, int j, int k) {
  if (C.split) return ((i + j + k) & 1) * C.half + C.margin + C.hx * (j + C.ny * k) + (i >> 1);
  return i + C.nx * (j + C.ny * k);
}

// A slot of a colour-split level: cell (i, j, k) of row r = j + ny k, its
// storage index and the base index of its neighbours in the other colour.
struct SCell {
  int i, j, k, r;
  int idx, ob;
  int par;  // i & 1
  bool ok;
};

// Lane 'lane' of colour c in segment sg = {row, segment in row, j, k}.
template <class LV>
__device__ __forceinline__ SCell scell(const LV& L, int4 sg, int c, int lane) {
  SCell e;
  const int s = sg.y * SEG_SLOTS + lane;
  e.j = sg.z;
  e.k = sg.w;
  e.r = sg.x;
  e.par = (c + e.j + e.k) & 1;
  e.i = 2 * s + e.par;
  e.ok = s < L.hx && e.i < L.nx;
  e.idx = c * L.half + L.margin + L.hx * e.r + min(s, L.hx - 1);
  e.ob = e.idx + (1 - 2 * c) * L.half;
  return e;
}

// Storage indices of the six neighbours (-x, +x, -y, +y, -z, +z), all in the
// other colour's half; addresses of neighbours off the grid are valid but their
// values are never used (the code bit is clear).
template <class LV>
__device__ __forceinline__ void snbr(const LV& L, const SCell& e, int (&nb)[6]) {
  const int pl = L.hx * L.ny;
  nb[0] = e.ob - 1 + e.par;
  nb[1] = e.ob + e.par;
  nb[2] = e.ob - L.hx;
  nb[3] = e.ob + L.hx;
  nb[4] = e.ob - pl;
  nb[5] = e.ob + pl;
}

// This CTA's slice [q0, q1) of a level's active segments.
__device__ __forceinline__ int2 seg_slice(const MgLevel& L) {
  const int n = (int)*L.nseg;
  const int per = (n + (int)team_size() - 1) / (int)team_size();
  const int q0 = min(n, (int)team_rank() * per);
  return make_int2(q0, min(n, q0 + per));
}

// Items (segment, colour) of this CTA for ncol colours: item t is segment
// t / ncol, colour t % ncol (ncol = 2) or the pass's colour (ncol = 1).  Each
// warp takes items first, first + PCG_WARPS, ...
struct Items {
  unsigned int first, end;
};

__device__ __forceinline__ Items seg_items(const MgLevel& L, int ncol) {
  const int2 q = seg_slice(L);
  return Items{(unsigned)(q.x * ncol + (int)(threadIdx.x >> 5)), (unsigned)(q.y * ncol)};
}

// Vectorised passes: a warp takes two segments (lanes 0-15 and 16-31), a lane two
// adjacent slots s, s + 1 of one colour (s even), read and written as 8-byte
// pairs.  Items are (segment pair, colour); item t is pair t / ncol.
__device__ __forceinline__ Items pair_items(int2 q, int ncol) {
  const int npairs = (q.y - q.x + 1) >> 1;
  return Items{(unsigned)(threadIdx.x >> 5), (unsigned)(npairs * ncol)};
}

// The two cells of a lane: slots s and s + 1 of colour c in one row.
struct PCell {
  int j, k, r, s, par;
  int iA;         // x of the first cell (the second is iA + 2)
  int idx, ob;    // storage index of slot s (even) and of slot s in the other colour
  bool okA, okB;  // inside the grid (and the lane's segment exists)
};

template <class LV>
__device__ __forceinline__ PCell pcell(const LV& L, int2 q, unsigned int pair, int c, int lane) {
  int sq = q.x + 2 * (int)pair + (lane >> 4);
  const bool seg_ok = sq < q.y;
  if (!seg_ok) sq = q.x;
  const int4 sg = L.seg[sq - L.seg_base];
  PCell e;
  e.j = sg.z;
  e.k = sg.w;
  e.r = sg.x;
  e.s = sg.y * SEG_SLOTS + 2 * (lane & 15);
  e.par = (c + e.j + e.k) & 1;
  e.iA = 2 * e.s + e.par;
  const bool s_ok = seg_ok && e.s < L.hx;
  e.okA = s_ok && e.iA < L.nx;
  e.okB = s_ok && e.iA + 2 < L.nx;
  e.idx = c * L.half + L.margin + L.hx * e.r + min(e.s, L.hx - 2);
  e.ob = e.idx + (1 - 2 * c) * L.half;
  return e;
}

// The other colour's values around a slot pair: xm/xp the -x/+x neighbours of
// cells A and B, ym, yp, zm, zp the pairs in the rows and planes next door.
struct Nbr2 {
  float xmA, xpA, xmB, xpB;
  float2 ym, yp, zm, zp;
};

template <class LV>
__device__ __forceinline__ Nbr2 load_nbr2(const LV& L, const float* x, const PCell& e) {
  const float2 m = *reinterpret_cast<const float2*>(x + e.ob);
  const float ex = x[e.ob - 1 + 3 * e.par];  // slot s - 1 (par 0) or s + 2 (par 1)
  Nbr2 n;
  if (e.par == 0) {
    n.xmA = ex; n.xpA = m.x; n.xmB = m.x; n.xpB = m.y;
  } else {
    n.xmA = m.x; n.xpA = m.y; n.xmB = m.y; n.xpB = ex;
  }
  const int pl = L.hx * L.ny;
  n.ym = *reinterpret_cast<const float2*>(x + e.ob - L.hx);
  n.yp = *reinterpret_cast<const float2*>(x + e.ob + L.hx);
  n.zm = *reinterpret_cast<const float2*>(x + e.ob - pl);
  n.zp = *reinterpret_cast<const float2*>(x + e.ob + pl);
  return n;
}

__device__ __forceinline__ void nbr_of(const Nbr2& n, int which, float (&xv)[6]) {
  if (which == 0) {
    xv[0] = n.xmA; xv[1] = n.xpA; xv[2] = n.ym.x; xv[3] = n.yp.x; xv[4] = n.zm.x; xv[5] = n.zp.x;
  } else {
    xv[0] = n.xmB; xv[1] = n.xpB; xv[2] = n.ym.y; xv[3] = n.yp.y; xv[4] = n.zm.y; xv[5] = n.zp.y;
  }
}

// ---------------------------------------------------------------- natural levels

struct Cell {
  int i, j, k, c;
  bool ok;
};

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

__device__ __forceinline__ Cell cell_at(const MgLevel& L, int c) {
  return Cell{c % L.nx, (c / L.nx) % L.ny, c / (L.nx * L.ny), c, true};
}

// Neighbour code of cell (i, j, k) from natural fluid flags fl (value 1 = fluid):
// bits 0..5 fluid neighbours inside the grid, bit 6 the cell itself, bits 8..10
// the number of neighbours inside the grid.
__device__ __forceinline__ unsigned int make_code(const MgLevel& L, const uint8_t* fl, int i, int j,
                                                  int k) {
  const int c = i + L.nx * (j + L.ny * k);
  const int sy = L.nx, sz = L.nx * L.ny;
  const bool in[6] = {i > 0, i < L.nx - 1, j > 0, j < L.ny - 1, k > 0, k < L.nz - 1};
  const int off[6] = {-1, 1, -sy, sy, -sz, sz};
  unsigned int code = (fl[c] == 1) ? CODE_SELF : 0u;
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    cnt += in[q];
    if (in[q] && fl[c + off[q]] == 1) code |= 1u << q;
  }
  return code | ((unsigned)cnt << 8);
}

// ---------------------------------------------------------------- arithmetic

enum SweepMode { FIRST = 0, NORMAL = 1, CORRECT = 2 };

__device__ __forceinline__ int code_cnt(unsigned int code) { return (int)((code >> 8) & 7u); }

// One Gauss-Seidel update of a cell of level l: x_c = b_c / (s_l n_c) + (sum of
// fluid neighbours' x) / n_c, with n_c the count of neighbours inside the grid.
__device__ __forceinline__ float gs_first(int l, int cnt, float bc) {
  return __fmul_rn(bc, s_inv_scnt[l][cnt]);
}

__device__ __forceinline__ float gs_sum(int l, int cnt, unsigned int code, float bc,
                                        const float (&xv)[6]) {
  const float base = __fmul_rn(bc, s_inv_scnt[l][cnt]);
  float sum = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) sum += ((code >> q) & 1u) ? xv[q] : 0.0f;
  return __fmaf_rn(sum, s_inv_cnt[cnt], base);
}

// Residual b - A x of a fluid cell, A x in difference form
// s (sum_fluid (x_c - x_n) + n_air x_c).
__device__ __forceinline__ float resid(float s, int cnt, unsigned int code, float bc, float xc,
                                       const float (&xv)[6]) {
  float d = 0.0f;
  int nfl = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const bool f = (code >> q) & 1u;
    d += f ? __fsub_rn(xc, xv[q]) : 0.0f;
    nfl += f;
  }
  return __fsub_rn(bc, __fmul_rn(s, __fmaf_rn((float)(cnt - nfl), xc, d)));
}

// resid for a cell whose six neighbours are all fluid (code CODE_FULL): the same
// operations without the masks (cnt - nfl = 0).
__device__ __forceinline__ float resid_full(float s, float bc, float xc, const float (&xv)[6]) {
  float d = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) d = __fadd_rn(d, __fsub_rn(xc, xv[q]));
  return __fsub_rn(bc, __fmul_rn(s, __fmaf_rn(0.0f, xc, d)));
}

// ---------------------------------------------------------------- sweeps

struct GsIn {
  int i, j, k, idx;
  bool ok;
  unsigned int code;
  float b;
  float xv[6];
  float pv[6];  // CORRECT: the neighbours' parents on the next coarser level
};

// Parents on level C of the six neighbours of cell (i, j, k) of a level with
// extents (nx, ny, nz); a neighbour off the grid is replaced by the cell itself
// (its value is unused).
__device__ __forceinline__ void parent_values(const PV& C, int nx, int ny, int nz, int i, int j,
                                              int k, float (&pv)[6]) {
  const int pi[6] = {max(i - 1, 0), min(i + 1, nx - 1), i, i, i, i};
  const int pj[6] = {j, j, max(j - 1, 0), min(j + 1, ny - 1), j, j};
  const int pk[6] = {k, k, k, k, max(k - 1, 0), min(k + 1, nz - 1)};
#pragma unroll
  for (int q = 0; q < 6; ++q) pv[q] = C.x[level_index(C, pi[q] >> 1, pj[q] >> 1, pk[q] >> 1)];
}

// The coarse values that the corrections of a slot pair's two cells (A at x = iA,
// B at iA + 2) read.  The twelve neighbours' parents are seven coarse cells: three
// in the pair's coarse row (x = s - 1 + par .. s + 1 + par, which hold A's and B's
// own parents, s and s + 1), and for A and B the parent in the other y row and in
// the other z plane (a neighbour's parent is the cell's own but for one neighbour
// per axis).  pr = {row x3, y-row A, y-row B, z-plane A, z-plane B}; coordinates of
// off-grid neighbours (never read unmasked) are clamped into the level.
template <class E>
__device__ __forceinline__ void pair_parents(const PV& C, const E& e, float (&pr)[7]) {
  const int J = e.j >> 1, K = e.k >> 1;
  const int Jy = min(max((e.j & 1) ? J + 1 : J - 1, 0), C.ny - 1);
  const int Kz = min(max((e.k & 1) ? K + 1 : K - 1, 0), C.nz - 1);
  const int a = min(e.s, C.nx - 1), b = min(e.s + 1, C.nx - 1);
#pragma unroll
  for (int q = 0; q < 3; ++q)
    pr[q] = C.x[level_index(C, min(max(e.s - 1 + e.par + q, 0), C.nx - 1), J, K)];
  pr[3] = C.x[level_index(C, a, Jy, K)];
  pr[4] = C.x[level_index(C, b, Jy, K)];
  pr[5] = C.x[level_index(C, a, J, Kz)];
  pr[6] = C.x[level_index(C, b, J, Kz)];
}

// The six neighbour parents (parent_values' order) of cell h (0: A, 1: B) of the
// pair, from pair_parents' seven values.
__device__ __forceinline__ void pair_parents_of(const float (&pr)[7], int par, int j, int k,
                                                int h, float (&pv)[6]) {
  const float own = (h == 0) ? (par ? pr[0] : pr[1]) : (par ? pr[1] : pr[2]);
  const float oy = (h == 0) ? pr[3] : pr[4], oz = (h == 0) ? pr[5] : pr[6];
  pv[0] = (h == 0) ? pr[0] : pr[1];
  pv[1] = (h == 0) ? pr[1] : pr[2];
  pv[2] = (j & 1) ? own : oy;
  pv[3] = (j & 1) ? oy : own;
  pv[4] = (k & 1) ? own : oz;
  pv[5] = (k & 1) ? oz : own;
}

template <int MODE>
__device__ __forceinline__ bool gs_apply(float* x, int l, float omega, GsIn& s, float& v) {
  if (!s.ok || !(s.code & CODE_SELF)) return false;
  if constexpr (MODE == CORRECT) {
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if ((s.code >> q) & 1u) s.xv[q] = __fmaf_rn(omega, s.pv[q], s.xv[q]);
  }
  v = gs_sum(l, code_cnt(s.code), s.code, s.b, s.xv);
  x[s.idx] = v;
  return true;
}

// Half-sweep of one colour over colour-split level l (description L; C is level
// l+1, read in CORRECT mode).  With rz, also accumulates b x over the updated
// cells.  Paired form: slots that are not fluid cells of the grid get 0.  (A
// grid-wide level never sweeps from zero here: its first red half-sweep is made
// by the pass that produces its right-hand side.)
template <int MODE, bool RZ>
__device__ __noinline__ void sweep_split_v(const MgArgs& M, const MgLevel& L, const MgLevel& C,
                                         int l, int colour, FF* rz) {
  static_assert(MODE != FIRST, "grid-wide levels start from the fused first half-sweep");
  constexpr int U = (MODE == CORRECT) ? 1 : 2;
  const int lane = threadIdx.x & 31;
  const SV v = sview(L);
  const PV cv = pview(C);
  const float omega = M.omega;
  const float inv6 = s_inv_cnt[6], invs6 = s_inv_scnt[l][6];
  const int2 q = seg_slice(L);
  const Items it = pair_items(q, 1);
  struct S {
    PCell e;
    unsigned int code2;
    float2 b;
    Nbr2 n;
    float pr[MODE == CORRECT ? 7 : 1];
  };
  FF acc;
  run_batched<U>(
      it.first, it.end, PCG_WARPS,
      [&](unsigned int t, bool ok) {
        S st;
        st.e = pcell(v, q, t, colour, lane);
        st.e.okA &= ok;
        st.e.okB &= ok;
        st.code2 = *reinterpret_cast<const unsigned int*>(v.code + st.e.idx);
        st.b = *reinterpret_cast<const float2*>(v.b + st.e.idx);
        st.n = load_nbr2(v, v.x, st.e);
        if constexpr (MODE == CORRECT) pair_parents(cv, st.e, st.pr);
        return st;
      },
      [&](S&) {},
      [&](S& st) {
        float out[2];
        {
          // a warp whose cells are all fluid with six fluid neighbours (the bulk of
          // the liquid): gs_sum's operations in its order, without masks or tables
          // (and the correction of every neighbour in CORRECT mode)
          const bool full = pair_full(st.code2) && st.e.okA && st.e.okB;
          if (__all_sync(0xffffffffu, full)) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float xv[6];
              nbr_of(st.n, h, xv);
              if constexpr (MODE == CORRECT) {
                float pv[6];
                pair_parents_of(st.pr, st.e.par, st.e.j, st.e.k, h, pv);
#pragma unroll
                for (int u = 0; u < 6; ++u) xv[u] = __fmaf_rn(omega, pv[u], xv[u]);
              }
              float sum = 0.0f;
#pragma unroll
              for (int u = 0; u < 6; ++u) sum = __fadd_rn(sum, xv[u]);
              const float bc = h == 0 ? st.b.x : st.b.y;
              out[h] = __fmaf_rn(sum, inv6, __fmul_rn(bc, invs6));
              if (RZ) acc.add_prod(bc, out[h]);
            }
            *reinterpret_cast<float2*>(v.x + st.e.idx) = make_float2(out[0], out[1]);
            return;
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned int code = h == 0 ? (st.code2 & 0xffffu) : (st.code2 >> 16);
          const bool ok = (h == 0 ? st.e.okA : st.e.okB) && (code & CODE_SELF);
          const float bc = h == 0 ? st.b.x : st.b.y;
          float xv[6];
          nbr_of(st.n, h, xv);
          if constexpr (MODE == CORRECT) {
            float pv[6];
            pair_parents_of(st.pr, st.e.par, st.e.j, st.e.k, h, pv);
#pragma unroll
            for (int u = 0; u < 6; ++u)
              if ((code >> u) & 1u) xv[u] = __fmaf_rn(omega, pv[u], xv[u]);
          }
          const float val = gs_sum(l, code_cnt(code), code, bc, xv);
          out[h] = ok ? val : 0.0f;
          if (RZ && ok) acc.add_prod(bc, val);
        }
        if (st.e.okA || st.e.okB)
          *reinterpret_cast<float2*>(v.x + st.e.idx) = make_float2(out[0], out[1]);
      });
  if constexpr (RZ) {
    rz->add_prod(acc.hi, 1.0f);
    rz->add_prod(acc.lo, 1.0f);
  }
}

// Scalar form: a lane takes one slot (levels with few segments per CTA, where
// more items in flight matter more than wider loads).
template <int MODE>
__device__ __noinline__ void sweep_split_s(const MgArgs& M, const MgLevel& L, const MgLevel& C,
                                         int l, int colour, FF* rz) {
  static_assert(MODE != FIRST, "grid-wide levels start from the fused first half-sweep");
  constexpr int U = (MODE == CORRECT) ? 1 : 2;
  const int lane = threadIdx.x & 31;
  const SV v = sview(L);
  const PV cv = pview(C);
  const int nz = L.nz;
  const float omega = M.omega;
  const Items it = seg_items(L, 1);
  const float inv6 = s_inv_cnt[6], invs6 = s_inv_scnt[l][6];
  FF acc;
  run_batched<U>(
      it.first, it.end, PCG_WARPS,
      [&](unsigned int t, bool ok) {
        const SCell e = scell(v, v.seg[t - v.seg_base], colour, lane);
        GsIn s;
        s.i = e.i;
        s.j = e.j;
        s.k = e.k;
        s.idx = e.idx;
        s.ok = e.ok && ok;
        s.code = v.code[e.idx];
        s.b = v.b[e.idx];
        int nb[6];
        snbr(v, e, nb);
#pragma unroll
        for (int q = 0; q < 6; ++q) s.xv[q] = v.x[nb[q]];
        if constexpr (MODE == CORRECT)
          parent_values(cv, v.nx, v.ny, nz, min(e.i, v.nx - 1), e.j, e.k, s.pv);
        return s;
      },
      [&](GsIn&) {},
      [&](GsIn& s) {
        // a warp whose cells are all fluid with six fluid neighbours: gs_apply's
        // operations in its order, without the masks
        if (__all_sync(0xffffffffu, s.ok && s.code == CODE_FULL)) {
          if constexpr (MODE == CORRECT) {
#pragma unroll
            for (int q = 0; q < 6; ++q) s.xv[q] = __fmaf_rn(omega, s.pv[q], s.xv[q]);
          }
          float sum = 0.0f;
#pragma unroll
          for (int q = 0; q < 6; ++q) sum = __fadd_rn(sum, s.xv[q]);
          const float xv = __fmaf_rn(sum, inv6, __fmul_rn(s.b, invs6));
          v.x[s.idx] = xv;
          if (rz) acc.add_prod(s.b, xv);
          return;
        }
        float xv;
        if (gs_apply<MODE>(v.x, l, omega, s, xv) && rz) acc.add_prod(s.b, xv);
      });
  if (rz) {
    rz->add_prod(acc.hi, 1.0f);
    rz->add_prod(acc.lo, 1.0f);
  }
}

// Levels with many segments per CTA take the paired form (8-byte accesses, half
// the load instructions); the others the scalar form.
constexpr int VEC_SEGS_PER_CTA = 256;

__device__ __forceinline__ bool use_pairs(const MgLevel& L) {
  return *L.nseg >= (unsigned)VEC_SEGS_PER_CTA * team_size();
}

template <int MODE>
__device__ __forceinline__ void sweep_split(const MgArgs& M, const MgLevel& L, const MgLevel& C,
                                            int l, int colour, FF* rz) {
  if (use_pairs(L)) {
    // the r.z accumulation only where asked (its registers would make the other
    // half-sweeps spill)
    if (rz) sweep_split_v<MODE, true>(M, L, C, l, colour, rz);
    else sweep_split_v<MODE, false>(M, L, C, l, colour, nullptr);
  }
  else sweep_split_s<MODE>(M, L, C, l, colour, rz);
}

// ---------------------------------------------------------------- restriction

// Residual of the red child (dy, dz) of coarse cell (I, J, K) on the
// colour-split fine level F.  The child's x offset dx makes its colour red:
// 2I+dx + 2J+dy + 2K+dz even, so its red slot is I.
struct ChildIn {
  bool ok;
  unsigned int code;
  float b, xc;
  float xv[6];
};

__device__ __forceinline__ void child_load(const SV& F, int fnz, int I, int J, int K, int dy,
                                           int dz, ChildIn& s) {
  const int dx = (dy + dz) & 1;
  const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
  s.ok = i < F.nx && j < F.ny && k < fnz;
  const int jj = min(j, F.ny - 1), kk = min(k, fnz - 1);
  const int idx = F.margin + F.hx * (jj + F.ny * kk) + min(I, F.hx - 1);
  const int ob = idx + F.half;
  s.code = F.code[idx];
  s.b = F.b[idx];
  s.xc = F.x[idx];
  const int nb[6] = {ob - 1 + dx, ob + dx, ob - F.hx, ob + F.hx, ob - F.pl, ob + F.pl};
#pragma unroll
  for (int q = 0; q < 6; ++q) s.xv[q] = F.x[nb[q]];
}

// b_C(I,J,K) = (1/16) sum over fluid children of the fine residual.  The
// restriction follows the pre-smoothing, whose last half-sweep is black: a black
// cell's update solves its own equation against the red neighbours it read, so
// its residual is exactly zero and only the red children contribute.  The four
// red children are loaded two at a time and summed in the order (dy, dz) =
// (0,0), (1,0), (0,1), (1,1).
__device__ __forceinline__ float restrict_sum(const SV& F, int fnz, int I, int J, int K) {
  float sum = 0.0f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    ChildIn ch[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) child_load(F, fnz, I, J, K, q, h, ch[q]);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const ChildIn& c = ch[q];
      if (!c.ok || !(c.code & CODE_SELF)) continue;
      sum = __fadd_rn(sum, resid(F.s, code_cnt(c.code), c.code, c.b, c.xc, c.xv));
    }
  }
  return __fmul_rn(sum, 0.0625f);
}

// Colour-split F -> colour-split C, over C's active segments; lanes take the
// segment's 64 cells in x order (so the fine red slots they read are contiguous).
// The pass also makes C's first red half-sweep from zero, x = b / (s_C n) on C's
// red fluid cells, which needs only the b it has just computed: C's
// pre-smoothing then starts with the black half-sweep, and the cycle meets one
// grid barrier fewer per level (the values are those the separate half-sweep
// computes; the slots of C's non-fluid cells, never read unmasked, are left).
__device__ __noinline__ void restrict_split(const MgLevel& Fl, const MgLevel& Cl) {
  const int lane = threadIdx.x & 31;
  const SV F = sview(Fl), C = sview(Cl);
  const int fnz = Fl.nz;
  const int lc = Cl.lvl;
  const Items it = seg_items(Cl, 1);
  for (unsigned int t = it.first; t < it.end; t += PCG_WARPS) {
    const int4 sg = C.seg[t - C.seg_base];
    const int J = sg.z, K = sg.w;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // every lane takes part (a lane past the row's end on its last cell, whose
      // result it drops), so that a warp can vote
      const int I = sg.y * (2 * SEG_SLOTS) + h * 32 + lane;
      const bool in = I < C.nx;
      const int Ic = in ? I : C.nx - 1;
      const int red = ((Ic + J + K) & 1) == 0;
      const int ci = (1 - red) * C.half + C.margin + C.hx * sg.x + (Ic >> 1);
      const unsigned int code = C.code[ci];
      // restrict_sum's sum over the red children; a pair of children that is all
      // interior fluid cells in every lane is added without the masks
      float sum = 0.0f;
#pragma unroll
      for (int hz = 0; hz < 2; ++hz) {
        ChildIn ch[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) child_load(F, fnz, Ic, J, K, q, hz, ch[q]);
        const bool full = ch[0].ok && ch[1].ok && ch[0].code == CODE_FULL && ch[1].code == CODE_FULL;
        if (__all_sync(0xffffffffu, full)) {
#pragma unroll
          for (int q = 0; q < 2; ++q)
            sum = __fadd_rn(sum, resid_full(F.s, ch[q].b, ch[q].xc, ch[q].xv));
        } else {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const ChildIn& c = ch[q];
            if (!c.ok || !(c.code & CODE_SELF)) continue;
            sum = __fadd_rn(sum, resid(F.s, code_cnt(c.code), c.code, c.b, c.xc, c.xv));
          }
        }
      }
      if (!in || !(code & CODE_SELF)) continue;
      const float bc = __fmul_rn(sum, 0.0625f);
      C.b[ci] = bc;
      if (red) C.x[ci] = gs_first(lc, code_cnt(code), bc);
    }
  }
}

// Colour-split F -> natural-layout C (the first CTA-local level, in global
// memory), over all of C's cells.
__device__ __noinline__ void restrict_split_nat(const MgLevel& Fl, const MgLevel& Cl) {
  const SV F = sview(Fl);
  const int fnz = Fl.nz;
  const int nx = Cl.nx, ny = Cl.ny;
  float* cb = Cl.b;
  const uint8_t* code = Cl.code;
  const Part p = level_part(Cl.ncells, false);
  for (int c = p.begin; c < p.end; c += p.stride) {
    if (!(code[c] & CODE_SELF)) continue;
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    cb[c] = restrict_sum(F, fnz, i, j, k);
  }
}

// ---------------------------------------------------------------- cycle pieces

__device__ __forceinline__ bool gsync(const PcgArgs& A) {
  return grid_barrier(A.bar, A.status, team_size(), A.timeout_ns);
}

// Pre-smoothing from zero and restriction, colour-split level l -> l+1.  The
// first red half-sweep from zero was made by the restriction into level l
// (restrict_split), behind the barrier that followed it.
__device__ __forceinline__ bool down_split(const PcgArgs& A, int l) {
  const MgArgs& M = A.mg;
  const MgLevel& L = M.lv[l];
  const MgLevel& C = M.lv[l + 1];
  sweep_split<NORMAL>(M, L, C, l, 1, nullptr);
  if (!gsync(A)) return false;
  for (int s = 1; s < M.nu; ++s) {
    sweep_split<NORMAL>(M, L, C, l, 0, nullptr);
    if (!gsync(A)) return false;
    sweep_split<NORMAL>(M, L, C, l, 1, nullptr);
    if (!gsync(A)) return false;
  }
  if (C.split) restrict_split(L, C);
  else restrict_split_nat(L, C);
  return gsync(A);
}

// Coarse correction from level l+1 and post-smoothing, colour-split level l.
__device__ __forceinline__ bool up_split(const PcgArgs& A, int l) {
  const MgArgs& M = A.mg;
  const MgLevel& L = M.lv[l];
  const MgLevel& C = M.lv[l + 1];
  sweep_split<CORRECT>(M, L, C, l, 1, nullptr);
  if (!gsync(A)) return false;
  sweep_split<NORMAL>(M, L, C, l, 0, nullptr);
  if (!gsync(A)) return false;
  for (int s = 1; s < M.nu; ++s) {
    sweep_split<NORMAL>(M, L, C, l, 1, nullptr);
    if (!gsync(A)) return false;
    sweep_split<NORMAL>(M, L, C, l, 0, nullptr);
    if (!gsync(A)) return false;
  }
  return true;
}

// ---------------------------------------------------------------- CTA-local levels

// The CTA-local levels [lgrid, nlev) live in CTA 0's (dynamic) shared memory:
// x, b and the neighbour codes of every such level (MG_CTA_CELLS cells in all),
// and per level and colour the list of its fluid cells, each as the packed
// coordinates i | j << bx | k << (bx + by) with bx, by the bits of nx - 1 and
// ny - 1 (at most 16 bits, since a CTA-local level has fewer than 2^13 cells).
// A half-sweep then visits exactly the fluid cells of its colour, with no
// divisions and no idle slots.
struct CtaMg {
  float x[MG_CTA_CELLS];
  float b[MG_CTA_CELLS];
  uint8_t code[MG_CTA_CELLS];
  uint16_t list[MG_CTA_CELLS];
  int off[MG_MAX_LEVELS][3];   // list of level l: colour 0 [off0, off1), colour 1 [off1, off2)
  int base[MG_MAX_LEVELS];     // first cell of level l in x, b, code
  int nx[MG_MAX_LEVELS], ny[MG_MAX_LEVELS], nz[MG_MAX_LEVELS];
  int bx[MG_MAX_LEVELS], by[MG_MAX_LEVELS];
  float s[MG_MAX_LEVELS];
};

// CTA 0's CTA-local levels sit at the start of the kernel's dynamic shared memory;
// reached through this (not a pointer argument) the compiler addresses them as
// shared memory.
__device__ __forceinline__ CtaMg& cta_mg() {
  extern __shared__ __align__(16) unsigned char mg_dyn[];
  return *reinterpret_cast<CtaMg*>(mg_dyn);
}

__device__ __forceinline__ int bits_for(int n) {  // bits of n - 1 (0 for n = 1)
  return n > 1 ? 32 - __clz(n - 1) : 0;
}

struct CtaCell {
  int i, j, k, c;
};

__device__ __forceinline__ CtaCell cta_cell(const CtaMg& sm, int l, unsigned int e) {
  const int bx = sm.bx[l], by = sm.by[l];
  CtaCell r;
  r.i = (int)(e & ((1u << bx) - 1u));
  r.j = (int)((e >> bx) & ((1u << by) - 1u));
  r.k = (int)(e >> (bx + by));
  r.c = r.i + sm.nx[l] * (r.j + sm.ny[l] * r.k);
  return r;
}

// Half-sweep of one colour over CTA-local level l (parents on level l + 1).
template <int MODE>
__device__ __noinline__ void sweep_cta(float omega, int l, int colour) {
  static_assert(MODE != FIRST, "the first half-sweep of a CTA-local level comes with its b");
  CtaMg& sm = cta_mg();
  const int nx = sm.nx[l], ny = sm.ny[l], nz = sm.nz[l], sy = nx, sz = nx * ny;
  float* x = sm.x + sm.base[l];
  const float* b = sm.b + sm.base[l];
  const uint8_t* code = sm.code + sm.base[l];
  const int e1 = sm.off[l][colour + 1];
  for (int e = sm.off[l][colour] + (int)threadIdx.x; e < e1; e += PCG_THREADS) {
    const CtaCell p = cta_cell(sm, l, sm.list[e]);
    const int cnt = (p.i > 0) + (p.i < nx - 1) + (p.j > 0) + (p.j < ny - 1) + (p.k > 0) +
                    (p.k < nz - 1);
    const unsigned int cd = code[p.c];
    const int off[6] = {-1, 1, -sy, sy, -sz, sz};
    float xv[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) xv[q] = ((cd >> q) & 1u) ? x[p.c + off[q]] : 0.0f;
    if constexpr (MODE == CORRECT) {
      const float* px = sm.x + sm.base[l + 1];
      const int pnx = sm.nx[l + 1], pny = sm.ny[l + 1];
      const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if ((cd >> q) & 1u) {
          const int pi = (p.i + di[q]) >> 1, pj = (p.j + dj[q]) >> 1, pk = (p.k + dk[q]) >> 1;
          xv[q] = __fmaf_rn(omega, px[pi + pnx * (pj + pny * pk)], xv[q]);
        }
    }
    x[p.c] = gs_sum(l, cnt, cd, b[p.c], xv);
  }
}

// b_{l+1} = (1/16) sum of the red fluid children's residuals, over level l+1's
// fluid cells (both colours), and the first red half-sweep of level l+1 from
// zero: x = gs_first(b) on its red cells.  Four consecutive lanes take the four
// red children of one coarse cell, and the group's first lane adds their
// residuals in child order.
__device__ __noinline__ void restrict_cta(int l) {
  CtaMg& sm = cta_mg();
  const int nx = sm.nx[l], ny = sm.ny[l], nz = sm.nz[l], sy = nx, sz = nx * ny;
  const int cnx = sm.nx[l + 1], cny = sm.ny[l + 1], cnz = sm.nz[l + 1];
  const float* x = sm.x + sm.base[l];
  const float* b = sm.b + sm.base[l];
  const uint8_t* code = sm.code + sm.base[l];
  float* cb = sm.b + sm.base[l + 1];
  float* cx = sm.x + sm.base[l + 1];
  const float sl = sm.s[l];
  const int e0 = sm.off[l + 1][0], ered = sm.off[l + 1][1];
  const int n4 = 4 * (sm.off[l + 1][2] - e0);
  const int lane = threadIdx.x & 31;
  for (int e4 = (int)threadIdx.x; e4 - lane < n4; e4 += PCG_THREADS) {  // warp-uniform bound
    const bool live = e4 < n4;
    float r = 0.0f;
    bool has = false;
    CtaCell P = {0, 0, 0, 0};
    if (live) {
      P = cta_cell(sm, l + 1, sm.list[e0 + (e4 >> 2)]);
      const int q = e4 & 3, dy = q & 1, dz = q >> 1, dx = (dy + dz) & 1;
      const int i = 2 * P.i + dx, j = 2 * P.j + dy, k = 2 * P.k + dz;
      if (i < nx && j < ny && k < nz) {
        const int fc = i + nx * (j + ny * k);
        const unsigned int cd = code[fc];
        if (cd & CODE_SELF) {
          const int off[6] = {-1, 1, -sy, sy, -sz, sz};
          float xv[6];
#pragma unroll
          for (int u = 0; u < 6; ++u) xv[u] = ((cd >> u) & 1u) ? x[fc + off[u]] : 0.0f;
          const int cnt = (i > 0) + (i < nx - 1) + (j > 0) + (j < ny - 1) + (k > 0) + (k < nz - 1);
          r = resid(sl, cnt, cd, b[fc], x[fc], xv);
          has = true;
        }
      }
    }
    const unsigned int hm = __ballot_sync(0xffffffffu, has) >> (lane & ~3);
    const float r1 = __shfl_down_sync(0xffffffffu, r, 1);
    const float r2 = __shfl_down_sync(0xffffffffu, r, 2);
    const float r3 = __shfl_down_sync(0xffffffffu, r, 3);
    if (live && (e4 & 3) == 0) {
      float sum = 0.0f;
      if (hm & 1u) sum = __fadd_rn(sum, r);
      if (hm & 2u) sum = __fadd_rn(sum, r1);
      if (hm & 4u) sum = __fadd_rn(sum, r2);
      if (hm & 8u) sum = __fadd_rn(sum, r3);
      const float bc = __fmul_rn(sum, 0.0625f);
      cb[P.c] = bc;
      if (e0 + (e4 >> 2) < ered) {
        const int cnt = (P.i > 0) + (P.i < cnx - 1) + (P.j > 0) + (P.j < cny - 1) + (P.k > 0) +
                        (P.k < cnz - 1);
        cx[P.c] = gs_first(l + 1, cnt, bc);
      }
    }
  }
}

// Points the shared level descriptions at the shared arrays, loads the codes and
// builds the fluid-cell lists (once per solve, after build_levels).  CTA 0 only.
__device__ __noinline__ void cta_levels_init(const MgArgs& M) {
  CtaMg& sm = cta_mg();
  __shared__ unsigned int s_wc[PCG_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    int off = 0;
    for (int l = M.lgrid; l < M.nlev; ++l) {
      sm.base[l] = off;
      sm.nx[l] = M.lv[l].nx;
      sm.ny[l] = M.lv[l].ny;
      sm.nz[l] = M.lv[l].nz;
      sm.bx[l] = bits_for(M.lv[l].nx);
      sm.by[l] = bits_for(M.lv[l].ny);
      sm.s[l] = M.lv[l].s;
      off += M.lv[l].ncells;
    }
  }
  __syncthreads();
  // Per level: each thread takes a contiguous run of cells, counts its fluid cells
  // of each colour (the two counts packed in one word: a level has fewer than 2^16
  // cells), a block-wide exclusive scan gives each run its place, and the runs
  // write their entries: colour 0's list then colour 1's, each in cell order.
  __shared__ unsigned int s_scan[PCG_WARPS];
  int pos = 0;  // next free list entry (same value in every thread)
  for (int l = M.lgrid; l < M.nlev; ++l) {
    const int n = M.lv[l].ncells, nx = sm.nx[l], ny = sm.ny[l], bl = sm.base[l];
    for (int c = threadIdx.x; c < n; c += PCG_THREADS) sm.code[bl + c] = M.lv[l].code[c];
    __syncthreads();
    const int per = (n + PCG_THREADS - 1) / PCG_THREADS;
    const int c0 = min(n, (int)threadIdx.x * per), c1 = min(n, c0 + per);
    unsigned int mine = 0;  // colour 0 in the low half, colour 1 in the high half
    for (int c = c0; c < c1; ++c) {
      const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
      if (sm.code[bl + c] & CODE_SELF) mine += ((i + j + k) & 1) ? 0x10000u : 1u;
    }
    unsigned int inc = mine;  // inclusive scan over the warp, then over the warps
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned int v = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += v;
    }
    if (lane == 31) s_scan[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const unsigned int t = lane < PCG_WARPS ? s_scan[lane] : 0u;
      unsigned int w = t;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += v;
      }
      if (lane < PCG_WARPS) s_scan[lane] = w - t;  // exclusive, per warp
      const unsigned int tot = __shfl_sync(0xffffffffu, w, 31);
      if (lane == 0) s_wc[0] = tot;
    }
    __syncthreads();
    const unsigned int before = s_scan[warp] + inc - mine, tot = s_wc[0];
    const int n0 = (int)(tot & 0xffffu), n1 = (int)(tot >> 16);
    int p0 = pos + (int)(before & 0xffffu), p1 = pos + n0 + (int)(before >> 16);
    for (int c = c0; c < c1; ++c) {
      if (!(sm.code[bl + c] & CODE_SELF)) continue;
      const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
      const uint16_t e = (uint16_t)(i | (j << sm.bx[l]) | (k << (sm.bx[l] + sm.by[l])));
      if ((i + j + k) & 1) sm.list[p1++] = e;
      else sm.list[p0++] = e;
    }
    if (threadIdx.x == 0) {
      sm.off[l][0] = pos;
      sm.off[l][1] = pos + n0;
      sm.off[l][2] = pos + n0 + n1;
    }
    pos += n0 + n1;
    __syncthreads();
  }
}

// The same cycle pieces as for the grid-wide levels, inside CTA 0.  The first
// red half-sweep of a level (from zero) is done where its b is made: in the
// copy-in for level lgrid, in the restriction for the levels below.
__device__ __forceinline__ void down_cta(const MgArgs& M, int l) {
  sweep_cta<NORMAL>(M.omega, l, 1);
  __syncthreads();
  for (int s = 1; s < M.nu; ++s) {
    sweep_cta<NORMAL>(M.omega, l, 0);
    __syncthreads();
    sweep_cta<NORMAL>(M.omega, l, 1);
    __syncthreads();
  }
  restrict_cta(l);
  __syncthreads();
}

__device__ __forceinline__ void up_cta(const MgArgs& M, int l) {
  sweep_cta<CORRECT>(M.omega, l, 1);
  __syncthreads();
  sweep_cta<NORMAL>(M.omega, l, 0);
  __syncthreads();
  for (int s = 1; s < M.nu; ++s) {
    sweep_cta<NORMAL>(M.omega, l, 1);
    __syncthreads();
    sweep_cta<NORMAL>(M.omega, l, 0);
    __syncthreads();
  }
}

// The coarsest level: MG_COARSE_SWEEPS (red, black) pairs from zero, then as many
// (black, red) pairs, run as one alternating sequence: the second of the two black
// half-sweeps in the middle would repeat the first on the same red values.
__device__ __forceinline__ void coarsest_cta(const MgArgs& M, int l) {
  for (int h = 1; h < 4 * MG_COARSE_SWEEPS - 1; ++h) {  // black, red, ..., red
    sweep_cta<NORMAL>(M.omega, l, h & 1);
    __syncthreads();
  }
}

// Levels [lgrid, nlev) inside CTA 0, from the right-hand side that the grid-wide
// restriction left in level lgrid's global b; leaves level lgrid's x in global
// memory for the correction of level lgrid - 1.
__device__ __noinline__ void cta_cycle(const PcgArgs& A) {
  const MgArgs& M = A.mg;
  CtaMg& sm = cta_mg();
  const int lg = M.lgrid;
  const int n = M.lv[lg].ncells;
  const float* gb = M.lv[lg].b;
  float* gx = M.lv[lg].x;
  // b of level lgrid (all loads of a thread before its stores), and the first red
  // half-sweep of level lgrid from zero on the same values
  constexpr int U = 4;
  float* sb = sm.b + sm.base[lg];
  for (int c0 = threadIdx.x; c0 < n; c0 += U * PCG_THREADS) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = c0 + u * PCG_THREADS;
      v[u] = c < n ? gb[c] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = c0 + u * PCG_THREADS;
      if (c < n) sb[c] = v[u];
    }
  }
  {
    const int nx = sm.nx[lg], ny = sm.ny[lg], nz = sm.nz[lg];
    float* sx = sm.x + sm.base[lg];
    const int e1 = sm.off[lg][1];
    for (int e = sm.off[lg][0] + (int)threadIdx.x; e < e1; e += PCG_THREADS) {
      const CtaCell p = cta_cell(sm, lg, sm.list[e]);
      const int cnt = (p.i > 0) + (p.i < nx - 1) + (p.j > 0) + (p.j < ny - 1) + (p.k > 0) +
                      (p.k < nz - 1);
      sx[p.c] = gs_first(lg, cnt, gb[p.c]);
    }
  }
  __syncthreads();
  for (int l = lg; l < M.nlev - 1; ++l) down_cta(M, l);
  coarsest_cta(M, M.nlev - 1);
  for (int l = M.nlev - 2; l >= lg; --l) up_cta(M, l);
  for (int c = threadIdx.x; c < n; c += PCG_THREADS) gx[c] = sm.x[sm.base[lg] + c];
}

// z = V(r), given that the first red half-sweep of level 0 (from zero) has been
// done in the phase that produced r, and that a grid barrier has passed since.
// The last black and the last red half-sweeps of level 0 accumulate r.z over
// their cells into rz.  The caller publishes rz and meets the next barrier.
// Returns false if a barrier failed.
__device__ bool vcycle_rest(const PcgArgs& A, FF& rz) {
  const MgArgs& M = A.mg;
  const MgLevel& L0 = M.lv[0];
  if (M.nlev == 1) {  // level 0 is the coarsest level
    // rest of the pre pairs (red, black) after the fused first red half-sweep
    for (int s = 0; s < MG_COARSE_SWEEPS; ++s) {
      sweep_split<NORMAL>(M, L0, L0, 0, 1, nullptr);
      if (!gsync(A)) return false;
      if (s + 1 < MG_COARSE_SWEEPS) {
        sweep_split<NORMAL>(M, L0, L0, 0, 0, nullptr);
        if (!gsync(A)) return false;
      }
    }
    // post pairs (black, red); the last black and the last red give r.z
    for (int s = 0; s < MG_COARSE_SWEEPS; ++s) {
      sweep_split<NORMAL>(M, L0, L0, 0, 1, s + 1 == MG_COARSE_SWEEPS ? &rz : nullptr);
      if (!gsync(A)) return false;
      if (s + 1 < MG_COARSE_SWEEPS) {
        sweep_split<NORMAL>(M, L0, L0, 0, 0, nullptr);
        if (!gsync(A)) return false;
      }
    }
    sweep_split<NORMAL>(M, L0, L0, 0, 0, &rz);
    return true;
  }
  const MgLevel& L1 = M.lv[1];
  sweep_split<NORMAL>(M, L0, L1, 0, 1, nullptr);
  if (!gsync(A)) return false;
  SOLVE_TRACE(TR_V_PRE1);
  for (int s = 1; s < M.nu; ++s) {
    sweep_split<NORMAL>(M, L0, L1, 0, 0, nullptr);
    if (!gsync(A)) return false;
    sweep_split<NORMAL>(M, L0, L1, 0, 1, nullptr);
    if (!gsync(A)) return false;
  }
  SOLVE_TRACE(TR_V_PRE);
  if (L1.split) restrict_split(L0, L1);
  else restrict_split_nat(L0, L1);
  if (!gsync(A)) return false;
  SOLVE_TRACE(TR_V_RESTRICT);
  for (int l = 1; l < M.lgrid; ++l) {
    if (!down_split(A, l)) return false;
    SOLVE_TRACE(TR_V_DOWN + min(l, 11));
  }
  if (team_rank() == 0) cta_cycle(A);
  if (!gsync(A)) return false;
  SOLVE_TRACE(TR_V_CTA);
  for (int l = M.lgrid - 1; l >= 1; --l) {
    if (!up_split(A, l)) return false;
    SOLVE_TRACE(TR_V_UP + min(l, 11));
  }
  sweep_split<CORRECT>(M, L0, L1, 0, 1, M.nu == 1 ? &rz : nullptr);
  if (!gsync(A)) return false;
  SOLVE_TRACE(TR_V_CORRECT);
  for (int s = 1; s < M.nu; ++s) {
    sweep_split<NORMAL>(M, L0, L1, 0, 0, nullptr);
    if (!gsync(A)) return false;
    sweep_split<NORMAL>(M, L0, L1, 0, 1, s + 1 == M.nu ? &rz : nullptr);
    if (!gsync(A)) return false;
  }
  SOLVE_TRACE(TR_V_POST);
  sweep_split<NORMAL>(M, L0, L1, 0, 0, &rz);  // the last red half-sweep
  return true;
}

// ---------------------------------------------------------------- level-0 passes

// Phase A with z from the V-cycle: p_new = z + beta p_old (recomputed for the
// neighbours), q = A p_new in difference form, partial p.q.  Both colours; paired
// form.
__device__ __noinline__ void phase_a_v(const PcgArgs& A, const float* pold, float* pnew, float beta,
                                     FF& pq) {
  const MgArgs& M = A.mg;
  const SV v = sview(M.lv[0]);
  const float* z = v.x;
  float* q0 = M.q0;
  const float s_a = A.s;
  const int lane = threadIdx.x & 31;
  const int2 q = seg_slice(M.lv[0]);
  const Items it = pair_items(q, 2);
  FF acc;
  for (unsigned int t = it.first; t < it.end; t += PCG_WARPS) {
    const PCell e = pcell(v, q, t >> 1, (int)(t & 1u), lane);
    const unsigned int code2 = *reinterpret_cast<const unsigned int*>(v.code + e.idx);
    const float2 zc = *reinterpret_cast<const float2*>(z + e.idx);
    const float2 pc = *reinterpret_cast<const float2*>(pold + e.idx);
    const Nbr2 nz = load_nbr2(v, z, e);
    const Nbr2 np = load_nbr2(v, pold, e);
    float pn[2], qn[2];
    // a warp whose cells are all fluid with six fluid neighbours: the same
    // operations in the same order without the masks (nfl = count = 6)
    const bool full = pair_full(code2) && e.okA && e.okB;
    if (__all_sync(0xffffffffu, full)) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float zv[6], pv[6];
        nbr_of(nz, h, zv);
        nbr_of(np, h, pv);
        const float p_c = __fmaf_rn(beta, h == 0 ? pc.x : pc.y, h == 0 ? zc.x : zc.y);
        float d = 0.0f;
#pragma unroll
        for (int u = 0; u < 6; ++u) d = __fadd_rn(d, __fsub_rn(p_c, __fmaf_rn(beta, pv[u], zv[u])));
        pn[h] = p_c;
        qn[h] = __fmul_rn(s_a, __fmaf_rn(0.0f, p_c, d));
        acc.add_prod(p_c, qn[h]);
      }
      *reinterpret_cast<float2*>(pnew + e.idx) = make_float2(pn[0], pn[1]);
      *reinterpret_cast<float2*>(q0 + e.idx) = make_float2(qn[0], qn[1]);
      continue;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned int code = h == 0 ? (code2 & 0xffffu) : (code2 >> 16);
      const bool ok = (h == 0 ? e.okA : e.okB) && (code & CODE_SELF);
      float zv[6], pv[6];
      nbr_of(nz, h, zv);
      nbr_of(np, h, pv);
      const float p_c = __fmaf_rn(beta, h == 0 ? pc.x : pc.y, h == 0 ? zc.x : zc.y);
      float d = 0.0f;
      int nfl = 0;
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        const bool f = (code >> u) & 1u;
        d += f ? __fsub_rn(p_c, __fmaf_rn(beta, pv[u], zv[u])) : 0.0f;
        nfl += f;
      }
      const float q_c = __fmul_rn(s_a, __fmaf_rn((float)(code_cnt(code) - nfl), p_c, d));
      pn[h] = ok ? p_c : 0.0f;
      qn[h] = ok ? q_c : 0.0f;
      if (ok) acc.add_prod(p_c, q_c);
    }
    if (e.okA || e.okB) {
      *reinterpret_cast<float2*>(pnew + e.idx) = make_float2(pn[0], pn[1]);
      *reinterpret_cast<float2*>(q0 + e.idx) = make_float2(qn[0], qn[1]);
    }
  }
  pq.add_prod(acc.hi, 1.0f);
  pq.add_prod(acc.lo, 1.0f);
}

// Phase B: d += alpha p, r -= alpha q, partial r.r, and the next V-cycle's first
// red half-sweep (from zero) z = r / (s n) on red cells.  Both colours.
__device__ __noinline__ void phase_b_v(const PcgArgs& A, const float* pnew, float alpha, FF& rr) {
  const MgArgs& M = A.mg;
  const SV v = sview(M.lv[0]);
  float* d0 = M.d0;
  const float* q0 = M.q0;
  const int lane = threadIdx.x & 31;
  const float invs6 = s_inv_scnt[0][6];
  const int2 q = seg_slice(M.lv[0]);
  const Items it = pair_items(q, 2);
  struct S {
    PCell e;
    int c;
    unsigned int code2;
    float2 d, p, qq, r;
  };
  FF acc;
  run_batched<2>(
      it.first, it.end, PCG_WARPS,
      [&](unsigned int t, bool ok) {
        S st;
        st.c = (int)(t & 1u);
        st.e = pcell(v, q, t >> 1, st.c, lane);
        st.e.okA &= ok;
        st.e.okB &= ok;
        st.code2 = *reinterpret_cast<const unsigned int*>(v.code + st.e.idx);
        st.d = *reinterpret_cast<const float2*>(d0 + st.e.idx);
        st.p = *reinterpret_cast<const float2*>(pnew + st.e.idx);
        st.qq = *reinterpret_cast<const float2*>(q0 + st.e.idx);
        st.r = *reinterpret_cast<const float2*>(v.b + st.e.idx);
        return st;
      },
      [&](S&) {},
      [&](S& st) {
        float dn[2], rn[2], zn[2];
        // a warp whose cells are all fluid with six fluid neighbours: no selects
        const bool full = pair_full(st.code2) && st.e.okA && st.e.okB;
        if (__all_sync(0xffffffffu, full)) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float dd = h == 0 ? st.d.x : st.d.y, pp = h == 0 ? st.p.x : st.p.y;
            const float qq = h == 0 ? st.qq.x : st.qq.y, r0 = h == 0 ? st.r.x : st.r.y;
            const float rc = __fmaf_rn(-alpha, qq, r0);
            dn[h] = __fmaf_rn(alpha, pp, dd);
            rn[h] = rc;
            zn[h] = __fmul_rn(rc, invs6);
            acc.add_prod(rc, rc);
          }
          *reinterpret_cast<float2*>(d0 + st.e.idx) = make_float2(dn[0], dn[1]);
          *reinterpret_cast<float2*>(v.b + st.e.idx) = make_float2(rn[0], rn[1]);
          if (st.c == 0) *reinterpret_cast<float2*>(v.x + st.e.idx) = make_float2(zn[0], zn[1]);
          return;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned int code = h == 0 ? (st.code2 & 0xffffu) : (st.code2 >> 16);
          const bool ok = (h == 0 ? st.e.okA : st.e.okB) && (code & CODE_SELF);
          const float dd = h == 0 ? st.d.x : st.d.y, pp = h == 0 ? st.p.x : st.p.y;
          const float qq = h == 0 ? st.qq.x : st.qq.y, r0 = h == 0 ? st.r.x : st.r.y;
          const float rc = __fmaf_rn(-alpha, qq, r0);
          dn[h] = ok ? __fmaf_rn(alpha, pp, dd) : dd;
          rn[h] = ok ? rc : r0;
          zn[h] = ok ? gs_first(0, code_cnt(code), rc) : 0.0f;
          if (ok) acc.add_prod(rc, rc);
        }
        if (st.e.okA || st.e.okB) {
          *reinterpret_cast<float2*>(d0 + st.e.idx) = make_float2(dn[0], dn[1]);
          *reinterpret_cast<float2*>(v.b + st.e.idx) = make_float2(rn[0], rn[1]);
          if (st.c == 0) *reinterpret_cast<float2*>(v.x + st.e.idx) = make_float2(zn[0], zn[1]);
        }
      });
  rr.add_prod(acc.hi, 1.0f);
  rr.add_prod(acc.lo, 1.0f);
}

// Phase A with z from the V-cycle: p_new = z + beta p_old (recomputed for the
// neighbours), q = A p_new in difference form, partial p.q.  Both colours.
__device__ __noinline__ void phase_a_s(const PcgArgs& A, const float* pold, float* pnew, float beta,
                                     FF& pq) {
  const MgArgs& M = A.mg;
  const SV v = sview(M.lv[0]);
  const float* z = v.x;
  float* q0 = M.q0;
  const float s_a = A.s;
  const int lane = threadIdx.x & 31;
  const Items it = seg_items(M.lv[0], 2);
  struct S {
    int idx;
    bool ok;
    unsigned int code;
    float zc, pc;
    float zv[6], pv[6];
  };
  FF acc;
  run_batched<1>(
      it.first, it.end, PCG_WARPS,
      [&](unsigned int t, bool ok) {
        const SCell e = scell(v, v.seg[(int)(t >> 1) - v.seg_base], (int)(t & 1u), lane);
        S s;
        s.idx = e.idx;
        s.ok = e.ok && ok;
        s.code = v.code[e.idx];
        s.zc = z[e.idx];
        s.pc = pold[e.idx];
        int nb[6];
        snbr(v, e, nb);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          s.zv[q] = z[nb[q]];
          s.pv[q] = pold[nb[q]];
        }
        return s;
      },
      [&](S&) {},
      [&](S& s) {
        if (!s.ok || !(s.code & CODE_SELF)) return;
        const int cnt = code_cnt(s.code);
        const float pc = __fmaf_rn(beta, s.pc, s.zc);
        float d = 0.0f;
        int nfl = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const bool f = (s.code >> q) & 1u;
          d += f ? __fsub_rn(pc, __fmaf_rn(beta, s.pv[q], s.zv[q])) : 0.0f;
          nfl += f;
        }
        const float qc = __fmul_rn(s_a, __fmaf_rn((float)(cnt - nfl), pc, d));
        pnew[s.idx] = pc;
        q0[s.idx] = qc;
        acc.add_prod(pc, qc);
      });
  pq.add_prod(acc.hi, 1.0f);
  pq.add_prod(acc.lo, 1.0f);
}

// Phase B: d += alpha p, r -= alpha q, partial r.r, and the next V-cycle's first
// red half-sweep (from zero) z = r / (s n) on red cells.  Both colours.
__device__ __noinline__ void phase_b_s(const PcgArgs& A, const float* pnew, float alpha, FF& rr) {
  const MgArgs& M = A.mg;
  const SV v = sview(M.lv[0]);
  float* d0 = M.d0;
  const float* q0 = M.q0;
  const int lane = threadIdx.x & 31;
  const Items it = seg_items(M.lv[0], 2);
  struct S {
    int idx, c;
    bool ok;
    unsigned int code;
    float d, p, q, r;
  };
  FF acc;
  run_batched<2>(
      it.first, it.end, PCG_WARPS,
      [&](unsigned int t, bool ok) {
        const SCell e = scell(v, v.seg[(int)(t >> 1) - v.seg_base], (int)(t & 1u), lane);
        S s;
        s.idx = e.idx;
        s.c = (int)(t & 1u);
        s.ok = e.ok && ok;
        s.code = v.code[e.idx];
        s.d = d0[e.idx];
        s.p = pnew[e.idx];
        s.q = q0[e.idx];
        s.r = v.b[e.idx];
        return s;
      },
      [&](S&) {},
      [&](S& s) {
        if (!s.ok || !(s.code & CODE_SELF)) return;
        d0[s.idx] = __fmaf_rn(alpha, s.p, s.d);
        const float rc = __fmaf_rn(-alpha, s.q, s.r);
        v.b[s.idx] = rc;
        if (s.c == 0) v.x[s.idx] = gs_first(0, code_cnt(s.code), rc);
        acc.add_prod(rc, rc);
      });
  rr.add_prod(acc.hi, 1.0f);
  rr.add_prod(acc.lo, 1.0f);
}

__device__ __forceinline__ void phase_a(const PcgArgs& A, const float* pold, float* pnew,
                                        float beta, FF& pq) {
  if (use_pairs(A.mg.lv[0])) phase_a_v(A, pold, pnew, beta, pq);
  else phase_a_s(A, pold, pnew, beta, pq);
}

__device__ __forceinline__ void phase_b(const PcgArgs& A, const float* pnew, float alpha, FF& rr) {
  if (use_pairs(A.mg.lv[0])) phase_b_v(A, pnew, alpha, rr);
  else phase_b_s(A, pnew, alpha, rr);
}

// One pass over this thread's fluid cells of level 0, both colours (start of the
// solve, the refinements and the end: not batched).  f(e, code, n) gets the slot,
// its code and the natural index n of the cell.
template <class F>
__device__ __forceinline__ void for_fluid0(const PcgArgs& A, F&& f) {
  const MgLevel& L0 = A.mg.lv[0];
  const SV v0 = sview(L0);
  const int lane = threadIdx.x & 31;
  const Items it = seg_items(L0, 2);
  for (unsigned int t = it.first; t < it.end; t += PCG_WARPS) {
    const SCell e = scell(v0, v0.seg[(int)(t >> 1) - v0.seg_base], (int)(t & 1u), lane);
    if (!e.ok) continue;
    const unsigned int code = L0.code16[e.idx];
    if (!(code & CODE_SELF)) continue;
    f(e, code, e.i + L0.nx * e.r);
  }
}

// Residual b - A x of one level-0 cell with x and b as float pairs (split
// layout); the arithmetic is residual_pair_cell's.
__device__ __forceinline__ float2 residual_pair(const SV& v, const float2* x2, const float2* b2,
                                                const SCell& e, unsigned int code, float s_hi,
                                                float s_lo) {
  int nb[6];
  snbr(v, e, nb);
  const float2 xc = x2[e.idx];
  float2 xn[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) xn[q] = x2[nb[q]];
  return residual_pair_cell(b2[e.idx], xc, xn, code & 63u, code_cnt(code), s_hi, s_lo);
}

// ---------------------------------------------------------------- set-up

// Whether segment g (flat: row g / nw, segment g % nw) of split level L meets a
// block holding fluid; sg receives {row, segment in row, j, k}.  Level 0 reads
// the binning's brick fluid counts.
__device__ __forceinline__ bool seg_active(const PcgArgs& A, const MgLevel& L, int l, int g,
                                           int4& sg) {
  const int r = g / L.nw, w = g - r * L.nw;
  const int j = r % L.ny, k = r / L.ny;
  sg = make_int4(r, w, j, k);
  const int by = j >> 3, bz = k >> 3;
  const int b0 = w * 8, b1 = min(L.nbx, b0 + 8);
  bool any = false;
  for (int bx = b0; bx < b1; ++bx) {
    const int bi = bx + L.nbx * (by + L.nby * bz);
    any |= (l == 0) ? (A.brick_fluid[bi] > 0u) : (L.bflag[bi] != 0);
  }
  return any;
}

// Builds, once per solve: the fluid flags of levels 1.. (a coarse cell is fluid
// when any child is) with their block flags, the active-segment lists of the
// colour-split levels (in segment order, so the work split is deterministic),
// the codes of every level.  Ends with a grid barrier.
__device__ __noinline__ bool build_levels(const PcgArgs& A, Shared& sh) {
  const MgArgs& M = A.mg;
  // block flags of the split coarse levels start clear
  for (int l = 1; l < M.lgrid; ++l) {
    const MgLevel& L = M.lv[l];
    const Part p = level_part(L.nbx * L.nby * L.nbz, false);
    for (int c = p.begin; c < p.end; c += p.stride) L.bflag[c] = 0;
  }
  if (!gsync(A)) return false;
  SOLVE_TRACE(TR_BFLAG);
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
      if (f && C.split) C.bflag[(i >> 3) + C.nbx * ((j >> 3) + C.nby * (k >> 3))] = 1;
    }
    if (!gsync(A)) return false;
    SOLVE_TRACE(TR_FLAGS + min(l, 11));
  }
  // active segments: count per CTA, then write them in segment order
  __shared__ unsigned int s_wsum[PCG_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int l = 0; l < M.lgrid; ++l) {
    const MgLevel& L = M.lv[l];
    const int nsegs = L.nw * L.ny * L.nz;
    const int per = (nsegs + (int)team_size() - 1) / (int)team_size();
    const int g0 = min(nsegs, (int)team_rank() * per), g1 = min(nsegs, g0 + per);
    unsigned int cnt = 0;
    for (int g = g0 + (int)threadIdx.x; g < g1; g += PCG_THREADS) {
      int4 sg;
      cnt += seg_active(A, L, l, g, sg);
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) s_wsum[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int tot = 0;
      for (int w = 0; w < PCG_WARPS; ++w) tot += s_wsum[w];
      M.segcount[l * team_size() + team_rank()] = tot;
    }
    __syncthreads();
  }
  if (!gsync(A)) return false;
  SOLVE_TRACE(TR_SEG_COUNT);
  for (int l = 0; l < M.lgrid; ++l) {
    const MgLevel& L = M.lv[l];
    const int nsegs = L.nw * L.ny * L.nz;
    const int per = (nsegs + (int)team_size() - 1) / (int)team_size();
    const int g0 = min(nsegs, (int)team_rank() * per), g1 = min(nsegs, g0 + per);
    // this CTA's offset: the counts of the CTAs before it
    if (warp == 0) {
      unsigned int before = 0, total = 0;
      for (unsigned int t = lane; t < team_size(); t += 32) {
        const unsigned int v = M.segcount[l * team_size() + t];
        total += v;
        before += (t < team_rank()) ? v : 0u;
      }
      before = __reduce_add_sync(0xffffffffu, before);
      total = __reduce_add_sync(0xffffffffu, total);
      if (lane == 0) {
        sh.dscal[0] = (double)before;
        if (team_rank() == 0) *L.nseg = total;
      }
    }
    __syncthreads();
    unsigned int base = (unsigned int)sh.dscal[0];
    __syncthreads();
    for (int g00 = g0; g00 < g1; g00 += PCG_THREADS) {
      const int g = g00 + (int)threadIdx.x;
      int4 sg = make_int4(0, 0, 0, 0);
      const bool act = g < g1 && seg_active(A, L, l, g, sg);
      const unsigned int bal = __ballot_sync(0xffffffffu, act);
      if (lane == 0) s_wsum[warp] = __popc(bal);
      __syncthreads();
      unsigned int off = 0, tot = 0;
      for (int w = 0; w < PCG_WARPS; ++w) {
        off += (w < warp) ? s_wsum[w] : 0u;
        tot += s_wsum[w];
      }
      if (act) L.seg[base + off + __popc(bal & ((1u << lane) - 1u))] = sg;
      base += tot;
      __syncthreads();
    }
  }
  if (!gsync(A)) return false;
  SOLVE_TRACE(TR_SEG_WRITE);
  // codes: split levels over their active segments, CTA-local levels over all cells
  for (int l = 0; l < M.lgrid; ++l) {
    const MgLevel& L = M.lv[l];
    const Items it = seg_items(L, 2);
    for (unsigned int t = it.first; t < it.end; t += PCG_WARPS) {
      const SCell e = scell(L, L.seg[t >> 1], (int)(t & 1u), lane);
      if (e.ok) L.code16[e.idx] = (uint16_t)make_code(L, L.t, e.i, e.j, e.k);
    }
  }
  for (int l = M.lgrid; l < M.nlev; ++l) {
    const MgLevel& L = M.lv[l];
    const Part p = level_part(L.ncells, false);
    for (int c = p.begin; c < p.end; c += p.stride) {
      const Cell cl = cell_at(L, c);
      L.code[c] = (uint8_t)(make_code(L, L.t, cl.i, cl.j, cl.k) & 0x7fu);
    }
  }
  const bool ok = gsync(A);
  SOLVE_TRACE(TR_CODES);
  return ok;
}

// Copies this CTA's slice of each grid-wide level's segment list into the
// shared-memory cache, level 0 first, while it fits (after build_levels).
__device__ __noinline__ void seg_cache_fill(const MgArgs& M, int4* cache) {
  int used = 0;
  for (int l = 0; l < M.lgrid; ++l) {
    const MgLevel& L = M.lv[l];
    const int2 q = seg_slice(L);
    const int n = q.y - q.x;
    const bool fits = used + n <= SEG_CACHE;
    if (fits)
      for (int i = threadIdx.x; i < n; i += PCG_THREADS) cache[used + i] = L.seg[q.x + i];
    if (threadIdx.x == 0) {
      s_segc[l] = fits ? cache + used : nullptr;
      s_segb[l] = q.x;
    }
    if (fits) used += n;
  }
  __syncthreads();
}

// The shared-memory cache of the segment slices sits after the CTA-local levels
// in the kernel's dynamic shared memory.
constexpr size_t MG_DYN_CTA = (sizeof(CtaMg) + 15) / 16 * 16;
constexpr size_t MG_DYN_BYTES = MG_DYN_CTA + sizeof(int4) * SEG_CACHE;

__device__ __forceinline__ int4* seg_cache_of(unsigned char* dyn) {
  return reinterpret_cast<int4*>(dyn + MG_DYN_CTA);
}

// The mixed mode's refinement, over level 0's slot pairs with two items in flight
// per warp (the per-cell arithmetic of the single-slot form, so the same values).
// refine_update: x += d as float pairs on fluid cells, d = 0 there.
__device__ __noinline__ void refine_update(const PcgArgs& A) {
  const MgArgs& M = A.mg;
  const SV v = sview(M.lv[0]);
  float* d0 = M.d0;
  float2* x2 = M.x2;
  const int lane = threadIdx.x & 31;
  const int2 q = seg_slice(M.lv[0]);
  const Items it = pair_items(q, 2);
  struct S {
    PCell e;
    unsigned int code2;
    float2 d;
    float4 x;  // the two slots' (hi, lo)
  };
  run_batched<2>(
      it.first, it.end, PCG_WARPS,
      [&](unsigned int t, bool ok) {
        S st;
        st.e = pcell(v, q, t >> 1, (int)(t & 1u), lane);
        st.e.okA &= ok;
        st.e.okB &= ok;
        st.code2 = *reinterpret_cast<const unsigned int*>(v.code + st.e.idx);
        st.d = *reinterpret_cast<const float2*>(d0 + st.e.idx);
        st.x = *reinterpret_cast<const float4*>(x2 + st.e.idx);
        return st;
      },
      [&](S&) {},
      [&](S& st) {
        if (!(st.e.okA || st.e.okB)) return;
        const bool fa = st.e.okA && (st.code2 & CODE_SELF);
        const bool fb = st.e.okB && ((st.code2 >> 16) & CODE_SELF);
        const float2 ta = two_sum(st.x.x, st.d.x), tb = two_sum(st.x.z, st.d.y);
        const float2 xa = fast_two_sum(ta.x, __fadd_rn(ta.y, st.x.y));
        const float2 xb = fast_two_sum(tb.x, __fadd_rn(tb.y, st.x.w));
        *reinterpret_cast<float4*>(x2 + st.e.idx) =
            make_float4(fa ? xa.x : st.x.x, fa ? xa.y : st.x.y, fb ? xb.x : st.x.z,
                        fb ? xb.y : st.x.w);
        *reinterpret_cast<float2*>(d0 + st.e.idx) =
            make_float2(fa ? 0.0f : st.d.x, fb ? 0.0f : st.d.y);
      });
}

// refine_residual: r = b - A x in float pairs (residual_pair_cell) on fluid cells,
// the next V-cycle's first red half-sweep z = r / (s n) on red ones, and r.r.
__device__ __noinline__ void refine_residual(const PcgArgs& A, FF& rr) {
  const MgArgs& M = A.mg;
  const MgLevel& L0 = M.lv[0];
  const SV v = sview(L0);
  const float2* x2 = M.x2;
  const float2* b2 = M.b2;
  float* r = L0.b;
  float* z = L0.x;
  const float s_hi = A.s, s_lo = A.s_lo;
  const int lane = threadIdx.x & 31;
  const int2 q = seg_slice(L0);
  const Items it = pair_items(q, 2);
  FF acc;
  for (unsigned int t = it.first; t < it.end; t += PCG_WARPS) {
    const int c = (int)(t & 1u);
    const PCell e = pcell(v, q, t >> 1, c, lane);
    const unsigned int code2 = *reinterpret_cast<const unsigned int*>(v.code + e.idx);
    const float4 bb = *reinterpret_cast<const float4*>(b2 + e.idx);
    const float4 xc = *reinterpret_cast<const float4*>(x2 + e.idx);
    // the other colour around the pair: slots s, s + 1 of this row, the one beyond
    // (s - 1 or s + 2), and the pairs in the rows and planes next door
    const float4 m = *reinterpret_cast<const float4*>(x2 + e.ob);
    const float2 ex = x2[e.ob - 1 + 3 * e.par];
    const float4 ym = *reinterpret_cast<const float4*>(x2 + e.ob - v.hx);
    const float4 yp = *reinterpret_cast<const float4*>(x2 + e.ob + v.hx);
    const float4 zm = *reinterpret_cast<const float4*>(x2 + e.ob - v.pl);
    const float4 zp = *reinterpret_cast<const float4*>(x2 + e.ob + v.pl);
    // a warp whose cells are all fluid with six fluid neighbours: the same cell
    // function with the mask and the count known
    const bool full = __all_sync(0xffffffffu, pair_full(code2) && e.okA && e.okB);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned int code = h == 0 ? (code2 & 0xffffu) : (code2 >> 16);
      if (!full && (!(h == 0 ? e.okA : e.okB) || !(code & CODE_SELF))) continue;
      const float2 m0 = make_float2(m.x, m.y), m1 = make_float2(m.z, m.w);
      float2 xn[6];
      if (h == 0) {
        xn[0] = e.par ? m0 : ex;
        xn[1] = e.par ? m1 : m0;
        xn[2] = make_float2(ym.x, ym.y);
        xn[3] = make_float2(yp.x, yp.y);
        xn[4] = make_float2(zm.x, zm.y);
        xn[5] = make_float2(zp.x, zp.y);
      } else {
        xn[0] = e.par ? m1 : m0;
        xn[1] = e.par ? ex : m1;
        xn[2] = make_float2(ym.z, ym.w);
        xn[3] = make_float2(yp.z, yp.w);
        xn[4] = make_float2(zm.z, zm.w);
        xn[5] = make_float2(zp.z, zp.w);
      }
      const float2 bc = h == 0 ? make_float2(bb.x, bb.y) : make_float2(bb.z, bb.w);
      const float2 xcc = h == 0 ? make_float2(xc.x, xc.y) : make_float2(xc.z, xc.w);
      const float2 rp = full ? residual_pair_cell(bc, xcc, xn, 63u, 6, s_hi, s_lo)
                             : residual_pair_cell(bc, xcc, xn, code & 63u, code_cnt(code), s_hi,
                                                  s_lo);
      const float r32 = __fadd_rn(rp.x, rp.y);
      r[e.idx + h] = r32;
      if (c == 0) z[e.idx + h] = gs_first(0, full ? 6 : code_cnt(code), r32);
      acc.add_prod(r32, r32);
    }
  }
  rr.add_prod(acc.hi, 1.0f);
  rr.add_prod(acc.lo, 1.0f);
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
// 3 = r.z (end of the V-cycle), 4 and 5 = ||b||^2 and ||r_0||^2 (start), 5 = the
// recomputed residual's norm (refinement).  A slot's readers always pass another barrier before the slot
// is written again.
template <bool MIXED>
__device__ void solve_mg(const PcgArgs& A, Shared& sh, int4* segc, SolveState& S) {
  const MgArgs& M = A.mg;
  const MgLevel& L0 = M.lv[0];
  float* d = M.d0;
  float* z = L0.x;
  float* r = L0.b;
  if (!build_levels(A, sh)) { S.ok = false; return; }
  seg_cache_fill(M, segc);
  SOLVE_TRACE(TR_SEG_CACHE);
  if (M.nlev > 1 && team_rank() == 0) cta_levels_init(M);
  SOLVE_TRACE(TR_CTA_LISTS);
  // ---- start: r = b (cold) or b - A x0 (warm start from the last solve's x),
  // p_old = 0, first red half-sweep of the V-cycle; mixed mode: b as a float pair,
  // the correction d = 0, and x = 0 unless warm
  const bool warm = A.warm_start != 0;
  {
    FF bb, rr0;
    const SV v0 = sview(L0);
    const float s_a = A.s;
    if (warm && MIXED) {  // b as a pair first: the residual pass below reads it
      for_fluid0(A, [&](const SCell& e, unsigned int, int n) {
        const double b64 = A.b64[n];
        const float bh = __double2float_rn(b64);
        M.b2[e.idx] = make_float2(bh, __double2float_rn(b64 - (double)bh));
      });
      if (!gsync(A)) { S.ok = false; return; }
    }
    for_fluid0(A, [&](const SCell& e, unsigned int code, int n) {
      float bc, rc;
      if constexpr (MIXED) {
        if (warm) {
          bc = M.b2[e.idx].x;
          const float2 rp = residual_pair(v0, M.x2, M.b2, e, code, s_a, A.s_lo);
          rc = __fadd_rn(rp.x, rp.y);
        } else {
          const double b64 = A.b64[n];
          bc = __double2float_rn(b64);
          M.b2[e.idx] = make_float2(bc, __double2float_rn(b64 - (double)bc));
          M.x2[e.idx] = make_float2(0.0f, 0.0f);
          rc = bc;
        }
        d[e.idx] = 0.0f;
      } else {
        bc = A.b32[n];
        rc = bc;
        if (warm) {
          int nb[6];
          snbr(v0, e, nb);
          float xv[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) xv[q] = d[nb[q]];
          rc = resid(s_a, code_cnt(code), code, bc, d[e.idx], xv);
        } else {
          d[e.idx] = 0.0f;
        }
      }
      r[e.idx] = rc;
      M.pa0[e.idx] = 0.0f;
      if (e.idx < L0.half) z[e.idx] = gs_first(0, code_cnt(code), rc);
      bb.add_prod(bc, bc);
      rr0.add_prod(rc, rc);
    });
    F2 v[2] = {f2_of(bb), f2_of(rr0)};
    publish<2>(A, 4, v, sh);
  }
  if (!gsync(A)) { S.ok = false; return; }
  SOLVE_TRACE(TR_START);
  double rz = 0.0, bnorm = 0.0, rnorm = 0.0, rmax = 0.0;
  const double target = MIXED ? A.ir_tol : A.tol;
  {
    double s0[2];
    gather<2>(A, 4, s0, sh);
    if (threadIdx.x == 0) {
      bnorm = sqrt(fmax(s0[0], 0.0));
      rnorm = rmax = sqrt(fmax(s0[1], 0.0));
      sh.flag = (bnorm == 0.0 || rnorm <= target * bnorm) ? 1 : 0;
    }
  }
  __syncthreads();
  int it = 0, refinements = 0;
  bool conv = sh.flag == 1, first = true;
  float* pold = M.pa0;
  float* pnew = M.pb0;
  while (!conv) {
    FF rzp;
    if (!vcycle_rest(A, rzp)) { S.ok = false; return; }
    {
      F2 v[1] = {f2_of(rzp)};
      publish<1>(A, 3, v, sh);
    }
    if (!gsync(A)) { S.ok = false; return; }
    if (it < 3) SOLVE_TRACE(TR_ITER + 3 * it);
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
    phase_a(A, pold, pnew, beta, pq);
    {
      F2 v[1] = {f2_of(pq)};
      publish<1>(A, 0, v, sh);
    }
    if (!gsync(A)) { S.ok = false; return; }
    if (it <= 3) SOLVE_TRACE(TR_ITER + 3 * (it - 1) + 1);
    {
      double s[1];
      gather<1>(A, 0, s, sh);
      if (threadIdx.x == 0) sh.alpha = (float)(rz / s[0]);
    }
    __syncthreads();
    const float alpha = sh.alpha;
    // ---- phase B (+ the next V-cycle's first red half-sweep)
    FF rr;
    phase_b(A, pnew, alpha, rr);
    {
      F2 v[1] = {f2_of(rr)};
      publish<1>(A, 1, v, sh);
    }
    if (!gsync(A)) { S.ok = false; return; }
    if (it <= 3) SOLVE_TRACE(TR_ITER + 3 * (it - 1) + 2);
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
        // ---- refinement: x += d, d = 0; r = b - A x in float pairs (+ first red
        // half-sweep)
        if (refinements == 0) SOLVE_TRACE(TR_REFINE);
        refine_update(A);
        if (!gsync(A)) { S.ok = false; return; }
        if (refinements == 0) SOLVE_TRACE(TR_REFINE + 1);
        FF rr64;
        refine_residual(A, rr64);
        F2 v[1] = {f2_of(rr64)};
        publish<1>(A, 5, v, sh);
        if (!gsync(A)) { S.ok = false; return; }
        if (refinements == 0) SOLVE_TRACE(TR_REFINE + 2);
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
  SOLVE_TRACE(TR_LOOP_END);
  // ---- the solution in natural layout: the FP32 pressure, or the float pair
  // (for G2P) and its FP64 value
  if constexpr (MIXED) {
    for_fluid0(A, [&](const SCell& e, unsigned int, int n) {
      float2 xp = M.x2[e.idx];
      if (!conv) {
        const float2 t = two_sum(xp.x, d[e.idx]);
        xp = fast_two_sum(t.x, __fadd_rn(t.y, xp.y));
        d[e.idx] = 0.0f;
      }
      A.pff[n] = xp;
      A.x64[n] = (double)xp.x + (double)xp.y;
    });
  } else {
    for_fluid0(A, [&](const SCell& e, unsigned int, int n) { A.x32[n] = d[e.idx]; });
  }
  SOLVE_TRACE(TR_END);
  S.iters = it;
  S.refinements = refinements;
  S.conv = conv;
  S.rel = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  S.bnorm = bnorm;
}

// The paper's GPU solver (Sec. 3.2.3): red-black Gauss-Seidel sweeps on A p = b
// from p = 0 (FP32), on the colour-split level-0 storage with the smoother's
// half-sweeps, until ||b - A p|| <= tol ||b||; the residual is taken every
// RBGS_CHECK sweep pairs and the sweep pairs are capped at max_iter.
constexpr int RBGS_CHECK = 8;

__device__ __noinline__ void solve_rbgs(const PcgArgs& A, Shared& sh, int4* segc, SolveState& S) {
  const MgArgs& M = A.mg;
  const MgLevel& L0 = M.lv[0];
  const MgLevel& L1 = M.nlev > 1 ? M.lv[1] : M.lv[0];
  float* z = L0.x;
  float* r = L0.b;
  if (!build_levels(A, sh)) { S.ok = false; return; }
  seg_cache_fill(M, segc);
  {
    FF bb;
    for_fluid0(A, [&](const SCell& e, unsigned int, int n) {
      const float bc = A.b32[n];
      r[e.idx] = bc;
      z[e.idx] = 0.0f;
      bb.add_prod(bc, bc);
    });
    F2 v[1] = {f2_of(bb)};
    publish<1>(A, 4, v, sh);
  }
  if (!gsync(A)) { S.ok = false; return; }
  double bnorm = 0.0, rnorm = 0.0;
  {
    double s0[1];
    gather<1>(A, 4, s0, sh);
    if (threadIdx.x == 0) {
      bnorm = sqrt(fmax(s0[0], 0.0));
      rnorm = bnorm;
      sh.flag = (bnorm == 0.0) ? 1 : 0;
    }
  }
  __syncthreads();
  bool conv = sh.flag == 1;
  int it = 0;
  while (!conv) {
    for (int k = 0; k < RBGS_CHECK; ++k) {
      sweep_split<NORMAL>(M, L0, L1, 0, 0, nullptr);
      if (!gsync(A)) { S.ok = false; return; }
      sweep_split<NORMAL>(M, L0, L1, 0, 1, nullptr);
      if (!gsync(A)) { S.ok = false; return; }
    }
    it += RBGS_CHECK;
    FF rr;
    const SV v0 = sview(L0);
    for_fluid0(A, [&](const SCell& e, unsigned int code, int) {
      int nb[6];
      snbr(v0, e, nb);
      float xv[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) xv[q] = z[nb[q]];
      const float rc = resid(A.s, code_cnt(code), code, r[e.idx], z[e.idx], xv);
      rr.add_prod(rc, rc);
    });
    {
      F2 v[1] = {f2_of(rr)};
      publish<1>(A, 5, v, sh);
    }
    if (!gsync(A)) { S.ok = false; return; }
    {
      double s[1];
      gather<1>(A, 5, s, sh);
      if (threadIdx.x == 0) {
        rnorm = sqrt(fmax(s[0], 0.0));
        if (rnorm <= A.tol * bnorm) sh.flag = 1;
        else if (it >= A.max_iter) sh.flag = 3;
        else sh.flag = 0;
      }
    }
    __syncthreads();
    if (sh.flag == 1) conv = true;
    if (sh.flag == 3) break;
  }
  for_fluid0(A, [&](const SCell& e, unsigned int, int n) { A.x32[n] = z[e.idx]; });
  S.iters = it;
  S.conv = conv;
  S.rel = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  S.bnorm = bnorm;
}

template <bool MIXED>
__device__ void solve_scene_mg(const PcgArgs& A, Shared& sh, unsigned char* dyn) {
  int4* segc = seg_cache_of(dyn);
  if (threadIdx.x < MG_MAX_LEVELS) s_segc[threadIdx.x] = nullptr;  // no cache until filled
  __syncthreads();
  const long long ncells = (long long)A.g.nx * A.g.ny * A.g.nz;
  const bool singular = A.check_singular && ((long long)A.stats->n_fluid == ncells);
  SolveState S;
  if (!singular) {
    if (!MIXED && A.precond == PRECOND_RBGS) solve_rbgs(A, sh, segc, S);
    else solve_mg<MIXED>(A, sh, segc, S);
  }
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
  extern __shared__ __align__(16) unsigned char mg_dyn[];
  team_enter(blockIdx.x, gridDim.x);
  SOLVE_TRACE(TR_ENTRY);
  load_tables(A.mg);
  SOLVE_TRACE(TR_TABLES);
  solve_scene_mg<MIXED>(A, sh, mg_dyn);
  SOLVE_TRACE(TR_EXIT);
}

// Several scenes in one launch: CTA b works on scene block_scene[b], in the team
// of CTAs team_first[s] .. team_first[s+1]-1.
template <bool MIXED>
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg_mg_batch(const __grid_constant__ PcgBatch B) {
  __shared__ Shared sh;
  extern __shared__ __align__(16) unsigned char mg_dyn[];
  const int s = B.block_scene[blockIdx.x];
  team_enter(blockIdx.x - B.team_first[s], B.team_first[s + 1] - B.team_first[s]);
  load_tables(B.args[s].mg);
  solve_scene_mg<MIXED>(B.args[s], sh, mg_dyn);
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
                                       dim3(PCG_THREADS), args, MG_DYN_BYTES, s);
  return cudaLaunchCooperativeKernel((const void*)k_pcg_mg<false>, dim3(nblocks),
                                     dim3(PCG_THREADS), args, MG_DYN_BYTES, s);
}

cudaError_t launch_pcg_mg_batch(const PcgBatch& b, bool mixed, int nblocks, cudaStream_t s) {
  void* args[] = {const_cast<PcgBatch*>(&b)};
  if (mixed)
    return cudaLaunchCooperativeKernel((const void*)k_pcg_mg_batch<true>, dim3(nblocks),
                                       dim3(PCG_THREADS), args, MG_DYN_BYTES, s);
  return cudaLaunchCooperativeKernel((const void*)k_pcg_mg_batch<false>, dim3(nblocks),
                                     dim3(PCG_THREADS), args, MG_DYN_BYTES, s);
}

// Opts the kernels in to the dynamic shared memory of the CTA-local levels and
// checks that one CTA per SM fits.
cudaError_t pcg_mg_check_occupancy() {
  const void* fns[4] = {(const void*)k_pcg_mg<false>, (const void*)k_pcg_mg<true>,
                        (const void*)k_pcg_mg_batch<false>, (const void*)k_pcg_mg_batch<true>};
  for (const void* f : fns) {
    cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MG_DYN_BYTES);
    if (e != cudaSuccess) return e;
    int a = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, f, PCG_THREADS, MG_DYN_BYTES);
    if (e != cudaSuccess) return e;
    if (a < 1) return cudaErrorInvalidConfiguration;
  }
  return cudaSuccess;
}

}  // namespace flipk

#ifdef FLIP_SOLVE_TRACE
// The stamps of the last solve (nanoseconds of the global timer; slots of
// flipk::TraceSlot; 0 where no stamp was taken since the library was loaded).
extern "C" int flip_solve_trace(unsigned long long* out, int n) {
  if (!out || n < 1 || n > 64) return 1;
  return cudaMemcpyFromSymbol(out, flipk::flip_trace_ns, sizeof(unsigned long long) * (size_t)n) ==
                 cudaSuccess
             ? 0
             : 3;
}
#endif
