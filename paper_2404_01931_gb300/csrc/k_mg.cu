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
#include "pcg_common.cuh"

namespace flipk {

namespace {

// ---------------------------------------------------------------- partitions

struct Part {
  int begin, end, stride;
};

// Dense cells of a level owned by this thread: a contiguous slice per CTA
// (grid-wide levels) or all cells by CTA 0's threads (CTA-local levels).
__device__ __forceinline__ Part level_part(int ncells, bool cta_local) {
  if (cta_local) return Part{(int)threadIdx.x, ncells, PCG_THREADS};
  int per = (ncells + (int)team_size() - 1) / (int)team_size();
  per = (per + 31) & ~31;
  const int b = min(ncells, (int)team_rank() * per);
  return Part{b + (int)threadIdx.x, min(ncells, b + per), PCG_THREADS};
}

struct LCell {
  int i, j, k, c;
};

template <class F>
__device__ __forceinline__ void for_level_cells(const MgLevel& L, const Part& p, F&& f) {
  for (int c = p.begin; c < p.end; c += p.stride) {
    if (L.t[c] != 1) continue;
    const int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
    f(LCell{i, j, k, c});
  }
}

__device__ __forceinline__ int lcount(const MgLevel& L, int i, int j, int k) {
  return (i > 0) + (i < L.nx - 1) + (j > 0) + (j < L.ny - 1) + (k > 0) + (k < L.nz - 1);
}

struct LNbr {
  int idx[6];
  bool fl[6];
};

__device__ __forceinline__ LNbr lneighbours(const MgLevel& L, int i, int j, int k, int c) {
  const int sy = L.nx, sz = L.nx * L.ny;
  const bool in[6] = {i > 0, i < L.nx - 1, j > 0, j < L.ny - 1, k > 0, k < L.nz - 1};
  const int off[6] = {-1, 1, -sy, sy, -sz, sz};
  LNbr n;
#pragma unroll
  for (int q = 0; q < 6; ++q) n.idx[q] = in[q] ? c + off[q] : c;
  uint8_t t[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) t[q] = L.t[n.idx[q]];
#pragma unroll
  for (int q = 0; q < 6; ++q) n.fl[q] = in[q] && t[q] == 1;
  return n;
}

// Index of the parent (level l+1 cell) of the level-l cell (i, j, k).
__device__ __forceinline__ int parent_index(const MgLevel& C, int i, int j, int k) {
  return (i >> 1) + C.nx * ((j >> 1) + C.ny * (k >> 1));
}

enum SweepMode { FIRST = 0, NORMAL = 1, CORRECT = 2 };

// One Gauss-Seidel update of a cell of the sweep colour:
//   x_c = b_c / (s n_c) + (sum of fluid neighbours' x) / n_c
// FIRST: all neighbours are still zero.  CORRECT: neighbours are read as
// x_n + omega x_{l+1}(parent(n)) (the coarse correction, applied on the fly).
template <int MODE>
__device__ __forceinline__ float gs_value(const MgArgs& M, int l, int i, int j, int k, int c,
                                          float bc) {
  const MgLevel& L = M.lv[l];
  const int cnt = lcount(L, i, j, k);
  const float base = __fmul_rn(bc, L.inv_scnt[cnt]);
  if constexpr (MODE == FIRST) return base;
  const LNbr n = lneighbours(L, i, j, k, c);
  float xv[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) xv[q] = L.x[n.idx[q]];
  if constexpr (MODE == CORRECT) {
    const MgLevel& C = M.lv[l + 1];
    const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (n.fl[q]) xv[q] = __fmaf_rn(M.omega, C.x[parent_index(C, i + di[q], j + dj[q], k + dk[q])], xv[q]);
  }
  float sum = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) sum += n.fl[q] ? xv[q] : 0.0f;
  return __fmaf_rn(sum, M.inv_cnt[cnt], base);
}

// Residual b - A x of a fluid cell of level l, with A x in difference form
// s (sum_fluid (x_c - x_n) + n_air x_c).
__device__ __forceinline__ float level_residual(const MgLevel& L, const float* b, int i, int j,
                                                int k, int c) {
  const LNbr n = lneighbours(L, i, j, k, c);
  const float xc = L.x[c];
  float xv[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) xv[q] = L.x[n.idx[q]];
  float d = 0.0f;
  int nfl = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    d += n.fl[q] ? __fsub_rn(xc, xv[q]) : 0.0f;
    nfl += n.fl[q];
  }
  const int cnt = lcount(L, i, j, k);
  return __fsub_rn(b[c], __fmul_rn(L.s, __fmaf_rn((float)(cnt - nfl), xc, d)));
}

// ---------------------------------------------------------------- sweeps

// Half-sweep of one colour over level l >= 1.  Threads map onto the cells of
// the sweep colour: each x-row has ceil(nx/2) slots, slot q of row (j, k) is
// x = 2q + parity (skipped when it falls off an odd-length row).
template <int MODE>
__device__ __forceinline__ void sweep_level(const MgArgs& M, int l, int colour, bool cta_local) {
  const MgLevel& L = M.lv[l];
  const int hx = (L.nx + 1) >> 1;
  const Part p = level_part(hx * L.ny * L.nz, cta_local);
  for (int e = p.begin; e < p.end; e += p.stride) {
    const int row = e / hx, q = e - row * hx;
    const int j = row % L.ny, k = row / L.ny;
    const int i = 2 * q + ((colour + j + k) & 1);
    if (i >= L.nx) continue;
    const int c = i + L.nx * row;
    if (L.t[c] != 1) continue;
    L.x[c] = gs_value<MODE>(M, l, i, j, k, c, L.b[c]);
  }
}

// Half-sweep of one colour over level 0; the right-hand side is the CG residual
// r.  Threads map straight onto the cells of the sweep colour: slot e of the
// colour's index space (256 cells per brick) is brick e/256, row m/4 of the
// brick (y fastest within z) and x position 2(m%4) + parity, so no lane idles on
// a cell of the other colour.  Slices are contiguous per CTA as for the CG.
template <int MODE>
__device__ __forceinline__ void sweep_level0(const PcgArgs& A, const Chunk& ch, int colour) {
  (void)ch;
  const MgArgs& M = A.mg;
  const MgLevel& L = M.lv[0];
  const Grid& g = A.g;
  const unsigned int nact = *A.n_active;
  const unsigned int total = nact * (BRICK_CELLS / 2);
  unsigned int per = (total + team_size() - 1) / team_size();
  per = (per + 31u) & ~31u;
  const unsigned int b = min(total, team_rank() * per), e_end = min(total, b + per);
  for (unsigned int e = b + threadIdx.x; e < e_end; e += PCG_THREADS) {
    const unsigned int brick = A.active[e >> 8];
    const int m = (int)(e & 255u);
    const int lj = (m >> 2) & 7, lk = m >> 5;
    const int li = 2 * (m & 3) + ((colour + lj + lk) & 1);
    const int i = (int)(brick % (unsigned)g.bx) * BRICK + li;
    const int j = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK + lj;
    const int k = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK + lk;
    if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
    const int c = i + g.nx * (j + g.ny * k);
    if (A.type[c] != 1) continue;
    L.x[c] = gs_value<MODE>(M, 0, i, j, k, c, A.r[c]);
  }
}

// b_{l+1} = (1/16) sum over fluid children of the level-l residual.  The
// restriction follows the pre-smoothing, whose last half-sweep is black: a black
// cell's update solves its own equation against the red neighbours it read, so
// its residual is exactly zero and only the red children contribute.
__device__ __forceinline__ void restrict_level(const PcgArgs& A, int l, bool cta_local) {
  const MgArgs& M = A.mg;
  const MgLevel& F = M.lv[l];
  const MgLevel& C = M.lv[l + 1];
  const float* fb = (l == 0) ? A.r : F.b;
  for_level_cells(C, level_part(C.ncells, cta_local), [&](const LCell& e) {
    float sum = 0.0f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        // the red child of row (dy, dz): x offset making 2I+dx+2J+dy+2K+dz even
        const int dx = (dy + dz) & 1;
        const int i = 2 * e.i + dx, j = 2 * e.j + dy, k = 2 * e.k + dz;
        if (i >= F.nx || j >= F.ny || k >= F.nz) continue;
        const int c = i + F.nx * (j + F.ny * k);
        if (F.t[c] != 1) continue;
        sum = __fadd_rn(sum, level_residual(F, fb, i, j, k, c));
      }
    C.b[e.c] = __fmul_rn(sum, 0.0625f);
  });
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

// Pre-smoothing of level l >= 1 from zero, then restriction to l+1.
__device__ __forceinline__ bool down_level(const PcgArgs& A, int l, bool cta_local) {
  const MgArgs& M = A.mg;
  const Sync sync{&A, cta_local};
  sweep_level<FIRST>(M, l, 0, cta_local);
  if (!sync()) return false;
  sweep_level<NORMAL>(M, l, 1, cta_local);
  if (!sync()) return false;
  for (int s = 1; s < M.nu; ++s) {
    sweep_level<NORMAL>(M, l, 0, cta_local);
    if (!sync()) return false;
    sweep_level<NORMAL>(M, l, 1, cta_local);
    if (!sync()) return false;
  }
  restrict_level(A, l, cta_local);
  return sync();
}

// Coarse correction + post-smoothing of level l >= 1.
__device__ __forceinline__ bool up_level(const PcgArgs& A, int l, bool cta_local) {
  const MgArgs& M = A.mg;
  const Sync sync{&A, cta_local};
  sweep_level<CORRECT>(M, l, 1, cta_local);
  if (!sync()) return false;
  sweep_level<NORMAL>(M, l, 0, cta_local);
  if (!sync()) return false;
  for (int s = 1; s < M.nu; ++s) {
    sweep_level<NORMAL>(M, l, 1, cta_local);
    if (!sync()) return false;
    sweep_level<NORMAL>(M, l, 0, cta_local);
    if (!sync()) return false;
  }
  return true;
}

// The coarsest level: MG_COARSE_SWEEPS (red, black) pairs from zero, then as many
// (black, red) pairs.
__device__ __forceinline__ bool coarsest_level(const PcgArgs& A, int l, bool cta_local) {
  const MgArgs& M = A.mg;
  const Sync sync{&A, cta_local};
  sweep_level<FIRST>(M, l, 0, cta_local);
  if (!sync()) return false;
  sweep_level<NORMAL>(M, l, 1, cta_local);
  if (!sync()) return false;
  for (int s = 1; s < MG_COARSE_SWEEPS; ++s) {
    sweep_level<NORMAL>(M, l, 0, cta_local);
    if (!sync()) return false;
    sweep_level<NORMAL>(M, l, 1, cta_local);
    if (!sync()) return false;
  }
  for (int s = 0; s < MG_COARSE_SWEEPS; ++s) {
    sweep_level<NORMAL>(M, l, 1, cta_local);
    if (!sync()) return false;
    sweep_level<NORMAL>(M, l, 0, cta_local);
    if (!sync()) return false;
  }
  return true;
}

// Levels [lgrid, nlev) inside CTA 0.
__device__ void cta_cycle(const PcgArgs& A) {
  const MgArgs& M = A.mg;
  for (int l = M.lgrid; l < M.nlev - 1; ++l) down_level(A, l, true);
  coarsest_level(A, M.nlev - 1, true);
  for (int l = M.nlev - 2; l >= M.lgrid; --l) up_level(A, l, true);
}

// z = V(r), given that the first red half-sweep of level 0 (from zero) has been
// done in the phase that produced r, and that a grid barrier has passed since.
// Ends with the last red half-sweep of
// level 0, which also accumulates r.z over all owned cells into rz.  The caller
// publishes rz and meets the next barrier.  Returns false if a barrier failed.
__device__ bool vcycle_rest(const PcgArgs& A, const Chunk& ch, FF& rz) {
  const MgArgs& M = A.mg;
  const Sync gsync{&A, false};
  const MgLevel& L0 = M.lv[0];
  if (M.nlev == 1) {  // level 0 is the coarsest level
    sweep_level0<NORMAL>(A, ch, 1);
    if (!gsync()) return false;
    for (int s = 1; s < MG_COARSE_SWEEPS; ++s) {
      sweep_level0<NORMAL>(A, ch, 0);
      if (!gsync()) return false;
      sweep_level0<NORMAL>(A, ch, 1);
      if (!gsync()) return false;
    }
    for (int s = 0; s < MG_COARSE_SWEEPS; ++s) {
      sweep_level0<NORMAL>(A, ch, 1);
      if (!gsync()) return false;
      if (s + 1 < MG_COARSE_SWEEPS) {
        sweep_level0<NORMAL>(A, ch, 0);
        if (!gsync()) return false;
      }
    }
  } else {
    sweep_level0<NORMAL>(A, ch, 1);
    if (!gsync()) return false;
    for (int s = 1; s < M.nu; ++s) {
      sweep_level0<NORMAL>(A, ch, 0);
      if (!gsync()) return false;
      sweep_level0<NORMAL>(A, ch, 1);
      if (!gsync()) return false;
    }
    restrict_level(A, 0, false);
    if (!gsync()) return false;
    for (int l = 1; l < M.lgrid; ++l)
      if (!down_level(A, l, false)) return false;
    if (team_rank() == 0) cta_cycle(A);
    if (!gsync()) return false;
    for (int l = M.lgrid - 1; l >= 1; --l)
      if (!up_level(A, l, false)) return false;
    sweep_level0<CORRECT>(A, ch, 1);
    if (!gsync()) return false;
    for (int s = 1; s < M.nu; ++s) {
      sweep_level0<NORMAL>(A, ch, 0);
      if (!gsync()) return false;
      sweep_level0<NORMAL>(A, ch, 1);
      if (!gsync()) return false;
    }
  }
  // last red half-sweep of level 0, with r.z over every owned cell
  for_my_cells(A, ch, [&](const CellRef& cr) {
    const float rc = A.r[cr.c];
    float zc;
    if (((cr.i + cr.j + cr.k) & 1) == 0) {
      zc = gs_value<NORMAL>(M, 0, cr.i, cr.j, cr.k, cr.c, rc);
      L0.x[cr.c] = zc;
    } else {
      zc = L0.x[cr.c];
    }
    rz.add_prod(rc, zc);
  });
  return true;
}

// Phase A with z from the V-cycle: p_new = z + beta p_old (recomputed for the
// neighbours), q = A p_new, partial p.q.
__device__ __forceinline__ void phase_a_mg(const PcgArgs& A, const CellRef& cr, const float* z,
                                           const float* pold, float* pnew, float beta, FF& pq) {
  const Nbrs n = neighbours(A, cr);
  const int cnt = nonsolid_count(A.g, cr.i, cr.j, cr.k);
  float zv[6], pv[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    zv[q] = z[n.idx[q]];
    pv[q] = pold[n.idx[q]];
  }
  const float pc = __fmaf_rn(beta, pold[cr.c], z[cr.c]);
  float d = 0.0f;  // difference form of (A p)_c, as in the Jacobi kernel
  int nfl = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    d += n.fl[q] ? __fsub_rn(pc, __fmaf_rn(beta, pv[q], zv[q])) : 0.0f;
    nfl += n.fl[q];
  }
  const float qc = __fmul_rn(A.s, __fmaf_rn((float)(cnt - nfl), pc, d));
  pnew[cr.c] = pc;
  A.q[cr.c] = qc;
  pq.add_prod(pc, qc);
}

// Builds the fluid flags of levels 1.. from level 0 (a coarse cell is fluid when
// any child is).
__device__ bool build_levels(const PcgArgs& A) {
  const MgArgs& M = A.mg;
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
  return true;
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
__device__ void solve_mg(const PcgArgs& A, const Chunk& ch, Shared& sh, SolveState& S) {
  float* x = A.x32;
  float* z = A.mg.lv[0].x;
  if (!build_levels(A)) { S.ok = false; return; }
  // ---- start: r = b, x = 0, p_old = 0, first red half-sweep of the V-cycle
  {
    FF bb;
    for_my_cells(A, ch, [&](const CellRef& cr) {
      const float bc = MIXED ? (float)A.b64[cr.c] : A.b32[cr.c];
      A.r[cr.c] = bc;
      x[cr.c] = 0.0f;
      A.pa[cr.c] = 0.0f;
      if (((cr.i + cr.j + cr.k) & 1) == 0) z[cr.c] = gs_value<FIRST>(A.mg, 0, cr.i, cr.j, cr.k, cr.c, bc);
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
    if (!vcycle_rest(A, ch, rzp)) { S.ok = false; return; }
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
    for_my_cells(A, ch, [&](const CellRef& cr) { phase_a_mg(A, cr, z, pold, pnew, beta, pq); });
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
    for_my_cells(A, ch, [&](const CellRef& cr) {
      const int c = cr.c;
      x[c] = __fmaf_rn(alpha, pnew[c], x[c]);
      const float rc = __fmaf_rn(-alpha, A.q[c], A.r[c]);
      A.r[c] = rc;
      if (((cr.i + cr.j + cr.k) & 1) == 0) z[c] = gs_value<FIRST>(A.mg, 0, cr.i, cr.j, cr.k, c, rc);
      rr.add_prod(rc, rc);
    });
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
        for_my_cells(A, ch, [&](const CellRef& cr) {
          A.x64[cr.c] += (double)x[cr.c];
          x[cr.c] = 0.0f;
        });
        if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
        FF rr64;
        for_my_cells(A, ch, [&](const CellRef& cr) {
          const float r32 = (float)residual64(A, cr);
          A.r[cr.c] = r32;
          if (((cr.i + cr.j + cr.k) & 1) == 0)
            z[cr.c] = gs_value<FIRST>(A.mg, 0, cr.i, cr.j, cr.k, cr.c, r32);
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
      for_my_cells(A, ch, [&](const CellRef& cr) {
        A.x64[cr.c] += (double)x[cr.c];
        x[cr.c] = 0.0f;
      });
    }
    for_my_cells(A, ch, [&](const CellRef& cr) {
      const double xv = A.x64[cr.c];
      const float hi = __double2float_rn(xv);
      const float lo = __double2float_rn(xv - (double)hi);
      A.pff[cr.c] = make_float2(hi, lo);
    });
  }
  S.iters = it;
  S.refinements = refinements;
  S.conv = conv;
  S.rel = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  S.bnorm = bnorm;
}

template <bool MIXED>
__device__ void solve_scene_mg(const PcgArgs& A, Shared& sh) {
  const unsigned int nact = *A.n_active;
  const long long ncells = (long long)A.g.nx * A.g.ny * A.g.nz;
  const bool singular = A.check_singular && ((long long)A.stats->n_fluid == ncells);
  SolveState S;
  if (!singular) solve_mg<MIXED>(A, my_chunk(nact), sh, S);
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
  team_enter(blockIdx.x, gridDim.x);
  solve_scene_mg<MIXED>(A, sh);
}

// Several scenes in one launch: CTA b works on scene block_scene[b], in the team
// of CTAs team_first[s] .. team_first[s+1]-1.
template <bool MIXED>
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg_mg_batch(const __grid_constant__ PcgBatch B) {
  __shared__ Shared sh;
  const int s = B.block_scene[blockIdx.x];
  team_enter(blockIdx.x - B.team_first[s], B.team_first[s + 1] - B.team_first[s]);
  solve_scene_mg<MIXED>(B.args[s], sh);
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
