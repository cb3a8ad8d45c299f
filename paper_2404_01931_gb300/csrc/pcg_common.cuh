// pcg_common.cuh — device helpers shared by the persistent PCG kernels
// (Jacobi in k_pcg.cu, multigrid in k_mg.cu): float-pair reductions, the
// ownership of cells by CTAs, neighbour gathering and the publish/gather of
// per-CTA partial sums around grid barriers.
#pragma once

#include "flip_kernels.cuh"

namespace flipk {

constexpr int PCG_THREADS = 1024;

// The CTAs that solve one scene form a team: the whole grid for a single scene,
// a slice of it when several scenes share one launch.  A CTA's rank and the
// team size are set once at kernel entry; barriers, reductions and the
// ownership of cells all use them instead of blockIdx / gridDim.
__shared__ unsigned int s_team_rank, s_team_size;

__device__ __forceinline__ unsigned int team_rank() { return s_team_rank; }
__device__ __forceinline__ unsigned int team_size() { return s_team_size; }

__device__ __forceinline__ void team_enter(unsigned int rank, unsigned int size) {
  if (threadIdx.x == 0) {
    s_team_rank = rank;
    s_team_size = size;
    s_bar_gen = 0u;  // grid barriers passed in this launch
  }
  __syncthreads();
}
constexpr int PCG_WARPS = PCG_THREADS / 32;

// ------------------------------------------------------------ float pairs

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
  const float hi = __fadd_rn(s, lo);
  return F2{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

__device__ __forceinline__ F2 f2_of(const FF& f) { return F2{f.hi, f.lo}; }

__device__ __forceinline__ F2 f2_warp_sum(F2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F2 w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = f2_add(v, w);
  }
  return v;
}

// CTA-wide sum of K float pairs; the result is valid in thread 0 only.
template <int K>
__device__ __forceinline__ void cta_sum(F2 (&v)[K], F2* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = f2_warp_sum(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) scratch[q * PCG_WARPS + warp] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      F2 s = (lane < PCG_WARPS) ? scratch[q * PCG_WARPS + lane] : F2{0.0f, 0.0f};
      v[q] = f2_warp_sum(s);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- float pairs

// Error-free transforms (Knuth's TwoSum, Dekker's FastTwoSum, the FMA product):
// a value is carried as hi + lo, ~48 significant bits, all on the FP32 pipes
// (GB300's FP64 pipe is narrow, and the refinement touches every fluid cell).
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv)));
}

__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ float2 pair_add(float2 x, float2 y) {
  const float2 t = two_sum(x.x, y.x);
  return fast_two_sum(t.x, __fadd_rn(t.y, __fadd_rn(x.y, y.y)));
}

__device__ __forceinline__ float2 pair_neg(float2 x) { return make_float2(-x.x, -x.y); }

// (hi, lo) * f for a float f, with the exact product of the hi parts.
__device__ __forceinline__ float2 pair_mul(float2 x, float f) {
  const float p = __fmul_rn(x.x, f);
  const float e = __fmaf_rn(x.x, f, -p);
  return fast_two_sum(p, __fmaf_rn(x.y, f, e));
}

// (hi, lo) * (s_hi, s_lo): the exact product of the hi parts plus the two cross
// terms (the lo * s_lo term is below the pair's precision).
__device__ __forceinline__ float2 pair_mul_pair(float2 x, float s_hi, float s_lo) {
  const float p = __fmul_rn(x.x, s_hi);
  const float e = __fmaf_rn(x.x, s_hi, -p);
  return fast_two_sum(p, __fmaf_rn(x.x, s_lo, __fmaf_rn(x.y, s_hi, e)));
}

// The mixed mode's residual of one cell, b - A x, with x, b and the operator's
// scale s = dt/(rho dx^2) as float pairs (Sec. 3.1.7's 7-point row): A x in
// difference form s ((cnt - nfl) x_c + sum over fluid neighbours (x_c - x_n)),
// bit q of `fluid` set when neighbour q is fluid, cnt the non-wall neighbours.
// The refinement of the multigrid solve and flip_residual_pairs both call it.
__device__ __forceinline__ float2 residual_pair_cell(float2 b, float2 xc, const float2 (&xn)[6],
                                                     unsigned int fluid, int cnt, float s_hi,
                                                     float s_lo) {
  float2 acc = make_float2(0.0f, 0.0f);
  int nfl = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (!((fluid >> q) & 1u)) continue;
    acc = pair_add(acc, pair_add(xc, pair_neg(xn[q])));
    ++nfl;
  }
  acc = pair_add(acc, pair_mul(xc, (float)(cnt - nfl)));
  return pair_add(b, pair_neg(pair_mul_pair(acc, s_hi, s_lo)));
}

// ------------------------------------------------------------ cell ownership

struct Chunk {
  unsigned int begin, end;  // slots of the active-cell index space
};

__device__ __forceinline__ Chunk my_chunk(unsigned int nact) {
  const unsigned int total = nact * BRICK_CELLS;
  unsigned int per = (total + team_size() - 1) / team_size();
  per = (per + 31u) & ~31u;
  const unsigned int b = min(total, team_rank() * per);
  return Chunk{b, min(total, b + per)};
}

struct CellRef {
  int i, j, k;
  int c;
};

template <class F>
__device__ __forceinline__ void for_my_cells(const PcgArgs& A, const Chunk& ch, F&& f) {
  const Grid& g = A.g;
  for (unsigned int e = ch.begin + threadIdx.x; e < ch.end; e += PCG_THREADS) {
    const unsigned int brick = A.active[e >> 9];
    const int l = (int)(e & 511u);
    const int i = (int)(brick % (unsigned)g.bx) * BRICK + (l & 7);
    const int j = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK + ((l >> 3) & 7);
    const int k = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK + (l >> 6);
    if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
    const int c = i + g.nx * (j + g.ny * k);
    if (A.type[c] != 1) continue;
    f(CellRef{i, j, k, c});
  }
}

// The six neighbours of a cell: index (the cell itself when outside the grid)
// and whether it is a fluid cell.  All loads are issued before any is used.
struct Nbrs {
  int idx[6];
  bool fl[6];
  int cnt[6];
};

__device__ __forceinline__ Nbrs neighbours(const PcgArgs& A, const CellRef& cr) {
  const Grid& g = A.g;
  const int sy = g.nx, sz = g.nx * g.ny;
  Nbrs n;
  const bool in[6] = {cr.i > 0, cr.i < g.nx - 1, cr.j > 0, cr.j < g.ny - 1, cr.k > 0,
                      cr.k < g.nz - 1};
  const int off[6] = {-1, 1, -sy, sy, -sz, sz};
#pragma unroll
  for (int q = 0; q < 6; ++q) n.idx[q] = in[q] ? cr.c + off[q] : cr.c;
  uint8_t t[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) t[q] = A.type[n.idx[q]];
#pragma unroll
  for (int q = 0; q < 6; ++q) n.fl[q] = in[q] && t[q] == 1;
  n.cnt[0] = nonsolid_count(g, cr.i - 1, cr.j, cr.k);
  n.cnt[1] = nonsolid_count(g, cr.i + 1, cr.j, cr.k);
  n.cnt[2] = nonsolid_count(g, cr.i, cr.j - 1, cr.k);
  n.cnt[3] = nonsolid_count(g, cr.i, cr.j + 1, cr.k);
  n.cnt[4] = nonsolid_count(g, cr.i, cr.j, cr.k - 1);
  n.cnt[5] = nonsolid_count(g, cr.i, cr.j, cr.k + 1);
  return n;
}

// p_new of a cell = z + beta p_old with z = r / diag.  One expression, so the
// owner of a cell and its neighbours compute the same bits.
__device__ __forceinline__ float p_update(float r, float pold, float minv, float beta) {
  return __fmaf_rn(beta, pold, __fmul_rn(r, minv));
}

__device__ __forceinline__ void phase_a_cell(const PcgArgs& A, const CellRef& cr,
                                             const float* pold, float* pnew, float beta,
                                             FF& pq) {
  const Nbrs n = neighbours(A, cr);
  const int cnt = nonsolid_count(A.g, cr.i, cr.j, cr.k);
  float rv[6], pv[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    rv[q] = A.r[n.idx[q]];
    pv[q] = pold[n.idx[q]];
  }
  const float pc = p_update(A.r[cr.c], pold[cr.c], A.minv_tab[cnt], beta);
  // (A p)_c in difference form, s * (sum_fluid (p_c - p_n) + n_air p_c): the
  // differences of neighbouring values are nearly exact, where n_c p_c - sum p_n
  // would cancel most of its digits.
  float d = 0.0f;
  int nfl = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float pn = p_update(rv[q], pv[q], A.minv_tab[n.cnt[q]], beta);
    d += n.fl[q] ? __fsub_rn(pc, pn) : 0.0f;
    nfl += n.fl[q];
  }
  const float qc = __fmul_rn(A.s, __fmaf_rn((float)(cnt - nfl), pc, d));
  pnew[cr.c] = pc;
  A.q[cr.c] = qc;
  pq.add_prod(pc, qc);
}

// FP64 residual of one cell for the refinement: b - A x with x in FP64.
__device__ __forceinline__ double residual64(const PcgArgs& A, const CellRef& cr) {
  const Nbrs n = neighbours(A, cr);
  const double xc = A.x64[cr.c];
  double xv[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) xv[q] = A.x64[n.idx[q]];
  double d = 0.0;
  int nfl = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    d += n.fl[q] ? xc - xv[q] : 0.0;
    nfl += n.fl[q];
  }
  const int cnt = nonsolid_count(A.g, cr.i, cr.j, cr.k);
  return A.b64[cr.c] - A.s64 * ((double)(cnt - nfl) * xc + d);
}

// ------------------------------------------------------------ reductions

struct Shared {
  F2 scratch[3 * PCG_WARPS];
  float alpha, beta;
  int flag;
  double dscal[4];
};

template <int K>
__device__ __forceinline__ void publish(const PcgArgs& A, int slot, F2 (&v)[K], Shared& sh) {
  cta_sum<K>(v, sh.scratch);
  if (threadIdx.x == 0) {
    float2* part = reinterpret_cast<float2*>(A.partials);
#pragma unroll
    for (int q = 0; q < K; ++q)
      part[(size_t)(slot + q) * team_size() + team_rank()] = make_float2(v[q].hi, v[q].lo);
  }
}

// After a barrier: the grid-wide sums of the published pairs, in FP64, valid in
// thread 0.  Every CTA adds the same pairs in the same order.
template <int K>
__device__ __forceinline__ void gather(const PcgArgs& A, int slot, double (&out)[K], Shared& sh) {
  const float2* part = reinterpret_cast<const float2*>(A.partials);
  F2 v[K];
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = F2{0.0f, 0.0f};
  if (threadIdx.x < 32) {
    for (unsigned int j = threadIdx.x; j < team_size(); j += 32)
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const float2 p = part[(size_t)(slot + q) * team_size() + j];
        v[q] = f2_add(v[q], F2{p.x, p.y});
      }
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = f2_warp_sum(v[q]);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = (double)v[q].hi + (double)v[q].lo;
  (void)sh;
}

}  // namespace flipk
