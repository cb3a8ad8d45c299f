// k_pcg.cu — matrix-free Jacobi-preconditioned conjugate gradient on A p = b
// (Sec. 3.1.7: 7-point Laplacian over fluid cells, p = 0 in air, walls
// dropped), as one persistent cooperative kernel per solve.
//
// All CTAs stay resident for the whole solve and meet at bounded grid barriers
// (two per iteration).  Work is the list of active 8x8x8 bricks, assigned to
// CTAs round-robin and kept by the same CTA in every phase, so a thread always
// owns the same cells.  Per iteration:
//   phase A  p_new = z + beta p_old, q = A p_new, partial p.q
//            (the p update of the previous iteration is folded into the stencil:
//             each neighbour's p_new is recomputed from its r and p_old, so p
//             needs no barrier of its own; p is double-buffered)
//   phase B  x += alpha p, r -= alpha q, z = r / diag, partials r.r and r.z
// Reductions are deterministic: per-thread float-pair accumulation, then FP64
// warp/block sums, one partial per CTA, and every CTA adds the partials in the
// same order after the barrier, so all CTAs take identical decisions.
//
// Mixed mode (FLIP_PREC_MIXED_IR) wraps the FP32 solve in iterative
// refinement: r = b - A x in FP64 with x in FP64, the FP32 PCG solves A d = r,
// x += d, until ||b - A x|| <= ir_tol ||b||.
#include "flip_kernels.cuh"

namespace flipk {

constexpr int PCG_THREADS = 256;

struct CellRef {
  int i, j, k;
  int c;
};

template <class F>
__device__ __forceinline__ void for_fluid_cells(const PcgArgs& A, unsigned int nact, F&& f) {
  const Grid& g = A.g;
  for (unsigned int bi = blockIdx.x; bi < nact; bi += gridDim.x) {
    const unsigned int brick = A.active[bi];
    const int b0 = (int)(brick % (unsigned)g.bx) * BRICK;
    const int b1 = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK;
    const int b2 = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK;
    for (int l = threadIdx.x; l < BRICK_CELLS; l += PCG_THREADS) {
      const int i = b0 + (l & 7), j = b1 + ((l >> 3) & 7), k = b2 + (l >> 6);
      if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
      const int c = i + g.nx * (j + g.ny * k);
      if (A.type[c] != 1) continue;
      f(CellRef{i, j, k, c});
    }
  }
}

__device__ __forceinline__ bool is_fluid(const PcgArgs& A, int c) { return A.type[c] == 1; }

// p_new of cell n = z_n + beta p_old_n with z_n = r_n / diag_n.  Written once
// here so that the owner of a cell and its neighbours compute the same bits.
__device__ __forceinline__ float p_update(const PcgArgs& A, const float* pold, int n, int cnt,
                                          float beta) {
  return __fmaf_rn(beta, __ldcg(pold + n), __fmul_rn(__ldcg(A.r + n), A.minv_tab[cnt]));
}

// Phase A for one fluid cell: returns p_new(c) and writes q(c).
__device__ __forceinline__ void phase_a_cell(const PcgArgs& A, const CellRef& cr,
                                             const float* pold, float* pnew, float beta,
                                             FF& pq) {
  const Grid& g = A.g;
  const int i = cr.i, j = cr.j, k = cr.k, c = cr.c;
  const int sx = 1, sy = g.nx, sz = g.nx * g.ny;
  const int cnt = nonsolid_count(g, i, j, k);
  const float pc = p_update(A, pold, c, cnt, beta);
  float nb = 0.0f;
  if (i > 0 && is_fluid(A, c - sx)) nb += p_update(A, pold, c - sx, nonsolid_count(g, i - 1, j, k), beta);
  if (i < g.nx - 1 && is_fluid(A, c + sx)) nb += p_update(A, pold, c + sx, nonsolid_count(g, i + 1, j, k), beta);
  if (j > 0 && is_fluid(A, c - sy)) nb += p_update(A, pold, c - sy, nonsolid_count(g, i, j - 1, k), beta);
  if (j < g.ny - 1 && is_fluid(A, c + sy)) nb += p_update(A, pold, c + sy, nonsolid_count(g, i, j + 1, k), beta);
  if (k > 0 && is_fluid(A, c - sz)) nb += p_update(A, pold, c - sz, nonsolid_count(g, i, j, k - 1), beta);
  if (k < g.nz - 1 && is_fluid(A, c + sz)) nb += p_update(A, pold, c + sz, nonsolid_count(g, i, j, k + 1), beta);
  const float qc = __fmaf_rn(A.diag_tab[cnt], pc, -__fmul_rn(A.s, nb));
  pnew[c] = pc;
  A.q[c] = qc;
  pq.add_prod(pc, qc);
}

template <int K>
__device__ __forceinline__ void publish_partials(const PcgArgs& A, int slot, double (&v)[K],
                                                 double* scratch) {
  block_sum<K>(v, scratch);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) A.partials[(size_t)(slot + q) * gridDim.x + blockIdx.x] = v[q];
}

template <int K>
__device__ __forceinline__ void gather_partials(const PcgArgs& A, int slot, double (&out)[K],
                                                double* scratch) {
  double v[K];
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = 0.0;
  for (unsigned int j = threadIdx.x; j < gridDim.x; j += PCG_THREADS)
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] += __ldcg(A.partials + (size_t)(slot + q) * gridDim.x + j);
  block_sum<K>(v, scratch);
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = v[q];
}

// FP32 PCG on A x32 = r (r, x32 = 0 and p_old = 0 already set on fluid cells;
// rz0 = r.z, rnorm0 = ||r||).  Returns false if a barrier failed.
__device__ bool pcg_fp32(const PcgArgs& A, unsigned int nact, double rz0, double rnorm0,
                         double tol, int max_iter, int* iters_out, bool* conv_out,
                         double* rel_out, double* scratch) {
  double rz = rz0;
  float beta = 0.0f;
  float* pold = A.pa;
  float* pnew = A.pb;
  int it = 0;
  bool conv = (rnorm0 == 0.0);
  double rnorm = rnorm0;
  while (!conv && it < max_iter) {
    ++it;
    FF pq;
    for_fluid_cells(A, nact, [&](const CellRef& cr) { phase_a_cell(A, cr, pold, pnew, beta, pq); });
    double va[1] = {pq.value()};
    publish_partials<1>(A, 0, va, scratch);
    if (!grid_barrier(A.bar, A.status, gridDim.x, A.timeout_ns)) return false;
    double pqs[1];
    gather_partials<1>(A, 0, pqs, scratch);
    const float alpha = (float)(rz / pqs[0]);
    FF rr, rzn;
    for_fluid_cells(A, nact, [&](const CellRef& cr) {
      const int c = cr.c;
      const int cnt = nonsolid_count(A.g, cr.i, cr.j, cr.k);
      A.x32[c] = __fmaf_rn(alpha, pnew[c], A.x32[c]);
      const float rc = __fmaf_rn(-alpha, A.q[c], A.r[c]);
      A.r[c] = rc;
      const float zc = __fmul_rn(rc, A.minv_tab[cnt]);
      rr.add_prod(rc, rc);
      rzn.add_prod(rc, zc);
    });
    double vb[2] = {rr.value(), rzn.value()};
    publish_partials<2>(A, 1, vb, scratch);
    if (!grid_barrier(A.bar, A.status, gridDim.x, A.timeout_ns)) return false;
    double sb[2];
    gather_partials<2>(A, 1, sb, scratch);
    rnorm = sqrt(fmax(sb[0], 0.0));
    if (rnorm <= tol * rnorm0) { conv = true; break; }
    beta = (float)(sb[1] / rz);
    rz = sb[1];
    float* t = pold; pold = pnew; pnew = t;
  }
  *iters_out = it;
  *conv_out = conv;
  *rel_out = rnorm0 > 0.0 ? rnorm / rnorm0 : 0.0;
  return true;
}

template <bool MIXED>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg(const __grid_constant__ PcgArgs A) {
  __shared__ double scratch[32 * 3];
  const unsigned int nact = *A.n_active;
  const long long ncells = (long long)A.g.nx * A.g.ny * A.g.nz;
  bool singular = false;
  if (A.check_singular) singular = ((long long)A.stats->n_fluid == ncells);
  int iters = 0, outer = 0;
  bool conv = false;
  double rel = 0.0, bnorm = 0.0;
  bool ok = true;

  if (!singular) {
    if constexpr (!MIXED) {
      // Phase I: r = b, x = 0, p_old = 0; ||b||^2 and r.z.
      FF bb, rz;
      for_fluid_cells(A, nact, [&](const CellRef& cr) {
        const float bc = A.b32[cr.c];
        A.r[cr.c] = bc;
        A.x32[cr.c] = 0.0f;
        A.pa[cr.c] = 0.0f;
        bb.add_prod(bc, bc);
        rz.add_prod(bc, __fmul_rn(bc, A.minv_tab[nonsolid_count(A.g, cr.i, cr.j, cr.k)]));
      });
      double v[2] = {bb.value(), rz.value()};
      publish_partials<2>(A, 1, v, scratch);
      ok = grid_barrier(A.bar, A.status, gridDim.x, A.timeout_ns);
      if (ok) {
        double s[2];
        gather_partials<2>(A, 1, s, scratch);
        bnorm = sqrt(fmax(s[0], 0.0));
        ok = pcg_fp32(A, nact, s[1], bnorm, A.tol, A.max_iter, &iters, &conv, &rel, scratch);
      }
    } else {
      // ||b||^2 in FP64 (once per solve).
      double bb = 0.0;
      for_fluid_cells(A, nact, [&](const CellRef& cr) {
        const double bc = A.b64[cr.c];
        bb = fma(bc, bc, bb);
      });
      double v0[1] = {bb};
      publish_partials<1>(A, 3, v0, scratch);
      ok = grid_barrier(A.bar, A.status, gridDim.x, A.timeout_ns);
      if (ok) {
        double s0[1];
        gather_partials<1>(A, 3, s0, scratch);
        bnorm = sqrt(fmax(s0[0], 0.0));
      }
      bool outer_conv = (bnorm == 0.0);
      while (ok && !outer_conv) {
        // Phase R: r = b - A x in FP64; inner start d = 0, p_old = 0.
        double rr64 = 0.0;
        FF rr32, rz32;
        const Grid& g = A.g;
        const int sy = g.nx, sz = g.nx * g.ny;
        for_fluid_cells(A, nact, [&](const CellRef& cr) {
          const int c = cr.c, i = cr.i, j = cr.j, k = cr.k;
          double nb = 0.0;
          if (i > 0 && is_fluid(A, c - 1)) nb += __ldcg(A.x64 + c - 1);
          if (i < g.nx - 1 && is_fluid(A, c + 1)) nb += __ldcg(A.x64 + c + 1);
          if (j > 0 && is_fluid(A, c - sy)) nb += __ldcg(A.x64 + c - sy);
          if (j < g.ny - 1 && is_fluid(A, c + sy)) nb += __ldcg(A.x64 + c + sy);
          if (k > 0 && is_fluid(A, c - sz)) nb += __ldcg(A.x64 + c - sz);
          if (k < g.nz - 1 && is_fluid(A, c + sz)) nb += __ldcg(A.x64 + c + sz);
          const int cnt = nonsolid_count(g, i, j, k);
          const double ax = A.s64 * ((double)cnt * __ldcg(A.x64 + c) - nb);
          const double rc = A.b64[c] - ax;
          rr64 = fma(rc, rc, rr64);
          const float r32 = (float)rc;
          A.r[c] = r32;
          A.x32[c] = 0.0f;
          A.pa[c] = 0.0f;
          rr32.add_prod(r32, r32);
          rz32.add_prod(r32, __fmul_rn(r32, A.minv_tab[cnt]));
        });
        double v[3] = {rr64, rr32.value(), rz32.value()};
        // Slots 4..6 are phase R's own: their previous readers finished before
        // the first barrier of the inner solve that followed.
        publish_partials<3>(A, 4, v, scratch);
        if (!(ok = grid_barrier(A.bar, A.status, gridDim.x, A.timeout_ns))) break;
        double s[3];
        gather_partials<3>(A, 4, s, scratch);
        rel = sqrt(fmax(s[0], 0.0)) / bnorm;
        if (rel <= A.ir_tol) { outer_conv = true; break; }
        if (outer >= A.ir_max_iter) break;
        ++outer;
        int it_in = 0;
        bool c_in = false;
        double rel_in = 0.0;
        ok = pcg_fp32(A, nact, s[2], sqrt(fmax(s[1], 0.0)), A.tol, A.max_iter, &it_in, &c_in,
                      &rel_in, scratch);
        iters += it_in;
        if (!ok) break;
        // Phase U: x += d.
        for_fluid_cells(A, nact, [&](const CellRef& cr) {
          A.x64[cr.c] += (double)A.x32[cr.c];
        });
        if (!(ok = grid_barrier(A.bar, A.status, gridDim.x, A.timeout_ns))) break;
      }
      conv = outer_conv;
      // Phase F: the solution as a float pair for the G2P gradient.
      for_fluid_cells(A, nact, [&](const CellRef& cr) {
        const double xv = A.x64[cr.c];
        const float hi = __double2float_rn(xv);
        const float lo = __double2float_rn(xv - (double)hi);
        A.pff[cr.c] = make_float2(hi, lo);
      });
    }
  }

  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int st = 0;
    if (singular) st |= DEV_SINGULAR;
    else if (ok && !conv) st |= DEV_NOT_CONVERGED;
    if (st) atomicOr(A.status, st);
    A.stats->cg_iters = iters;
    A.stats->ir_iters = outer;
    A.stats->cg_iters_total += iters;
    A.stats->ir_iters_total += outer;
    A.stats->rel_res = rel;
    A.stats->bnorm = bnorm;
  }
}

int pcg_block_size() { return PCG_THREADS; }

cudaError_t pcg_max_blocks(int* max_blocks, int* sm_count) {
  int dev = 0, sms = 0, per_sm_a = 0, per_sm_b = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, k_pcg<false>, PCG_THREADS, 0);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_pcg<true>, PCG_THREADS, 0);
  if (e != cudaSuccess) return e;
  int per_sm = per_sm_a < per_sm_b ? per_sm_a : per_sm_b;
  if (per_sm > 4) per_sm = 4;  // fewer partials per reduction; 1024 threads per SM
  *max_blocks = per_sm * sms;
  *sm_count = sms;
  return cudaSuccess;
}

cudaError_t launch_pcg(const PcgArgs& a, bool mixed, int nblocks, cudaStream_t s) {
  void* args[] = {const_cast<PcgArgs*>(&a)};
  if (mixed)
    return cudaLaunchCooperativeKernel((const void*)k_pcg<true>, dim3(nblocks), dim3(PCG_THREADS),
                                       args, 0, s);
  return cudaLaunchCooperativeKernel((const void*)k_pcg<false>, dim3(nblocks), dim3(PCG_THREADS),
                                     args, 0, s);
}

// ---- helpers of the standalone solve: active bricks straight from cell types

__global__ void k_mark_bricks(const Grid g, const uint8_t* __restrict__ type,
                              unsigned int* __restrict__ brick_fluid) {
  const unsigned int brick = blockIdx.x;
  const int b0 = (int)(brick % (unsigned)g.bx) * BRICK;
  const int b1 = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK;
  const int b2 = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK;
  const int l = threadIdx.x;
  const int i = b0 + (l & 7), j = b1 + ((l >> 3) & 7), k = b2 + (l >> 6);
  int f = 0;
  if (i < g.nx && j < g.ny && k < g.nz) f = (type[i + g.nx * (j + g.ny * k)] == 1);
  const int tot = __syncthreads_count(f);
  if (l == 0) brick_fluid[brick] = (unsigned)tot;
}

__global__ void k_compact_bricks(const Grid g, const unsigned int* __restrict__ brick_fluid,
                                 unsigned int* __restrict__ active, DevStats* st) {
  __shared__ unsigned int warp_tot[32];
  __shared__ unsigned int fl_tot;
  const unsigned int nb = (unsigned)g.bx * g.by * g.bz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) fl_tot = 0;
  unsigned int run = 0, fluid = 0;
  for (unsigned int base = 0; base < nb; base += blockDim.x) {
    const unsigned int idx = base + threadIdx.x;
    const unsigned int f = idx < nb ? brick_fluid[idx] : 0u;
    const unsigned int flag = f > 0;
    unsigned int incl = flag;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    fluid += f;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned int woff = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) woff += warp_tot[w];
      tot += warp_tot[w];
    }
    if (flag) active[run + woff + incl - 1] = idx;
    run += tot;
    __syncthreads();  // warp_tot is rewritten in the next round
  }
  atomicAdd(&fl_tot, fluid);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->n_active = run;
    st->n_fluid = fl_tot;
  }
}

__global__ void k_zero_off_fluid(const Grid g, const uint8_t* __restrict__ type,
                                 float* __restrict__ p, unsigned int* bar) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    p[c] = 0.0f;
  if (blockIdx.x == 0 && threadIdx.x == 0) bar[0] = 0u;
  (void)type;
}

void launch_mark_bricks(const Grid& g, const uint8_t* type, unsigned int* brick_fluid,
                        cudaStream_t s) {
  const unsigned int nb = (unsigned)g.bx * g.by * g.bz;
  k_mark_bricks<<<nb, BRICK_CELLS, 0, s>>>(g, type, brick_fluid);
}

void launch_compact_bricks(const Grid& g, const unsigned int* brick_fluid, unsigned int* active,
                           DevStats* st, cudaStream_t s) {
  k_compact_bricks<<<1, 1024, 0, s>>>(g, brick_fluid, active, st);
}

void launch_zero_off_fluid(const Grid& g, const uint8_t* type, float* p, unsigned int* bar,
                           cudaStream_t s) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_zero_off_fluid<<<(unsigned)blocks, 256, 0, s>>>(g, type, p, bar);
}

}  // namespace flipk
