// k_pcg.cu — matrix-free Jacobi-preconditioned conjugate gradient on A p = b
// (Sec. 3.1.7: 7-point Laplacian over fluid cells, p = 0 in air, walls
// dropped), as one persistent cooperative kernel per solve.
//
// One CTA of 1024 threads per SM stays resident for the whole solve; CTAs meet
// at bounded grid barriers (two per iteration).  The cells of the active bricks
// form one index space (brick slot * 512 + local cell) that is cut into equal
// contiguous chunks, one per CTA, so every thread owns the same cells in every
// phase.  Per iteration:
//   phase A  p_new = z + beta p_old, q = A p_new, partial p.q
//            (the p update of the previous iteration is folded into the stencil:
//             each neighbour's p_new is recomputed from its r and p_old, so p
//             needs no barrier of its own; p is double-buffered)
//   phase B  x += alpha p, r -= alpha q, z = r / diag, partials r.r and r.z
// Reductions run on the FP32 pipes: each thread, then each warp and the CTA,
// sums exact float pairs (FMA-split products, TwoSum additions); CTAs publish one
// pair each, and after the barrier every CTA adds the published pairs in the
// same order, so all CTAs take identical decisions.  Only thread 0 turns the
// sums into the FP64 scalars alpha, beta and the stopping test.
//
// Mixed mode (FLIP_PREC_MIXED_IR): the same FP32 iteration works on a
// correction d; whenever the recursive residual has dropped by the factor
// delta = cg_tol since the last refinement (or reaches the target), the correction is
// folded into the FP64 solution (x += d, d = 0) and the residual is replaced by
// the true one, r = b - A x, evaluated in FP64 — iterative refinement without
// restarting the Krylov direction.  The solve stops when the FP64 residual
// satisfies ||b - A x|| <= ir_tol ||b||.
#include "pcg_common.cuh"

namespace flipk {

// ------------------------------------------------------------ the solve

struct SolveState {
  int iters = 0;
  int refinements = 0;
  bool conv = false;
  bool ok = true;
  double rel = 0.0;
  double bnorm = 0.0;
};

// Partial-sum slots (float pairs): 0 = p.q; 1,2 = r.r, r.z (phase B and the FP32
// start); 3,4 = ||b||^2 and r.z of the mixed start; 5,6 = FP64 residual norm and
// r.z after a refinement.  A slot's readers always pass one more barrier before
// the slot is written again.
template <bool MIXED>
__device__ void solve(const PcgArgs& A, const Chunk& ch, Shared& sh, SolveState& S) {
  float* x = A.x32;
  // ---- start: r = b (or float(b)), x = 0, p_old = 0; ||b||, r.z
  {
    FF bb, rz;
    for_my_cells(A, ch, [&](const CellRef& cr) {
      const float bc = MIXED ? (float)A.b64[cr.c] : A.b32[cr.c];
      A.r[cr.c] = bc;
      x[cr.c] = 0.0f;
      A.pa[cr.c] = 0.0f;
      bb.add_prod(bc, bc);
      rz.add_prod(bc, __fmul_rn(bc, A.minv_tab[nonsolid_count(A.g, cr.i, cr.j, cr.k)]));
    });
    F2 v[2] = {f2_of(bb), f2_of(rz)};
    publish<2>(A, 1, v, sh);
  }
  if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
  double s0[2];
  gather<2>(A, 1, s0, sh);
  // thread 0 owns the scalars
  double rz = s0[1];
  double bnorm = sqrt(fmax(s0[0], 0.0));
  double rnorm = bnorm, rmax = bnorm;
  const double target = MIXED ? A.ir_tol : A.tol;
  if (threadIdx.x == 0) {
    sh.flag = (bnorm == 0.0) ? 1 : 0;
    sh.beta = 0.0f;
  }
  __syncthreads();
  S.bnorm = bnorm;
  bool conv = sh.flag != 0;
  int it = 0, refinements = 0;
  float* pold = A.pa;
  float* pnew = A.pb;
  while (!conv && it < A.max_iter) {
    ++it;
    const float beta = sh.beta;
    // ---- phase A
    FF pq;
    for_my_cells(A, ch, [&](const CellRef& cr) { phase_a_cell(A, cr, pold, pnew, beta, pq); });
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
    // ---- phase B
    FF rr, rzn;
    for_my_cells(A, ch, [&](const CellRef& cr) {
      const int c = cr.c;
      x[c] = __fmaf_rn(alpha, pnew[c], x[c]);
      const float rc = __fmaf_rn(-alpha, A.q[c], A.r[c]);
      A.r[c] = rc;
      rr.add_prod(rc, rc);
      rzn.add_prod(rc, __fmul_rn(rc, A.minv_tab[nonsolid_count(A.g, cr.i, cr.j, cr.k)]));
    });
    {
      F2 v[2] = {f2_of(rr), f2_of(rzn)};
      publish<2>(A, 1, v, sh);
    }
    if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
    {
      double s[2];
      gather<2>(A, 1, s, sh);
      if (threadIdx.x == 0) {
        rnorm = sqrt(fmax(s[0], 0.0));
        int f = 0;  // 0 continue, 1 converged, 2 refine
        if (rnorm <= target * bnorm) f = MIXED ? 2 : 1;
        else if (MIXED && rnorm <= A.tol * rmax) f = 2;
        if (f == 0) {
          sh.beta = (float)(s[1] / rz);
          rz = s[1];
        }
        sh.flag = f;
      }
    }
    __syncthreads();
    int f = sh.flag;
    if constexpr (MIXED) {
      if (f == 2) {
        // ---- refinement: x64 += d, d = 0; then r = b - A x64 in FP64
        for_my_cells(A, ch, [&](const CellRef& cr) {
          A.x64[cr.c] += (double)x[cr.c];
          x[cr.c] = 0.0f;
        });
        if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
        FF rr64, rz2;  // the norm of the FP64 residual is accumulated from its float value
        double rr_exact = 0.0;
        for_my_cells(A, ch, [&](const CellRef& cr) {
          const double rc = residual64(A, cr);
          const float r32 = (float)rc;
          A.r[cr.c] = r32;
          rr64.add_prod(r32, r32);
          rz2.add_prod(r32, __fmul_rn(r32, A.minv_tab[nonsolid_count(A.g, cr.i, cr.j, cr.k)]));
        });
        (void)rr_exact;
        F2 v[2] = {f2_of(rr64), f2_of(rz2)};
        publish<2>(A, 5, v, sh);
        if (!grid_barrier(A.bar, A.status, team_size(), A.timeout_ns)) { S.ok = false; return; }
        double s[2];
        gather<2>(A, 5, s, sh);
        ++refinements;
        if (threadIdx.x == 0) {
          rnorm = sqrt(fmax(s[0], 0.0));
          rmax = rnorm;
          if (rnorm <= target * bnorm) {
            sh.flag = 1;
          } else if (refinements >= A.ir_max_iter) {
            sh.flag = 3;  // refinement cap: stop with the current solution
          } else {
            sh.flag = 0;
            sh.beta = (float)(s[1] / rz);
            rz = s[1];
          }
        }
        __syncthreads();
        f = sh.flag;
      }
    }
    if (f == 1) { conv = true; break; }
    if (f == 3) break;
    float* t = pold; pold = pnew; pnew = t;
  }
  if constexpr (MIXED) {
    if (!conv) {  // cap reached: keep the last iterate
      for_my_cells(A, ch, [&](const CellRef& cr) {
        A.x64[cr.c] += (double)x[cr.c];
        x[cr.c] = 0.0f;
      });
    }
    // the solution as a float pair for the G2P pressure gradient
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
}

template <bool MIXED>
__device__ void solve_scene(const PcgArgs& A, Shared& sh) {
  const unsigned int nact = *A.n_active;
  const long long ncells = (long long)A.g.nx * A.g.ny * A.g.nz;
  const bool singular = A.check_singular && ((long long)A.stats->n_fluid == ncells);
  SolveState S;
  if (!singular) solve<MIXED>(A, my_chunk(nact), sh, S);
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
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg(const __grid_constant__ PcgArgs A) {
  __shared__ Shared sh;
  team_enter(blockIdx.x, gridDim.x);
  solve_scene<MIXED>(A, sh);
}

// Several scenes in one launch (see k_pcg_mg_batch).
template <bool MIXED>
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg_batch(const __grid_constant__ PcgBatch B) {
  __shared__ Shared sh;
  const int s = B.block_scene[blockIdx.x];
  team_enter(blockIdx.x - B.team_first[s], B.team_first[s + 1] - B.team_first[s]);
  solve_scene<MIXED>(B.args[s], sh);
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
  const int per_sm = per_sm_a < per_sm_b ? per_sm_a : per_sm_b;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *max_blocks = sms;  // one CTA per SM
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

cudaError_t launch_pcg_batch(const PcgBatch& b, bool mixed, int nblocks, cudaStream_t s) {
  void* args[] = {const_cast<PcgBatch*>(&b)};
  if (mixed)
    return cudaLaunchCooperativeKernel((const void*)k_pcg_batch<true>, dim3(nblocks),
                                       dim3(PCG_THREADS), args, 0, s);
  return cudaLaunchCooperativeKernel((const void*)k_pcg_batch<false>, dim3(nblocks),
                                     dim3(PCG_THREADS), args, 0, s);
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
  if (blockIdx.x == 0 && threadIdx.x < BAR_WORDS) bar[threadIdx.x] = 0u;
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
