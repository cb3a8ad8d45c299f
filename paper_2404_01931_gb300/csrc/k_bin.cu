// k_bin.cu — particle binning (Sec. 3.1.5 "space hash", Sec. 3.2.2: cell index
// -> prefix sum over per-cell counts -> reorder into a double buffer).
//
// A counting sort keyed by the brick-major cell key.  The per-cell histogram is
// built by the atomics of the step that moved the particles (the G2P epilogue,
// or k_rebin after creation / a write), whose return value is the particle's
// rank inside its cell.  Then:
//   k_cell_local_scan  one CTA per 8x8x8 brick: exclusive scan of its 512
//                      counts (local offsets), the brick total, cell types
//                      (fluid = count > 0), and clears the counts for the next
//                      step's atomics
//   k_brick_scan       one CTA: exclusive scan of the brick totals, the list of
//                      active bricks, the fluid-cell count
//   k_scatter          particle p goes to brick_start + local_start + rank
// The paper scans with a work-efficient balanced-tree (Blelloch) scan; here the
// scan is split by the brick structure instead (warp-shuffle scans inside a
// brick, one small scan over bricks), which needs no global tree passes.
#include "flip_kernels.cuh"

namespace flipk {

__global__ void k_rebin(const Grid g, const PartView p, const BinView b, long long np) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int ci = cell_of(p.x[i], g.inv_dx, g.nx);
  const int cj = cell_of(p.y[i], g.inv_dx, g.ny);
  const int ck = cell_of(p.z[i], g.inv_dx, g.nz);
  const unsigned int key = brick_key(g, ci, cj, ck);
  b.key[i] = key;
  b.rank[i] = atomicAdd(b.cell_count + key, 1u);
}

__global__ void __launch_bounds__(BRICK_CELLS) k_cell_local_scan(const Grid g, const BinView b,
                                                                   uint8_t* __restrict__ type) {
  __shared__ unsigned int warp_tot[BRICK_CELLS / 32];
  const unsigned int brick = blockIdx.x;
  const int l = threadIdx.x, lane = l & 31, warp = l >> 5;
  const unsigned int key = brick * BRICK_CELLS + (unsigned)l;
  const unsigned int cnt = b.cell_count[key];
  b.cell_count[key] = 0u;
  unsigned int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  unsigned int woff = 0;
#pragma unroll
  for (int w = 0; w < BRICK_CELLS / 32; ++w) woff += (w < warp) ? warp_tot[w] : 0u;
  const unsigned int excl = woff + incl - cnt;
  b.local_start[key] = excl;
  if (l == BRICK_CELLS - 1) b.brick_count[brick] = excl + cnt;
  const int i = (int)(brick % (unsigned)g.bx) * BRICK + (l & 7);
  const int j = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK + ((l >> 3) & 7);
  const int k = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK + (l >> 6);
  const bool inside = (i < g.nx && j < g.ny && k < g.nz);
  if (inside) type[i + g.nx * (j + g.ny * k)] = (cnt > 0u) ? 1 : 0;
  const int nfl = __syncthreads_count(inside && cnt > 0u);
  if (l == 0) b.brick_fluid[brick] = (unsigned)nfl;
}

// One CTA of 1024 threads walks all bricks in chunks: exclusive scan of the
// brick totals (particle offsets), compaction of the bricks holding particles.
__global__ void __launch_bounds__(1024) k_brick_scan(const Grid g, const BinView b, DevStats* st) {
  __shared__ unsigned int wc[32], wf[32];
  __shared__ unsigned int fl_tot;
  const unsigned int nb = (unsigned)g.bx * g.by * g.bz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) fl_tot = 0;
  unsigned int run = 0, run_act = 0, fluid = 0;
  for (unsigned int base = 0; base < nb; base += blockDim.x) {
    const unsigned int idx = base + threadIdx.x;
    const unsigned int c = idx < nb ? b.brick_count[idx] : 0u;
    const unsigned int flag = c > 0u;
    fluid += idx < nb ? b.brick_fluid[idx] : 0u;
    unsigned int ic = c, iff = flag;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t1 = __shfl_up_sync(0xffffffffu, ic, o);
      const unsigned int t2 = __shfl_up_sync(0xffffffffu, iff, o);
      if (lane >= o) { ic += t1; iff += t2; }
    }
    if (lane == 31) { wc[warp] = ic; wf[warp] = iff; }
    __syncthreads();
    unsigned int oc = 0, of = 0, tc = 0, tf = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) { oc += wc[w]; of += wf[w]; }
      tc += wc[w];
      tf += wf[w];
    }
    if (idx < nb) b.brick_start[idx] = run + oc + ic - c;
    if (flag) b.active[run_act + of + iff - 1] = idx;
    run += tc;
    run_act += tf;
    __syncthreads();
  }
  atomicAdd(&fl_tot, fluid);
  __syncthreads();
  if (threadIdx.x == 0) {
    b.brick_start[nb] = run;
    st->n_active = run_act;
    st->n_fluid = fl_tot;
  }
}

__global__ void k_scatter(const PartView src, const PartView dst, const BinView b, long long np) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const unsigned int key = b.key[i];
  const unsigned int d = b.brick_start[key / BRICK_CELLS] + b.local_start[key] + b.rank[i];
  dst.x[d] = src.x[i];
  dst.y[d] = src.y[i];
  dst.z[d] = src.z[i];
  dst.u[d] = src.u[i];
  dst.v[d] = src.v[i];
  dst.w[d] = src.w[i];
  dst.id[d] = src.id[i];
}

__global__ void k_iota(int* id, long long np) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < np) id[i] = (int)i;
}

static unsigned int blocks_for(long long n, int t) {
  long long b = (n + t - 1) / t;
  return (unsigned int)(b < 1 ? 1 : b);
}

void launch_rebin(const Grid& g, const PartView& p, const BinView& b, long long np,
                  cudaStream_t s) {
  if (np > 0) k_rebin<<<blocks_for(np, 256), 256, 0, s>>>(g, p, b, np);
}

void launch_bin(const Grid& g, const BinView& b, uint8_t* type, DevStats* st, cudaStream_t s) {
  const unsigned int nb = (unsigned)g.bx * g.by * g.bz;
  k_cell_local_scan<<<nb, BRICK_CELLS, 0, s>>>(g, b, type);
  k_brick_scan<<<1, 1024, 0, s>>>(g, b, st);
}

void launch_scatter(const PartView& src, const PartView& dst, const BinView& b, long long np,
                    cudaStream_t s) {
  if (np > 0) k_scatter<<<blocks_for(np, 256), 256, 0, s>>>(src, dst, b, np);
}

void launch_iota(int* id, long long np, cudaStream_t s) {
  if (np > 0) k_iota<<<blocks_for(np, 256), 256, 0, s>>>(id, np);
}

}  // namespace flipk
