// k_bin.cu — particle binning (Sec. 3.1.5 "space hash", Sec. 3.2.2: cell index
// -> prefix sum over per-cell counts -> reorder into a double buffer).
//
// A counting sort keyed by the brick-major cell key.  The per-cell histogram is
// built by the atomics of the step that moved the particles (the G2P epilogue,
// or k_rebin after creation / a write), whose return value is the particle's
// rank inside its cell.  Then:
//   k_cell_local_scan  one warp per 8x8x8 brick: exclusive scan of its 512
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

__global__ void k_rebin(const Grid g, const PartView p, const BinView b, long long np,
                        unsigned int* __restrict__ st_speed) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float s2 = 0.0f;
  if (i < np) {
    const int ci = cell_of(p.x[i], g.inv_dx, g.nx);
    const int cj = cell_of(p.y[i], g.inv_dx, g.ny);
    const int ck = cell_of(p.z[i], g.inv_dx, g.nz);
    const unsigned int key = brick_key(g, ci, cj, ck);
    b.key[i] = key;
    b.rank[i] = atomicAdd(b.cell_count + key, 1u);
    const float u = p.u[i], v = p.v[i], w = p.w[i];
    s2 = u * u + v * v + w * w;
  }
  // the particles' largest speed: the first adaptive time step's input
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 = fmaxf(s2, __shfl_xor_sync(0xffffffffu, s2, o));
  if ((threadIdx.x & 31) == 0 && s2 > 0.0f) atomicMax(st_speed, __float_as_uint(sqrtf(s2)));
}

// One warp per brick: lane l owns the 16 consecutive keys 16l .. 16l+15 (two
// x-rows of the brick), read and written as four 16-byte vectors.
constexpr int SCAN_THREADS = 256;

// cmax: particles a cell keeps (reseeding's upper bound; ~0u when off); the
// excess is counted into st->removed_total and dropped by the scatter.
// Body of one CTA (block `blk` of the scene's launch).
__device__ __forceinline__ void cell_local_scan(const Grid& g, const BinView& b,
                                                uint8_t* __restrict__ type, unsigned int nb,
                                                unsigned int cmax, DevStats* st,
                                                unsigned int blk) {
  const int lane = threadIdx.x & 31;
  const unsigned int brick = blk * (SCAN_THREADS / 32) + (threadIdx.x >> 5);
  if (brick >= nb) return;
  const unsigned int key0 = brick * BRICK_CELLS + 16u * (unsigned)lane;
  uint4* cnt4 = reinterpret_cast<uint4*>(b.cell_count + key0);
  uint4* st4 = reinterpret_cast<uint4*>(b.local_start + key0);
  unsigned int c[16];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const uint4 t = cnt4[v];
    c[4 * v] = t.x;
    c[4 * v + 1] = t.y;
    c[4 * v + 2] = t.z;
    c[4 * v + 3] = t.w;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) cnt4[v] = make_uint4(0u, 0u, 0u, 0u);
  if (cmax != ~0u) {
    unsigned int drop = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const unsigned int keep = min(c[q], cmax);
      drop += c[q] - keep;
      c[q] = keep;
    }
    drop = __reduce_add_sync(0xffffffffu, drop);
    if (lane == 0 && drop) atomicAdd((unsigned long long*)&st->removed_total, (unsigned long long)drop);
  }
  unsigned int tot = 0;
#pragma unroll
  for (int q = 0; q < 16; ++q) tot += c[q];
  unsigned int incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  unsigned int run = incl - tot;
  unsigned int ex[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    ex[q] = run;
    run += c[q];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) st4[v] = make_uint4(ex[4 * v], ex[4 * v + 1], ex[4 * v + 2], ex[4 * v + 3]);
  if (lane == 31) b.brick_count[brick] = incl;
  // cell types of the two rows (fluid = count > 0) and the brick's fluid count
  const int i0 = (int)(brick % (unsigned)g.bx) * BRICK;
  const int j0 = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK;
  const int k0 = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK;
  const int k = k0 + (lane >> 2);
  int nfl = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = j0 + ((2 * lane + h) & 7);
    if (j >= g.ny || k >= g.nz) continue;
    uint8_t* row = type + (size_t)g.nx * (j + (size_t)g.ny * k);
    if (i0 + BRICK <= g.nx && (reinterpret_cast<uintptr_t>(row + i0) & 7u) == 0) {
      // the row's eight types in one 8-byte store (byte x = cell i0 + x)
      unsigned long long word = 0ull;
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        const bool f = c[8 * h + x] > 0u;
        word |= (unsigned long long)f << (8 * x);
        nfl += f;
      }
      *reinterpret_cast<unsigned long long*>(row + i0) = word;
      continue;
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const int i = i0 + x;
      if (i >= g.nx) continue;
      const bool f = c[8 * h + x] > 0u;
      row[i] = f ? 1 : 0;
      nfl += f;
    }
  }
  nfl = __reduce_add_sync(0xffffffffu, (unsigned)nfl);
  if (lane == 0) b.brick_fluid[brick] = (unsigned)nfl;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_cell_local_scan(const Grid g, const BinView b,
                                                                    uint8_t* __restrict__ type,
                                                                    unsigned int nb,
                                                                    unsigned int cmax,
                                                                    DevStats* st) {
  cell_local_scan(g, b, type, nb, cmax, st, blockIdx.x);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_cell_local_scan_batch(const BatchLaunch L) {
  const int s = batch_scene(L, blockIdx.x);
  const SceneDev& S = L.scenes[s];
  cell_local_scan(S.g, S.B, S.type, S.nbricks, ~0u, S.st, blockIdx.x - L.first[s]);
}

// One CTA of 1024 threads walks all bricks in chunks of 8 per thread: exclusive
// scan of the brick totals (particle offsets), compaction of the bricks holding
// particles.  A thread scans its 8 consecutive bricks serially, the CTA scans the
// thread totals.
constexpr int BSCAN_PER = 8;
__device__ __forceinline__ void brick_scan(const Grid& g, const BinView& b, DevStats* st) {
  __shared__ unsigned int wc[32], wf[32];
  __shared__ unsigned int fl_tot;
  const unsigned int nb = (unsigned)g.bx * g.by * g.bz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) fl_tot = 0;
  unsigned int run = 0, run_act = 0, fluid = 0;
  const unsigned int chunk = blockDim.x * BSCAN_PER;
  for (unsigned int base = 0; base < nb; base += chunk) {
    const unsigned int i0 = base + threadIdx.x * BSCAN_PER;
    unsigned int c[BSCAN_PER];
    unsigned int tc = 0, tf = 0;
#pragma unroll
    for (int q = 0; q < BSCAN_PER; ++q) {
      const unsigned int idx = i0 + q;
      c[q] = idx < nb ? b.brick_count[idx] : 0u;
      fluid += idx < nb ? b.brick_fluid[idx] : 0u;
      tc += c[q];
      tf += c[q] > 0u;
    }
    unsigned int ic = tc, iff = tf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t1 = __shfl_up_sync(0xffffffffu, ic, o);
      const unsigned int t2 = __shfl_up_sync(0xffffffffu, iff, o);
      if (lane >= o) { ic += t1; iff += t2; }
    }
    if (lane == 31) { wc[warp] = ic; wf[warp] = iff; }
    __syncthreads();
    unsigned int oc = 0, of = 0, sc = 0, sf = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) { oc += wc[w]; of += wf[w]; }
      sc += wc[w];
      sf += wf[w];
    }
    unsigned int pc = run + oc + ic - tc, pf = run_act + of + iff - tf;
#pragma unroll
    for (int q = 0; q < BSCAN_PER; ++q) {
      const unsigned int idx = i0 + q;
      if (idx >= nb) break;
      b.brick_start[idx] = pc;
      pc += c[q];
      if (c[q]) b.active[pf++] = idx;
    }
    run += sc;
    run_act += sf;
    __syncthreads();
  }
  atomicAdd(&fl_tot, fluid);
  __syncthreads();
  if (threadIdx.x == 0) {
    b.brick_start[nb] = run;
    st->n_active = run_act;
    st->n_fluid = fl_tot;
    st->np_layout = run;
  }
}

__global__ void __launch_bounds__(1024) k_brick_scan(const Grid g, const BinView b, DevStats* st) {
  brick_scan(g, b, st);
}

// CTA s scans scene s.
__global__ void __launch_bounds__(1024) k_brick_scan_batch(const BatchLaunch L) {
  const SceneDev& S = L.scenes[blockIdx.x];
  brick_scan(S.g, S.B, S.st);
}

// Two particles per thread (i and i + stride), so each thread has two
// dependent gather chains (key -> offsets -> 7 moves) in flight.
// np_dev (nullable): the source count in device memory, bounding np; particles
// of rank >= rank_max in their cell are dropped (reseeding's upper bound).
__device__ __forceinline__ void scatter(const PartView& src, const PartView& dst, const BinView& b,
                                        long long np, const long long* np_dev,
                                        unsigned int rank_max, unsigned int blk,
                                        unsigned int nblk) {
  if (np_dev) np = min(np, *np_dev);
  const long long stride = (long long)nblk * blockDim.x;
  const long long i0 = blk * (long long)blockDim.x + threadIdx.x;
  unsigned int d[2];
  bool ok[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const long long i = i0 + u * stride;
    ok[u] = i < np;
    const unsigned int key = ok[u] ? b.key[i] : 0u;
    const unsigned int r = ok[u] ? b.rank[i] : 0u;
    ok[u] = ok[u] && r < rank_max;
    d[u] = ok[u] ? b.brick_start[key / BRICK_CELLS] + b.local_start[key] + r : 0u;
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    if (!ok[u]) continue;
    const long long i = i0 + u * stride;
    const float x = src.x[i], y = src.y[i], z = src.z[i];
    const float vu = src.u[i], vv = src.v[i], vw = src.w[i];
    const int id = src.id[i];
    dst.x[d[u]] = x;
    dst.y[d[u]] = y;
    dst.z[d[u]] = z;
    dst.u[d[u]] = vu;
    dst.v[d[u]] = vv;
    dst.w[d[u]] = vw;
    dst.id[d[u]] = id;
  }
}

__global__ void k_scatter(const PartView src, const PartView dst, const BinView b, long long np,
                          const long long* np_dev, unsigned int rank_max) {
  scatter(src, dst, b, np, np_dev, rank_max, blockIdx.x, gridDim.x);
}

__global__ void k_scatter_batch(const BatchLaunch L) {
  const int s = batch_scene(L, blockIdx.x);
  const SceneDev& S = L.scenes[s];
  scatter(S.src, S.dst, S.B, S.np, nullptr, ~0u, blockIdx.x - L.first[s],
          L.first[s + 1] - L.first[s]);
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
                  unsigned int* st_speed,
                  cudaStream_t s) {
  if (np > 0) k_rebin<<<blocks_for(np, 256), 256, 0, s>>>(g, p, b, np, st_speed);
}

void launch_bin(const Grid& g, const BinView& b, uint8_t* type, DevStats* st, cudaStream_t s,
                unsigned int cmax) {
  const unsigned int nb = (unsigned)g.bx * g.by * g.bz;
  k_cell_local_scan<<<(nb + SCAN_THREADS / 32 - 1) / (SCAN_THREADS / 32), SCAN_THREADS, 0, s>>>(
      g, b, type, nb, cmax, st);
  k_brick_scan<<<1, 1024, 0, s>>>(g, b, st);
}

void launch_scatter(const PartView& src, const PartView& dst, const BinView& b, long long np,
                    cudaStream_t s, const long long* np_dev, unsigned int rank_max) {
  if (np > 0)
    k_scatter<<<blocks_for((np + 1) / 2, 256), 256, 0, s>>>(src, dst, b, np, np_dev, rank_max);
}

void launch_bin_batch(const BatchLaunch& L_scan, unsigned int ctas_scan, const BatchLaunch& L_one,
                      cudaStream_t s) {
  if (ctas_scan) k_cell_local_scan_batch<<<ctas_scan, SCAN_THREADS, 0, s>>>(L_scan);
  if (L_one.n > 0) k_brick_scan_batch<<<(unsigned)L_one.n, 1024, 0, s>>>(L_one);
}

void launch_scatter_batch(const BatchLaunch& L, unsigned int ctas, cudaStream_t s) {
  if (ctas) k_scatter_batch<<<ctas, 256, 0, s>>>(L);
}

void launch_iota(int* id, long long np, cudaStream_t s) {
  if (np > 0) k_iota<<<blocks_for(np, 256), 256, 0, s>>>(id, np);
}

}  // namespace flipk
