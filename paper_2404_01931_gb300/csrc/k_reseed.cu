// k_reseed.cu — reseeding of under-filled fluid cells (Sec. 3.1.2: a fluid cell
// should hold no fewer than three particles; one that falls short is reseeded).
//
// Runs after G2P, whose histogram (cell_count, the next step's binning input)
// gives each cell's count.  A cell holding c in [1, ppc_min) particles gets
// ppc_min - c new ones, appended after the current buffer's particles with the
// next slots of the cell's histogram (key and rank), so the next step's
// counting sort places them like any other particle:
//   position  uniform in the cell: SplitMix64 with counter
//             ((step * n_cells + cell) * 64 + slot) * 3 + axis, slot = c + s;
//             U = top 53 bits * 2^-53, x = (i + U) dx in FP64 rounded to float,
//             moved by one float at a time back into the cell, clamped to
//             [skin, n dx - skin] like the advection
//   velocity  the projected grid velocity at that position (Eq. 4 weights on
//             the Eq. 5 face values, as G2P interpolates U)
//   id        next_id + (its place among this step's new particles)
// The per-cell atomic that reserves the slots makes the placement order in the
// buffer (and so the ids) vary from run to run; positions and velocities do not.
#include "flip_kernels.cuh"

namespace flipk {

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): output number `counter` of the stream at seed * G.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long counter) {
  const unsigned long long G = 0x9E3779B97F4A7C15ull;
  unsigned long long z = seed * G + (counter + 1ull) * G;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long counter) {
  return (double)(splitmix64(seed, counter) >> 11) * 0x1.0p-53;
}

// Coordinate of a new particle on one axis of cell index i.
__device__ __forceinline__ float spawn_coord(int i, double U, double dx, float inv, int n,
                                             float lo, float hi) {
  float x = (float)(((double)i + U) * dx);
  while (cell_of(x, inv, n) > i) x = nextafterf(x, 0.0f);
  while (cell_of(x, inv, n) < i) x = nextafterf(x, 3.0e38f);
  return fminf(fmaxf(x, lo), hi);
}

// Component D of the projected velocity at a point of cell (ci, cj, ck).
template <int D, bool PAIR>
__device__ __forceinline__ float interp_unew(const Grid& g, const StepConsts& K,
                                             const float* __restrict__ uo, float x, float y,
                                             float z, int ci, int cj, int ck, const float* p32,
                                             const float2* pff) {
  const AxisW ax = axis_weights<D, 0>(x, g.inv_dx, ci, g.nx);
  const AxisW ay = axis_weights<D, 1>(y, g.inv_dx, cj, g.ny);
  const AxisW az = axis_weights<D, 2>(z, g.inv_dx, ck, g.nz);
  const int a0 = (D == 0) ? ci : ci - 1 + ax.off;
  const int b0 = (D == 1) ? cj : cj - 1 + ay.off;
  const int c0 = (D == 2) ? ck : ck - 1 + az.off;
  const int FX = g.nx + (D == 0), FY = g.ny + (D == 1);
  const float wx[2] = {ax.w0, ax.w1}, wy[2] = {ay.w0, ay.w1}, wz[2] = {az.w0, az.w1};
  float s = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const float wyz = __fmul_rn(wy[dy], wz[dz]);
#pragma unroll
      for (int dxi = 0; dxi < 2; ++dxi) {
        const int a = a0 + dxi, b = b0 + dy, c = c0 + dz;
        const long long f = a + (long long)FX * (b + (long long)FY * c);
        const float un = face_unew<D, PAIR>(g, K, uo[f], a, b, c, p32, pff);
        s = __fmaf_rn(__fmul_rn(wx[dxi], wyz), un, s);
      }
    }
  return s;
}

template <bool PAIR>
__global__ void k_spawn(const Grid g, const StepConsts K0, const PartView p, const BinView b,
                        const float* __restrict__ uo0, const float* __restrict__ uo1,
                        const float* __restrict__ uo2, const float* __restrict__ p32,
                        const float2* __restrict__ pff, DevStats* st, const ReseedArgs r,
                        long long nkeys) {
  const double dx = r.dx;
  const long long key = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (key >= nkeys) return;
  const unsigned int c = b.cell_count[key];
  if (c == 0u || c >= (unsigned)r.ppc_min) return;
  const StepConsts K = step_consts(K0);
  const unsigned int brick = (unsigned int)(key / BRICK_CELLS), local = (unsigned int)(key % BRICK_CELLS);
  const int ci = (int)(brick % (unsigned)g.bx) * BRICK + (int)(local & 7u);
  const int cj = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK + (int)((local >> 3) & 7u);
  const int ck = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK + (int)(local >> 6);
  const unsigned int want = (unsigned)r.ppc_min - c;
  const long long np0 = st->np_layout;
  const unsigned long long first = atomicAdd(&st->spawn_req, (unsigned long long)want);
  const unsigned long long cell =
      (unsigned long long)ci + (unsigned long long)g.nx * ((unsigned long long)cj + (unsigned long long)g.ny * ck);
  const unsigned long long ncells = (unsigned long long)g.nx * g.ny * g.nz;
  unsigned int made = 0;
  for (unsigned int s = 0; s < want; ++s) {
    const long long idx = np0 + (long long)(first + s);
    if (idx >= r.capacity) break;
    const unsigned long long ctr =
        (((unsigned long long)r.step * ncells + cell) * 64ull + (unsigned long long)(c + s)) * 3ull;
    const float x = spawn_coord(ci, uniform01(r.seed, ctr), dx, g.inv_dx, g.nx, g.skin, g.hi[0]);
    const float y = spawn_coord(cj, uniform01(r.seed, ctr + 1), dx, g.inv_dx, g.ny, g.skin, g.hi[1]);
    const float z = spawn_coord(ck, uniform01(r.seed, ctr + 2), dx, g.inv_dx, g.nz, g.skin, g.hi[2]);
    p.x[idx] = x;
    p.y[idx] = y;
    p.z[idx] = z;
    p.u[idx] = interp_unew<0, PAIR>(g, K, uo0, x, y, z, ci, cj, ck, p32, pff);
    p.v[idx] = interp_unew<1, PAIR>(g, K, uo1, x, y, z, ci, cj, ck, p32, pff);
    p.w[idx] = interp_unew<2, PAIR>(g, K, uo2, x, y, z, ci, cj, ck, p32, pff);
    p.id[idx] = (int)(st->next_id + (long long)(first + s));
    {  // the next adaptive time step sees the new particles' speeds too
      const float su = p.u[idx], sv = p.v[idx], sw = p.w[idx];
      const float s2 = su * su + sv * sv + sw * sw;
      if (s2 > 0.0f) atomicMax(&st->max_speed_bits, __float_as_uint(sqrtf(s2)));
    }
    b.key[idx] = (unsigned int)key;
    b.rank[idx] = c + s;
    ++made;
  }
  if (made) {
    b.cell_count[key] = c + made;
    atomicAdd((unsigned long long*)&st->added_total, (unsigned long long)made);
  }
}

// The buffer's count after the spawn; capacity overflow raises DEV_CAPACITY.
__global__ void k_spawn_finalize(DevStats* st, long long capacity) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const long long req = (long long)st->spawn_req;
  const long long room = capacity - st->np_layout;
  const long long made = req < room ? req : (room > 0 ? room : 0);
  st->np_buffer = st->np_layout + made;
  st->next_id += made;
  if (made < req) atomicOr(&st->status, DEV_CAPACITY);
  st->spawn_req = 0ull;
}

void launch_spawn(const Grid& g, const StepConsts& k, const PartView& p, const BinView& b,
                  const float* const uo[3], const float* p32, const float2* pff, DevStats* st,
                  const ReseedArgs& r, long long nkeys, cudaStream_t s) {
  if (r.ppc_min > 0) {
    const unsigned int blocks = (unsigned int)((nkeys + 255) / 256);
    if (pff)
      k_spawn<true><<<blocks, 256, 0, s>>>(g, k, p, b, uo[0], uo[1], uo[2], p32, pff, st, r, nkeys);
    else
      k_spawn<false><<<blocks, 256, 0, s>>>(g, k, p, b, uo[0], uo[1], uo[2], p32, pff, st, r, nkeys);
  }
  k_spawn_finalize<<<1, 32, 0, s>>>(st, r.capacity);
}

}  // namespace flipk
