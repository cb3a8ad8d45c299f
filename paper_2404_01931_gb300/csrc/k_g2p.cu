// k_g2p.cu — grid-to-particle transfer with the PIC/FLIP blend (Sec. 2.1.4,
// 3.1.8), forward-Euler advection and the wall clamp (Sec. 3.1.3), fused with
// the histogram of the next step's binning.
//
// One CTA takes one active 8x8x8 brick at a time (its particles are one
// contiguous range after binning).  It first stages in shared memory the
// pressure of the brick plus a one-cell halo, then, for every component, the
// face nodes any of the brick's particles can reach (the 9x10x10 tile P2G also
// uses): u_new (Eq. 5 with gravity and walls, face_unew's arithmetic) and
// u_new - u_old.  Each face value is so computed once per brick instead of once
// per particle that touches it.  Then one thread per particle interpolates
//     U = interp(u_new),  dU = interp(u_new - u_old)
//     v <- r (v + dU) + (1 - r) U
//     x <- clamp(x + dt v, skin, n dx - skin)     (or dt U with grid advection)
// and computes the key of the cell it moved to and its rank there.  Ranks come
// from one histogram atomic per distinct key in a warp (lanes with the same key
// take consecutive ranks), which is all the next step's counting sort needs.
#include "flip_kernels.cuh"

namespace flipk {

constexpr int G2P_THREADS = 256;
constexpr int G2P_TILE = 904;     // >= 9 * 10 * 10 face nodes per component
constexpr int G2P_PTILE = 1000;   // 10 * 10 * 10 cells of pressure

template <int D>
struct FaceTile {
  static constexpr int X = (D == 0) ? 9 : 10;
  static constexpr int Y = (D == 1) ? 9 : 10;
  static constexpr int Z = (D == 2) ? 9 : 10;
  static constexpr int N = X * Y * Z;
};

template <bool PAIR>
struct PTile;
template <>
struct PTile<true> {
  using T = float2;
};
template <>
struct PTile<false> {
  using T = float;
};

// Pressure difference p(+) - p(-) in the arithmetic of face_unew.
__device__ __forceinline__ float pdiff(float2 hp, float2 hm) {
  return __fadd_rn(__fsub_rn(hp.x, hm.x), __fsub_rn(hp.y, hm.y));
}
__device__ __forceinline__ float pdiff(float hp, float hm) { return __fsub_rn(hp, hm); }

// Stages component D's face tile: node (a, b, c) with a in [o0, o0 + X) etc.,
// o = brick origin on the own axis and origin - 1 on the others.  Nodes outside
// the face grid are never interpolated (the clamped weights keep every node in
// range) and are set to 0.
template <int D, bool PAIR>
__device__ __forceinline__ void stage_faces(const Grid& g, const StepConsts& K, int b0, int b1,
                                            int b2, const float* __restrict__ uo,
                                            const typename PTile<PAIR>::T* sp, float* su,
                                            float* sd) {
  constexpr int TX = FaceTile<D>::X, TY = FaceTile<D>::Y, N = FaceTile<D>::N;
  const int o0 = (D == 0) ? b0 : b0 - 1, o1 = (D == 1) ? b1 : b1 - 1, o2 = (D == 2) ? b2 : b2 - 1;
  const int FX = g.nx + (D == 0), FY = g.ny + (D == 1), FZ = g.nz + (D == 2);
  const int nmax = (D == 0) ? g.nx : (D == 1) ? g.ny : g.nz;
  for (int t = threadIdx.x; t < N; t += G2P_THREADS) {
    const int ta = t % TX, tb = (t / TX) % TY, tc = t / (TX * TY);
    const int a = o0 + ta, b = o1 + tb, c = o2 + tc;
    float un = 0.0f, du = 0.0f;
    if (a >= 0 && b >= 0 && c >= 0 && a < FX && b < FY && c < FZ) {
      const float uov = __ldg(uo + (a + FX * (b + FY * c)));
      const int nd = (D == 0) ? a : (D == 1) ? b : c;
      if (nd != 0 && nd != nmax) {
        // pressure tile cell of (a, b, c) is (a - b0 + 1, ...); the minus cell
        // is one step down along D
        const int pc = (a - b0 + 1) + 10 * ((b - b1 + 1) + 10 * (c - b2 + 1));
        const int pm = pc - ((D == 0) ? 1 : (D == 1) ? 10 : 100);
        const float dp = pdiff(sp[pc], sp[pm]);
        un = __fsub_rn(__fadd_rn(uov, K.gdt[D]), __fmul_rn(K.pscale, dp));
      }
      du = __fsub_rn(un, uov);
    }
    su[t] = un;
    sd[t] = du;
  }
}

// Interpolates component D of U and dU at a particle of cell (ci, cj, ck),
// local (li, lj, lk) in the brick, from the staged tile.
template <int D>
__device__ __forceinline__ void interp_tile(const Grid& g, float px, float py, float pz, int ci,
                                            int cj, int ck, int li, int lj, int lk,
                                            const float* su, const float* sd, float& U,
                                            float& dU) {
  constexpr int TX = FaceTile<D>::X, TY = FaceTile<D>::Y;
  const AxisW ax = axis_weights<D, 0>(px, g.inv_dx, ci, g.nx);
  const AxisW ay = axis_weights<D, 1>(py, g.inv_dx, cj, g.ny);
  const AxisW az = axis_weights<D, 2>(pz, g.inv_dx, ck, g.nz);
  const int t0 = (li + ax.off) + TX * ((lj + ay.off) + TY * (lk + az.off));
  const float wx[2] = {ax.w0, ax.w1}, wy[2] = {ay.w0, ay.w1}, wz[2] = {az.w0, az.w1};
  float s_u = 0.0f, s_d = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const float wyz = __fmul_rn(wy[dy], wz[dz]);
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float w = __fmul_rn(wx[dx], wyz);
        const int t = t0 + dx + TX * (dy + TY * dz);
        s_u = __fmaf_rn(w, su[t], s_u);
        s_d = __fmaf_rn(w, sd[t], s_d);
      }
    }
  U = s_u;
  dU = s_d;
}

template <bool PAIR>
__global__ void __launch_bounds__(G2P_THREADS, 6) k_g2p(const Grid g, const StepConsts K0,
                                                     const PartView P, const BinView B,
                                                     const float* __restrict__ uo0,
                                                     const float* __restrict__ uo1,
                                                     const float* __restrict__ uo2,
                                                     const float* __restrict__ p32,
                                                     const float2* __restrict__ pff,
                                                     DevStats* st) {
  const StepConsts K = step_consts(K0);
  using PT = typename PTile<PAIR>::T;
  __shared__ PT sp[G2P_PTILE];
  __shared__ float su[3][G2P_TILE];
  __shared__ float sd[3][G2P_TILE];
  const int lane = threadIdx.x & 31;
  const unsigned int nact = st->n_active;
  float speed2 = 0.0f;
  for (unsigned int bi = blockIdx.x; bi < nact; bi += gridDim.x) {
    const unsigned int brick = B.active[bi];
    const int b0 = (int)(brick % (unsigned)g.bx) * BRICK;
    const int b1 = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK;
    const int b2 = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK;
    // pressure of cells [b - 1, b + 8] per axis (0 outside the grid: never used)
    for (int t = threadIdx.x; t < G2P_PTILE; t += G2P_THREADS) {
      const int i = b0 - 1 + t % 10, j = b1 - 1 + (t / 10) % 10, k = b2 - 1 + t / 100;
      PT v{};
      if (i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz) {
        const int c = i + g.nx * (j + g.ny * k);
        if constexpr (PAIR) v = pff[c];
        else v = p32[c];
      }
      sp[t] = v;
    }
    __syncthreads();
    stage_faces<0, PAIR>(g, K, b0, b1, b2, uo0, sp, su[0], sd[0]);
    stage_faces<1, PAIR>(g, K, b0, b1, b2, uo1, sp, su[1], sd[1]);
    stage_faces<2, PAIR>(g, K, b0, b1, b2, uo2, sp, su[2], sd[2]);
    __syncthreads();
    const unsigned int bstart = B.brick_start[brick], bend = B.brick_start[brick + 1];
    // warp-uniform trip count, so every lane takes part in the key match
    for (unsigned int base = bstart + (threadIdx.x & ~31u); base < bend; base += G2P_THREADS) {
      const unsigned int q = base + (unsigned)lane;
      const bool valid = q < bend;
      unsigned int key = 0xffffffffu;
      if (valid) {
        float x = P.x[q], y = P.y[q], z = P.z[q];
        const float vp[3] = {P.u[q], P.v[q], P.w[q]};
        const int ci = cell_of(x, g.inv_dx, g.nx);
        const int cj = cell_of(y, g.inv_dx, g.ny);
        const int ck = cell_of(z, g.inv_dx, g.nz);
        // the particle's cell lies in this brick (its key was taken by the
        // same cell_of on the same coordinates); the clamp only keeps the
        // shared-memory indices in range
        const int li = min(max(ci - b0, 0), BRICK - 1);
        const int lj = min(max(cj - b1, 0), BRICK - 1);
        const int lk = min(max(ck - b2, 0), BRICK - 1);
        float U[3], dU[3];
        interp_tile<0>(g, x, y, z, ci, cj, ck, li, lj, lk, su[0], sd[0], U[0], dU[0]);
        interp_tile<1>(g, x, y, z, ci, cj, ck, li, lj, lk, su[1], sd[1], U[1], dU[1]);
        interp_tile<2>(g, x, y, z, ci, cj, ck, li, lj, lk, su[2], sd[2], U[2], dU[2]);
        const float r = K.flip_ratio, r1 = 1.0f - K.flip_ratio;
        float vn[3], adv[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          vn[d] = __fadd_rn(__fmul_rn(r, __fadd_rn(vp[d], dU[d])), __fmul_rn(r1, U[d]));
          adv[d] = K.advect_grid ? U[d] : vn[d];
        }
        x = fminf(fmaxf(__fmaf_rn(K.dt, adv[0], x), g.skin), g.hi[0]);
        y = fminf(fmaxf(__fmaf_rn(K.dt, adv[1], y), g.skin), g.hi[1]);
        z = fminf(fmaxf(__fmaf_rn(K.dt, adv[2], z), g.skin), g.hi[2]);
        P.x[q] = x;
        P.y[q] = y;
        P.z[q] = z;
        P.u[q] = vn[0];
        P.v[q] = vn[1];
        P.w[q] = vn[2];
        speed2 = fmaxf(speed2, vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
        key = brick_key(g, cell_of(x, g.inv_dx, g.nx), cell_of(y, g.inv_dx, g.ny),
                        cell_of(z, g.inv_dx, g.nz));
      }
      // one histogram atomic per distinct key of the warp
      const unsigned int same = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(same) - 1;
      unsigned int first = 0u;
      if (valid && lane == leader) first = atomicAdd(B.cell_count + key, (unsigned)__popc(same));
      first = __shfl_sync(0xffffffffu, first, leader);
      if (valid) {
        B.key[q] = key;
        B.rank[q] = first + (unsigned)__popc(same & ((1u << lane) - 1u));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) speed2 = fmaxf(speed2, __shfl_xor_sync(0xffffffffu, speed2, o));
  if (lane == 0 && speed2 > 0.0f) atomicMax(&st->max_speed_bits, __float_as_uint(sqrtf(speed2)));
}

int g2p_blocks(int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_g2p<true>, G2P_THREADS, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return sm_count * per_sm;
}

void launch_g2p(const Grid& g, const StepConsts& k, const PartView& p, const BinView& b,
                const float* const uo[3], const float* p32, const float2* pff, DevStats* st,
                long long np, int nblocks, cudaStream_t s) {
  if (np <= 0) return;
  if (pff)
    k_g2p<true><<<nblocks, G2P_THREADS, 0, s>>>(g, k, p, b, uo[0], uo[1], uo[2], p32, pff, st);
  else
    k_g2p<false><<<nblocks, G2P_THREADS, 0, s>>>(g, k, p, b, uo[0], uo[1], uo[2], p32, pff, st);
}

}  // namespace flipk
