// k_g2p.cu — grid-to-particle transfer with the PIC/FLIP blend (Sec. 2.1.4,
// 3.1.8), forward-Euler advection and the wall clamp (Sec. 3.1.3), fused with
// the histogram of the next step's binning.
//
// One CTA takes one active 8x8x8 brick at a time (its particles are one
// contiguous range after binning; they stream into shared memory by bulk copies,
// see below).  It first stages in shared memory the
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
//
// The pressure slab of a brick (the 10 x 10 x 10 cells [b - 1, b + 8] per axis)
// is staged by one TMA tensor copy (cp.async.bulk.tensor) when the handle has a
// tensor map of its pressure (row pitches a multiple of 16 bytes): the copy starts
// at x = b0 - XOFF so that its first coordinate is 16-byte aligned, rows are SPX
// cells wide, and cells outside the grid arrive as 0.  Otherwise, and in the
// batched kernel, the same tile is filled with plain loads.
#include <cudaTypedefs.h>

#include <cstring>

#include "flip_kernels.cuh"

namespace flipk {

constexpr int G2P_THREADS = 256;
constexpr int G2P_TILE = 904;     // >= 9 * 10 * 10 face nodes per component

template <int D>
struct FaceTile {
  static constexpr int X = (D == 0) ? 9 : 10;
  static constexpr int Y = (D == 1) ? 9 : 10;
  static constexpr int Z = (D == 2) ? 9 : 10;
  static constexpr int N = X * Y * Z;
};

// The staged pressure tile: element type (the float pair of mixed mode, or FP32),
// row width SPX and the x offset XOFF of its first cell from the brick origin, so
// that XOFF * sizeof(T) and SPX * sizeof(T) are multiples of 16 bytes.
template <bool PAIR>
struct PTile;
template <>
struct PTile<true> {
  using T = float2;
  static constexpr int SPX = 12, XOFF = 2;
};
template <>
struct PTile<false> {
  using T = float;
  static constexpr int SPX = 16, XOFF = 4;
};
template <bool PAIR>
constexpr int PTILE_N = 10 * 10 * PTile<PAIR>::SPX;

// ---------------------------------------------------------------- bulk copies
// Particles stream into shared memory in chunks of G2P_THREADS (one per thread)
// by cp.async.bulk (the Blackwell/Hopper bulk-copy engine), double-buffered and
// tracked by an mbarrier per buffer, so a chunk's loads are in flight while the
// previous chunk is processed.  A bulk copy starts and ends on 16-byte
// boundaries: a chunk [q0, q1) is copied as [q0 & ~3, (q1 + 3) & ~3), which stays
// inside its array (every array of the arena is padded to 256 bytes).
constexpr int G2P_CHUNK_PAD = G2P_THREADS + 8;
// After a wait has given up (StepConsts::wait_ns), the copies still in flight are
// waited for once more, up to this limit, before the CTA leaves: its shared memory
// must not be handed to another CTA while the copy engine still writes into it.
constexpr unsigned long long G2P_DRAIN_NS = 1000000000ull;

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of the barrier; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int parity,
                                          unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_timer_ns() - t0 > limit_ns) return false;
  return true;
}

// One 3-D tiled tensor copy of the box at (x, y, z) into dst, completing on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned int bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One thread: copy particles [q0, q1) of x, y, z, u, v, w into `dst` (the
// buffer then starts at particle q0 rounded down to 4), completing on `bar`.
__device__ __forceinline__ void issue_chunk(const PartView& P, unsigned int q0, unsigned int q1,
                                            float (*dst)[G2P_CHUNK_PAD],
                                            unsigned long long* bar) {
  const unsigned int a0 = q0 & ~3u, a1 = (q1 + 3u) & ~3u;
  const unsigned int bytes = 4u * (a1 - a0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, 6u * bytes);
  const float* src[6] = {P.x, P.y, P.z, P.u, P.v, P.w};
#pragma unroll
  for (int a = 0; a < 6; ++a) bulk_g2s(dst[a], src[a] + a0, bytes, bar);
}

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
                                            const typename PTile<PAIR>::T* sp, float2* sud) {
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
        // pressure tile cell of (a, b, c) is (a - b0 + XOFF, b - b1 + 1, c - b2 + 1);
        // the minus cell is one step down along D
        constexpr int SPX = PTile<PAIR>::SPX, XOFF = PTile<PAIR>::XOFF;
        const int pc = (a - b0 + XOFF) + SPX * ((b - b1 + 1) + 10 * (c - b2 + 1));
        const int pm = pc - ((D == 0) ? 1 : (D == 1) ? SPX : 10 * SPX);
        const float dp = pdiff(sp[pc], sp[pm]);
        un = __fsub_rn(__fadd_rn(uov, K.gdt[D]), __fmul_rn(K.pscale, dp));
      }
      du = __fsub_rn(un, uov);
    }
    sud[t] = make_float2(un, du);
  }
}

// Interpolates component D of U and dU at a particle of cell (ci, cj, ck),
// local (li, lj, lk) in the brick, from the staged tile.
// The particle's weights on each axis, computed once: `face` for the component
// whose faces are normal to that axis, `cen` (cell-centred nodes) for the others.
struct PartW {
  AxisW face[3], cen[3];
};

template <int D>
__device__ __forceinline__ void interp_tile(const PartW& W, int li, int lj, int lk,
                                            const float2* sud, float& U, float& dU) {
  constexpr int TX = FaceTile<D>::X, TY = FaceTile<D>::Y;
  const AxisW& ax = (D == 0) ? W.face[0] : W.cen[0];
  const AxisW& ay = (D == 1) ? W.face[1] : W.cen[1];
  const AxisW& az = (D == 2) ? W.face[2] : W.cen[2];
  const int t0 = (li + ax.off) + TX * ((lj + ay.off) + TY * (lk + az.off));
  const float wx[2] = {ax.w0, ax.w1}, wy[2] = {ay.w0, ay.w1}, wz[2] = {az.w0, az.w1};
  // (U, dU) accumulate together: one packed two-lane FMA per node, each lane
  // rounded like __fmaf_rn
  float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const float wyz = __fmul_rn(wy[dy], wz[dz]);
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float w = __fmul_rn(wx[dx], wyz);
        const int t = t0 + dx + TX * (dy + TY * dz);
        s = __ffma2_rn(make_float2(w, w), sud[t], s);
      }
    }
  U = s.x;
  dU = s.y;
}

// Shared memory of a G2P CTA: the brick's staged tiles and the particle buffers.
template <bool PAIR>
struct G2pShared {
  __align__(128) typename PTile<PAIR>::T sp[PTILE_N<PAIR>];  // the pressure slab
  float2 sud[3][G2P_TILE];  // (u_new, u_new - u_old) per face node
  __align__(16) float pbuf[2][6][G2P_CHUNK_PAD];
  __align__(8) unsigned long long bar[3];  // particle buffers 0, 1; the pressure slab
  int abort;
};

// A CTA's streaming state, kept across bricks (and across scenes in a batched
// launch): the mbarrier phases, the buffer of the next chunk, and (thread 0) which
// barriers have a copy that nobody has waited for.
struct G2pCta {
  unsigned int phase[3] = {0u, 0u, 0u};
  unsigned int kbuf = 0;
  bool inflight[3] = {false, false, false};
};

template <bool PAIR>
__device__ __forceinline__ void g2p_init(G2pShared<PAIR>& sh) {
  if (threadIdx.x == 0) {
    mbar_init(&sh.bar[0], 1);
    mbar_init(&sh.bar[1], 1);
    mbar_init(&sh.bar[2], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh.abort = 0;
  }
  __syncthreads();
}

// One brick of one scene (pmap: the tensor map of the scene's pressure, or
// nullptr for plain loads).  CTA-uniform; returns false once a wait has given up
// (DEV_TIMEOUT set in the scene's status), after which the CTA takes no more bricks.
template <bool PAIR>
__device__ __forceinline__ bool g2p_brick(const Grid& g, const StepConsts& K, const PartView& P,
                                          const BinView& B, const float* __restrict__ uo0,
                                          const float* __restrict__ uo1,
                                          const float* __restrict__ uo2,
                                          const float* __restrict__ p32,
                                          const float2* __restrict__ pff, DevStats* st,
                                          const CUtensorMap* pmap, unsigned int brick,
                                          G2pShared<PAIR>& sh, G2pCta& cs, float& speed2) {
  using PT = typename PTile<PAIR>::T;
  const int lane = threadIdx.x & 31;
  const int b0 = (int)(brick % (unsigned)g.bx) * BRICK;
  const int b1 = (int)((brick / (unsigned)g.bx) % (unsigned)g.by) * BRICK;
  const int b2 = (int)(brick / ((unsigned)g.bx * (unsigned)g.by)) * BRICK;
  const unsigned int bstart = B.brick_start[brick], bend = B.brick_start[brick + 1];
  // the brick's first chunk streams in while the tiles are staged
  if (threadIdx.x == 0 && bstart < bend) {
    issue_chunk(P, bstart, min(bend, bstart + G2P_THREADS), sh.pbuf[cs.kbuf], &sh.bar[cs.kbuf]);
    cs.inflight[cs.kbuf] = true;
  }
  // pressure of cells [b0 - XOFF, b0 - XOFF + SPX) x [b1 - 1, b1 + 9) x [b2 - 1, b2 + 9)
  // (0 outside the grid: never used)
  constexpr int SPX = PTile<PAIR>::SPX, XOFF = PTile<PAIR>::XOFF;
  if (pmap) {
    if (threadIdx.x == 0) {
      // the tile's readers of the previous brick passed the __syncthreads that
      // ended it; order their generic-proxy reads before the async-proxy write
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&sh.bar[2], (unsigned)sizeof(sh.sp));
      tma_load_3d(sh.sp, pmap, b0 - XOFF, b1 - 1, b2 - 1, &sh.bar[2]);
      cs.inflight[2] = true;
    }
    if (mbar_wait(&sh.bar[2], cs.phase[2], K.wait_ns)) {
      cs.phase[2] ^= 1u;
      cs.inflight[2] = false;
    } else {
      atomicOr(&st->status, DEV_TIMEOUT);
      sh.abort = 1;
    }
  } else {
    for (int t = threadIdx.x; t < PTILE_N<PAIR>; t += G2P_THREADS) {
      const int i = b0 - XOFF + t % SPX, j = b1 - 1 + (t / SPX) % 10, k = b2 - 1 + t / (10 * SPX);
      PT v{};
      if (i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz) {
        const int c = i + g.nx * (j + g.ny * k);
        if constexpr (PAIR) v = pff[c];
        else v = p32[c];
      }
      sh.sp[t] = v;
    }
  }
  __syncthreads();
  if (sh.abort) return false;
  stage_faces<0, PAIR>(g, K, b0, b1, b2, uo0, sh.sp, sh.sud[0]);
  stage_faces<1, PAIR>(g, K, b0, b1, b2, uo1, sh.sp, sh.sud[1]);
  stage_faces<2, PAIR>(g, K, b0, b1, b2, uo2, sh.sp, sh.sud[2]);
  __syncthreads();
  // chunk loop: CTA-uniform trip count, so every lane takes part in the key match
  for (unsigned int c0 = bstart; c0 < bend; c0 += G2P_THREADS) {
    const unsigned int cur = cs.kbuf;
    cs.kbuf ^= 1u;
    // the next chunk goes into the other buffer, whose readers passed the
    // __syncthreads that ended the previous chunk
    const unsigned int n0 = c0 + G2P_THREADS;
    if (threadIdx.x == 0 && n0 < bend) {
      issue_chunk(P, n0, min(bend, n0 + G2P_THREADS), sh.pbuf[cs.kbuf], &sh.bar[cs.kbuf]);
      cs.inflight[cs.kbuf] = true;
    }
    // a thread whose wait gives up reads nothing of the chunk; one whose wait
    // succeeded saw the whole chunk land
    if (mbar_wait(&sh.bar[cur], cs.phase[cur], K.wait_ns)) {
      cs.phase[cur] ^= 1u;
      cs.inflight[cur] = false;
    } else {
      atomicOr(&st->status, DEV_TIMEOUT);
      sh.abort = 1;
    }
    const float(*pb)[G2P_CHUNK_PAD] = sh.pbuf[cur];
    const unsigned int a0 = c0 & ~3u;
    const unsigned int q = c0 + threadIdx.x;
    const bool valid = q < bend && !sh.abort;
    unsigned int key = 0xffffffffu;
    if (valid) {
      const unsigned int o = q - a0;
      float x = pb[0][o], y = pb[1][o], z = pb[2][o];
      const float vp[3] = {pb[3][o], pb[4][o], pb[5][o]};
      const int ci = cell_of(x, g.inv_dx, g.nx);
      const int cj = cell_of(y, g.inv_dx, g.ny);
      const int ck = cell_of(z, g.inv_dx, g.nz);
      // the particle's cell lies in this brick (its key was taken by the
      // same cell_of on the same coordinates); the clamp only keeps the
      // shared-memory indices in range
      const int li = min(max(ci - b0, 0), BRICK - 1);
      const int lj = min(max(cj - b1, 0), BRICK - 1);
      const int lk = min(max(ck - b2, 0), BRICK - 1);
      PartW W;
      W.face[0] = axis_weights<0, 0>(x, g.inv_dx, ci, g.nx);
      W.face[1] = axis_weights<1, 1>(y, g.inv_dx, cj, g.ny);
      W.face[2] = axis_weights<2, 2>(z, g.inv_dx, ck, g.nz);
      W.cen[0] = axis_weights<1, 0>(x, g.inv_dx, ci, g.nx);
      W.cen[1] = axis_weights<0, 1>(y, g.inv_dx, cj, g.ny);
      W.cen[2] = axis_weights<0, 2>(z, g.inv_dx, ck, g.nz);
      float U[3], dU[3];
      interp_tile<0>(W, li, lj, lk, sh.sud[0], U[0], dU[0]);
      interp_tile<1>(W, li, lj, lk, sh.sud[1], U[1], dU[1]);
      interp_tile<2>(W, li, lj, lk, sh.sud[2], U[2], dU[2]);
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
    __syncthreads();
    if (sh.abort) break;
  }
  __syncthreads();
  return !sh.abort;
}

// After an abort, thread 0 drains the copies it issued and nobody waited for
// (the chunk whose wait gave up, the one issued after it), boundedly; the CTA's
// shared memory stays allocated until thread 0 leaves.
template <bool PAIR>
__device__ __forceinline__ void g2p_drain(G2pShared<PAIR>& sh, const G2pCta& cs) {
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (cs.inflight[k]) (void)mbar_wait(&sh.bar[k], cs.phase[k], G2P_DRAIN_NS);
}

// The largest particle speed a CTA saw in a scene, into the scene's statistics.
// CTA-uniform (every warp takes part).
__device__ __forceinline__ void g2p_flush_speed(float& speed2, DevStats* st) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) speed2 = fmaxf(speed2, __shfl_xor_sync(0xffffffffu, speed2, o));
  if ((threadIdx.x & 31) == 0 && speed2 > 0.0f)
    atomicMax(&st->max_speed_bits, __float_as_uint(sqrtf(speed2)));
  speed2 = 0.0f;
}

template <bool PAIR>
__global__ void __launch_bounds__(G2P_THREADS, 5) k_g2p(const Grid g, const StepConsts K0,
                                                     const PartView P, const BinView B,
                                                     const float* __restrict__ uo0,
                                                     const float* __restrict__ uo1,
                                                     const float* __restrict__ uo2,
                                                     const float* __restrict__ p32,
                                                     const float2* __restrict__ pff,
                                                     DevStats* st,
                                                     const __grid_constant__ CUtensorMap pmap,
                                                     int use_tma) {
  __shared__ G2pShared<PAIR> sh;
  const StepConsts K = step_consts(K0);
  const unsigned int nact = st->n_active;
  g2p_init(sh);
  G2pCta cs;
  float speed2 = 0.0f;
  const CUtensorMap* map = use_tma ? &pmap : nullptr;
  for (unsigned int bi = blockIdx.x; bi < nact; bi += gridDim.x)
    if (!g2p_brick<PAIR>(g, K, P, B, uo0, uo1, uo2, p32, pff, st, map, B.active[bi], sh, cs,
                         speed2))
      break;
  g2p_drain(sh, cs);
  g2p_flush_speed(speed2, st);
}

// All scenes' active bricks as one list (L.first from k_active_prefix): the CTAs
// share every scene's bricks evenly.  A CTA that gives up on a wait marks every
// scene whose bricks it leaves undone.
template <bool PAIR>
__global__ void __launch_bounds__(G2P_THREADS, 5) k_g2p_batch(const BatchLaunch L) {
  __shared__ G2pShared<PAIR> sh;
  g2p_init(sh);
  G2pCta cs;
  float speed2 = 0.0f;
  int cur = -1;
  const unsigned int g0 = L.first[0], g1 = L.first[L.n];
  unsigned int gb = g0 + blockIdx.x;
  for (; gb < g1; gb += gridDim.x) {
    const int s = batch_scene(L, gb);
    const SceneDev& S = L.scenes[s];
    if (s != cur) {
      if (cur >= 0) g2p_flush_speed(speed2, L.scenes[cur].st);
      cur = s;
    }
    if (!g2p_brick<PAIR>(S.g, step_consts(S.K), S.dst, S.B, S.uo[0], S.uo[1], S.uo[2], S.x32,
                         S.pff, S.st, nullptr, S.B.active[gb - L.first[s]], sh, cs, speed2))
      break;
  }
  g2p_drain(sh, cs);
  if (cur >= 0) g2p_flush_speed(speed2, L.scenes[cur].st);
  if (gb < g1 && threadIdx.x == 0)  // aborted: the scenes of the bricks left undone
    for (gb += gridDim.x; gb < g1; gb += gridDim.x)
      atomicOr(&L.scenes[batch_scene(L, gb)].st->status, DEV_TIMEOUT);
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

void launch_g2p_batch(const BatchLaunch& L, unsigned int ctas, bool pair, cudaStream_t s) {
  if (!ctas) return;
  if (pair) k_g2p_batch<true><<<ctas, G2P_THREADS, 0, s>>>(L);
  else k_g2p_batch<false><<<ctas, G2P_THREADS, 0, s>>>(L);
}

void launch_g2p(const Grid& g, const StepConsts& k, const PartView& p, const BinView& b,
                const float* const uo[3], const float* p32, const float2* pff, DevStats* st,
                long long np, int nblocks, const CUtensorMap* pmap, cudaStream_t s) {
  if (np <= 0) return;
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  const CUtensorMap& m = pmap ? *pmap : none;
  const int tma = pmap ? 1 : 0;
  if (pff)
    k_g2p<true><<<nblocks, G2P_THREADS, 0, s>>>(g, k, p, b, uo[0], uo[1], uo[2], p32, pff, st, m,
                                               tma);
  else
    k_g2p<false><<<nblocks, G2P_THREADS, 0, s>>>(g, k, p, b, uo[0], uo[1], uo[2], p32, pff, st, m,
                                                tma);
}

bool encode_pressure_map(const Grid& g, void* base, bool pair, CUtensorMap* out) {
  // row and plane pitches must be multiples of 16 bytes; the box (SPX x 10 x 10)
  // must fit the grid
  const size_t elem = pair ? 8 : 4;
  const int spx = pair ? PTile<true>::SPX : PTile<false>::SPX;
  if (!base || (reinterpret_cast<uintptr_t>(base) & 15u) || ((size_t)g.nx * elem) % 16 != 0 ||
      g.nx < spx || g.ny < 10 || g.nz < 10)
    return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = (PFN_cuTensorMapEncodeTiled_v12000)f;
    cudaGetLastError();
    looked_up = true;
  }
  if (!encode) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.nx * elem, (cuuint64_t)g.nx * g.ny * elem};
  const cuuint32_t box[3] = {(cuuint32_t)spx, 10u, 10u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return encode(out, pair ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace flipk
