// k_surface.cu — surface reconstruction (Sec. 3.3): the particles' signed
// distance field on a sampling grid (Sec. 3.3.1), marching cubes over it and
// inverse-area-weighted vertex normals (Sec. 3.3.2).  C ABI: include/flip_surface.h.
//
// Pipeline of flip_surface_sdf (all on the surface's stream):
//   k_sbin_count    particle -> bin of edge R/2 over the corner box grown by R;
//                   the histogram atomic returns its rank in the bin
//   scan            exclusive scan of the bin counts (tile scan below)
//   k_sbin_scatter  positions into bin order as float4
//   k_sdf           one warp per 4 corners along x: the bin rows that meet their
//                   balls of radius R, read as coalesced particle ranges; kernel
//                   sums of k and k (x_i - x), phi = |sum k d| / sum k - r
// Pipeline of flip_surface_mesh:
//   tile scan over corners of one packed count per corner: (vertices on the
//   corner's 3 outgoing edges) + (triangles of the cube it is the lowest corner
//   of) << 32; the last pass stores each corner's offsets and its crossing /
//   case code and writes the vertices; then one pass writes triangles, one the
//   per-triangle weighted normals n/A, and one gathers them per vertex from the
//   four cubes around its edge in a fixed order (deterministic sums).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/flip_surface.h"
#include "flip_kernels.cuh"

void flip_set_last_error_(const std::string& msg);

using namespace flipk;

namespace {

int sfail(int code, const std::string& msg) {
  flip_set_last_error_(msg);
  return code;
}

int scuda(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? FLIP_E_OOM : FLIP_E_CUDA;
  return sfail(code, std::string(what) + ": " + cudaGetErrorName(e));
}

#define SURF_CUDA(call)                            \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return scuda(e_, #call); \
  } while (0)

// ------------------------------------------------------------------ case table
//
// Local cube numbering: corner c has offset (c & 1, (c >> 1) & 1, c >> 2).  Edge
// e runs along axis a = e / 4 from the corner with bit a clear; its bits on the
// other two axes (ascending) are e & 1 and (e >> 1) & 1.
constexpr int MC_MAXT = 12;

struct McTable {
  uint8_t ntri[256];
  uint8_t tri[256][MC_MAXT][3];
};

__constant__ McTable c_mc;

int edge_of(int c0, int c1) {
  const int d = c0 ^ c1;
  const int a = (d == 1) ? 0 : (d == 2) ? 1 : 2;
  const int lo = (a == 0) ? 1 : 0, hi = (a == 2) ? 1 : 2;
  return 4 * a + ((c0 >> lo) & 1) + 2 * ((c0 >> hi) & 1);
}

void edge_ends(int e, int& c0, int& c1) {
  const int a = e / 4;
  const int lo = (a == 0) ? 1 : 0, hi = (a == 2) ? 1 : 2;
  c0 = ((e & 1) << lo) | (((e >> 1) & 1) << hi);
  c1 = c0 | (1 << a);
}

bool build_table(McTable& T) {
  std::memset(&T, 0, sizeof(T));
  for (int cs = 0; cs < 256; ++cs) {
    auto in = [&](int c) { return (cs >> c) & 1; };
    // face segments: each crossing edge gets one partner per face it lies on
    int partner[12][2];
    int np_[12] = {0};
    for (int f = 0; f < 6; ++f) {
      const int a = f / 2, s = f % 2;
      const int u = (a == 0) ? 1 : 0, v = (a == 2) ? 1 : 2;
      int P[4];
      const int cyc[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
      for (int q = 0; q < 4; ++q) P[q] = (s << a) | (cyc[q][0] << u) | (cyc[q][1] << v);
      int E[4], X[4], nx = 0;
      for (int q = 0; q < 4; ++q) {
        E[q] = edge_of(P[q], P[(q + 1) & 3]);
        X[q] = in(P[q]) != in(P[(q + 1) & 3]);
        nx += X[q];
      }
      auto link = [&](int e0, int e1) {
        partner[e0][np_[e0]++] = e1;
        partner[e1][np_[e1]++] = e0;
      };
      if (nx == 2) {
        int k0 = -1, k1 = -1;
        for (int q = 0; q < 4; ++q)
          if (X[q]) (k0 < 0 ? k0 : k1) = q;
        link(E[k0], E[k1]);
      } else if (nx == 4) {
        for (int q = 0; q < 4; ++q)
          if (in(P[q])) link(E[(q + 3) & 3], E[q]);  // cut off each inside corner
      }
    }
    bool used[12] = {false};
    int nt = 0;
    for (int e0 = 0; e0 < 12; ++e0) {
      if (np_[e0] == 0 || used[e0]) continue;
      if (np_[e0] != 2) return false;
      int loop[12], len = 0, prev = -1, cur = e0;
      do {
        if (len == 12) return false;
        loop[len++] = cur;
        used[cur] = true;
        const int nxt = (partner[cur][0] != prev) ? partner[cur][0] : partner[cur][1];
        prev = cur;
        cur = nxt;
      } while (cur != e0);
      if (len < 3) return false;
      // winding: Newell normal of the edge midpoints against inside -> outside
      double N[3] = {0, 0, 0}, D[3] = {0, 0, 0}, M[12][3];
      for (int q = 0; q < len; ++q) {
        int c0, c1;
        edge_ends(loop[q], c0, c1);
        for (int d = 0; d < 3; ++d) {
          const double p0 = (c0 >> d) & 1, p1 = (c1 >> d) & 1;
          M[q][d] = 0.5 * (p0 + p1);
          D[d] += in(c0) ? (p1 - p0) : (p0 - p1);
        }
      }
      for (int q = 0; q < len; ++q) {
        const double* A = M[q];
        const double* B = M[(q + 1) % len];
        N[0] += (A[1] - B[1]) * (A[2] + B[2]);
        N[1] += (A[2] - B[2]) * (A[0] + B[0]);
        N[2] += (A[0] - B[0]) * (A[1] + B[1]);
      }
      const double nd = N[0] * D[0] + N[1] * D[1] + N[2] * D[2];
      if (std::fabs(nd) < 1e-9) return false;
      if (nd < 0) std::reverse(loop, loop + len);
      // fan apex: the lowest edge on no face the loop crosses twice (a face holding
      // four of its edges); a fan from there puts no triangle inside a cube face
      int on_face[6] = {0, 0, 0, 0, 0, 0};
      auto faces_of = [](int e, int& f0, int& f1) {
        const int a = e / 4;
        const int lo = (a == 0) ? 1 : 0, hi = (a == 2) ? 1 : 2;
        f0 = 2 * lo + (e & 1);
        f1 = 2 * hi + ((e >> 1) & 1);
      };
      for (int q = 0; q < len; ++q) {
        int f0, f1;
        faces_of(loop[q], f0, f1);
        ++on_face[f0];
        ++on_face[f1];
      }
      int r0 = -1;
      for (int q = 0; q < len; ++q) {
        int f0, f1;
        faces_of(loop[q], f0, f1);
        if (on_face[f0] < 4 && on_face[f1] < 4 && (r0 < 0 || loop[q] < loop[r0])) r0 = q;
      }
      if (r0 < 0) r0 = (int)(std::min_element(loop, loop + len) - loop);
      std::rotate(loop, loop + r0, loop + len);
      for (int q = 1; q + 1 < len; ++q) {
        if (nt == MC_MAXT) return false;
        T.tri[cs][nt][0] = (uint8_t)loop[0];
        T.tri[cs][nt][1] = (uint8_t)loop[q];
        T.tri[cs][nt][2] = (uint8_t)loop[q + 1];
        ++nt;
      }
    }
    T.ntri[cs] = (uint8_t)nt;
  }
  return true;
}

// The table is generated once per process and uploaded to each device that
// creates a surface object (constant memory is per device).
std::mutex g_table_mutex;
bool g_table_built = false, g_table_ok = false;
McTable g_table;
std::vector<int> g_table_devices;

int ensure_table() {
  std::lock_guard<std::mutex> lock(g_table_mutex);
  if (!g_table_built) {
    g_table_ok = build_table(g_table);
    g_table_built = true;
  }
  if (!g_table_ok) return sfail(FLIP_E_CUDA, "marching-cubes table generation failed");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return scuda(e, "cudaGetDevice");
  if (std::find(g_table_devices.begin(), g_table_devices.end(), dev) != g_table_devices.end())
    return FLIP_OK;
  e = cudaMemcpyToSymbol(c_mc, &g_table, sizeof(g_table));
  if (e != cudaSuccess) return scuda(e, "cudaMemcpyToSymbol(case table)");
  g_table_devices.push_back(dev);
  return FLIP_OK;
}

// ------------------------------------------------------------------ geometry

struct SGrid {
  int n[3];           // cells per axis
  int c[3];           // corners per axis (n + 1)
  long long ncorners;
  float o[3];         // origin
  float h;
  float iso;
};

struct SBins {
  int nb[3];
  long long nbins;
  float o[3];         // bin-grid origin (corner origin - R)
  float b;            // bin edge
  float inv_b;
  float R, R2, inv_R2, r;
};

__device__ __forceinline__ void corner_ijk(const SGrid& g, long long c, int& i, int& j, int& k) {
  i = (int)(c % g.c[0]);
  const long long t = c / g.c[0];
  j = (int)(t % g.c[1]);
  k = (int)(t / g.c[1]);
}

// ------------------------------------------------------------------ tile scan
//
// An exclusive scan over n items of a per-item count computed by a functor:
// pass 1 reduces tiles of SC_TILE items, pass 2 (one CTA) scans the tile sums,
// pass 3 recomputes the counts, scans them within the tile and hands each item
// its exclusive prefix.  The counts are never stored.
constexpr int SC_THREADS = 256;
constexpr int SC_ROWS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ROWS;
typedef unsigned long long u64;

__device__ __forceinline__ u64 block_excl_scan(u64 v, u64& total, u64* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) sm[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    u64 w = (lane < SC_THREADS / 32) ? sm[lane] : 0ull;
    u64 wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < SC_THREADS / 32) sm[32 + lane] = wi - w;
    if (lane == SC_THREADS / 32 - 1) sm[64] = wi;
  }
  __syncthreads();
  total = sm[64];
  return sm[32 + warp] + incl - v;
}

template <class F>
__global__ void __launch_bounds__(SC_THREADS) k_tile_reduce(F f, long long n, u64* tile_sum) {
  __shared__ u64 sm[72];
  const long long base = (long long)blockIdx.x * SC_TILE;
  u64 s = 0;
#pragma unroll
  for (int r = 0; r < SC_ROWS; ++r) {
    const long long i = base + r * SC_THREADS + threadIdx.x;
    if (i < n) s += f.count(i);
  }
  u64 tot;
  block_excl_scan(s, tot, sm);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SC_THREADS) k_tile_scan(u64* tile_sum, long long ntiles,
                                                          u64* total) {
  __shared__ u64 sm[72];
  u64 carry = 0;
  for (long long b = 0; b < ntiles; b += SC_THREADS) {
    const long long i = b + threadIdx.x;
    const u64 v = (i < ntiles) ? tile_sum[i] : 0ull;
    u64 tot;
    const u64 ex = block_excl_scan(v, tot, sm);
    if (i < ntiles) tile_sum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

template <class F>
__global__ void __launch_bounds__(SC_THREADS) k_tile_apply(F f, long long n, const u64* tile_off) {
  __shared__ u64 sm[72];
  const long long base = (long long)blockIdx.x * SC_TILE;
  u64 run = tile_off[blockIdx.x];
  for (int r = 0; r < SC_ROWS; ++r) {
    const long long i = base + r * SC_THREADS + threadIdx.x;
    const u64 c = (i < n) ? f.count(i) : 0ull;
    u64 tot;
    const u64 ex = block_excl_scan(c, tot, sm);
    if (i < n) f.apply(i, run + ex);
    run += tot;
  }
}

template <class F>
void tile_scan(const F& f, long long n, u64* tile_sum, u64* total, cudaStream_t s) {
  const long long ntiles = (n + SC_TILE - 1) / SC_TILE;
  k_tile_reduce<F><<<(unsigned)ntiles, SC_THREADS, 0, s>>>(f, n, tile_sum);
  k_tile_scan<<<1, SC_THREADS, 0, s>>>(tile_sum, ntiles, total);
  k_tile_apply<F><<<(unsigned)ntiles, SC_THREADS, 0, s>>>(f, n, tile_sum);
}

// ------------------------------------------------------------------ binning + SDF

__device__ __forceinline__ int bin_coord(float x, const SBins& B, int a) {
  const float t = floorf((x - B.o[a]) * B.inv_b);
  return (t >= 0.0f && t < (float)B.nb[a]) ? (int)t : -1;
}

__global__ void k_sbin_count(const PartView p, long long np, const SBins B,
                             unsigned int* __restrict__ count, int* __restrict__ pbin,
                             unsigned int* __restrict__ prank) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int bx = bin_coord(p.x[i], B, 0), by = bin_coord(p.y[i], B, 1),
            bz = bin_coord(p.z[i], B, 2);
  int b = -1;
  if (bx >= 0 && by >= 0 && bz >= 0) {
    b = bx + B.nb[0] * (by + B.nb[1] * bz);
    prank[i] = atomicAdd(count + b, 1u);
  }
  pbin[i] = b;
}

// Scans nbins + 1 items so that start[nbins] is the total.
struct BinScan {
  const unsigned int* cnt;
  unsigned int* start;
  long long nbins;
  __device__ u64 count(long long i) const { return i < nbins ? cnt[i] : 0u; }
  __device__ void apply(long long i, u64 ex) const { start[i] = (unsigned int)ex; }
};

__global__ void k_fill(float* __restrict__ p, long long n, float v) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_sbin_scatter(const PartView p, long long np, const int* __restrict__ pbin,
                               const unsigned int* __restrict__ prank,
                               const unsigned int* __restrict__ start, float4* __restrict__ pos) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int b = pbin[i];
  if (b < 0) return;
  pos[start[b] + prank[i]] = make_float4(p.x[i], p.y[i], p.z[i], 0.0f);
}

// One warp per group of SDF_G corners consecutive along x (same j, k).  With bins
// of edge R/2 the balls meet at most 5 bins along y and along z, so at most 25 bin
// rows (fixed y, z bin): lane r finds row r's particle range (the row's bins
// within the balls' x extent are one contiguous range), a warp scan lays the rows
// end to end in a per-warp shared table, and the lanes stride over that flat
// range, so every load is independent and a warp's loads are consecutive
// float4s.  Each particle is tested against all SDF_G corners, whose sums stay in
// registers until a warp reduction.  A bin whose nearest point is R or farther
// from the corners holds no particle closer than R and is skipped.
constexpr int SDF_G = 4;
constexpr int SDF_THREADS = 256;
constexpr int SDF_WARPS = SDF_THREADS / 32;

__global__ void __launch_bounds__(SDF_THREADS) k_sdf(const SGrid g, const SBins B,
                                                     const unsigned int* __restrict__ start,
                                                     const float4* __restrict__ pos,
                                                     float* __restrict__ phi) {
  __shared__ unsigned int s_end[SDF_WARPS][32], s_beg[SDF_WARPS][32], s_p0[SDF_WARPS][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gx = (g.c[0] + SDF_G - 1) / SDF_G;
  const long long ngroups = (long long)gx * g.c[1] * g.c[2];
  const long long warps = (long long)gridDim.x * SDF_WARPS;
  constexpr float Rb = 2.0f;  // R in bins (the bin edge is R/2)
  for (long long grp = blockIdx.x * (long long)SDF_WARPS + wid; grp < ngroups; grp += warps) {
    const int i0 = (int)(grp % gx) * SDF_G;
    const int j = (int)((grp / gx) % g.c[1]);
    const int k = (int)(grp / ((long long)gx * g.c[1]));
    const int ng = min(SDF_G, g.c[0] - i0);
    const float x0 = g.o[0] + g.h * (float)i0, xl = g.o[0] + g.h * (float)(i0 + ng - 1);
    const float yc = g.o[1] + g.h * (float)j, zc = g.o[2] + g.h * (float)k;
    const float ry = (yc - B.o[1]) * B.inv_b, rz = (zc - B.o[2]) * B.inv_b;
    const int by0 = max(0, (int)floorf(ry - Rb)), by1 = min(B.nb[1] - 1, (int)floorf(ry + Rb));
    const int bz0 = max(0, (int)floorf(rz - Rb)), bz1 = min(B.nb[2] - 1, (int)floorf(rz + Rb));
    const int nyr = max(by1 - by0 + 1, 1);
    const int nrows = min(nyr * (bz1 - bz0 + 1), 32);
    unsigned int p0 = 0, cnt = 0;
    if (lane < nrows) {
      const int by = by0 + lane % nyr, bz = bz0 + lane / nyr;
      const float dy = fmaxf(fmaxf(B.o[1] + B.b * by - yc, yc - (B.o[1] + B.b * (by + 1))), 0.0f);
      const float dz = fmaxf(fmaxf(B.o[2] + B.b * bz - zc, zc - (B.o[2] + B.b * (bz + 1))), 0.0f);
      const float dyz = dy * dy + dz * dz;
      if (dyz < B.R2) {
        const float rx = sqrtf(B.R2 - dyz) * B.inv_b;
        const int bx0 = max(0, (int)floorf((x0 - B.o[0]) * B.inv_b - rx));
        const int bx1 = min(B.nb[0] - 1, (int)floorf((xl - B.o[0]) * B.inv_b + rx));
        if (bx0 <= bx1) {
          const long long row = (long long)B.nb[0] * (by + (long long)B.nb[1] * bz);
          p0 = start[row + bx0];
          cnt = start[row + bx1 + 1] - p0;
        }
      }
    }
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    s_end[wid][lane] = incl;
    s_beg[wid][lane] = incl - cnt;
    s_p0[wid][lane] = p0;
    __syncwarp();
    // per corner q: (sum k, sum k ex) and (sum k ey, sum k ez); corners go in
    // pairs through packed two-lane FP32 operations, each lane rounded like the
    // scalar operation
    static_assert(SDF_G % 2 == 0, "corners in pairs");
    float2 a01[SDF_G], a23[SDF_G];
    float2 xq[SDF_G / 2];  // minus the corners' x (P.x + (-x) rounds as P.x - x)
#pragma unroll
    for (int q = 0; q < SDF_G; ++q) a01[q] = a23[q] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int u = 0; u < SDF_G / 2; ++u)
      xq[u] = make_float2(-(x0 + g.h * (float)(2 * u)), -(x0 + g.h * (float)(2 * u + 1)));
    const float2 one = make_float2(1.0f, 1.0f), m_inv = make_float2(-B.inv_R2, -B.inv_R2);
    int r = 0;  // this lane's current row: only moves forward
    for (unsigned int f = lane; f < total; f += 32) {
      while (f >= s_end[wid][r]) ++r;
      const float4 P = pos[s_p0[wid][r] + (f - s_beg[wid][r])];
      const float ey = __fsub_rn(P.y, yc), ez = __fsub_rn(P.z, zc);
      const float r2 = __fmaf_rn(ez, ez, __fmul_rn(ey, ey));
      const float2 eyz = make_float2(ey, ez);
#pragma unroll
      for (int u = 0; u < SDF_G / 2; ++u) {
        const float2 ex = __fadd2_rn(make_float2(P.x, P.x), xq[u]);
        const float2 dd = __ffma2_rn(ex, ex, make_float2(r2, r2));
        const float2 t = __ffma2_rn(dd, m_inv, one);
        float2 kk = __fmul2_rn(__fmul2_rn(t, t), t);
        if (!(2 * u < ng && dd.x < B.R2)) kk.x = 0.0f;
        if (!(2 * u + 1 < ng && dd.y < B.R2)) kk.y = 0.0f;
        a01[2 * u] = __ffma2_rn(make_float2(kk.x, kk.x), make_float2(1.0f, ex.x), a01[2 * u]);
        a23[2 * u] = __ffma2_rn(make_float2(kk.x, kk.x), eyz, a23[2 * u]);
        a01[2 * u + 1] = __ffma2_rn(make_float2(kk.y, kk.y), make_float2(1.0f, ex.y), a01[2 * u + 1]);
        a23[2 * u + 1] = __ffma2_rn(make_float2(kk.y, kk.y), eyz, a23[2 * u + 1]);
      }
    }
    float sk[SDF_G], s0[SDF_G], s1[SDF_G], s2[SDF_G];
#pragma unroll
    for (int q = 0; q < SDF_G; ++q) {
      sk[q] = a01[q].x;
      s0[q] = a01[q].y;
      s1[q] = a23[q].x;
      s2[q] = a23[q].y;
    }
#pragma unroll
    for (int q = 0; q < SDF_G; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sk[q] += __shfl_xor_sync(0xffffffffu, sk[q], o);
        s0[q] += __shfl_xor_sync(0xffffffffu, s0[q], o);
        s1[q] += __shfl_xor_sync(0xffffffffu, s1[q], o);
        s2[q] += __shfl_xor_sync(0xffffffffu, s2[q], o);
      }
    }
    if (lane < ng) {
      float a = 0.0f, b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
#pragma unroll
      for (int q = 0; q < SDF_G; ++q)
        if (q == lane) {
          a = sk[q];
          b0 = s0[q];
          b1 = s1[q];
          b2 = s2[q];
        }
      const float v = (a > 0.0f) ? sqrtf(b0 * b0 + b1 * b1 + b2 * b2) / a - B.r : B.R - B.r;
      phi[(i0 + lane) + (long long)g.c[0] * (j + (long long)g.c[1] * k)] = v;
    }
  }
}

int sdf_blocks() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sdf, SDF_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    return 152 * 8;
  }
  return std::max(1, sms * std::max(per, 1));
}

// ------------------------------------------------------------------ marching cubes

struct McScan {
  SGrid g;
  const float* phi;
  unsigned int* voff;
  unsigned int* toff;
  uint16_t* code;     // bits 0..2: crossing edges along x, y, z; bits 8..15: cube case
  float* vert;
  long long* vedge;

  __device__ __forceinline__ void classify(long long c, int& flags, int& cs) const {
    int i, j, k;
    corner_ijk(g, c, i, j, k);
    const long long sx = 1, sy = g.c[0], sz = (long long)g.c[0] * g.c[1];
    const bool in0 = phi[c] < g.iso;
    flags = 0;
    if (i < g.n[0] && ((phi[c + sx] < g.iso) != in0)) flags |= 1;
    if (j < g.n[1] && ((phi[c + sy] < g.iso) != in0)) flags |= 2;
    if (k < g.n[2] && ((phi[c + sz] < g.iso) != in0)) flags |= 4;
    cs = 0;
    if (i < g.n[0] && j < g.n[1] && k < g.n[2]) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const long long cq = c + (q & 1) * sx + ((q >> 1) & 1) * sy + ((q >> 2) & 1) * sz;
        cs |= (phi[cq] < g.iso) << q;
      }
    }
  }
  __device__ u64 count(long long c) const {
    int flags, cs;
    classify(c, flags, cs);
    return (u64)__popc(flags) | ((u64)c_mc.ntri[cs] << 32);
  }
  __device__ void apply(long long c, u64 ex) const {
    int flags, cs;
    classify(c, flags, cs);
    const unsigned int v0 = (unsigned int)(ex & 0xffffffffull);
    voff[c] = v0;
    toff[c] = (unsigned int)(ex >> 32);
    code[c] = (uint16_t)(flags | (cs << 8));
    if (!flags) return;
    int ijk[3];
    corner_ijk(g, c, ijk[0], ijk[1], ijk[2]);
    const long long st[3] = {1, g.c[0], (long long)g.c[0] * g.c[1]};
    const float pa = phi[c];
    unsigned int v = v0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!((flags >> a) & 1)) continue;
      const float pb = phi[c + st[a]];
      const float t = (g.iso - pa) / (pb - pa);
#pragma unroll
      for (int d = 0; d < 3; ++d)
        vert[3 * (size_t)v + d] = g.o[d] + g.h * ((float)ijk[d] + (d == a ? t : 0.0f));
      vedge[v] = 3 * c + a;
      ++v;
    }
  }
};

__device__ __forceinline__ unsigned int vertex_of_edge(const SGrid& g, long long c, int e,
                                                       const unsigned int* voff,
                                                       const uint16_t* code) {
  const int a = e >> 2;
  const int lo = (a == 0) ? 1 : 0, hi = (a == 2) ? 1 : 2;
  int off[3] = {0, 0, 0};
  off[lo] = e & 1;
  off[hi] = (e >> 1) & 1;
  const long long cc = c + off[0] + (long long)g.c[0] * (off[1] + (long long)g.c[1] * off[2]);
  const int fl = code[cc] & 7;
  return voff[cc] + __popc(fl & ((1 << a) - 1));
}

__global__ void k_mc_triangles(const SGrid g, const unsigned int* __restrict__ voff,
                               const unsigned int* __restrict__ toff,
                               const uint16_t* __restrict__ code, int* __restrict__ tri) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncorners) return;
  const int cs = code[c] >> 8;
  const int nt = c_mc.ntri[cs];
  const unsigned int t0 = toff[c];
  for (int t = 0; t < nt; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      tri[3 * ((size_t)t0 + t) + q] = (int)vertex_of_edge(g, c, c_mc.tri[cs][t][q], voff, code);
}

// n / A for a triangle of unit normal n and area A: 2 (e1 x e2) / |e1 x e2|^2.
__global__ void k_mc_tri_weights(long long nt, const float* __restrict__ vert,
                                 const int* __restrict__ tri, float* __restrict__ tw) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
  const float ax = vert[3 * (size_t)a], ay = vert[3 * (size_t)a + 1], az = vert[3 * (size_t)a + 2];
  const float e1x = vert[3 * (size_t)b] - ax, e1y = vert[3 * (size_t)b + 1] - ay,
              e1z = vert[3 * (size_t)b + 2] - az;
  const float e2x = vert[3 * (size_t)c] - ax, e2y = vert[3 * (size_t)c + 1] - ay,
              e2z = vert[3 * (size_t)c + 2] - az;
  const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  const float l2 = nx * nx + ny * ny + nz * nz;
  const float s = (l2 > 0.0f) ? 2.0f / l2 : 0.0f;
  tw[3 * t] = s * nx;
  tw[3 * t + 1] = s * ny;
  tw[3 * t + 2] = s * nz;
}

__global__ void k_mc_normals(const SGrid g, long long nv,
                             const long long* __restrict__ vedge,
                             const unsigned int* __restrict__ toff,
                             const uint16_t* __restrict__ code, const int* __restrict__ tri,
                             const float* __restrict__ tw, float* __restrict__ nrm) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const long long e = vedge[v];
  const long long c = e / 3;
  const int a = (int)(e % 3);
  int ijk[3];
  corner_ijk(g, c, ijk[0], ijk[1], ijk[2]);
  const int u = (a == 0) ? 1 : 0, w = (a == 2) ? 1 : 2;
  const long long st[3] = {1, g.c[0], (long long)g.c[0] * g.c[1]};
  float sx = 0.0f, sy = 0.0f, sz = 0.0f;
  for (int q = 0; q < 4; ++q) {
    const int bu = q & 1, bw = q >> 1;
    if (ijk[u] - bu < 0 || ijk[w] - bw < 0 || ijk[u] - bu >= g.n[u] || ijk[w] - bw >= g.n[w])
      continue;
    const long long cc = c - bu * st[u] - bw * st[w];
    const unsigned int t0 = toff[cc];
    const int nt = c_mc.ntri[code[cc] >> 8];
    for (int t = 0; t < nt; ++t) {
      const size_t tt = (size_t)t0 + t;
      if (tri[3 * tt] == (int)v || tri[3 * tt + 1] == (int)v || tri[3 * tt + 2] == (int)v) {
        sx += tw[3 * tt];
        sy += tw[3 * tt + 1];
        sz += tw[3 * tt + 2];
      }
    }
  }
  const float l = sqrtf(sx * sx + sy * sy + sz * sz);
  const float s = (l > 0.0f) ? 1.0f / l : 0.0f;
  nrm[3 * v] = sx * s;
  nrm[3 * v + 1] = sy * s;
  nrm[3 * v + 2] = sz * s;
}

unsigned int blocks_for(long long n, int threads) {
  return (unsigned int)std::max<long long>(1, (n + threads - 1) / threads);
}

}  // namespace

// ------------------------------------------------------------------ object

struct flip_surface {
  flip_surface_params prm{};
  SGrid g{};
  SBins B{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* phi = nullptr;
  // bins (grow with the particle count)
  unsigned int* bin_count = nullptr;
  unsigned int* bin_start = nullptr;
  long long part_cap = 0;
  int* pbin = nullptr;
  unsigned int* prank = nullptr;
  float4* pos = nullptr;
  // marching cubes
  unsigned int* voff = nullptr;
  unsigned int* toff = nullptr;
  uint16_t* code = nullptr;
  u64* tile = nullptr;       // tile sums + the total
  long long tile_cap = 0;
  long long vcap = 0, tcap = 0;
  float* vert = nullptr;
  float* nrm = nullptr;
  long long* vedge = nullptr;
  int* tri = nullptr;
  float* tw = nullptr;
  long long nv = 0, nt = 0;
  u64* htotal = nullptr;     // pinned
};

namespace {

void sfree(void* p) {
  if (p) cudaFree(p);
}

// Replaces p by a fresh device array of n (>= 1) elements.
template <class T>
int realloc_n(T*& p, long long n) {
  sfree(p);
  p = nullptr;
  SURF_CUDA(cudaMalloc(reinterpret_cast<void**>(&p), sizeof(T) * (size_t)std::max<long long>(n, 1)));
  return FLIP_OK;
}

}  // namespace

namespace flipk {
bool handle_particles(flip_handle* h, PartView* p, long long* np, cudaStream_t* s);
}

extern "C" {

void flip_surface_default_params(const flip_params* p, flip_surface_params* out) {
  if (!out) return;
  std::memset(out, 0, sizeof(*out));
  if (!p) return;
  for (int a = 0; a < 3; ++a) {
    out->n[a] = p->n[a];
    out->origin[a] = 0.0;
  }
  out->h = p->dx;
  out->radius = 0.5 * p->dx;
  out->search_radius = 2.0 * p->dx;
  out->iso = 0.0;
}

int flip_surface_create(const flip_surface_params* sp, void* stream, flip_surface** out) {
  if (!sp || !out) return sfail(FLIP_E_ARG, "params or out is NULL");
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (sp->n[a] < 1 || sp->n[a] > 1024) return sfail(FLIP_E_ARG, "n must be in [1, 1024]");
  if (!(sp->h > 0.0) || !std::isfinite(sp->h)) return sfail(FLIP_E_ARG, "h must be > 0");
  if (!(sp->search_radius > 0.0) || !std::isfinite(sp->search_radius))
    return sfail(FLIP_E_ARG, "search_radius must be > 0");
  if (!(sp->radius >= 0.0) || !(sp->radius < sp->search_radius))
    return sfail(FLIP_E_ARG, "radius must be in [0, search_radius)");
  if (!std::isfinite(sp->iso)) return sfail(FLIP_E_ARG, "iso must be finite");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(sp->origin[a])) return sfail(FLIP_E_ARG, "origin must be finite");
  {
    // particle bins (edge search_radius / 2) are indexed in 32 bits
    const double bb = (double)(0.5f * (float)sp->search_radius);  // the bin edge used below
    double nbins = 1.0;
    for (int a = 0; a < 3; ++a)
      nbins *= std::ceil((sp->n[a] * sp->h + 2.0 * sp->search_radius) / bb) + 1.0;
    if (!(nbins <= 2147483647.0))
      return sfail(FLIP_E_ARG, "bin grid too large (over 2^31 bins): search_radius is too small "
                               "for the sampling grid");
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return sfail(FLIP_E_NOGPU, "no CUDA device");
  if (int rc = ensure_table()) return rc;
  flip_surface* s = new (std::nothrow) flip_surface;
  if (!s) return sfail(FLIP_E_OOM, "host allocation failed");
  s->prm = *sp;
  SGrid& g = s->g;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = sp->n[a];
    g.c[a] = sp->n[a] + 1;
    g.o[a] = (float)sp->origin[a];
  }
  g.ncorners = (long long)g.c[0] * g.c[1] * g.c[2];
  g.h = (float)sp->h;
  g.iso = (float)sp->iso;
  SBins& B = s->B;
  B.R = (float)sp->search_radius;
  B.R2 = B.R * B.R;
  B.inv_R2 = 1.0f / B.R2;
  B.r = (float)sp->radius;
  B.b = 0.5f * B.R;
  B.inv_b = 1.0f / B.b;
  B.nbins = 1;
  for (int a = 0; a < 3; ++a) {
    B.o[a] = g.o[a] - B.R;
    B.nb[a] = (int)std::ceil((sp->n[a] * sp->h + 2.0 * sp->search_radius) / B.b) + 1;
    B.nbins *= B.nb[a];
  }
  int rc = FLIP_OK;
  auto step = [&](cudaError_t e, const char* what) {
    if (rc == FLIP_OK && e != cudaSuccess) rc = scuda(e, what);
  };
  if (stream) {
    s->stream = static_cast<cudaStream_t>(stream);
  } else {
    step(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    s->own_stream = rc == FLIP_OK;
  }
  const long long nc = g.ncorners;
  step(cudaMalloc(&s->phi, sizeof(float) * nc), "cudaMalloc(phi)");
  step(cudaMalloc(&s->voff, sizeof(unsigned int) * nc), "cudaMalloc(voff)");
  step(cudaMalloc(&s->toff, sizeof(unsigned int) * nc), "cudaMalloc(toff)");
  step(cudaMalloc(&s->code, sizeof(uint16_t) * nc), "cudaMalloc(code)");
  step(cudaMalloc(&s->bin_count, sizeof(unsigned int) * B.nbins), "cudaMalloc(bins)");
  step(cudaMalloc(&s->bin_start, sizeof(unsigned int) * (B.nbins + 1)), "cudaMalloc(bins)");
  step(cudaMallocHost(&s->htotal, sizeof(u64)), "cudaMallocHost");
  if (rc == FLIP_OK) {
    const long long ntiles = (std::max(nc, B.nbins + 1) + SC_TILE - 1) / SC_TILE;
    rc = realloc_n(s->tile, ntiles + 1);
    if (rc == FLIP_OK) s->tile_cap = ntiles + 1;
  }
  if (rc == FLIP_OK) {
    // corners start outside: phi = R - r until a field is computed or set
    k_fill<<<blocks_for(nc, 256), 256, 0, s->stream>>>(s->phi, nc, B.R - B.r);
    step(cudaGetLastError(), "k_fill");
    step(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
  }
  if (rc != FLIP_OK) {
    flip_surface_destroy(s);
    return rc;
  }
  *out = s;
  return FLIP_OK;
}

int flip_surface_case_table(uint8_t ntri[256], uint8_t* tri) {
  if (!ntri || !tri) return sfail(FLIP_E_ARG, "NULL output");
  static_assert(MC_MAXT == FLIP_SURF_MAX_TRI, "table width");
  McTable T;
  if (!build_table(T)) return sfail(FLIP_E_CUDA, "marching-cubes table generation failed");
  std::memcpy(ntri, T.ntri, sizeof(T.ntri));
  std::memcpy(tri, T.tri, sizeof(T.tri));
  return FLIP_OK;
}

void flip_surface_destroy(flip_surface* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (void* p : {(void*)s->phi, (void*)s->bin_count, (void*)s->bin_start, (void*)s->pbin,
                  (void*)s->prank, (void*)s->pos, (void*)s->voff, (void*)s->toff,
                  (void*)s->code, (void*)s->tile, (void*)s->vert, (void*)s->nrm,
                  (void*)s->vedge, (void*)s->tri, (void*)s->tw})
    sfree(p);
  if (s->htotal) cudaFreeHost(s->htotal);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

int flip_surface_sdf(flip_surface* s, flip_handle* h) {
  if (!s || !h) return sfail(FLIP_E_ARG, "surface or handle is NULL");
  PartView P;
  long long np = 0;
  cudaStream_t hs = nullptr;
  if (!handle_particles(h, &P, &np, &hs)) return sfail(FLIP_E_ARG, "bad handle");
  // order after the handle's queued work
  cudaEvent_t ev;
  SURF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  SURF_CUDA(cudaEventRecord(ev, hs));
  SURF_CUDA(cudaStreamWaitEvent(s->stream, ev, 0));
  cudaEventDestroy(ev);
  if (np > s->part_cap) {
    s->part_cap = 0;
    if (int rc = realloc_n(s->pbin, np)) return rc;
    if (int rc = realloc_n(s->prank, np)) return rc;
    if (int rc = realloc_n(s->pos, np)) return rc;
    s->part_cap = np;
  }
  const cudaStream_t st = s->stream;
  SURF_CUDA(cudaMemsetAsync(s->bin_count, 0, sizeof(unsigned int) * s->B.nbins, st));
  if (np > 0) {
    k_sbin_count<<<blocks_for(np, 256), 256, 0, st>>>(P, np, s->B, s->bin_count, s->pbin,
                                                      s->prank);
  }
  BinScan bs{s->bin_count, s->bin_start, s->B.nbins};
  tile_scan(bs, s->B.nbins + 1, s->tile, s->tile + s->tile_cap - 1, st);
  if (np > 0) {
    k_sbin_scatter<<<blocks_for(np, 256), 256, 0, st>>>(P, np, s->pbin, s->prank, s->bin_start,
                                                        s->pos);
  }
  k_sdf<<<sdf_blocks(), SDF_THREADS, 0, st>>>(s->g, s->B, s->bin_start, s->pos, s->phi);
  SURF_CUDA(cudaGetLastError());
  return FLIP_OK;
}

int flip_surface_set_field(flip_surface* s, const float* phi, int32_t src_is_device) {
  if (!s || !phi) return sfail(FLIP_E_ARG, "surface or phi is NULL");
  SURF_CUDA(cudaMemcpyAsync(s->phi, phi, sizeof(float) * s->g.ncorners,
                            src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s->stream));
  SURF_CUDA(cudaStreamSynchronize(s->stream));
  return FLIP_OK;
}

int flip_surface_mesh(flip_surface* s, int64_t* n_vertices, int64_t* n_triangles) {
  if (!s) return sfail(FLIP_E_ARG, "surface is NULL");
  const cudaStream_t st = s->stream;
  const long long nc = s->g.ncorners;
  McScan f{s->g, s->phi, s->voff, s->toff, s->code, nullptr, nullptr};
  const long long ntiles = (nc + SC_TILE - 1) / SC_TILE;
  u64* total = s->tile + s->tile_cap - 1;
  k_tile_reduce<McScan><<<(unsigned)ntiles, SC_THREADS, 0, st>>>(f, nc, s->tile);
  k_tile_scan<<<1, SC_THREADS, 0, st>>>(s->tile, ntiles, total);
  SURF_CUDA(cudaMemcpyAsync(s->htotal, total, sizeof(u64), cudaMemcpyDeviceToHost, st));
  SURF_CUDA(cudaStreamSynchronize(st));
  // Vertices (crossing edges, at most 3 per corner) never exceed 2^32, so the low
  // word is exact.  Each crossing edge is a vertex of one fan polygon in each of at
  // most 4 cubes, and a k-gon gives k - 2 triangles, so triangles <= 4 * vertices:
  // below 2^31 vertices / 4 the high word cannot have wrapped either.
  const long long nv = (long long)(*s->htotal & 0xffffffffull);
  const long long nt = (long long)(*s->htotal >> 32);
  if (4 * nv >= (1ll << 31) || nt >= (1ll << 31))
    return sfail(FLIP_E_SIZE, "mesh too large for int32 indices (2^29 vertices or more)");
  if (nv > s->vcap) {
    s->vcap = 0;
    s->nv = 0;
    if (int rc = realloc_n(s->vert, 3 * nv)) return rc;
    if (int rc = realloc_n(s->nrm, 3 * nv)) return rc;
    if (int rc = realloc_n(s->vedge, nv)) return rc;
    s->vcap = nv;
  }
  if (nt > s->tcap) {
    s->tcap = 0;
    s->nt = 0;
    if (int rc = realloc_n(s->tri, 3 * nt)) return rc;
    if (int rc = realloc_n(s->tw, 3 * nt)) return rc;
    s->tcap = nt;
  }
  f.vert = s->vert;
  f.vedge = s->vedge;
  k_tile_apply<McScan><<<(unsigned)ntiles, SC_THREADS, 0, st>>>(f, nc, s->tile);
  if (nt > 0) {
    k_mc_triangles<<<blocks_for(nc, 256), 256, 0, st>>>(s->g, s->voff, s->toff, s->code, s->tri);
    k_mc_tri_weights<<<blocks_for(nt, 256), 256, 0, st>>>(nt, s->vert, s->tri, s->tw);
  }
  if (nv > 0)
    k_mc_normals<<<blocks_for(nv, 256), 256, 0, st>>>(s->g, nv, s->vedge, s->toff, s->code,
                                                      s->tri, s->tw, s->nrm);
  SURF_CUDA(cudaGetLastError());
  SURF_CUDA(cudaStreamSynchronize(st));
  s->nv = nv;
  s->nt = nt;
  if (n_vertices) *n_vertices = nv;
  if (n_triangles) *n_triangles = nt;
  return FLIP_OK;
}

size_t flip_surface_bytes(const flip_surface* s, flip_surface_field which) {
  if (!s) return 0;
  switch (which) {
    case FLIP_SURF_FIELD: return sizeof(float) * (size_t)s->g.ncorners;
    case FLIP_SURF_VERTICES: case FLIP_SURF_NORMALS: return 12 * (size_t)s->nv;
    case FLIP_SURF_TRIANGLES: return 12 * (size_t)s->nt;
    case FLIP_SURF_VERTEX_EDGE: return 8 * (size_t)s->nv;
    default: return 0;
  }
}

int flip_surface_read(flip_surface* s, flip_surface_field which, void* dst, size_t bytes,
                      int32_t dst_is_device) {
  if (!s) return sfail(FLIP_E_ARG, "surface is NULL");
  if (which < FLIP_SURF_FIELD || which > FLIP_SURF_VERTEX_EDGE)
    return sfail(FLIP_E_ARG, "unknown field");
  const size_t need = flip_surface_bytes(s, which);
  if (bytes != need) return sfail(FLIP_E_SIZE, "bytes must be " + std::to_string(need));
  if (need == 0) return FLIP_OK;
  if (!dst) return sfail(FLIP_E_ARG, "dst is NULL");
  const void* src = nullptr;
  switch (which) {
    case FLIP_SURF_FIELD: src = s->phi; break;
    case FLIP_SURF_VERTICES: src = s->vert; break;
    case FLIP_SURF_NORMALS: src = s->nrm; break;
    case FLIP_SURF_TRIANGLES: src = s->tri; break;
    case FLIP_SURF_VERTEX_EDGE: src = s->vedge; break;
  }
  SURF_CUDA(cudaMemcpyAsync(dst, src, bytes,
                            dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s->stream));
  SURF_CUDA(cudaStreamSynchronize(s->stream));
  return FLIP_OK;
}

}  // extern "C"
