// k_g2p.cu — grid-to-particle transfer with the PIC/FLIP blend (Sec. 2.1.4,
// 3.1.8), forward-Euler advection and the wall clamp (Sec. 3.1.3), fused with
// the histogram of the next step's binning.
//
// One thread per particle, particles in cell-sorted order.  For every
// component the eight face nodes around the particle are read once: u_old (the
// P2G result) and the projected u_new (Eq. 5, evaluated on the fly from u_old
// and the pressure, so u_new is never stored).  The particle receives
//     U = interp(u_new),  dU = interp(u_new - u_old)
//     v <- r (v + dU) + (1 - r) U
//     x <- clamp(x + dt v, skin, n dx - skin)     (or dt U with grid advection)
// and then the key of the cell it moved to plus its rank there (an atomic on
// the histogram), which is all the next step's counting sort needs.
#include "flip_kernels.cuh"

namespace flipk {

constexpr int G2P_THREADS = 256;

template <int D, bool PAIR>
__device__ __forceinline__ void g2p_comp(const Grid& g, const StepConsts& K,
                                         const float* __restrict__ uo,
                                         const float* __restrict__ p32,
                                         const float2* __restrict__ pff, float px, float py,
                                         float pz, int ci, int cj, int ck, float& U, float& dU) {
  const AxisW ax = axis_weights<D, 0>(px, g.inv_dx, ci, g.nx);
  const AxisW ay = axis_weights<D, 1>(py, g.inv_dx, cj, g.ny);
  const AxisW az = axis_weights<D, 2>(pz, g.inv_dx, ck, g.nz);
  const int a0 = (D == 0) ? ci : ci - 1 + ax.off;
  const int b0 = (D == 1) ? cj : cj - 1 + ay.off;
  const int c0 = (D == 2) ? ck : ck - 1 + az.off;
  const float wx[2] = {ax.w0, ax.w1}, wy[2] = {ay.w0, ay.w1}, wz[2] = {az.w0, az.w1};
  const int FX = g.nx + (D == 0), FY = g.ny + (D == 1);
  float su = 0.0f, sd = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const float wyz = __fmul_rn(wy[dy], wz[dz]);
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float w = __fmul_rn(wx[dx], wyz);
        const int a = a0 + dx, b = b0 + dy, c = c0 + dz;
        const float uov = __ldg(uo + (a + FX * (b + FY * c)));
        const float un = face_unew<D, PAIR>(g, K, uov, a, b, c, p32, pff);
        su = __fmaf_rn(w, un, su);
        sd = __fmaf_rn(w, __fsub_rn(un, uov), sd);
      }
    }
  U = su;
  dU = sd;
}

template <bool PAIR>
__global__ void __launch_bounds__(G2P_THREADS) k_g2p(const Grid g, const StepConsts K,
                                                     const PartView P, const BinView B,
                                                     const float* __restrict__ uo0,
                                                     const float* __restrict__ uo1,
                                                     const float* __restrict__ uo2,
                                                     const float* __restrict__ p32,
                                                     const float2* __restrict__ pff,
                                                     DevStats* st, long long np) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float speed2 = 0.0f;
  if (i < np) {
    float x = P.x[i], y = P.y[i], z = P.z[i];
    const float vp[3] = {P.u[i], P.v[i], P.w[i]};
    const int ci = cell_of(x, g.inv_dx, g.nx);
    const int cj = cell_of(y, g.inv_dx, g.ny);
    const int ck = cell_of(z, g.inv_dx, g.nz);
    float U[3], dU[3];
    g2p_comp<0, PAIR>(g, K, uo0, p32, pff, x, y, z, ci, cj, ck, U[0], dU[0]);
    g2p_comp<1, PAIR>(g, K, uo1, p32, pff, x, y, z, ci, cj, ck, U[1], dU[1]);
    g2p_comp<2, PAIR>(g, K, uo2, p32, pff, x, y, z, ci, cj, ck, U[2], dU[2]);
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
    P.x[i] = x;
    P.y[i] = y;
    P.z[i] = z;
    P.u[i] = vn[0];
    P.v[i] = vn[1];
    P.w[i] = vn[2];
    speed2 = vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2];
    const unsigned int key = brick_key(g, cell_of(x, g.inv_dx, g.nx), cell_of(y, g.inv_dx, g.ny),
                                       cell_of(z, g.inv_dx, g.nz));
    B.key[i] = key;
    B.rank[i] = atomicAdd(B.cell_count + key, 1u);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) speed2 = fmaxf(speed2, __shfl_xor_sync(0xffffffffu, speed2, o));
  if ((threadIdx.x & 31) == 0 && speed2 > 0.0f)
    atomicMax(&st->max_speed_bits, __float_as_uint(sqrtf(speed2)));
}

void launch_g2p(const Grid& g, const StepConsts& k, const PartView& p, const BinView& b,
                const float* const uo[3], const float* p32, const float2* pff, DevStats* st,
                long long np, cudaStream_t s) {
  if (np <= 0) return;
  const unsigned int blocks = (unsigned int)((np + G2P_THREADS - 1) / G2P_THREADS);
  if (pff)
    k_g2p<true><<<blocks, G2P_THREADS, 0, s>>>(g, k, p, b, uo[0], uo[1], uo[2], p32, pff, st, np);
  else
    k_g2p<false><<<blocks, G2P_THREADS, 0, s>>>(g, k, p, b, uo[0], uo[1], uo[2], p32, pff, st, np);
}

}  // namespace flipk
