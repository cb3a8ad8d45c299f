// k_diag.cu — diagnostics over the particle set: the total mechanical energy
// the paper tracks to compare its CPU and GPU runs (Sec. 4, Fig. 10).
//
// With particle mass m and body acceleration g,
//   kinetic   = m/2 * sum_p |v_p|^2
//   potential = -m * g . sum_p x_p       (zero at the origin)
// The potential needs only the three position sums.  Every thread keeps the
// four sums (|v|^2, x, y, z) as float pairs: squares are split exactly by an
// FMA and added with TwoSum, so a thread's pair carries the exact sum of its
// particles' terms up to ~2^-48 relative, without FP64 arithmetic per particle.
// The pairs are then summed in FP64, per CTA and then over CTAs in a fixed
// order.  Particles are read as 16-byte vectors: 24 bytes per particle, one pass.
#include <algorithm>

#include "flip_kernels.cuh"

namespace flipk {

constexpr int DIAG_THREADS = 1024;

__device__ __forceinline__ void energy_terms(FF (&a)[4], float x, float y, float z, float u,
                                             float v, float w) {
  a[0].add_prod(u, u);
  a[0].add_prod(v, v);
  a[0].add_prod(w, w);
  a[1].add(x);
  a[2].add(y);
  a[3].add(z);
}

__global__ void __launch_bounds__(DIAG_THREADS) k_energy_partial(const PartView p, long long np,
                                                                  double* __restrict__ partials) {
  __shared__ double scratch[32 * 4];
  FF a[4];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nv = np >> 2;  // whole 4-particle vectors (arrays are 256-byte aligned)
  const float4* x4 = reinterpret_cast<const float4*>(p.x);
  const float4* y4 = reinterpret_cast<const float4*>(p.y);
  const float4* z4 = reinterpret_cast<const float4*>(p.z);
  const float4* u4 = reinterpret_cast<const float4*>(p.u);
  const float4* v4 = reinterpret_cast<const float4*>(p.v);
  const float4* w4 = reinterpret_cast<const float4*>(p.w);
  for (long long i = t0; i < nv; i += stride) {
    const float4 X = __ldcs(x4 + i), Y = __ldcs(y4 + i), Z = __ldcs(z4 + i);
    const float4 U = __ldcs(u4 + i), V = __ldcs(v4 + i), W = __ldcs(w4 + i);
    energy_terms(a, X.x, Y.x, Z.x, U.x, V.x, W.x);
    energy_terms(a, X.y, Y.y, Z.y, U.y, V.y, W.y);
    energy_terms(a, X.z, Y.z, Z.z, U.z, V.z, W.z);
    energy_terms(a, X.w, Y.w, Z.w, U.w, V.w, W.w);
  }
  for (long long i = 4 * nv + t0; i < np; i += stride)
    energy_terms(a, p.x[i], p.y[i], p.z[i], p.u[i], p.v[i], p.w[i]);
  double v[4] = {a[0].value(), a[1].value(), a[2].value(), a[3].value()};
  block_sum<4>(v, scratch);
  if (threadIdx.x < 4) partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = v[threadIdx.x];
}

// Thread q sums quantity q over the CTAs in CTA order.
__global__ void k_energy_final(const double* __restrict__ partials, int nblocks,
                               double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= 4) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[(size_t)q * nblocks + b];
  out[q] = s;
}

__global__ void k_cfl_dt(DevStats* st, double g0, double g1, double g2, double dt_max,
                         double alpha_dx) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float vmax = __uint_as_float(st->max_speed_bits);
  double dt = dt_max;
  if (vmax > 0.0f) dt = fmin(dt_max, alpha_dx / (double)vmax);
  st->dt_cur = dt;
  st->dyn[0] = (float)(g0 * dt);
  st->dyn[1] = (float)(g1 * dt);
  st->dyn[2] = (float)(g2 * dt);
  st->dyn[3] = (float)dt;
}

void launch_cfl_dt(DevStats* st, const double g[3], double dt_max, double alpha_dx,
                   cudaStream_t s) {
  k_cfl_dt<<<1, 32, 0, s>>>(st, g[0], g[1], g[2], dt_max, alpha_dx);
}

template <class T>
__global__ void k_scale(T* out, long long n, double f) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (T)((double)out[i] * f);
}

void launch_scale(float* out, long long n, double f, cudaStream_t s) {
  if (n > 0) k_scale<float><<<(unsigned)std::min<long long>((n + 255) / 256, 65535), 256, 0, s>>>(out, n, f);
}
void launch_scale(double* out, long long n, double f, cudaStream_t s) {
  if (n > 0) k_scale<double><<<(unsigned)std::min<long long>((n + 255) / 256, 65535), 256, 0, s>>>(out, n, f);
}

int energy_blocks(int sm_count) { return sm_count > 0 ? sm_count : 1; }

void launch_energy(const PartView& p, long long np, double* partials, int nblocks, double* out,
                   cudaStream_t s) {
  k_energy_partial<<<nblocks, DIAG_THREADS, 0, s>>>(p, np, partials);
  k_energy_final<<<1, 32, 0, s>>>(partials, nblocks, out);
}

}  // namespace flipk
