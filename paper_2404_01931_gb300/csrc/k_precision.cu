// k_precision.cu — the two extended-precision steps of the mixed-precision solve,
// run on caller data so that their arithmetic can be checked against exact sums:
//   flip_dot_f32:        the CG's dot product (float-pair accumulation per
//                        thread, float-pair sums over warps and CTAs, FP64 at the
//                        end), the reduction every solve of this library uses;
//   flip_residual_pairs: the refinement's residual b - A x (Sec. 3.1.7's 7-point
//                        row) with x, b and the scale as float pairs, the
//                        function the mixed-mode multigrid solve calls per cell.
// Both call the same device functions as the solvers (FF::add_prod, cta_sum,
// publish/gather, residual_pair_cell); only the indexing is plain here.
#include <cuda_runtime.h>

#include <string>

#include "../../include/flip.h"
#include "flip_api_internal.cuh"
#include "pcg_common.cuh"

namespace flipk {
namespace {

// Each CTA takes a contiguous slice of [0, n) (a multiple of 32 long, like the
// solver's share of cells) and its threads stride through it.
__global__ void __launch_bounds__(PCG_THREADS, 1) k_dot_partial(const __grid_constant__ PcgArgs A,
                                                              const float* __restrict__ a,
                                                              const float* __restrict__ b,
                                                              long long n) {
  __shared__ Shared sh;
  team_enter(blockIdx.x, gridDim.x);
  long long per = (n + gridDim.x - 1) / gridDim.x;
  per = (per + 31) & ~31LL;
  const long long lo = min(n, (long long)blockIdx.x * per), hi = min(n, lo + per);
  FF acc;
  for (long long i = lo + threadIdx.x; i < hi; i += PCG_THREADS) acc.add_prod(a[i], b[i]);
  F2 v[1] = {f2_of(acc)};
  publish<1>(A, 0, v, sh);
}

// One warp adds the published pairs in the solver's order (gather) and writes
// the FP64 value.
__global__ void k_dot_final(const __grid_constant__ PcgArgs A, unsigned int parts, double* out) {
  __shared__ Shared sh;
  team_enter(0, parts);
  double s[1];
  gather<1>(A, 0, s, sh);
  if (threadIdx.x == 0) *out = s[0];
}

__global__ void k_residual_pairs(const Grid g, float s_hi, float s_lo,
                                 const uint8_t* __restrict__ type, const float* __restrict__ xh,
                                 const float* __restrict__ xl, const float* __restrict__ bh,
                                 const float* __restrict__ bl, float* __restrict__ rh,
                                 float* __restrict__ rl) {
  const long long nc = (long long)g.nx * g.ny * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    float2 r = make_float2(0.0f, 0.0f);
    if (type[c] == 1) {
      const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((long long)g.nx * g.ny));
      const long long sy = g.nx, sz = (long long)g.nx * g.ny;
      // neighbours in the solver's order: -x, +x, -y, +y, -z, +z
      const bool in[6] = {i > 0, i < g.nx - 1, j > 0, j < g.ny - 1, k > 0, k < g.nz - 1};
      const long long off[6] = {-1, 1, -sy, sy, -sz, sz};
      float2 xn[6];
      unsigned int fluid = 0;
      int cnt = 0;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const long long nb = in[q] ? c + off[q] : c;
        xn[q] = make_float2(xh[nb], xl[nb]);
        cnt += in[q];
        if (in[q] && type[nb] == 1) fluid |= 1u << q;
      }
      r = residual_pair_cell(make_float2(bh[c], bl[c]), make_float2(xh[c], xl[c]), xn, fluid, cnt,
                             s_hi, s_lo);
    }
    rh[c] = r.x;
    rl[c] = r.y;
  }
}

}  // namespace
}  // namespace flipk

using namespace flipk;

void flip_set_last_error_(const std::string& msg);

extern "C" {

int flip_dot_f32(const float* a, const float* b, int64_t n, double* out, void* stream) {
  auto err = [](int code, const std::string& msg) {
    flip_set_last_error_("flip_dot_f32: " + msg);
    return code;
  };
  if (!out) return err(FLIP_E_ARG, "out is NULL");
  if (n < 0 || n > 2147483647LL) return err(FLIP_E_ARG, "n must be in [0, 2^31-1]");
  if (n > 0 && (!a || !b)) return err(FLIP_E_ARG, "a and b must be device pointers");
  if (int rc = api_check_device()) return rc;
  int blocks = 0, sms = 0;
  if (cudaError_t e = pcg_max_blocks(&blocks, &sms); e != cudaSuccess) {
    cudaGetLastError();
    return err(FLIP_E_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
  }
  const cudaStream_t s = (cudaStream_t)stream;
  void* scratch = nullptr;  // the CTAs' pairs, then the result
  const size_t part_bytes = sizeof(double) * (size_t)blocks;
  cudaError_t e = cudaMallocAsync(&scratch, part_bytes + sizeof(double), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return err(e == cudaErrorMemoryAllocation ? FLIP_E_OOM : FLIP_E_CUDA,
               std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
  PcgArgs A{};
  A.partials = (double*)scratch;
  double* d_out = (double*)((char*)scratch + part_bytes);
  k_dot_partial<<<blocks, PCG_THREADS, 0, s>>>(A, a, b, (long long)n);
  k_dot_final<<<1, 32, 0, s>>>(A, (unsigned)blocks, d_out);
  e = cudaGetLastError();
  double h = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_out, sizeof(double), cudaMemcpyDeviceToHost, s);
  const cudaError_t e2 = cudaFreeAsync(scratch, s);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = e3;
  if (e != cudaSuccess) return err(FLIP_E_CUDA, cudaGetErrorString(e));
  *out = h;
  return FLIP_OK;
}

int flip_residual_pairs(const flip_params* params, const uint8_t* type, const float* x_hi,
                        const float* x_lo, const float* b_hi, const float* b_lo, float* r_hi,
                        float* r_lo, void* stream) {
  auto err = [](int code, const std::string& msg) {
    flip_set_last_error_("flip_residual_pairs: " + msg);
    return code;
  };
  if (int rc = api_check_params(params, false)) return rc;
  if (!type || !x_hi || !x_lo || !b_hi || !b_lo || !r_hi || !r_lo)
    return err(FLIP_E_ARG, "every array must be a device pointer");
  if (int rc = api_check_device()) return rc;
  const Grid g = api_make_grid(*params);
  PcgArgs t{};
  api_fill_pcg_tables(t, *params);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaStream_t s = (cudaStream_t)stream;
  k_residual_pairs<<<4 * (sms > 0 ? sms : 1), 256, 0, s>>>(g, t.s, t.s_lo, type, x_hi, x_lo, b_hi,
                                                          b_lo, r_hi, r_lo);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(FLIP_E_CUDA, cudaGetErrorString(e));
  return FLIP_OK;
}

}  // extern "C"
