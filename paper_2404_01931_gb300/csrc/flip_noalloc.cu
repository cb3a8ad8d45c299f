// flip_noalloc.cu — flip_solve_pressure_noalloc: the standalone pressure solve
// without any device allocation.
//
// Some callers cannot allocate device memory while they run: a plug-in inside a
// host application whose memory is owned by that application's allocator under a
// fixed budget, or a latency-critical loop where cudaMalloc/cudaFree are not
// allowed because they can synchronise the whole device.  This entry point lets
// them run the same PCG as flip_solve_pressure: its scratch (CG vectors, brick
// list, reduction slots, barrier, statistics) lives in one file-scope device
// array of fixed size, reserved when the library's device code is loaded and held
// by every GPU that loads it until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/flip.h"
#include "flip_kernels.cuh"

using namespace flipk;

namespace {

constexpr long long kMaxCells = FLIP_NOALLOC_MAX_CELLS;
constexpr unsigned int kMaxBricks = FLIP_NOALLOC_MAX_BRICKS;
constexpr int kMaxBlocks = 2048;
constexpr int kMaxDevices = 64;

constexpr size_t kAlign = 256;
constexpr size_t al(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of the sub-buffers inside the array.
constexpr size_t kOffR = 0;
constexpr size_t kOffPa = kOffR + al(sizeof(float) * kMaxCells);
constexpr size_t kOffPb = kOffPa + al(sizeof(float) * kMaxCells);
constexpr size_t kOffQ = kOffPb + al(sizeof(float) * kMaxCells);
constexpr size_t kOffBrickFluid = kOffQ + al(sizeof(float) * kMaxCells);
constexpr size_t kOffActive = kOffBrickFluid + al(sizeof(unsigned int) * kMaxBricks);
constexpr size_t kOffPartials = kOffActive + al(sizeof(unsigned int) * kMaxBricks);
constexpr size_t kOffBar = kOffPartials + al(sizeof(double) * PCG_SLOTS * kMaxBlocks);
constexpr size_t kOffStats = kOffBar + al(sizeof(unsigned int) * BAR_WORDS);
constexpr size_t kScratchBytes = kOffStats + al(sizeof(DevStats));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
char* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

// Records the message returned by flip_last_error (defined with the other entry points).
void flip_set_last_error_(const std::string& msg);

extern "C" int flip_solve_pressure_noalloc(const flip_params* params, const uint8_t* type,
                                           const float* b, float* p, void* stream,
                                           int32_t* iterations, double* rel_residual) {
  auto err = [](int code, const std::string& msg) {
    flip_set_last_error_("flip_solve_pressure_noalloc: " + msg);
    return code;
  };
  if (!params || !type || !b || !p) return err(FLIP_E_ARG, "params, type, b and p are required");
  for (int a = 0; a < 3; ++a)
    if (params->n[a] < 2 || params->n[a] > 2048) return err(FLIP_E_ARG, "n[a] must be in [2, 2048]");
  if (params->precision != FLIP_PREC_FP32) return err(FLIP_E_ARG, "FP32 solver only");
  if (!(params->dx > 0.0) || !(params->dt > 0.0) || !(params->rho > 0.0) ||
      !(params->cg_tol > 0.0) || params->cg_max_iter < 1)
    return err(FLIP_E_ARG, "dx, dt, rho, cg_tol must be > 0 and cg_max_iter >= 1");
  const long long nc = (long long)params->n[0] * params->n[1] * params->n[2];
  Grid g{};
  g.nx = params->n[0];
  g.ny = params->n[1];
  g.nz = params->n[2];
  g.bx = (g.nx + BRICK - 1) / BRICK;
  g.by = (g.ny + BRICK - 1) / BRICK;
  g.bz = (g.nz + BRICK - 1) / BRICK;
  g.inv_dx = (float)(1.0 / params->dx);
  g.dx = (float)params->dx;
  const unsigned long long nb = (unsigned long long)g.bx * g.by * g.bz;
  // Sizes beyond the fixed scratch are refused before any device work.
  if (nc > kMaxCells || nb > kMaxBricks)
    return err(FLIP_E_SIZE, "grid of " + std::to_string(nc) + " cells / " + std::to_string(nb) +
                                " bricks exceeds the fixed scratch (" + std::to_string(kMaxCells) +
                                " cells, " + std::to_string(kMaxBricks) + " bricks)");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return err(FLIP_E_NOGPU, "no usable CUDA device");
  }
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      major != 10 || minor != 3)
    return err(FLIP_E_NOGPU, "built for sm_103a (GB300)");
  char* base = nullptr;
  {
    // One-time set-up per device, with that device current: the host-side name of
    // the array is only a stand-in, so its device address is looked up here.
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return err(FLIP_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_scratch_ptr[dev] = (char*)ptr;
    }
    base = g_scratch_ptr[dev];
  }
  int blocks = 0, sms = 0;
  if (pcg_max_blocks(&blocks, &sms) != cudaSuccess || blocks > kMaxBlocks)
    return err(FLIP_E_CUDA, "occupancy query failed");

  const cudaStream_t s = (cudaStream_t)stream;
  float* r = (float*)(base + kOffR);
  float* pa = (float*)(base + kOffPa);
  float* pb = (float*)(base + kOffPb);
  float* q = (float*)(base + kOffQ);
  unsigned int* bf = (unsigned int*)(base + kOffBrickFluid);
  unsigned int* act = (unsigned int*)(base + kOffActive);
  double* part = (double*)(base + kOffPartials);
  unsigned int* bar = (unsigned int*)(base + kOffBar);
  DevStats* st = (DevStats*)(base + kOffStats);

  // The array keeps the previous call's contents: clear what must start at zero
  // (statistics and status; the barrier counter is reset by k_zero_off_fluid).
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStats), s);
  if (e == cudaSuccess) {
    launch_zero_off_fluid(g, type, p, bar, s);
    launch_mark_bricks(g, type, bf, s);
    launch_compact_bricks(g, bf, act, st, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    PcgArgs a{};
    a.g = g;
    const double sc = params->dt / (params->rho * params->dx * params->dx);
    a.s = (float)sc;
    a.s64 = sc;
    for (int c = 0; c < 8; ++c) {
      a.diag_tab[c] = (float)(sc * c);
      a.minv_tab[c] = c > 0 ? (float)(1.0 / (sc * c)) : 0.0f;
    }
    a.type = type;
    a.active = act;
    a.n_active = &st->n_active;
    a.b32 = b;
    a.x32 = p;
    a.r = r;
    a.pa = pa;
    a.pb = pb;
    a.q = q;
    a.partials = part;
    a.bar = bar;
    a.status = &st->status;
    a.stats = st;
    a.tol = params->cg_tol;
    a.max_iter = params->cg_max_iter;
    a.check_singular = 1;
    a.timeout_ns = 5000000000ull;
    e = launch_pcg(a, false, blocks, s);
  }
  DevStats hst{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, st, sizeof(DevStats), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(FLIP_E_CUDA, cudaGetErrorString(e));
  if (iterations) *iterations = hst.cg_iters;
  if (rel_residual) *rel_residual = hst.rel_res;
  if (hst.status & DEV_TIMEOUT) return err(FLIP_E_TIMEOUT, "a device-side wait timed out");
  if (hst.status & DEV_SINGULAR) return err(FLIP_E_ARG, "every cell is fluid: A is singular");
  if (hst.status & DEV_NOT_CONVERGED) return err(FLIP_E_NOT_CONVERGED, "iteration cap reached");
  return FLIP_OK;
}
