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
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/flip.h"
#include "flip_api_internal.cuh"
#include "flip_kernels.cuh"

using namespace flipk;

namespace {

constexpr long long kMaxCells = FLIP_NOALLOC_MAX_CELLS;
constexpr unsigned int kMaxBricks = FLIP_NOALLOC_MAX_BRICKS;
constexpr int kMaxBlocks = 2048;  // reduction slots: one per co-resident solver CTA
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

// The array's device address per device, with the id of the context it was looked
// up in: a context created after cudaDeviceReset may place the array elsewhere, so
// a cached address is only used while the same context is current.
struct ScratchAddr {
  char* ptr = nullptr;
  unsigned long long ctx = 0;
};
std::mutex g_mu;
ScratchAddr g_scratch[kMaxDevices];

// Id of the current context (unique per context over the process's life), 0 when
// none is current or the driver does not provide one.  Driver entry points are
// taken through the runtime, so the library links no driver library.
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = (PFN_cuCtxGetCurrent_v4000)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (PFN_cuCtxGetId_v12000)f;
    cudaGetLastError();
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

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
  // The same checks as flip_solve_pressure, so both refuse the same inputs.
  if (int rc = api_check_params(params, false)) return rc;
  if (params->precision != FLIP_PREC_FP32)
    return err(FLIP_E_ARG, "runs the FP32 solver only");
  if (!type || !b || !p) return err(FLIP_E_ARG, "type, b and p must be device pointers");
  const long long nc = (long long)params->n[0] * params->n[1] * params->n[2];
  const Grid g = api_make_grid(*params);
  const unsigned long long nb = (unsigned long long)g.bx * g.by * g.bz;
  // Sizes beyond the fixed scratch are refused before any device work.
  if (nc > kMaxCells || nb > kMaxBricks)
    return err(FLIP_E_SIZE, "grid of " + std::to_string(nc) + " cells / " + std::to_string(nb) +
                                " bricks exceeds the fixed scratch (" + std::to_string(kMaxCells) +
                                " cells, " + std::to_string(kMaxBricks) + " bricks)");
  if (int rc = api_check_device()) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return err(FLIP_E_NOGPU, "no usable CUDA device");
  }
  char* base = nullptr;
  {
    // Set-up per device (and per context of that device), with the device
    // current: the host-side name of the array is only a stand-in, so its device
    // address is looked up here.  The first call on a device does it.
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr& sa = g_scratch[dev];
    const unsigned long long ctx = current_context_id();
    if (!sa.ptr || ctx == 0 || ctx != sa.ctx) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        sa = ScratchAddr{};
        return err(FLIP_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      sa.ptr = (char*)ptr;
      sa.ctx = current_context_id();  // the look-up made the device's context current
    }
    base = sa.ptr;
  }
  int blocks = 0, sms = 0;
  if (cudaError_t e = pcg_max_blocks(&blocks, &sms); e != cudaSuccess) {
    cudaGetLastError();
    return err(FLIP_E_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
  }
  if (blocks > kMaxBlocks)
    return err(FLIP_E_CUDA, "the device holds " + std::to_string(blocks) +
                                " co-resident solver CTAs, more than the fixed scratch's " +
                                std::to_string(kMaxBlocks) + " reduction slots");

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
    api_fill_pcg_tables(a, *params);
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
    a.timeout_ns = api_barrier_wait_ns();
    e = launch_pcg(a, false, blocks, s);
  }
  DevStats hst{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, st, sizeof(DevStats), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(FLIP_E_CUDA, cudaGetErrorString(e));
  if (iterations) *iterations = hst.cg_iters;
  if (rel_residual) *rel_residual = hst.rel_res;
  return api_status_to_code(hst.status);
}
