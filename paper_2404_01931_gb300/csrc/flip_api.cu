// flip_api.cu — the C ABI of include/flip.h: handle lifetime, device memory,
// and the stream-ordered sequence of kernels that makes one FLIP step
// (Sec. 3 of the paper, order: bin -> P2G -> gravity/walls + divergence ->
// PCG -> G2P blend + advection).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/flip.h"
#include "flip_api_internal.cuh"
#include "flip_kernels.cuh"

using namespace flipk;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? FLIP_E_OOM : FLIP_E_CUDA;
  return fail(code, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                        cudaGetErrorString(e) + ")");
}

#define FLIP_CUDA(call)                              \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// The same, for functions that return a count or -status.
#define FLIP_CUDA_NEG(call)                               \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return -cuda_fail(e_, #call);  \
  } while (0)

constexpr size_t kAlign = 256;

// Default limits of the bounded device-side waits: a grid barrier of the solve,
// and G2P's wait for a bulk copy of particles (flip_set_wait_timeout changes both).
constexpr unsigned long long kBarrierWaitNs = 5000000000ull;
constexpr unsigned long long kG2pWaitNs = 1000000000ull;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Carves sub-buffers out of one arena; first pass measures, second assigns.
struct Carver {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += align_up(sizeof(T) * std::max<size_t>(count, 1));
    return p;
  }
};

}  // namespace

struct flip_handle {
  flip_params prm;
  Grid g;
  StepConsts K;
  long long np = 0, ncells = 0, nkeys = 0, nf[3] = {0, 0, 0};
  long long cap = 0;          // particle capacity (np, or more when reseeding)
  long long steps_done = 0;   // steps taken (the reseeding generator's step index)
  long long serial = 0;       // creation number (distinguishes a handle reusing an address)
  unsigned int nbricks = 0;
  bool mixed = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  flip_alloc alloc{};
  bool has_alloc = false;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  PartView P[2];
  int cur = 0;
  BinView B;
  uint8_t* type = nullptr;
  // the bricks near the liquid (launch_finalize_near): marks kept across steps,
  // this step's list; near_stale after a step of the fused batch form, whose
  // whole-grid kernels leave the marks behind (the next step sweeps the grid)
  uint8_t* hmark = nullptr;
  unsigned int* hrow = nullptr;
  unsigned int* hlist = nullptr;
  unsigned int* hlist_n = nullptr;
  bool near_stale = false;
  float2* acc[3] = {nullptr, nullptr, nullptr};
  float* uo[3] = {nullptr, nullptr, nullptr};
  float* b32 = nullptr;
  double* b64 = nullptr;
  float* x32 = nullptr;
  double* x64 = nullptr;
  float2* pff = nullptr;
  float* r = nullptr;
  float* pa = nullptr;
  float* pb = nullptr;
  float* q = nullptr;
  double* partials = nullptr;
  MgArgs mg{};            // level shapes and scales (pointers filled by carve)
  int mg_dims[MG_MAX_LEVELS][3] = {};
  unsigned int* bar = nullptr;
  DevStats* dstats = nullptr;
  DevStats* hstats = nullptr;  // pinned
  double* norms = nullptr;
  double* diag = nullptr;      // energy sums: 4 per CTA, then the 4 totals
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  int pcg_blocks = 0, sm_count = 0, p2g_blocks = 0, g2p_blocks = 0;
  int p2g_per_sm = 0, g2p_per_sm = 0;  // flip_set_transfer_ctas (0: the defaults)
  int solver_blocks = 0;      // CTAs of a single solve (0: pcg_blocks)
  int launches = 0;
  bool stepped = false;
  unsigned long long wait_ns = 0;  // flip_set_wait_timeout (0: the defaults)
  CUtensorMap pmap{};              // the pressure field for G2P's TMA slab staging
  bool has_pmap = false;           // pmap is valid (the grid's pitches allow one)
  // timing of flip_step calls with statistics: 5 events per step plus one, kept
  // for the handle's life so a timed call creates none once the pool is large enough
  std::vector<cudaEvent_t> tev;
  std::vector<double> step_ms;  // device time of each step of the last timed call
};

void flip_set_last_error_(const std::string& msg) { g_last_error = msg; }

// P2G's default grid: 8 CTAs per SM, twice the co-resident 4, so that CTAs
// taking heavy bricks are balanced by the scheduler (the kernel loops over the
// active bricks; measured 8 % faster than one wave on a 128^3 dam break, equal on
// the 256^3 pool).  G2P's: its co-resident count.
constexpr int kP2gPerSm = 8;

void set_transfer_grids(flip_handle* h) {
  h->p2g_blocks = h->sm_count * (h->p2g_per_sm > 0 ? h->p2g_per_sm : kP2gPerSm);
  h->g2p_blocks = h->g2p_per_sm > 0 ? h->sm_count * h->g2p_per_sm : g2p_blocks(h->sm_count);
}

extern "C" {

int flip_abi_version(void) { return FLIP_ABI_VERSION; }

const char* flip_last_error(void) { return g_last_error.c_str(); }

const char* flip_strerror(int status) {
  switch (status) {
    case FLIP_OK: return "ok";
    case FLIP_E_ARG: return "invalid argument or unsolvable state";
    case FLIP_E_OOM: return "device allocation failed";
    case FLIP_E_CUDA: return "CUDA error";
    case FLIP_E_NOT_CONVERGED: return "pressure solve hit its iteration cap";
    case FLIP_E_TIMEOUT: return "device-side wait timed out";
    case FLIP_E_SIZE: return "buffer size does not match the field";
    case FLIP_E_NOGPU: return "no usable sm_103 CUDA device";
    case FLIP_E_CAPACITY: return "reseeding reached the particle capacity (warning)";
    default: return "unknown status";
  }
}

void flip_default_params(flip_params* p, int32_t nx, int32_t ny, int32_t nz) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n[0] = nx;
  p->n[1] = ny;
  p->n[2] = nz;
  const int m = std::max(nx, std::max(ny, nz));
  p->dx = m > 0 ? 1.0 / m : 0.0;
  p->dt = 1.0 / 240.0;
  p->gravity[1] = -9.81;
  p->rho = 1.0;
  p->flip_ratio = 0.95;
  p->skin = 1e-3 * p->dx;
  p->cg_tol = 1e-6;
  p->ir_tol = 1e-8;
  p->cg_max_iter = 20 * m;
  p->ir_max_iter = 100;
  p->precision = FLIP_PREC_FP32;
  p->advect_source = FLIP_ADVECT_PARTICLE;
  p->preconditioner = FLIP_PRECOND_MG;
  p->mg_smooth = 2;
  p->warm_start = 0;
}

}  // extern "C"

namespace {

int check_params(const flip_params* p, bool need_particles_prm) {
  if (!p) return fail(FLIP_E_ARG, "params is NULL");
  for (int a = 0; a < 3; ++a)
    if (p->n[a] < 2 || p->n[a] > 2048) return fail(FLIP_E_ARG, "n[a] must be in [2, 2048]");
  const long long nc = (long long)p->n[0] * p->n[1] * p->n[2];
  const long long nfmax = (long long)(p->n[0] + 1) * (p->n[1] + 1) * (p->n[2] + 1);
  if (nfmax >= (1LL << 31)) return fail(FLIP_E_ARG, "grid too large (face count >= 2^31)");
  (void)nc;
  if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return fail(FLIP_E_ARG, "dx must be > 0");
  // 1/dx must be an integer (to rounding: 1/(1/n) need not give n exactly in FP64)
  const double inv = 1.0 / p->dx;
  const double inv_int = std::round(inv);
  if (!(std::fabs(inv - inv_int) <= 1e-9 * inv_int) || inv_int < 1.0 || inv_int > 16777216.0)
    return fail(FLIP_E_ARG, "1/dx must be an integer <= 2^24");
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return fail(FLIP_E_ARG, "dt must be > 0");
  if (!(p->rho > 0.0)) return fail(FLIP_E_ARG, "rho must be > 0");
  if (!(p->cg_tol > 0.0) || p->cg_max_iter < 1) return fail(FLIP_E_ARG, "bad PCG tolerance/cap");
  if (p->precision != FLIP_PREC_FP32 && p->precision != FLIP_PREC_MIXED_IR)
    return fail(FLIP_E_ARG, "unknown precision mode");
  if (p->precision == FLIP_PREC_MIXED_IR && (!(p->ir_tol > 0.0) || !(p->cg_tol < 1.0)))
    return fail(FLIP_E_ARG, "mixed mode needs ir_tol > 0 and a refinement trigger cg_tol < 1");
  if (need_particles_prm) {
    if (p->preconditioner != FLIP_PRECOND_JACOBI && p->preconditioner != FLIP_PRECOND_MG &&
        p->preconditioner != FLIP_PRECOND_RBGS)
      return fail(FLIP_E_ARG, "unknown preconditioner");
    if (p->preconditioner == FLIP_PRECOND_RBGS && p->precision != FLIP_PREC_FP32)
      return fail(FLIP_E_ARG, "the red-black Gauss-Seidel solver runs in FP32 precision only");
    if (p->preconditioner == FLIP_PRECOND_MG && (p->mg_smooth < 1 || p->mg_smooth > 8))
      return fail(FLIP_E_ARG, "mg_smooth must be in [1, 8]");
    if (p->warm_start != 0 && p->warm_start != 1)
      return fail(FLIP_E_ARG, "warm_start must be 0 or 1");
    if (!(p->cfl >= 0.0) || !std::isfinite(p->cfl))
      return fail(FLIP_E_ARG, "cfl must be finite and >= 0");
    if (p->ppc_min < 0 || p->ppc_min > 64) return fail(FLIP_E_ARG, "ppc_min must be in [0, 64]");
    if (p->ppc_max < 0 || (p->ppc_max > 0 && p->ppc_max < std::max(p->ppc_min, 1)))
      return fail(FLIP_E_ARG, "ppc_max must be 0 or >= max(ppc_min, 1)");
    if (p->max_particles < 0 || p->max_particles > 2147483647LL)
      return fail(FLIP_E_ARG, "max_particles must be in [0, 2^31-1]");
    if (!(p->flip_ratio >= 0.0 && p->flip_ratio <= 1.0))
      return fail(FLIP_E_ARG, "flip_ratio must be in [0, 1]");
    if (!(p->skin > 0.0 && p->skin < p->dx)) return fail(FLIP_E_ARG, "skin must be in (0, dx)");
    if (p->advect_source != FLIP_ADVECT_PARTICLE && p->advect_source != FLIP_ADVECT_GRID)
      return fail(FLIP_E_ARG, "unknown advect_source");
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(p->gravity[a])) return fail(FLIP_E_ARG, "gravity must be finite");
  }
  return FLIP_OK;
}

int check_device() {
  int dev = 0, n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(FLIP_E_NOGPU, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  FLIP_CUDA(cudaGetDevice(&dev));
  int major = 0, minor = 0, coop = 0;
  FLIP_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  FLIP_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  FLIP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (major != 10 || minor != 3)
    return fail(FLIP_E_NOGPU, "this library is built for sm_103a (GB300); device is sm_" +
                                  std::to_string(major) + std::to_string(minor));
  if (!coop) return fail(FLIP_E_NOGPU, "device lacks cooperative launch");
  return FLIP_OK;
}

Grid make_grid(const flip_params& p) {
  Grid g{};
  g.nx = p.n[0];
  g.ny = p.n[1];
  g.nz = p.n[2];
  g.bx = (g.nx + BRICK - 1) / BRICK;
  g.by = (g.ny + BRICK - 1) / BRICK;
  g.bz = (g.nz + BRICK - 1) / BRICK;
  g.inv_dx = (float)std::round(1.0 / p.dx);  // an integer: the binning is exact
  g.dx = (float)p.dx;
  for (int a = 0; a < 3; ++a) g.hi[a] = (float)((double)p.n[a] * p.dx - p.skin);
  g.skin = (float)p.skin;
  return g;
}

// The parameters the pressure solve and Eq. 5 see.  With an adaptive time step
// (cfl > 0) they run on q = dt p / (rho dx^2), which is what a solve with
// dt = rho dx^2 produces: L q = b and u_new = u* - dx (q+ - q-), free of the
// step's dt.  The pressure is p = q rho dx^2 / dt when it is read.
flip_params solver_params(const flip_params& p) {
  flip_params q = p;
  if (p.cfl > 0.0) q.dt = p.rho * p.dx * p.dx;
  return q;
}

StepConsts make_consts(const flip_params& p) {
  StepConsts k{};
  const flip_params q = solver_params(p);
  for (int a = 0; a < 3; ++a) k.gdt[a] = (float)(p.gravity[a] * p.dt);
  k.pscale = (float)(q.dt / (q.rho * q.dx));
  k.pscale64 = q.dt / (q.rho * q.dx);
  k.flip_ratio = (float)p.flip_ratio;
  k.advect_grid = p.advect_source == FLIP_ADVECT_GRID;
  k.dt = (float)p.dt;
  k.wait_ns = kG2pWaitNs;
  return k;
}

// Level shapes and scales of the multigrid hierarchy (pointers left empty).
void setup_mg(MgArgs& m, int dims[MG_MAX_LEVELS][3], const flip_params& p) {
  m.nlev = mg_level_dims(p.n[0], p.n[1], p.n[2], dims);
  m.nu = p.mg_smooth;
  m.omega = MG_OMEGA;
  for (int c = 0; c < 8; ++c) m.inv_cnt[c] = c > 0 ? 1.0f / (float)c : 0.0f;
  m.lgrid = m.nlev;
  for (int l = 0; l < m.nlev; ++l) {
    MgLevel& L = m.lv[l];
    L.lvl = l;
    L.nx = dims[l][0];
    L.ny = dims[l][1];
    L.nz = dims[l][2];
    L.ncells = L.nx * L.ny * L.nz;
    const double h = p.dx * (double)(1 << l);
    const double s = p.dt / (p.rho * h * h);
    L.s = (float)s;
    for (int c = 0; c < 8; ++c) L.inv_scnt[c] = c > 0 ? (float)(1.0 / (s * c)) : 0.0f;
  }
  // the CTA-local levels: the longest tail of levels whose cells fit in MG_CTA_CELLS
  long long tail = 0;
  for (int l = m.nlev - 1; l >= 1; --l) {
    tail += m.lv[l].ncells;
    if (tail > MG_CTA_CELLS) break;
    m.lgrid = l;
  }
  if (m.nlev == 1) m.lgrid = 1;
  // the grid-wide levels are stored colour-split (MgLevel)
  for (int l = 0; l < m.nlev; ++l) {
    MgLevel& L = m.lv[l];
    L.split = l < m.lgrid;
    L.hx = ((L.nx + 1) / 2 + 1) & ~1;  // even, so pairs of slots are 8-byte aligned
    L.margin = L.hx * L.ny + 2;
    L.half = L.hx * L.ny * L.nz + 2 * L.margin;
    L.nw = (L.hx + 31) / 32;
    L.nbx = (L.nx + 7) / 8;
    L.nby = (L.ny + 7) / 8;
    L.nbz = (L.nz + 7) / 8;
  }
}

void fill_pcg_tables(PcgArgs& a, const flip_params& p) {
  const double s = p.dt / (p.rho * p.dx * p.dx);
  a.s = (float)s;
  a.s_lo = (float)(s - (double)a.s);
  a.s64 = s;
  for (int c = 0; c < 8; ++c) {
    a.diag_tab[c] = (float)(s * c);
    a.minv_tab[c] = c > 0 ? (float)(1.0 / (s * c)) : 0.0f;
  }
}

// Lays out (or measures) every device buffer of a handle.
void carve(flip_handle* h, Carver& cv) {
  const size_t np = (size_t)h->cap, nc = (size_t)h->ncells, nk = (size_t)h->nkeys,
               nb = h->nbricks;
  for (int b = 0; b < 2; ++b) {
    h->P[b].x = cv.take<float>(np);
    h->P[b].y = cv.take<float>(np);
    h->P[b].z = cv.take<float>(np);
    h->P[b].u = cv.take<float>(np);
    h->P[b].v = cv.take<float>(np);
    h->P[b].w = cv.take<float>(np);
    h->P[b].id = cv.take<int>(np);
  }
  h->B.key = cv.take<unsigned int>(np);
  h->B.rank = cv.take<unsigned int>(np);
  h->B.cell_count = cv.take<unsigned int>(nk);
  h->B.local_start = cv.take<unsigned int>(nk);
  h->B.brick_count = cv.take<unsigned int>(nb);
  h->B.brick_fluid = cv.take<unsigned int>(nb);
  h->B.brick_start = cv.take<unsigned int>(nb + 1);
  h->B.active = cv.take<unsigned int>(nb);
  h->type = cv.take<uint8_t>(nc);
  h->hmark = cv.take<uint8_t>(nb);
  h->hrow = cv.take<unsigned int>((nb + 31) / 32);  // brick-rows <= bricks
  h->hlist = cv.take<unsigned int>(nb);
  h->hlist_n = cv.take<unsigned int>(1);
  for (int d = 0; d < 3; ++d) {
    h->acc[d] = cv.take<float2>((size_t)h->nf[d]);
    h->uo[d] = cv.take<float>((size_t)h->nf[d]);
  }
  h->x32 = cv.take<float>(nc);
  if (h->mixed) {
    h->b64 = cv.take<double>(nc);
    h->x64 = cv.take<double>(nc);
    h->pff = cv.take<float2>(nc);
  } else {
    h->b32 = cv.take<float>(nc);
  }
  h->partials = cv.take<double>((size_t)PCG_SLOTS * (size_t)h->pcg_blocks);
  if (h->prm.preconditioner != FLIP_PRECOND_JACOBI) {
    MgArgs& m = h->mg;
    for (int l = 0; l < m.nlev; ++l) {
      MgLevel& L = m.lv[l];
      const size_t n = (size_t)L.ncells;
      if (L.split) {
        const size_t ns = 2 * (size_t)L.half;
        L.x = cv.take<float>(ns);
        L.b = cv.take<float>(ns);
        L.code16 = cv.take<uint16_t>(ns);
        L.seg = cv.take<int4>((size_t)L.nw * L.ny * L.nz);
        L.nseg = cv.take<unsigned int>(1);
        if (l > 0) {
          L.t = cv.take<uint8_t>(n);
          L.bflag = cv.take<uint8_t>((size_t)L.nbx * L.nby * L.nbz);
        }
        if (l == 0) {
          m.pa0 = cv.take<float>(ns);
          m.pb0 = cv.take<float>(ns);
          m.q0 = cv.take<float>(ns);
          m.d0 = cv.take<float>(ns);
          if (h->mixed) {
            m.x2 = cv.take<float2>(ns);
            m.b2 = cv.take<float2>(ns);
          }
        }
      } else {
        L.x = cv.take<float>(n);
        L.b = cv.take<float>(n);
        L.t = cv.take<uint8_t>(n);
        L.code = cv.take<uint8_t>(n);
      }
    }
    m.segcount = cv.take<unsigned int>((size_t)MG_MAX_LEVELS * (size_t)h->pcg_blocks);
  } else {
    h->r = cv.take<float>(nc);
    h->pa = cv.take<float>(nc);
    h->pb = cv.take<float>(nc);
    h->q = cv.take<float>(nc);
  }
  h->bar = cv.take<unsigned int>(BAR_WORDS);
  h->dstats = cv.take<DevStats>(1);
  h->norms = cv.take<double>(2);
  h->diag = cv.take<double>(4 * (size_t)energy_blocks(h->sm_count) + 4);
  const size_t nfmax = (size_t)std::max(h->nf[0], std::max(h->nf[1], h->nf[2]));
  h->tmp_bytes = std::max(nfmax * sizeof(float), nc * sizeof(double));
  h->tmp = cv.take<char>(h->tmp_bytes);
}

int upload(void* dst, const void* src, size_t bytes, int src_dev, cudaStream_t s) {
  if (bytes == 0) return FLIP_OK;
  if (!src) return fail(FLIP_E_ARG, "source pointer is NULL");
  FLIP_CUDA(cudaMemcpyAsync(dst, src, bytes,
                            src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return FLIP_OK;
}

bool reseeding(const flip_handle* h) { return h->prm.ppc_min > 0 || h->prm.ppc_max > 0; }

// Particle capacity: max_particles, or np without reseeding, or room for a full
// refill of every occupied cell (np + ppc_min * min(np, cells)), at least 2 np.
long long default_capacity(const flip_params& p, long long np) {
  if (p.max_particles > 0) return std::max<long long>(p.max_particles, np);
  if (p.ppc_min <= 0 && p.ppc_max <= 0) return np;
  const long long cells = (long long)p.n[0] * p.n[1] * p.n[2];
  const long long want = std::max<long long>(
      {2 * np, np + (long long)p.ppc_min * std::min(np, cells), 1024LL});
  return std::min<long long>(want, 2147483647LL);
}

unsigned int cell_cap(const flip_handle* h) {
  return h->prm.ppc_max > 0 ? (unsigned int)h->prm.ppc_max : ~0u;
}

// The particle count: with reseeding it lives on the device (read back here,
// synchronising the stream), otherwise it is np.
int refresh_np(flip_handle* h) {
  if (!reseeding(h)) return FLIP_OK;
  long long v = 0;
  FLIP_CUDA(cudaMemcpyAsync(&v, &h->dstats->np_buffer, sizeof(v), cudaMemcpyDeviceToHost,
                            h->stream));
  FLIP_CUDA(cudaStreamSynchronize(h->stream));
  h->np = v;
  return FLIP_OK;
}

int rebin(flip_handle* h) {
  if (reseeding(h)) {  // the buffer holds h->np particles, all of them binned below
    FLIP_CUDA(cudaMemcpyAsync(&h->dstats->np_layout, &h->np, sizeof(long long),
                              cudaMemcpyHostToDevice, h->stream));
    FLIP_CUDA(cudaMemcpyAsync(&h->dstats->np_buffer, &h->np, sizeof(long long),
                              cudaMemcpyHostToDevice, h->stream));
  }
  FLIP_CUDA(cudaMemsetAsync(h->B.cell_count, 0, sizeof(unsigned int) * (size_t)h->nkeys,
                            h->stream));
  FLIP_CUDA(cudaMemsetAsync(&h->dstats->max_speed_bits, 0, sizeof(unsigned int), h->stream));
  launch_rebin(h->g, h->P[h->cur], h->B, h->np, &h->dstats->max_speed_bits, h->stream);
  FLIP_CUDA(cudaGetLastError());
  return FLIP_OK;
}

PcgArgs pcg_args(flip_handle* h) {
  PcgArgs a{};
  a.g = h->g;
  fill_pcg_tables(a, solver_params(h->prm));
  a.type = h->type;
  a.active = h->B.active;
  a.n_active = &h->dstats->n_active;
  a.brick_fluid = h->B.brick_fluid;
  a.b32 = h->b32;
  a.b64 = h->b64;
  a.x32 = h->x32;
  a.x64 = h->x64;
  a.pff = h->pff;
  a.r = h->r;
  a.pa = h->pa;
  a.pb = h->pb;
  a.q = h->q;
  a.partials = h->partials;
  a.bar = h->bar;
  a.status = &h->dstats->status;
  a.stats = h->dstats;
  a.tol = h->prm.cg_tol;
  a.ir_tol = h->prm.ir_tol;
  a.max_iter = h->prm.cg_max_iter;
  a.ir_max_iter = h->prm.ir_max_iter;
  a.check_singular = 1;
  a.timeout_ns = h->wait_ns ? h->wait_ns : kBarrierWaitNs;
  a.precond = h->prm.preconditioner;
  a.warm_start = h->prm.warm_start;
  if (a.precond != FLIP_PRECOND_JACOBI) {
    a.mg = h->mg;
    a.mg.lv[0].t = h->type;
  }
  return a;
}

// Adaptive time step (Sec. 3.1.4): the step's dt from the particles' largest
// speed, before anything of the step uses it.
void launch_step_dt(flip_handle* h) {
  if (h->prm.cfl <= 0.0) return;
  launch_cfl_dt(h->dstats, h->prm.gravity, h->prm.dt, h->prm.cfl * h->prm.dx, h->stream);
  h->launches += 1;
}

// Pressure units of the stored solution: 1, or rho dx^2 / dt of the last step
// when the solve runs on q (adaptive time step).  Synchronises the stream.
int pressure_factor(flip_handle* h, double* f) {
  *f = 1.0;
  if (h->prm.cfl <= 0.0) return FLIP_OK;
  double dt = 0.0;
  FLIP_CUDA(cudaMemcpyAsync(&dt, &h->dstats->dt_cur, sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  FLIP_CUDA(cudaStreamSynchronize(h->stream));
  if (dt > 0.0) *f = h->prm.rho * h->prm.dx * h->prm.dx / dt;
  return FLIP_OK;
}

// The front of a step: adaptive dt, binning (with reseeding's upper bound) and
// the counting-sort scatter into the other buffer.
void launch_front(flip_handle* h, cudaStream_t s) {
  launch_step_dt(h);
  launch_bin(h->g, h->B, h->type, h->dstats, s, cell_cap(h));
  if (reseeding(h))
    launch_scatter(h->P[h->cur], h->P[1 - h->cur], h->B, h->cap, s, &h->dstats->np_buffer,
                   cell_cap(h));
  else
    launch_scatter(h->P[h->cur], h->P[1 - h->cur], h->B, h->np, s);
  h->cur = 1 - h->cur;
  h->launches += 2 + (h->np > 0 || reseeding(h));
}

// Particles G2P walks (its launch is skipped for 0).
long long g2p_count(const flip_handle* h) { return reseeding(h) ? h->cap : h->np; }

// The back of a step, after G2P: reseeding's spawn into under-filled cells.
void launch_back(flip_handle* h, cudaStream_t s) {
  if (reseeding(h)) {
    const float* uo[3] = {h->uo[0], h->uo[1], h->uo[2]};
    ReseedArgs r{h->prm.ppc_min, h->prm.reseed_seed, h->steps_done, h->cap, h->prm.dx};
    launch_spawn(h->g, h->K, h->P[h->cur], h->B, uo, h->mixed ? nullptr : h->x32, h->pff,
                 h->dstats, r, h->nkeys, s);
    h->launches += 1 + (h->prm.ppc_min > 0);
  }
  ++h->steps_done;
}

int status_to_code(int st) {
  if (st & DEV_CAPACITY && !(st & (DEV_TIMEOUT | DEV_SINGULAR | DEV_NOT_CONVERGED)))
    return fail(FLIP_E_CAPACITY, "reseeding reached max_particles; some new particles were skipped");
  if (st & DEV_TIMEOUT) return fail(FLIP_E_TIMEOUT, "a device-side wait in the PCG timed out");
  if (st & DEV_SINGULAR)
    return fail(FLIP_E_ARG, "every cell is fluid: the pressure system is singular");
  if (st & DEV_NOT_CONVERGED) return fail(FLIP_E_NOT_CONVERGED, "PCG hit its iteration cap");
  return FLIP_OK;
}

// Reads and clears the sticky device status; the stream must be idle.
int take_status(flip_handle* h) {
  FLIP_CUDA(cudaMemcpyAsync(h->hstats, h->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost,
                            h->stream));
  FLIP_CUDA(cudaMemsetAsync(&h->dstats->status, 0, sizeof(int), h->stream));
  FLIP_CUDA(cudaStreamSynchronize(h->stream));
  if (reseeding(h)) h->np = h->hstats->np_buffer;
  return status_to_code(h->hstats->status);
}

}  // namespace

extern "C" {

int flip_create(const flip_params* params, const float* x, const float* y, const float* z,
                const float* u, const float* v, const float* w, int64_t np,
                int32_t src_is_device, const flip_alloc* alloc, void* stream,
                flip_handle** out) {
  if (!out) return fail(FLIP_E_ARG, "out is NULL");
  *out = nullptr;
  int rc = check_params(params, true);
  if (rc) return rc;
  if (np < 0 || np > 2147483647LL) return fail(FLIP_E_ARG, "np must be in [0, 2^31-1]");
  if (params->max_particles > 0 && params->max_particles < np)
    return fail(FLIP_E_ARG, "max_particles must be >= np");
  if (alloc && (!alloc->alloc || !alloc->free))
    return fail(FLIP_E_ARG, "flip_alloc needs both alloc and free");
  rc = check_device();
  if (rc) return rc;

  flip_handle* h = new (std::nothrow) flip_handle();
  if (!h) return fail(FLIP_E_OOM, "host allocation failed");
  h->prm = *params;
  {
    static std::atomic<long long> next_serial{1};
    h->serial = next_serial.fetch_add(1);
  }
  h->g = make_grid(*params);
  h->K = make_consts(*params);
  h->np = np;
  h->cap = default_capacity(*params, np);
  h->ncells = (long long)h->g.nx * h->g.ny * h->g.nz;
  h->nbricks = (unsigned)h->g.bx * h->g.by * h->g.bz;
  h->nkeys = (long long)h->nbricks * BRICK_CELLS;
  for (int d = 0; d < 3; ++d) h->nf[d] = n_faces(h->g, d);
  h->mixed = params->precision == FLIP_PREC_MIXED_IR;
  if (alloc) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  auto cleanup = [&](int code) {
    flip_destroy(h);
    return code;
  };
  cudaError_t e;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamCreate"));
    h->own_stream = true;
  }
  e = pcg_max_blocks(&h->pcg_blocks, &h->sm_count);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "occupancy query"));
  if (params->preconditioner != FLIP_PRECOND_JACOBI) {
    e = pcg_mg_check_occupancy();
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "multigrid kernel occupancy"));
    setup_mg(h->mg, h->mg_dims, solver_params(*params));
  }
  set_transfer_grids(h);

  Carver measure;
  carve(h, measure);
  h->arena_bytes = measure.off;
  if (h->has_alloc) {
    h->arena = h->alloc.alloc(h->alloc.ctx, h->arena_bytes, (void*)h->stream);
    if (!h->arena) return cleanup(fail(FLIP_E_OOM, "allocator callback returned NULL"));
  } else {
    e = cudaMallocAsync(&h->arena, h->arena_bytes, h->stream);
    if (e != cudaSuccess) {
      h->arena = nullptr;
      return cleanup(cuda_fail(e, "cudaMallocAsync(arena)"));
    }
  }
  Carver assign;
  assign.base = (char*)h->arena;
  carve(h, assign);
  h->has_pmap = encode_pressure_map(h->g, h->mixed ? (void*)h->pff : (void*)h->x32, h->mixed,
                                    &h->pmap);
  h->K.dyn = params->cfl > 0.0 ? h->dstats->dyn : nullptr;
  e = cudaMallocHost((void**)&h->hstats, sizeof(DevStats));
  if (e != cudaSuccess) {
    h->hstats = nullptr;
    return cleanup(cuda_fail(e, "cudaMallocHost"));
  }
  // Zero everything once: histogram, accumulators, fields, barrier, stats.
  e = cudaMemsetAsync(h->arena, 0, h->arena_bytes, h->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMemsetAsync(arena)"));
  const size_t pb = sizeof(float) * (size_t)np;
  const float* src[6] = {x, y, z, u, v, w};
  float* dst[6] = {h->P[0].x, h->P[0].y, h->P[0].z, h->P[0].u, h->P[0].v, h->P[0].w};
  for (int a = 0; a < 6; ++a) {
    rc = upload(dst[a], src[a], pb, src_is_device, h->stream);
    if (rc) return cleanup(rc);
  }
  launch_iota(h->P[0].id, np, h->stream);
  {
    long long next_id = np;  // pageable source: the copy is staged before the call returns
    e = cudaMemcpyAsync(&h->dstats->next_id, &next_id, sizeof(next_id), cudaMemcpyHostToDevice,
                        h->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMemcpyAsync(next_id)"));
  }
  rc = rebin(h);
  if (rc) return cleanup(rc);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "flip_create"));
  *out = h;
  return FLIP_OK;
}

void flip_destroy(flip_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->arena) {
    if (h->has_alloc) h->alloc.free(h->alloc.ctx, h->arena, h->arena_bytes, (void*)h->stream);
    else cudaFreeAsync(h->arena, h->stream);
  }
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->hstats) cudaFreeHost(h->hstats);
  for (cudaEvent_t e : h->tev)
    if (e) cudaEventDestroy(e);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int flip_step(flip_handle* h, int32_t nsteps, flip_stats* stats) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (nsteps < 0) return fail(FLIP_E_ARG, "nsteps must be >= 0");
  const cudaStream_t s = h->stream;
  const bool timed = stats != nullptr;
  // Step st is bracketed by events E[5 st] .. E[5 st + 5] (its stages in between;
  // a step's last event is the next step's first).  Nothing waits on them until
  // every step is enqueued, so the host never stalls the stream inside the call.
  if (timed) {
    const size_t need = std::max<size_t>(5 * (size_t)nsteps + 1, 256);
    while (h->tev.size() < need) {
      cudaEvent_t e = nullptr;
      FLIP_CUDA(cudaEventCreate(&e));
      h->tev.push_back(e);
    }
  }
  cudaEvent_t* E = timed ? h->tev.data() : nullptr;
  const int launches0 = h->launches;
  if (timed) {
    FLIP_CUDA(cudaMemcpyAsync(&h->dstats->cg_iters_mark, &h->dstats->cg_iters_total,
                              2 * sizeof(long long), cudaMemcpyDeviceToDevice, s));
    FLIP_CUDA(cudaMemcpyAsync(&h->dstats->added_mark, &h->dstats->added_total,
                              2 * sizeof(long long), cudaMemcpyDeviceToDevice, s));
  }
  const float* uo[3] = {h->uo[0], h->uo[1], h->uo[2]};
  PcgArgs pa = pcg_args(h);
  int rc = FLIP_OK;
  for (int st = 0; st < nsteps; ++st) {
    cudaEvent_t* ev = timed ? E + 5 * (size_t)st : nullptr;
    if (timed && st == 0) FLIP_CUDA(cudaEventRecord(ev[0], s));
    launch_step_dt(h);
    launch_front(h, s);
    if (timed) FLIP_CUDA(cudaEventRecord(ev[1], s));
    launch_p2g(h->g, h->P[h->cur], h->B, h->acc, h->dstats, h->p2g_blocks, s);
    FLIP_CUDA(launch_finalize_near(h->g, h->B.brick_count, h->hmark, h->hrow, h->hlist,
                                   h->hlist_n, h->acc, h->uo, h->bar, h->dstats, h->sm_count,
                                   h->near_stale, s));
    h->launches += 3;
    if (timed) FLIP_CUDA(cudaEventRecord(ev[2], s));
    launch_divergence_near(h->g, h->K, h->type, uo, h->b32, h->b64, h->x32, h->x64, h->pff,
                           h->bar, h->dstats, h->hlist, h->hlist_n, h->sm_count, h->near_stale,
                           s);
    h->near_stale = false;
    h->launches += 1;
    if (timed) FLIP_CUDA(cudaEventRecord(ev[3], s));
    const int nsb = h->solver_blocks > 0 ? h->solver_blocks : h->pcg_blocks;
    if (pa.precond != FLIP_PRECOND_JACOBI) FLIP_CUDA(launch_pcg_mg(pa, h->mixed, nsb, s));
    else FLIP_CUDA(launch_pcg(pa, h->mixed, nsb, s));
    h->launches += 1;
    if (timed) FLIP_CUDA(cudaEventRecord(ev[4], s));
    launch_g2p(h->g, h->K, h->P[h->cur], h->B, uo, h->mixed ? nullptr : h->x32, h->pff,
               h->dstats, g2p_count(h), h->g2p_blocks, h->has_pmap ? &h->pmap : nullptr, s);
    h->launches += (g2p_count(h) > 0);
    launch_back(h, s);
    if (timed) FLIP_CUDA(cudaEventRecord(ev[5], s));
    FLIP_CUDA(cudaGetLastError());
    h->stepped = true;
  }
  if (timed) {
    double ms[5] = {0, 0, 0, 0, 0};
    double ms_total = 0.0;
    h->step_ms.assign((size_t)nsteps, 0.0);
    if (nsteps > 0) FLIP_CUDA(cudaEventSynchronize(E[5 * (size_t)nsteps]));
    for (int st = 0; st < nsteps; ++st) {
      const cudaEvent_t* ev = E + 5 * (size_t)st;
      for (int q = 0; q < 5; ++q) {
        float t = 0.0f;
        FLIP_CUDA(cudaEventElapsedTime(&t, ev[q], ev[q + 1]));
        ms[q] += t;
      }
      float t = 0.0f;
      FLIP_CUDA(cudaEventElapsedTime(&t, ev[0], ev[5]));
      h->step_ms[(size_t)st] = t;
    }
    if (nsteps > 0) {
      float t = 0.0f;
      FLIP_CUDA(cudaEventElapsedTime(&t, E[0], E[5 * (size_t)nsteps]));
      ms_total = t;
    }
    std::memset(stats, 0, sizeof(*stats));
    FLIP_CUDA(cudaMemsetAsync(h->norms, 0, 2 * sizeof(double), s));
    if (h->stepped) {
      launch_div_norms(h->g, h->K, h->type, uo, h->mixed ? nullptr : h->x32, h->x64, h->norms, s);
      FLIP_CUDA(cudaGetLastError());
      h->launches += 1;
    }
    double norms[2] = {0.0, 0.0};
    FLIP_CUDA(cudaMemcpyAsync(norms, h->norms, sizeof(norms), cudaMemcpyDeviceToHost, s));
    rc = take_status(h);
    const DevStats& d = *h->hstats;
    stats->steps = nsteps;
    stats->n_particles = h->np;
    stats->particles_added = d.added_total - d.added_mark;
    stats->particles_removed = d.removed_total - d.removed_mark;
    stats->n_fluid_cells = d.n_fluid;
    stats->n_active_bricks = d.n_active;
    stats->cg_iterations = d.cg_iters_total - d.cg_iters_mark;
    stats->ir_iterations = (int32_t)(d.ir_iters_total - d.ir_iters_mark);
    stats->kernel_launches = h->launches - launches0;
    stats->cg_rel_residual = d.rel_res;
    stats->rel_divergence = norms[0] > 0.0 ? std::sqrt(norms[1] / norms[0]) : 0.0;
    float ms_f;
    std::memcpy(&ms_f, &d.max_speed_bits, sizeof(float));
    stats->max_speed = ms_f;
    stats->dt_last = h->prm.cfl > 0.0 ? d.dt_cur : h->prm.dt;
    stats->ms_bin = ms[0];
    stats->ms_p2g = ms[1];
    stats->ms_divergence = ms[2];
    stats->ms_pcg = ms[3];
    stats->ms_g2p = ms[4];
    stats->ms_total = ms_total;
  }
  return rc;
}

int flip_set_wait_timeout(flip_handle* h, uint64_t timeout_ns) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  h->wait_ns = timeout_ns;
  h->K.wait_ns = timeout_ns ? timeout_ns : kG2pWaitNs;
  return FLIP_OK;
}

int32_t flip_step_times(const flip_handle* h, double* ms, int32_t n) {
  if (!h) return -fail(FLIP_E_ARG, "handle is NULL");
  const int32_t count = (int32_t)h->step_ms.size();
  if (ms)
    for (int32_t q = 0; q < std::min(n, count); ++q) ms[q] = h->step_ms[(size_t)q];
  return count;
}

int flip_set_solver_blocks(flip_handle* h, int32_t nblocks) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (nblocks < 0 || nblocks > h->pcg_blocks)
    return fail(FLIP_E_ARG, "nblocks must be in [0, " + std::to_string(h->pcg_blocks) + "]");
  h->solver_blocks = nblocks;
  return FLIP_OK;
}

int flip_autotune_solver(flip_handle* h, int32_t steps_per_candidate, int32_t* nblocks) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (steps_per_candidate < 1) return fail(FLIP_E_ARG, "steps_per_candidate must be >= 1");
  const int m = h->pcg_blocks;
  const int cand[4] = {m, std::max(1, m / 2), std::max(1, m / 4), std::max(1, m / 8)};
  int best = h->solver_blocks > 0 ? h->solver_blocks : m, first_warning = FLIP_OK;
  double best_ms = -1.0;
  for (int c : cand) {
    h->solver_blocks = c;
    flip_stats st;
    const int rc = flip_step(h, steps_per_candidate, &st);
    if (rc == FLIP_E_NOT_CONVERGED || rc == FLIP_E_CAPACITY) {
      if (first_warning == FLIP_OK) first_warning = rc;
    } else if (rc != FLIP_OK) {
      h->solver_blocks = best;
      return rc;
    }
    if (best_ms < 0.0 || st.ms_pcg < best_ms) {
      best_ms = st.ms_pcg;
      best = c;
    }
  }
  h->solver_blocks = best;
  if (nblocks) *nblocks = best;
  return first_warning;
}

int flip_set_transfer_ctas(flip_handle* h, int32_t p2g_per_sm, int32_t g2p_per_sm) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (p2g_per_sm < 0 || p2g_per_sm > 64 || g2p_per_sm < 0 || g2p_per_sm > 64)
    return fail(FLIP_E_ARG, "CTAs per SM must be in [0, 64]");
  h->p2g_per_sm = p2g_per_sm;
  h->g2p_per_sm = g2p_per_sm;
  set_transfer_grids(h);
  return FLIP_OK;
}

int flip_get_transfer_ctas(const flip_handle* h, int32_t* p2g_per_sm, int32_t* g2p_per_sm) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  const int sm = std::max(h->sm_count, 1);
  if (p2g_per_sm) *p2g_per_sm = h->p2g_blocks / sm;
  if (g2p_per_sm) *g2p_per_sm = h->g2p_blocks / sm;
  return FLIP_OK;
}

}  // extern "C"

namespace {

// The candidates of the launch-shape autotuners: P2G at 4, 8 and 16 CTAs per SM,
// G2P at 1, 2 and 4 times its co-resident count, taken in pairs (the two stages are
// timed apart, so each keeps its own best).
struct TransferCand {
  int p2g, g2p;
};

void transfer_candidates(TransferCand (&c)[3]) {
  const int g = g2p_blocks(1);  // G2P's co-resident CTAs per SM
  c[0] = {4, g};
  c[1] = {8, 2 * g};
  c[2] = {16, 4 * g};
}

}  // namespace

extern "C" {

int flip_autotune_transfers(flip_handle* h, int32_t steps_per_candidate, int32_t* p2g_per_sm,
                            int32_t* g2p_per_sm) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (steps_per_candidate < 1) return fail(FLIP_E_ARG, "steps_per_candidate must be >= 1");
  TransferCand cand[3];
  transfer_candidates(cand);
  const int keep_p = h->p2g_per_sm, keep_g = h->g2p_per_sm;
  double p_ms[3] = {}, g_ms[3] = {};
  int first_warning = FLIP_OK;
  // forward then reverse (the scene evolves while it is timed)
  for (int t = 0; t < 6; ++t) {
    const int c = t < 3 ? t : 5 - t;
    h->p2g_per_sm = cand[c].p2g;
    h->g2p_per_sm = cand[c].g2p;
    set_transfer_grids(h);
    flip_stats st;
    const int rc = flip_step(h, steps_per_candidate, &st);
    if (rc == FLIP_E_NOT_CONVERGED || rc == FLIP_E_CAPACITY) {
      if (first_warning == FLIP_OK) first_warning = rc;
    } else if (rc != FLIP_OK) {
      h->p2g_per_sm = keep_p;
      h->g2p_per_sm = keep_g;
      set_transfer_grids(h);
      return rc;
    }
    p_ms[c] += st.ms_p2g;
    g_ms[c] += st.ms_g2p;
  }
  int bp = 0, bg = 0;
  for (int c = 1; c < 3; ++c) {
    if (p_ms[c] < p_ms[bp]) bp = c;
    if (g_ms[c] < g_ms[bg]) bg = c;
  }
  h->p2g_per_sm = cand[bp].p2g;
  h->g2p_per_sm = cand[bg].g2p;
  set_transfer_grids(h);
  if (p2g_per_sm) *p2g_per_sm = cand[bp].p2g;
  if (g2p_per_sm) *g2p_per_sm = cand[bg].g2p;
  return first_warning;
}

int flip_energy(flip_handle* h, double particle_mass, double out[3]) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (!out) return fail(FLIP_E_ARG, "out is NULL");
  if (!(particle_mass >= 0.0) || !std::isfinite(particle_mass))
    return fail(FLIP_E_ARG, "particle_mass must be finite and >= 0");
  if (int rc = refresh_np(h)) return rc;
  double sums[4] = {0.0, 0.0, 0.0, 0.0};
  if (h->np > 0) {
    const int nb = energy_blocks(h->sm_count);
    double* tot = h->diag + 4 * (size_t)nb;
    launch_energy(h->P[h->cur], h->np, h->diag, nb, tot, h->stream);
    FLIP_CUDA(cudaGetLastError());
    h->launches += 2;
    FLIP_CUDA(cudaMemcpyAsync(sums, tot, sizeof(sums), cudaMemcpyDeviceToHost, h->stream));
  }
  FLIP_CUDA(cudaStreamSynchronize(h->stream));
  const double* g = h->prm.gravity;
  out[0] = 0.5 * particle_mass * sums[0];
  out[1] = -particle_mass * (g[0] * sums[1] + g[1] * sums[2] + g[2] * sums[3]);
  out[2] = out[0] + out[1];
  return FLIP_OK;
}

size_t flip_footprint_bytes(const flip_params* params, int64_t np) {
  if (check_params(params, true) != FLIP_OK || np < 0 || np > 2147483647LL) return 0;
  if (check_device() != FLIP_OK) return 0;
  flip_handle tmp;
  tmp.prm = *params;
  tmp.g = make_grid(*params);
  tmp.np = np;
  tmp.cap = default_capacity(*params, np);
  tmp.ncells = (long long)tmp.g.nx * tmp.g.ny * tmp.g.nz;
  tmp.nbricks = (unsigned)tmp.g.bx * tmp.g.by * tmp.g.bz;
  tmp.nkeys = (long long)tmp.nbricks * BRICK_CELLS;
  for (int d = 0; d < 3; ++d) tmp.nf[d] = n_faces(tmp.g, d);
  tmp.mixed = params->precision == FLIP_PREC_MIXED_IR;
  if (pcg_max_blocks(&tmp.pcg_blocks, &tmp.sm_count) != cudaSuccess) return 0;
  if (params->preconditioner != FLIP_PRECOND_JACOBI) setup_mg(tmp.mg, tmp.mg_dims, *params);
  Carver measure;
  carve(&tmp, measure);
  return measure.off;
}

int flip_sync(flip_handle* h) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  FLIP_CUDA(cudaStreamSynchronize(h->stream));
  return take_status(h);
}

size_t flip_field_bytes(const flip_handle* h, flip_field which) {
  if (!h) return 0;
  if (which <= FLIP_FIELD_PID && refresh_np(const_cast<flip_handle*>(h)) != FLIP_OK) return 0;
  switch (which) {
    case FLIP_FIELD_PX: case FLIP_FIELD_PY: case FLIP_FIELD_PZ:
    case FLIP_FIELD_PU: case FLIP_FIELD_PV: case FLIP_FIELD_PW:
    case FLIP_FIELD_PID:
      return 4 * (size_t)h->np;
    case FLIP_FIELD_U_OLD: case FLIP_FIELD_U_NEW: return 4 * (size_t)h->nf[0];
    case FLIP_FIELD_V_OLD: case FLIP_FIELD_V_NEW: return 4 * (size_t)h->nf[1];
    case FLIP_FIELD_W_OLD: case FLIP_FIELD_W_NEW: return 4 * (size_t)h->nf[2];
    case FLIP_FIELD_PRESSURE: case FLIP_FIELD_RHS: return 4 * (size_t)h->ncells;
    case FLIP_FIELD_PRESSURE_F64: return 8 * (size_t)h->ncells;
    case FLIP_FIELD_CELL_TYPE: return (size_t)h->ncells;
    default: return 0;
  }
}

int flip_read(flip_handle* h, flip_field which, void* dst, size_t bytes, int32_t dst_is_device) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  const size_t need = flip_field_bytes(h, which);
  if (which < 0 || which >= FLIP_FIELD_COUNT_) return fail(FLIP_E_ARG, "unknown field");
  if (bytes != need) return fail(FLIP_E_SIZE, "bytes must be " + std::to_string(need));
  if (need == 0) return FLIP_OK;
  if (!dst) return fail(FLIP_E_ARG, "dst is NULL");
  const cudaStream_t s = h->stream;
  const void* src = nullptr;
  const PartView& P = h->P[h->cur];
  switch (which) {
    case FLIP_FIELD_PX: src = P.x; break;
    case FLIP_FIELD_PY: src = P.y; break;
    case FLIP_FIELD_PZ: src = P.z; break;
    case FLIP_FIELD_PU: src = P.u; break;
    case FLIP_FIELD_PV: src = P.v; break;
    case FLIP_FIELD_PW: src = P.w; break;
    case FLIP_FIELD_PID: src = P.id; break;
    case FLIP_FIELD_U_OLD: src = h->uo[0]; break;
    case FLIP_FIELD_V_OLD: src = h->uo[1]; break;
    case FLIP_FIELD_W_OLD: src = h->uo[2]; break;
    case FLIP_FIELD_U_NEW: case FLIP_FIELD_V_NEW: case FLIP_FIELD_W_NEW: {
      const int d = which - FLIP_FIELD_U_NEW;
      launch_u_new(h->g, h->K, d, h->uo[d], h->mixed ? nullptr : h->x32, h->pff, (float*)h->tmp, s);
      src = h->tmp;
      break;
    }
    case FLIP_FIELD_PRESSURE: {
      double f = 1.0;
      if (int rc = pressure_factor(h, &f)) return rc;
      if (h->mixed) {
        launch_f64_to_f32(h->x64, (float*)h->tmp, h->ncells, s);
        src = h->tmp;
      } else if (f != 1.0) {
        FLIP_CUDA(cudaMemcpyAsync(h->tmp, h->x32, sizeof(float) * h->ncells,
                                  cudaMemcpyDeviceToDevice, s));
        src = h->tmp;
      } else {
        src = h->x32;
      }
      if (f != 1.0) launch_scale((float*)h->tmp, h->ncells, f, s);
      break;
    }
    case FLIP_FIELD_PRESSURE_F64: {
      double f = 1.0;
      if (int rc = pressure_factor(h, &f)) return rc;
      if (h->mixed && f == 1.0) {
        src = h->x64;
      } else {
        if (h->mixed)
          FLIP_CUDA(cudaMemcpyAsync(h->tmp, h->x64, sizeof(double) * h->ncells,
                                    cudaMemcpyDeviceToDevice, s));
        else
          launch_f32_to_f64(h->x32, (double*)h->tmp, h->ncells, s);
        if (f != 1.0) launch_scale((double*)h->tmp, h->ncells, f, s);
        src = h->tmp;
      }
      break;
    }
    case FLIP_FIELD_RHS:
      if (h->mixed) {
        launch_f64_to_f32(h->b64, (float*)h->tmp, h->ncells, s);
        src = h->tmp;
      } else {
        src = h->b32;
      }
      break;
    case FLIP_FIELD_CELL_TYPE: src = h->type; break;
    default: return fail(FLIP_E_ARG, "unknown field");
  }
  FLIP_CUDA(cudaGetLastError());
  FLIP_CUDA(cudaMemcpyAsync(dst, src, need,
                            dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  FLIP_CUDA(cudaStreamSynchronize(s));
  return FLIP_OK;
}

int flip_write(flip_handle* h, flip_field which, const void* src, size_t bytes,
               int32_t src_is_device) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (which < FLIP_FIELD_PX || which > FLIP_FIELD_PID)
    return fail(FLIP_E_ARG, "only particle fields can be written");
  const size_t need = flip_field_bytes(h, which);
  if (bytes != need) return fail(FLIP_E_SIZE, "bytes must be " + std::to_string(need));
  const PartView& P = h->P[h->cur];
  void* dst = nullptr;
  switch (which) {
    case FLIP_FIELD_PX: dst = P.x; break;
    case FLIP_FIELD_PY: dst = P.y; break;
    case FLIP_FIELD_PZ: dst = P.z; break;
    case FLIP_FIELD_PU: dst = P.u; break;
    case FLIP_FIELD_PV: dst = P.v; break;
    case FLIP_FIELD_PW: dst = P.w; break;
    default: dst = P.id; break;
  }
  int rc = upload(dst, src, need, src_is_device, h->stream);
  if (rc) return rc;
  if (which <= FLIP_FIELD_PZ) {
    rc = rebin(h);
    if (rc) return rc;
  }
  FLIP_CUDA(cudaStreamSynchronize(h->stream));
  return FLIP_OK;
}

int flip_read_particles(flip_handle* h, float* x, float* y, float* z, float* u, float* v,
                        float* w, int32_t* id, int32_t dst_is_device) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (int rc = refresh_np(h)) return rc;
  const PartView& P = h->P[h->cur];
  void* dst[7] = {x, y, z, u, v, w, id};
  const void* src[7] = {P.x, P.y, P.z, P.u, P.v, P.w, P.id};
  const size_t nb = 4 * (size_t)h->np;
  for (int a = 0; a < 7; ++a) {
    if (!dst[a]) {
      if (a < 6 && nb) return fail(FLIP_E_ARG, "particle destination is NULL");
      continue;
    }
    if (nb)
      FLIP_CUDA(cudaMemcpyAsync(dst[a], src[a], nb,
                                dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream));
  }
  FLIP_CUDA(cudaStreamSynchronize(h->stream));
  return FLIP_OK;
}

int flip_write_particles(flip_handle* h, const float* x, const float* y, const float* z,
                         const float* u, const float* v, const float* w, int32_t src_is_device) {
  if (!h) return fail(FLIP_E_ARG, "handle is NULL");
  if (int rc = refresh_np(h)) return rc;
  const PartView& P = h->P[h->cur];
  float* dst[6] = {P.x, P.y, P.z, P.u, P.v, P.w};
  const float* src[6] = {x, y, z, u, v, w};
  for (int a = 0; a < 6; ++a) {
    const int rc = upload(dst[a], src[a], 4 * (size_t)h->np, src_is_device, h->stream);
    if (rc) return rc;
  }
  const int rc = rebin(h);
  if (rc) return rc;
  FLIP_CUDA(cudaStreamSynchronize(h->stream));
  return FLIP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches

struct flip_batch {
  int capacity = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  PcgArgs* d_args = nullptr;     // [capacity]
  int* d_block_scene = nullptr;  // [max CTAs]
  int* d_team_first = nullptr;   // [capacity + 1]
  int max_blocks = 0;
  std::vector<cudaEvent_t> ev;   // one per scene slot
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
  cudaEvent_t ev_solved = nullptr;
  std::vector<cudaEvent_t> pev;  // timed calls: the batched solves' start and end per step
  double team_exponent = 1.0;    // team size proportional to particles^exponent
  // two steps of a fixed set of scenes captured as one CUDA graph (untimed calls)
  cudaGraphExec_t graph = nullptr;
  std::vector<unsigned long long> graph_key;
  std::vector<int> graph_launches;  // kernel launches per scene in the captured pair
  int graph_batch_launches = 0;
  bool graph_off = false;           // capture failed once: use the plain path
  bool graphs = false;              // graph replay requested (flip_batch_set_graphs)
  // one launch per step kernel across all scenes (flip_batch_set_fused); off by
  // default: per-scene launches on per-scene streams measured 3-4 % faster on the
  // 64-scene batch (cross-stage overlap between scenes), and the autotuner chooses
  bool fused = false;
  SceneDev* d_scenes = nullptr;     // [2 * capacity]: the scene table for either buffer parity
  unsigned int* d_first = nullptr;  // [kFusedLaunches * (capacity + 1)] CTA ranges
};

namespace {

// Runs `pairs` pairs of batched steps as a CUDA graph: two steps of the scenes
// captured from enqueue_step (the particle double buffers are back in place
// after two steps), cached on the batch for the same scenes, buffer parity and
// CTA split.  Host-side state the capture moved (buffer index, step and launch
// counters) is restored and advanced per replay.  Returns the steps done (0 when
// the graph path is unavailable: the caller steps normally), or -status.
template <class F>
int batch_graph_steps(flip_batch* b, flip_handle* const* hs, int n, int pairs,
                      const std::vector<int>& first_all, F& enqueue_step, int* batch_launches) {
  const cudaStream_t bs = b->stream;
  std::vector<unsigned long long> key;
  key.push_back((unsigned long long)n);
  key.push_back(b->fused ? 1ull : 0ull);  // the form the graph captured
  for (int s = 0; s < n; ++s) {
    key.push_back((unsigned long long)(uintptr_t)hs[s]);
    key.push_back((unsigned long long)hs[s]->serial);
    key.push_back((unsigned long long)hs[s]->cur);
    key.push_back((unsigned long long)hs[s]->p2g_blocks);  // the captured launch shapes
    key.push_back((unsigned long long)hs[s]->g2p_blocks);
    key.push_back(hs[s]->near_stale ? 1ull : 0ull);  // whether the first step sweeps the grid
  }
  for (int v : first_all) key.push_back((unsigned long long)v);
  // the batch stream starts after every scene stream's earlier work
  for (int s = 0; s < n; ++s) {
    FLIP_CUDA_NEG(cudaEventRecord(b->ev[s], hs[s]->stream));
    FLIP_CUDA_NEG(cudaStreamWaitEvent(bs, b->ev[s], 0));
  }
  if (!b->graph || b->graph_key != key) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    std::vector<int> cur(n), launches(n);
    std::vector<long long> steps(n);
    std::vector<char> stepped(n);
    for (int s = 0; s < n; ++s) {
      cur[s] = hs[s]->cur;
      launches[s] = hs[s]->launches;
      steps[s] = hs[s]->steps_done;
      stepped[s] = hs[s]->stepped;
    }
    const int bl0 = *batch_launches;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal);
    int rc = FLIP_OK;
    if (e == cudaSuccess) {
      // fork the scene streams into the capture, two steps, join them back
      e = cudaEventRecord(b->ev_solved, bs);
      for (int s = 0; s < n && e == cudaSuccess; ++s)
        e = cudaStreamWaitEvent(hs[s]->stream, b->ev_solved, 0);
      if (e == cudaSuccess) rc = enqueue_step();
      if (e == cudaSuccess && rc == FLIP_OK) rc = enqueue_step();
      for (int s = 0; s < n && e == cudaSuccess && rc == FLIP_OK; ++s) {
        e = cudaEventRecord(b->ev[s], hs[s]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, b->ev[s], 0);
      }
      const cudaError_t e2 = cudaStreamEndCapture(bs, &g);
      if (e == cudaSuccess) e = e2;
    }
    b->graph_launches.assign(n, 0);
    for (int s = 0; s < n; ++s) {
      b->graph_launches[s] = hs[s]->launches - launches[s];
      hs[s]->cur = cur[s];
      hs[s]->launches = launches[s];
      hs[s]->steps_done = steps[s];
      hs[s]->stepped = stepped[s];
    }
    b->graph_batch_launches = *batch_launches - bl0;
    *batch_launches = bl0;
    if (e == cudaSuccess && rc == FLIP_OK && g)
      e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || rc != FLIP_OK || !b->graph) {
      cudaGetLastError();  // not sticky: the plain path takes over
      b->graph = nullptr;
      b->graph_off = true;
      return 0;
    }
    b->graph_key = key;
  }
  for (int p = 0; p < pairs; ++p) FLIP_CUDA_NEG(cudaGraphLaunch(b->graph, bs));
  for (int s = 0; s < n; ++s) {
    hs[s]->launches += pairs * b->graph_launches[s];
    hs[s]->steps_done += 2LL * pairs;
    hs[s]->stepped = true;
  }
  *batch_launches += pairs * b->graph_batch_launches;
  // every scene stream continues after the graph
  FLIP_CUDA_NEG(cudaEventRecord(b->ev_solved, bs));
  for (int s = 0; s < n; ++s) FLIP_CUDA_NEG(cudaStreamWaitEvent(hs[s]->stream, b->ev_solved, 0));
  return 2 * pairs;
}

// The batched (fused) step kernels: CTA ranges of each launch, in this order.
// FL_ACT is the running sum of the scenes' active bricks, written on the device
// each step, which P2G and G2P share out.
enum FusedLaunch { FL_SCAN = 0, FL_ONE, FL_SCATTER, FL_FINALIZE, FL_DIV, FL_ACT,
                   kFusedLaunches };

// Scenes a fused step can take: fixed time step, no reseeding.
bool fusable(const flip_handle* h) { return h->prm.cfl <= 0.0 && !reseeding(h); }

// The table entry of a scene for a step that starts with particle buffer `cur`.
SceneDev scene_dev(const flip_handle* h, int cur) {
  SceneDev d{};
  d.g = h->g;
  d.K = h->K;
  d.src = h->P[cur];
  d.dst = h->P[1 - cur];
  d.B = h->B;
  d.type = h->type;
  for (int a = 0; a < 3; ++a) {
    d.acc[a] = h->acc[a];
    d.uo[a] = h->uo[a];
  }
  d.b32 = h->b32;
  d.b64 = h->b64;
  d.x32 = h->mixed ? nullptr : h->x32;
  d.x64 = h->x64;
  d.pff = h->pff;
  d.bar = h->bar;
  d.st = h->dstats;
  d.np = h->np;
  d.nbricks = h->nbricks;
  return d;
}

// Splits max_blocks CTAs over scenes in proportion to their particle counts
// raised to `exponent`, at least one each (n <= max_blocks).  first has n+1
// entries.
void assign_teams(const std::vector<flip_handle*>& hs, int max_blocks, std::vector<int>& first,
                  double exponent) {
  const int n = (int)hs.size();
  std::vector<double> w(n);
  double tot = 0.0;
  for (int s = 0; s < n; ++s) {
    w[s] = std::pow((double)std::max<long long>(hs[s]->np, 1), exponent);
    tot += w[s];
  }
  std::vector<int> cnt(n, 1);
  int left = max_blocks - n;
  std::vector<std::pair<double, int>> rem;
  for (int s = 0; s < n; ++s) {
    const double share = left * w[s] / tot;
    const int extra = (int)std::floor(share);
    cnt[s] += extra;
    rem.push_back({share - extra, s});
  }
  int used = 0;
  for (int s = 0; s < n; ++s) used += cnt[s];
  std::sort(rem.begin(), rem.end(), [](auto& x, auto& y) { return x.first > y.first; });
  for (size_t q = 0; q < rem.size() && used < max_blocks; ++q, ++used) cnt[rem[q].second] += 1;
  first.assign(n + 1, 0);
  for (int s = 0; s < n; ++s) first[s + 1] = first[s] + cnt[s];
}

}  // namespace

extern "C" {

int flip_batch_create(int32_t capacity, void* stream, flip_batch** out) {
  if (!out) return fail(FLIP_E_ARG, "out is NULL");
  *out = nullptr;
  if (capacity < 1 || capacity > 4096) return fail(FLIP_E_ARG, "capacity must be in [1, 4096]");
  int rc = check_device();
  if (rc) return rc;
  flip_batch* b = new (std::nothrow) flip_batch();
  if (!b) return fail(FLIP_E_OOM, "host allocation failed");
  b->capacity = capacity;
  int sms = 0;
  cudaError_t e = pcg_max_blocks(&b->max_blocks, &sms);
  auto bail = [&](cudaError_t err, const char* what) {
    flip_batch_destroy(b);
    return cuda_fail(err, what);
  };
  if (e != cudaSuccess) return bail(e, "occupancy query");
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(e, "cudaStreamCreate");
    b->own_stream = true;
  }
  if ((e = cudaMalloc(&b->d_args, sizeof(PcgArgs) * (size_t)capacity)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_block_scene, sizeof(int) * (size_t)b->max_blocks)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_team_first, sizeof(int) * (size_t)(capacity + 1))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_scenes, sizeof(SceneDev) * 2 * (size_t)capacity)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_first, sizeof(unsigned int) * kFusedLaunches *
                                       (size_t)(capacity + 1))) != cudaSuccess)
    return bail(e, "cudaMalloc(batch)");
  b->ev.resize(capacity, nullptr);
  for (auto& ev : b->ev)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return bail(e, "cudaEventCreate");
  if ((e = cudaEventCreate(&b->ev_begin)) != cudaSuccess ||
      (e = cudaEventCreate(&b->ev_end)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_solved, cudaEventDisableTiming)) != cudaSuccess)
    return bail(e, "cudaEventCreate");
  *out = b;
  return FLIP_OK;
}

int flip_batch_graph_active(const flip_batch* b) { return (b && b->graph) ? 1 : 0; }

int flip_batch_set_graphs(flip_batch* b, int32_t enable) {
  if (!b) return fail(FLIP_E_ARG, "batch is NULL");
  b->graphs = enable != 0;
  return FLIP_OK;
}

int flip_batch_set_fused(flip_batch* b, int32_t enable) {
  if (!b) return fail(FLIP_E_ARG, "batch is NULL");
  b->fused = enable != 0;
  return FLIP_OK;
}

int flip_batch_set_team_exponent(flip_batch* b, double exponent) {
  if (!b) return fail(FLIP_E_ARG, "batch is NULL");
  if (!(exponent >= 0.0 && exponent <= 3.0)) return fail(FLIP_E_ARG, "exponent must be in [0, 3]");
  b->team_exponent = exponent;
  return FLIP_OK;
}

int flip_batch_autotune(flip_batch* b, flip_handle* const* hs, int32_t n,
                        int32_t steps_per_candidate, double* exponent) {
  if (!b) return fail(FLIP_E_ARG, "batch is NULL");
  if (steps_per_candidate < 1) return fail(FLIP_E_ARG, "steps_per_candidate must be >= 1");
  // The scenes evolve while they are timed (a spreading fluid covers more cells), so
  // each candidate is timed twice, in the order c1..cK then cK..c1, and the two
  // times are added: a cost that drifts linearly with the step cancels out of the
  // comparison.
  static const double cand[] = {0.5, 0.75, 1.0, 1.25, 1.5, 2.0, 2.5};
  constexpr int NC = 7;
  std::vector<flip_stats> st((size_t)std::max(n, 1));
  const double keep = b->team_exponent;
  double sum_ms[NC] = {};
  int first_warning = FLIP_OK;
  for (int pass = 0; pass < 2; ++pass)
    for (int q = 0; q < NC; ++q) {
      const int c = pass == 0 ? q : NC - 1 - q;
      b->team_exponent = cand[c];
      const int rc = flip_batch_step(b, hs, n, steps_per_candidate, st.data());
      if (rc == FLIP_E_NOT_CONVERGED || rc == FLIP_E_CAPACITY) {
        if (first_warning == FLIP_OK) first_warning = rc;
      } else if (rc != FLIP_OK) {
        b->team_exponent = keep;
        return rc;
      }
      sum_ms[c] += n > 0 ? st[0].ms_pcg : 0.0;
    }
  int bc = 0;
  for (int c = 1; c < NC; ++c)
    if (sum_ms[c] < sum_ms[bc]) bc = c;
  const double best = cand[bc];
  b->team_exponent = best;
  if (exponent) *exponent = best;
  // Then the step's form: fused or per-scene launches, each stream-ordered or
  // replayed as CUDA graphs, timed over 2 * steps_per_candidate untimed steps with
  // events on the batch stream (the call joins every scene stream at its end),
  // after one 2-step call that warms the form (and captures its graph).
  struct Form {
    bool fused, graphs;
  };
  static const Form forms[4] = {{true, false}, {true, true}, {false, false}, {false, true}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FLIP_CUDA(cudaEventCreate(&e0));
  FLIP_CUDA(cudaEventCreate(&e1));
  const Form keep_form{b->fused, b->graphs};
  float form_ms[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  int rc = FLIP_OK;
  for (int t = 0; t < 8 && rc == FLIP_OK; ++t) {  // forms 0..3 then 3..0, times added
    const int fi = t < 4 ? t : 7 - t;
    const Form& f = forms[fi];
    b->fused = f.fused;
    b->graphs = f.graphs;
    rc = flip_batch_step(b, hs, n, 2, nullptr);
    cudaError_t e = rc == FLIP_OK ? cudaEventRecord(e0, b->stream) : cudaSuccess;
    if (rc == FLIP_OK && e == cudaSuccess) rc = flip_batch_step(b, hs, n, 2 * steps_per_candidate, nullptr);
    if (rc == FLIP_OK && e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (rc == FLIP_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (rc == FLIP_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rc == FLIP_OK && e != cudaSuccess) rc = cuda_fail(e, "flip_batch_autotune timing");
    if (rc == FLIP_OK) form_ms[fi] += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != FLIP_OK) {
    b->fused = keep_form.fused;
    b->graphs = keep_form.graphs;
    return rc;
  }
  int bf = 0;
  for (int fi = 1; fi < 4; ++fi)
    if (form_ms[fi] < form_ms[bf]) bf = fi;
  b->fused = forms[bf].fused;
  b->graphs = forms[bf].graphs;
  // Then the transfers' launch shapes, the same for every scene: each candidate
  // pair over steps_per_candidate steps with statistics, forward then reverse.  In
  // the fused form each stage keeps its fastest count by the batch-wide stage
  // times; in the per-scene form (stages on the scenes' streams, overlapping) the
  // pair whose calls took least wall time is kept.
  TransferCand tc[3];
  transfer_candidates(tc);
  std::vector<int> keep_p(n), keep_g(n);
  for (int s = 0; s < n; ++s) {
    keep_p[s] = hs[s]->p2g_per_sm;
    keep_g[s] = hs[s]->g2p_per_sm;
  }
  double p_ms[3] = {}, g_ms[3] = {};
  for (int t = 0; t < 6; ++t) {
    const int c = t < 3 ? t : 5 - t;
    for (int s = 0; s < n; ++s) {
      hs[s]->p2g_per_sm = tc[c].p2g;
      hs[s]->g2p_per_sm = tc[c].g2p;
      set_transfer_grids(hs[s]);
    }
    rc = flip_batch_step(b, hs, n, steps_per_candidate, st.data());
    if (rc == FLIP_E_NOT_CONVERGED || rc == FLIP_E_CAPACITY) {
      if (first_warning == FLIP_OK) first_warning = rc;
    } else if (rc != FLIP_OK) {
      for (int s = 0; s < n; ++s) {
        hs[s]->p2g_per_sm = keep_p[s];
        hs[s]->g2p_per_sm = keep_g[s];
        set_transfer_grids(hs[s]);
      }
      return rc;
    }
    if (n > 0) {
      p_ms[c] += b->fused ? st[0].ms_p2g : st[0].ms_total;
      g_ms[c] += b->fused ? st[0].ms_g2p : st[0].ms_total;
    }
  }
  int bp = 0, bg = 0;
  for (int c = 1; c < 3; ++c) {
    if (p_ms[c] < p_ms[bp]) bp = c;
    if (g_ms[c] < g_ms[bg]) bg = c;
  }
  for (int s = 0; s < n; ++s) {
    hs[s]->p2g_per_sm = tc[bp].p2g;
    hs[s]->g2p_per_sm = tc[bg].g2p;
    set_transfer_grids(hs[s]);
  }
  // the device-side conditions of the untimed calls
  for (int s = 0; s < n; ++s) {
    const int r2 = flip_sync(hs[s]);
    if (r2 == FLIP_E_NOT_CONVERGED || r2 == FLIP_E_CAPACITY) {
      if (first_warning == FLIP_OK) first_warning = r2;
    } else if (r2 != FLIP_OK) {
      return r2;
    }
  }
  return first_warning;
}

int flip_batch_get_form(const flip_batch* b, int32_t* fused, int32_t* graphs) {
  if (!b) return fail(FLIP_E_ARG, "batch is NULL");
  if (fused) *fused = b->fused ? 1 : 0;
  if (graphs) *graphs = b->graphs ? 1 : 0;
  return FLIP_OK;
}

void flip_batch_destroy(flip_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto ev : b->ev)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : {b->ev_begin, b->ev_end, b->ev_solved})
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : b->pev)
    if (ev) cudaEventDestroy(ev);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->d_args) cudaFree(b->d_args);
  if (b->d_block_scene) cudaFree(b->d_block_scene);
  if (b->d_team_first) cudaFree(b->d_team_first);
  if (b->d_scenes) cudaFree(b->d_scenes);
  if (b->d_first) cudaFree(b->d_first);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"

namespace {

// flip_batch_step; with join = false (untimed calls only) the batch stream does not
// wait for the scenes' G2P at the end, so the next call's uploads and solve can be
// enqueued behind this call's solve while its G2P still runs on the scene streams
// (the server's overlapped batches).  The caller then learns of each scene's end
// from an event on the scene's stream.
int batch_step_impl(flip_batch* b, flip_handle* const* hs, int32_t n, int32_t nsteps,
                    flip_stats* stats, bool join) {
  if (!b || (!hs && n > 0)) return fail(FLIP_E_ARG, "batch or handles are NULL");
  if (!join && stats) return fail(FLIP_E_ARG, "statistics need the joined form");
  if (n < 0 || n > b->capacity) return fail(FLIP_E_ARG, "n must be in [0, capacity]");
  if (nsteps < 0) return fail(FLIP_E_ARG, "nsteps must be >= 0");
  for (int s = 0; s < n; ++s) {
    if (!hs[s]) return fail(FLIP_E_ARG, "a handle is NULL");
    for (int t = 0; t < s; ++t)
      if (hs[t] == hs[s]) return fail(FLIP_E_ARG, "a scene appears twice in the batch");
  }
  if (n == 0) return FLIP_OK;
  const cudaStream_t bs = b->stream;
  // Group the scenes by solver kernel (precision x preconditioner); each group is
  // one cooperative launch, in chunks of at most max_blocks scenes.
  struct Launch {
    bool mixed, mg;
    std::vector<int> scenes;
    int arg0;  // offset of the group's argument blocks
  };
  std::vector<Launch> launches;
  for (int g = 0; g < 4; ++g) {
    const bool mixed = g & 1, mg = g & 2;
    std::vector<int> sc;
    for (int s = 0; s < n; ++s)
      if (hs[s]->mixed == mixed && (hs[s]->prm.preconditioner != FLIP_PRECOND_JACOBI) == mg)
        sc.push_back(s);
    for (size_t c = 0; c < sc.size(); c += (size_t)b->max_blocks) {
      Launch L{mixed, mg, {}, 0};
      L.scenes.assign(sc.begin() + c, sc.begin() + std::min(sc.size(), c + (size_t)b->max_blocks));
      launches.push_back(L);
    }
  }
  // Argument blocks, CTA->scene tables: uploaded once for the call.
  std::vector<PcgArgs> args;
  std::vector<int> block_scene_all, first_all;
  std::vector<int> bs_off, tf_off;
  for (auto& L : launches) {
    L.arg0 = (int)args.size();
    std::vector<flip_handle*> hv;
    for (int s : L.scenes) {
      hv.push_back(hs[s]);
      args.push_back(pcg_args(hs[s]));
    }
    std::vector<int> first;
    assign_teams(hv, b->max_blocks, first, b->team_exponent);
    bs_off.push_back((int)block_scene_all.size());
    tf_off.push_back((int)first_all.size());
    for (int t = 0; t < (int)hv.size(); ++t)
      for (int c = first[t]; c < first[t + 1]; ++c) block_scene_all.push_back(t);
    first_all.insert(first_all.end(), first.begin(), first.end());
  }
  if ((int)block_scene_all.size() > b->max_blocks * (int)launches.size() ||
      (int)first_all.size() > b->capacity + 1 + (int)launches.size())
    return fail(FLIP_E_ARG, "batch tables overflow");
  // one table region per launch: block_scene entries need max_blocks per launch
  std::vector<int*> d_bs(launches.size()), d_tf(launches.size());
  std::vector<int*> tmp_alloc;
  for (size_t q = 0; q < launches.size(); ++q) {
    if (q == 0) {
      d_bs[q] = b->d_block_scene;
      d_tf[q] = b->d_team_first;
    } else {  // rare: mixed groups in one call; small stream-ordered buffers
      int* p1 = nullptr;
      int* p2 = nullptr;
      FLIP_CUDA(cudaMallocAsync(&p1, sizeof(int) * (size_t)b->max_blocks, bs));
      FLIP_CUDA(cudaMallocAsync(&p2, sizeof(int) * (size_t)(b->capacity + 1), bs));
      tmp_alloc.push_back(p1);
      tmp_alloc.push_back(p2);
      d_bs[q] = p1;
      d_tf[q] = p2;
    }
    const size_t nb = (q + 1 < launches.size() ? bs_off[q + 1] : block_scene_all.size()) - bs_off[q];
    const size_t nf = (q + 1 < launches.size() ? tf_off[q + 1] : first_all.size()) - tf_off[q];
    FLIP_CUDA(cudaMemcpyAsync(d_bs[q], block_scene_all.data() + bs_off[q], sizeof(int) * nb,
                              cudaMemcpyHostToDevice, bs));
    FLIP_CUDA(cudaMemcpyAsync(d_tf[q], first_all.data() + tf_off[q], sizeof(int) * nf,
                              cudaMemcpyHostToDevice, bs));
  }
  FLIP_CUDA(cudaMemcpyAsync(b->d_args, args.data(), sizeof(PcgArgs) * args.size(),
                            cudaMemcpyHostToDevice, bs));
  const bool timed = stats != nullptr;
  std::vector<int> launches0(n);
  for (int s = 0; s < n; ++s) launches0[s] = hs[s]->launches;
  int batch_launches = 0;
  if (timed) {
    // events per step around the batched solves (fused form: around every stage),
    // read once after the call
    while (b->pev.size() < 6 * (size_t)nsteps) {
      cudaEvent_t e = nullptr;
      FLIP_CUDA(cudaEventCreate(&e));
      b->pev.push_back(e);
    }
    FLIP_CUDA(cudaEventRecord(b->ev_begin, bs));
    for (int s = 0; s < n; ++s) {
      FLIP_CUDA(cudaMemcpyAsync(&hs[s]->dstats->cg_iters_mark, &hs[s]->dstats->cg_iters_total,
                                2 * sizeof(long long), cudaMemcpyDeviceToDevice, bs));
      FLIP_CUDA(cudaMemcpyAsync(&hs[s]->dstats->added_mark, &hs[s]->dstats->added_total,
                                2 * sizeof(long long), cudaMemcpyDeviceToDevice, bs));
    }
  }
  // Fused form: every step kernel of every scene in one launch on the batch
  // stream, over a table of the scenes (single-precision scenes first, then the
  // mixed ones, so G2P runs as one launch per precision).
  bool fused = b->fused;
  for (int s = 0; s < n; ++s) fused = fused && fusable(hs[s]);
  std::vector<flip_handle*> order;
  std::vector<unsigned int> first;
  int n32 = 0;
  std::vector<int> cur0(n);
  for (int s = 0; s < n; ++s) cur0[s] = hs[s]->cur;
  if (fused) {
    // the batch stream starts after each scene stream's earlier work
    for (int s = 0; s < n; ++s) {
      FLIP_CUDA(cudaEventRecord(b->ev[s], hs[s]->stream));
      FLIP_CUDA(cudaStreamWaitEvent(bs, b->ev[s], 0));
    }
    for (int s = 0; s < n; ++s)
      if (!hs[s]->mixed) order.push_back(hs[s]);
    n32 = (int)order.size();
    for (int s = 0; s < n; ++s)
      if (hs[s]->mixed) order.push_back(hs[s]);
    std::vector<SceneDev> tab(2 * (size_t)n);
    for (int q = 0; q < n; ++q) {
      tab[q] = scene_dev(order[q], order[q]->cur);
      tab[n + q] = scene_dev(order[q], 1 - order[q]->cur);
    }
    const size_t W = (size_t)n + 1;
    first.assign(kFusedLaunches * W, 0u);
    for (int q = 0; q < n; ++q) {
      const flip_handle* h = order[q];
      const long long faces = h->nf[0] + h->nf[1] + h->nf[2];
      const unsigned int cnt[5] = {(h->nbricks + 7u) / 8u, 1u,
                                   (unsigned int)((h->np + 511) / 512),
                                   (unsigned int)((faces + 1023) / 1024),
                                   (unsigned int)h->g.ny * (unsigned int)h->g.nz};
      const int which[5] = {FL_SCAN, FL_ONE, FL_SCATTER, FL_FINALIZE, FL_DIV};
      for (int k = 0; k < 5; ++k) first[which[k] * W + q + 1] = first[which[k] * W + q] + cnt[k];
    }
    FLIP_CUDA(cudaMemcpyAsync(b->d_scenes, tab.data(), sizeof(SceneDev) * tab.size(),
                              cudaMemcpyHostToDevice, bs));
    FLIP_CUDA(cudaMemcpyAsync(b->d_first, first.data(), sizeof(unsigned int) * first.size(),
                              cudaMemcpyHostToDevice, bs));
  }
  // every scene stream starts after the call's uploads (and the begin event)
  FLIP_CUDA(cudaEventRecord(b->ev_solved, bs));
  for (int s = 0; s < n; ++s) FLIP_CUDA(cudaStreamWaitEvent(hs[s]->stream, b->ev_solved, 0));
  float ms_pcg = 0.0f;
  float ms_stage[5] = {0, 0, 0, 0, 0};  // fused form: bin, P2G, divergence, solve, G2P
  int timed_steps = 0;
  // One step of every scene in the fused form, all on the batch stream.
  auto enqueue_fused = [&]() -> int {
    const size_t W = (size_t)n + 1;
    const int par = (hs[0]->cur == cur0[0]) ? 0 : 1;  // every scene flips its buffers per step
    const SceneDev* tab = b->d_scenes + (size_t)par * n;
    auto L = [&](int k, int off, int cnt) {
      return BatchLaunch{tab + off, b->d_first + k * W + off, cnt};
    };
    auto total = [&](int k, int off, int cnt) { return first[k * W + off + cnt] - first[k * W + off]; };
    cudaEvent_t* E = timed ? b->pev.data() + 6 * (size_t)timed_steps : nullptr;
    if (timed) FLIP_CUDA(cudaEventRecord(E[0], bs));
    unsigned int* act = b->d_first + FL_ACT * W;  // the active bricks' running sum
    launch_bin_batch(L(FL_SCAN, 0, n), total(FL_SCAN, 0, n), L(FL_ONE, 0, n), bs);
    launch_active_prefix(tab, n, act, bs);
    launch_scatter_batch(L(FL_SCATTER, 0, n), total(FL_SCATTER, 0, n), bs);
    for (auto* h : order) h->cur = 1 - h->cur;
    if (timed) FLIP_CUDA(cudaEventRecord(E[1], bs));
    launch_p2g_batch(BatchLaunch{tab, act, n}, (unsigned)order[0]->p2g_blocks, bs);
    launch_finalize_batch(L(FL_FINALIZE, 0, n), total(FL_FINALIZE, 0, n), bs);
    if (timed) FLIP_CUDA(cudaEventRecord(E[2], bs));
    launch_divergence_batch(L(FL_DIV, 0, n), total(FL_DIV, 0, n), bs);
    batch_launches += 7;
    if (timed) FLIP_CUDA(cudaEventRecord(E[3], bs));
    for (size_t q = 0; q < launches.size(); ++q) {
      const Launch& Lq = launches[q];
      PcgBatch pb{b->d_args + Lq.arg0, d_bs[q], d_tf[q], (int)Lq.scenes.size()};
      const int nblk = first_all[tf_off[q] + (int)Lq.scenes.size()];
      if (Lq.mg) FLIP_CUDA(launch_pcg_mg_batch(pb, Lq.mixed, nblk, bs));
      else FLIP_CUDA(launch_pcg_batch(pb, Lq.mixed, nblk, bs));
      ++batch_launches;
    }
    if (timed) FLIP_CUDA(cudaEventRecord(E[4], bs));
    // G2P reads its scenes from the table offset by the group's first scene
    if (n32 > 0) {
      launch_g2p_batch(BatchLaunch{tab, act, n32}, (unsigned)order[0]->g2p_blocks, false, bs);
      ++batch_launches;
    }
    if (n32 < n) {
      launch_g2p_batch(BatchLaunch{tab + n32, act + n32, n - n32},
                       (unsigned)order[0]->g2p_blocks, true, bs);
      ++batch_launches;
    }
    if (timed) FLIP_CUDA(cudaEventRecord(E[5], bs));
    for (auto* h : order) {
      ++h->steps_done;
      h->stepped = true;
      h->near_stale = true;  // the whole-grid batch kernels ran, not the marks
    }
    FLIP_CUDA(cudaGetLastError());
    if (timed) ++timed_steps;
    return FLIP_OK;
  };
  // One step of every scene, enqueued on the scene streams and the batch stream.
  auto enqueue_step = [&]() -> int {
    if (fused) return enqueue_fused();
    for (int s = 0; s < n; ++s) {
      flip_handle* h = hs[s];
      const float* uo[3] = {h->uo[0], h->uo[1], h->uo[2]};
      launch_front(h, h->stream);
      launch_p2g(h->g, h->P[h->cur], h->B, h->acc, h->dstats, h->p2g_blocks, h->stream);
      FLIP_CUDA(launch_finalize_near(h->g, h->B.brick_count, h->hmark, h->hrow, h->hlist,
                                     h->hlist_n, h->acc, h->uo, h->bar, h->dstats, h->sm_count,
                                     h->near_stale, h->stream));
      launch_divergence_near(h->g, h->K, h->type, uo, h->b32, h->b64, h->x32, h->x64, h->pff,
                             h->bar, h->dstats, h->hlist, h->hlist_n, h->sm_count,
                             h->near_stale, h->stream);
      h->near_stale = false;
      h->launches += 4;
      FLIP_CUDA(cudaEventRecord(b->ev[s], h->stream));
      FLIP_CUDA(cudaStreamWaitEvent(bs, b->ev[s], 0));
    }
    if (timed) FLIP_CUDA(cudaEventRecord(b->pev[2 * (size_t)timed_steps], bs));
    for (size_t q = 0; q < launches.size(); ++q) {
      const Launch& L = launches[q];
      PcgBatch pb{b->d_args + L.arg0, d_bs[q], d_tf[q], (int)L.scenes.size()};
      const int nblk = first_all[tf_off[q] + (int)L.scenes.size()];
      if (L.mg) FLIP_CUDA(launch_pcg_mg_batch(pb, L.mixed, nblk, bs));
      else FLIP_CUDA(launch_pcg_batch(pb, L.mixed, nblk, bs));
      ++batch_launches;
    }
    if (timed) FLIP_CUDA(cudaEventRecord(b->pev[2 * (size_t)timed_steps + 1], bs));
    FLIP_CUDA(cudaEventRecord(b->ev_solved, bs));
    for (int s = 0; s < n; ++s) {
      flip_handle* h = hs[s];
      const float* uo[3] = {h->uo[0], h->uo[1], h->uo[2]};
      FLIP_CUDA(cudaStreamWaitEvent(h->stream, b->ev_solved, 0));
      launch_g2p(h->g, h->K, h->P[h->cur], h->B, uo, h->mixed ? nullptr : h->x32, h->pff,
                 h->dstats, g2p_count(h), h->g2p_blocks, h->has_pmap ? &h->pmap : nullptr,
                 h->stream);
      h->launches += (g2p_count(h) > 0);
      launch_back(h, h->stream);
      h->stepped = true;
    }
    FLIP_CUDA(cudaGetLastError());
    if (timed) ++timed_steps;
    return FLIP_OK;
  };
  int done = 0;
  if (b->graphs && !timed && nsteps >= 2 && tmp_alloc.empty() && !b->graph_off) {
    bool reseed = false;
    for (int s = 0; s < n; ++s) reseed |= reseeding(hs[s]);
    if (!reseed) {
      int rc = batch_graph_steps(b, hs, n, nsteps / 2, first_all, enqueue_step, &batch_launches);
      if (rc < 0) return -rc;
      done = rc;
    }
  }
  for (int st = done; st < nsteps; ++st)
    if (int rc = enqueue_step()) return rc;
  for (void* p : tmp_alloc) FLIP_CUDA(cudaFreeAsync(p, bs));
  // fused: the scene streams continue after the batch stream's work
  if (fused) {
    FLIP_CUDA(cudaEventRecord(b->ev_solved, bs));
    for (int s = 0; s < n; ++s) FLIP_CUDA(cudaStreamWaitEvent(hs[s]->stream, b->ev_solved, 0));
  }
  // the batch stream joins every scene stream at the end of the call
  if (join && !fused)
    for (int s = 0; s < n; ++s) {
      FLIP_CUDA(cudaEventRecord(b->ev[s], hs[s]->stream));
      FLIP_CUDA(cudaStreamWaitEvent(bs, b->ev[s], 0));
    }
  if (!timed) return FLIP_OK;
  FLIP_CUDA(cudaEventRecord(b->ev_end, bs));
  FLIP_CUDA(cudaEventSynchronize(b->ev_end));
  float ms_total = 0.0f;
  FLIP_CUDA(cudaEventElapsedTime(&ms_total, b->ev_begin, b->ev_end));
  for (int st = 0; st < timed_steps; ++st) {
    if (fused) {
      const cudaEvent_t* E = b->pev.data() + 6 * (size_t)st;
      for (int q = 0; q < 5; ++q) {
        float t = 0.0f;
        FLIP_CUDA(cudaEventElapsedTime(&t, E[q], E[q + 1]));
        ms_stage[q] += t;
      }
    } else {
      float t = 0.0f;
      FLIP_CUDA(cudaEventElapsedTime(&t, b->pev[2 * (size_t)st], b->pev[2 * (size_t)st + 1]));
      ms_pcg += t;
    }
  }
  if (fused) ms_pcg = ms_stage[3];
  int first_rc = FLIP_OK;
  for (int s = 0; s < n; ++s) {
    flip_handle* h = hs[s];
    flip_stats* o = stats + s;
    std::memset(o, 0, sizeof(*o));
    const float* uo[3] = {h->uo[0], h->uo[1], h->uo[2]};
    FLIP_CUDA(cudaMemsetAsync(h->norms, 0, 2 * sizeof(double), h->stream));
    if (h->stepped) {
      launch_div_norms(h->g, h->K, h->type, uo, h->mixed ? nullptr : h->x32, h->x64, h->norms,
                       h->stream);
      h->launches += 1;
    }
    double norms[2] = {0.0, 0.0};
    FLIP_CUDA(cudaMemcpyAsync(norms, h->norms, sizeof(norms), cudaMemcpyDeviceToHost, h->stream));
    const int rc = take_status(h);
    if (rc != FLIP_OK && first_rc == FLIP_OK) first_rc = rc;
    const DevStats& d = *h->hstats;
    o->steps = nsteps;
    o->n_particles = h->np;
    o->particles_added = d.added_total - d.added_mark;
    o->particles_removed = d.removed_total - d.removed_mark;
    o->n_fluid_cells = d.n_fluid;
    o->n_active_bricks = d.n_active;
    o->cg_iterations = d.cg_iters_total - d.cg_iters_mark;
    o->ir_iterations = (int32_t)(d.ir_iters_total - d.ir_iters_mark);
    o->kernel_launches = h->launches - launches0[s] + (s == 0 ? batch_launches : 0);
    o->cg_rel_residual = d.rel_res;
    o->rel_divergence = norms[0] > 0.0 ? std::sqrt(norms[1] / norms[0]) : 0.0;
    float msf;
    std::memcpy(&msf, &d.max_speed_bits, sizeof(float));
    o->max_speed = msf;
    o->dt_last = h->prm.cfl > 0.0 ? d.dt_cur : h->prm.dt;
    o->ms_pcg = ms_pcg;
    o->ms_total = ms_total;
    if (fused) {  // the batch-wide stage times (every scene's stages run in one launch)
      o->ms_bin = ms_stage[0];
      o->ms_p2g = ms_stage[1];
      o->ms_divergence = ms_stage[2];
      o->ms_g2p = ms_stage[4];
    }
  }
  return first_rc;
}

}  // namespace

extern "C" int flip_batch_step(flip_batch* b, flip_handle* const* hs, int32_t n, int32_t nsteps,
                               flip_stats* stats) {
  return batch_step_impl(b, hs, n, nsteps, stats, true);
}

namespace flipk {
// One step of the scenes on the batch, without the final join (see batch_step_impl).
int batch_step_overlapped(flip_batch* b, flip_handle* const* hs, int n) {
  return batch_step_impl(b, hs, n, 1, nullptr, false);
}
// The stream a handle's kernels run on.
cudaStream_t handle_stream(const flip_handle* h) { return h ? h->stream : nullptr; }
// The device address of a handle's sticky status word (DEV_* bits).
int* handle_status_word(const flip_handle* h) { return h ? &h->dstats->status : nullptr; }
}  // namespace flipk

extern "C" {

int flip_solve_pressure(const flip_params* params, const uint8_t* type, const float* b, float* p,
                        void* stream, int32_t* iterations, double* rel_residual) {
  int rc = check_params(params, false);
  if (rc) return rc;
  if (params->precision != FLIP_PREC_FP32)
    return fail(FLIP_E_ARG, "flip_solve_pressure runs the FP32 solver only");
  if (!type || !b || !p) return fail(FLIP_E_ARG, "type, b and p must be device pointers");
  rc = check_device();
  if (rc) return rc;
  const cudaStream_t s = (cudaStream_t)stream;
  const Grid g = make_grid(*params);
  const long long nc = (long long)g.nx * g.ny * g.nz;
  const unsigned int nb = (unsigned)g.bx * g.by * g.bz;
  int blocks = 0, sms = 0;
  FLIP_CUDA(pcg_max_blocks(&blocks, &sms));
  // scratch: r, p_a, p_b, q, brick flags, active list, partials, barrier, stats
  Carver cv;
  auto lay = [&](Carver& c, float** r, float** pa, float** pb, float** q, unsigned int** bf,
                 unsigned int** act, double** part, unsigned int** bar, DevStats** st) {
    *r = c.take<float>((size_t)nc);
    *pa = c.take<float>((size_t)nc);
    *pb = c.take<float>((size_t)nc);
    *q = c.take<float>((size_t)nc);
    *bf = c.take<unsigned int>(nb);
    *act = c.take<unsigned int>(nb);
    *part = c.take<double>((size_t)PCG_SLOTS * blocks);
    *bar = c.take<unsigned int>(BAR_WORDS);
    *st = c.take<DevStats>(1);
  };
  float *r, *pa_, *pb_, *q;
  unsigned int *bf, *act, *bar;
  double* part;
  DevStats* st;
  lay(cv, &r, &pa_, &pb_, &q, &bf, &act, &part, &bar, &st);
  void* arena = nullptr;
  FLIP_CUDA(cudaMallocAsync(&arena, cv.off, s));
  Carver as;
  as.base = (char*)arena;
  lay(as, &r, &pa_, &pb_, &q, &bf, &act, &part, &bar, &st);
  DevStats hst{};
  cudaError_t e = cudaMemsetAsync(arena, 0, cv.off, s);
  if (e == cudaSuccess) {
    launch_zero_off_fluid(g, type, p, bar, s);
    launch_mark_bricks(g, type, bf, s);
    launch_compact_bricks(g, bf, act, st, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    PcgArgs a{};
    a.g = g;
    fill_pcg_tables(a, *params);
    a.type = type;
    a.active = act;
    a.n_active = &st->n_active;
    a.b32 = b;
    a.x32 = p;
    a.r = r;
    a.pa = pa_;
    a.pb = pb_;
    a.q = q;
    a.partials = part;
    a.bar = bar;
    a.status = &st->status;
    a.stats = st;
    a.tol = params->cg_tol;
    a.max_iter = params->cg_max_iter;
    a.check_singular = 1;
    a.timeout_ns = kBarrierWaitNs;
    e = launch_pcg(a, false, blocks, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, st, sizeof(DevStats), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaFreeAsync(arena, s);
  cudaError_t e3 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "flip_solve_pressure");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  if (e3 != cudaSuccess) return cuda_fail(e3, "flip_solve_pressure sync");
  if (iterations) *iterations = hst.cg_iters;
  if (rel_residual) *rel_residual = hst.rel_res;
  return status_to_code(hst.status);
}

}  // extern "C"

namespace flipk {
int api_check_params(const flip_params* p, bool with_particles) {
  return check_params(p, with_particles);
}
int api_check_device() { return check_device(); }
Grid api_make_grid(const flip_params& p) { return make_grid(p); }
void api_fill_pcg_tables(PcgArgs& a, const flip_params& p) { fill_pcg_tables(a, p); }
int api_status_to_code(int dev_status) { return status_to_code(dev_status); }
unsigned long long api_barrier_wait_ns() { return kBarrierWaitNs; }

// The current particle buffer of a handle and its stream (for k_surface.cu).
bool handle_particles(flip_handle* h, PartView* p, long long* np, cudaStream_t* s) {
  if (!h || refresh_np(h) != FLIP_OK) return false;
  *p = h->P[h->cur];
  *np = h->np;
  *s = h->stream;
  return true;
}
}  // namespace flipk
