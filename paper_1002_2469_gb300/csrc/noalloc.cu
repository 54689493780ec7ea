// noalloc.cu -- dichotomy_solve_noalloc: a single-system solve that allocates nothing.
//
// Some callers cannot allocate device memory at all: code that runs under a framework whose
// allocator owns the whole device, plugins that may not call cudaMalloc, or callers that must
// not allocate inside a latency-critical or restricted section.  For them this entry point
// takes only the coefficients, the size and the caller's F and x.  The plan record, its tables
// and the device status word live in one file-scope __device__ array of fixed size
// (kNoAllocScratchBytes) that every GPU loading this library keeps until the process exits;
// the host-side staging copy lives in a static host buffer.  No cudaMalloc, cudaFree or
// other allocating routine is called.
//
// Sharing: every call writes the plan of its own system into the same array (the device
// status word included, cleared on every call), so two calls whose kernels overlap on the
// GPU -- different streams, or different host threads -- race on it; calls on one stream are
// ordered and safe.  The first call on a device looks the array's device address up
// (cudaGetSymbolAddress, with that device current).  The plan goes from the static host buffer
// to the array by a copy from pageable memory, which may hold the host until the stream has
// reached it; a stream that is being captured is refused (the captured copy would replay the
// buffer's later contents).  No device status is reported: the word is cleared by every call.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/dichotomy.h"
#include "launch.cuh"
#include "planner.cuh"

using namespace dich;
using namespace dich::plan;

constexpr size_t kNoAllocScratchBytes = 256 * 1024;

// The scratch array: plan record, status word and tables of the most recent call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr size_t kRecBytes = 512;       // plan record region
constexpr size_t kStatusOff = 512;      // device status word
constexpr size_t kTabOff = 768;         // tables
constexpr int kMaxDevices = 64;

static_assert(sizeof(SysPlan) <= kRecBytes, "plan record must fit its region");

std::mutex g_mu;                         // guards the set-up table and the host staging buffer
void* g_addr[kMaxDevices] = {nullptr};   // device address of g_noalloc_scratch per device
alignas(256) unsigned char g_stage[kNoAllocScratchBytes];

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) return DICH_ERR_UNSUPPORTED;
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DICH_OK;
}

}  // namespace

extern "C" int dichotomy_solve_noalloc(double t_m1, double t_0, double t_1, int64_t N, const double* d_F,
                                       double* d_x, void* stream) {
  if (N < 0) return DICH_ERR_ARG;
  int rc = validate_t(t_m1, t_0, t_1);
  if (rc) return rc;
  if (N == 0) return DICH_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // the staging copy reads the static host buffer, which the next call overwrites: a captured
  // copy would replay whatever plan the buffer holds then, so a capturing stream is refused
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(st, &cap);
  if (ce != cudaSuccess) return cuda_fail(ce);
  if (cap != cudaStreamCaptureStatusNone) return DICH_ERR_UNSUPPORTED;
  if (!d_F || !d_x || !aligned8(d_F) || !aligned8(d_x)) return DICH_ERR_ARG;
  const size_t nb = sizeof(double) * (size_t)N;
  if (overlap(d_F, nb, d_x, nb)) return DICH_ERR_ALIAS;
  if (!is_device_ptr(d_F) || !is_device_ptr(d_x)) return DICH_ERR_ARG;

  std::lock_guard<std::mutex> lock(g_mu);
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;

  // plan (the Toeplitz preliminary step) into the static host staging buffer
  Opts o;
  o.prec = DICH_PREC_AUTO;
  const Roots r = toeplitz_roots(t_m1, t_0, t_1);
  const int form = pick_form(o.prec, r);
  const int NT = default_threads(form);
  std::memset(g_stage, 0, kTabOff);
  SysBuild sb;
  sb.ext = reinterpret_cast<double*>(g_stage + kTabOff);
  sb.ext_cap = (kNoAllocScratchBytes - kTabOff) / sizeof(double);
  int n = 2;
  if (N >= 2) {
    const int nmax = max_rows(NT, form, kSmemBudget);
    n = choose_n(N, window_blocks(NT, form), nmax, 0, default_rows(form));
    rc = build_system(t_m1, t_0, t_1, N, NT, form, n, o, true, sb);
    if (rc) return rc;                                  // DICH_ERR_WORKSPACE: tables exceed the array
  } else {
    sb.rec.N = N;
    sb.rec.t0 = t_0;
    sb.ext_used = 0;
  }
  sb.rec.tab = 0;
  std::memcpy(g_stage, &sb.rec, sizeof(SysPlan));
  const size_t bytes = kTabOff + sizeof(double) * sb.ext_used;
  // general path: per-block beta and first/last values and the chunk scan after the tables
  const int64_t P = (N >= 2) ? sb.rec.P : 0;
  const size_t off_beta = align_up(bytes);
  const size_t off_iface = align_up(off_beta + sizeof(double) * 2 * (size_t)P);
  const size_t off_scan = align_up(off_iface + sizeof(double) * 2 * (size_t)P);
  const size_t end_general = off_scan + sizeof(double) * 6 * (size_t)ceil_div(P, kScanChunk);
  if (sb.path == PATH_GENERAL && end_general > kNoAllocScratchBytes) return DICH_ERR_WORKSPACE;
  // pageable source: the call returns once the staging buffer has been consumed
  cudaError_t e = cudaMemcpyAsync(base, g_stage, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);

  const SysPlan* d_plan = reinterpret_cast<const SysPlan*>(base);
  if (N == 1) {
    e = launch_trivial(d_plan, nullptr, 1, d_F, d_x, nullptr, nullptr, nullptr, 0, st);
    return e == cudaSuccess ? DICH_OK : cuda_fail(e);
  }
  WinArgs a{};
  a.plans = d_plan;
  a.tabs = reinterpret_cast<const double*>(static_cast<unsigned char*>(base) + kTabOff);
  a.items = nullptr;
  a.F = d_F;
  a.x = d_x;
  a.status = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(base) + kStatusOff);
  a.mode = MODE_FULL;
  a.n_smem = n;
  a.bulk = 1;   // F and x are device memory (checked above)
  const int64_t tiles = ceil_div(sb.rec.P, sb.rec.own);
  const size_t smem = smem_bytes(NT, n, form);
  auto launch = [&](const WinArgs& w) {
    return (form == FORM_F64) ? launch_window_f64(NT, (int)tiles, smem, st, w)
                              : launch_window_mixed(NT, (int)tiles, smem, st, w);
  };
  unsigned char* b = static_cast<unsigned char*>(base);
  if (sb.path != PATH_GENERAL) {
    e = launch(a);
  } else {
    double* beta = reinterpret_cast<double*>(b + off_beta);
    double* iface = reinterpret_cast<double*>(b + off_iface);
    WinArgs w = a;
    w.mode = MODE_BETA;
    w.beta = beta;
    e = launch(w);
    if (e == cudaSuccess)
      e = launch_block_scan(d_plan, a.tabs, P, beta, iface, reinterpret_cast<double*>(b + off_scan), st);
    if (e == cudaSuccess) {
      a.mode = MODE_APPLY;
      a.iface = iface;
      e = launch(a);
    }
  }
  return e == cudaSuccess ? DICH_OK : cuda_fail(e);
}
