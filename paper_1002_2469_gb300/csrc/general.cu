// general.cu -- general (non-Toeplitz) tridiagonal systems behind the dichotomy_gen_* entry
// points of include/dichotomy.h: the O(N) preliminary step of the Dichotomy Algorithm (Sec. 2.3)
// on the host at plan time or on the device at bind time (gen_prelim.cuh), the choice of the
// precision form and of the path, the solves by the window kernels of window_gen.cuh (FP64 or
// float-float), and the a posteriori residual check for matrices without dominance.
//
// Preliminary step, in the terms of the Toeplitz restatement (exterior ratios and block maps
// from the homogeneous solutions phi, vanishing left of row 0, and psi, vanishing right of row
// N-1): the whole-system forward elimination factors cp_i = c_i / (b_i - a_i cp_{i-1}) give
// phi_i / phi_{i+1} = -cp_i, the backward ones cq_i = a_i / (b_i - c_i cq_{i+1}) give
// psi_i / psi_{i-1} = -cq_i.  Per block m = [s, e]:
//   kL = -cp_{s-1}, kR = -cq_{e+1} (zero at the system ends),
//   a = prod_{i=s+1..e+1} (-cq_i), b = kR, c = prod_{i=s-1..e-1} (-cp_i), d = kL,
//   tL = prod_{i=s..e-1} (-cp_i) = phi_s / phi_e, tR = prod_{i=s+1..e} (-cq_i) = psi_e / psi_s,
//   the block's own Thomas factors and spikes v = T_m^-1 (-a_s e_0), w = T_m^-1 (-c_e e_{n-1}),
//   M = (I - [[kL v_0, kR w_0], [kL v_end, kR w_end]])^-1 (eq. 16 restated).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/dichotomy.h"
#include "launch.cuh"
#include "planner.cuh"
#include "gen_prelim.cuh"
#include "window_gen.cuh"

using namespace dich;
using namespace dich::plan;

namespace dich {

template <int NT>
static cudaError_t launch_gen_one(int grid, int grid_y, size_t smem, cudaStream_t st, const GenArgs& a) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_window_gen<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, grid_y);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_window_gen<NT>, a);
}

template <int NT>
static cudaError_t launch_gen_ff_one(int grid, int grid_y, size_t smem, cudaStream_t st, const GenArgs& a) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_window_gen_ff<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, grid_y);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_window_gen_ff<NT>, a);
}

static cudaError_t launch_window_gen(int NT, int grid, size_t smem, cudaStream_t st, const GenArgs& a, int grid_y,
                                     int form) {
  if (form == FORM_MIXED) {
    switch (NT) {
      case 64: return launch_gen_ff_one<64>(grid, grid_y, smem, st, a);
      case 128: return launch_gen_ff_one<128>(grid, grid_y, smem, st, a);
      case 256: return launch_gen_ff_one<256>(grid, grid_y, smem, st, a);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (NT) {
    case 64: return launch_gen_one<64>(grid, grid_y, smem, st, a);
    case 128: return launch_gen_one<128>(grid, grid_y, smem, st, a);
    case 256: return launch_gen_one<256>(grid, grid_y, smem, st, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dich

namespace dich {

// the a posteriori check: max |F - A x|, max |x|, max |F| (bits of non-negative doubles)
__global__ void __launch_bounds__(256) k_gen_residual(int64_t N, const double* a, const double* b, const double* c,
                                                       const double* F, const double* x, unsigned long long* res) {
  double r = 0.0, xm = 0.0, fm = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double ax = b[i] * x[i];
    if (i > 0) ax = fma(a[i], x[i - 1], ax);
    if (i + 1 < N) ax = fma(c[i], x[i + 1], ax);
    r = fmax(r, fabs(F[i] - ax));
    xm = fmax(xm, fabs(x[i]));
    fm = fmax(fm, fabs(F[i]));
  }
  for (int d = 16; d > 0; d >>= 1) {
    r = fmax(r, __shfl_xor_sync(0xffffffffu, r, d));
    xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, d));
    fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, d));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&res[0], (unsigned long long)__double_as_longlong(r));
    atomicMax(&res[1], (unsigned long long)__double_as_longlong(xm));
    atomicMax(&res[2], (unsigned long long)__double_as_longlong(fm));
  }
}

}  // namespace dich

struct dich_gen_s {
  int64_t N = 0;
  Opts opts;
  int NT = 64;
  int path = PATH_SINGLE;
  int form = FORM_F64;                // FP64 or MIXED (float-float rows)
  int64_t tiles = 0;
  int64_t stride = 0;                 // doubles per per-row field
  SysPlan rec{};                      // geometry record read by the kernels
  std::vector<double> recs;           // block records, kBC doubles per block (host preliminary)
  std::vector<double> rows;           // per-row fields (window_gen.cuh layout; host preliminary)
  bool device_prelim = false;         // preliminary step on the device at bind time
  double norm_inf = 0.0;              // ||A||_inf, for the backward error of the residual check
  double gamma = 1.0;                 // largest block map factor (at least 1): the a priori growth base
  size_t off_res = 0;                 // residual check: 3 maxima
  std::vector<double> ha, hb, hc;     // the matrix, kept for the device preliminary
  size_t ws_bytes = 0, off_plan = 0, off_status = 0, off_recs = 0, off_rows = 0, off_beta = 0, off_iface = 0,
         off_scan = 0, off_raw = 0, off_comp = 0, off_chunk = 0, off_max = 0;
  char* d_ws = nullptr;
};

namespace {

// default geometry (measured on GB300 at N = 2^24): the FP64 kernel is bound by its FP64 pipe and
// prefers 32-row blocks in 64-thread windows; the float-float kernel, bound by the latency of its
// coefficient loads, prefers 16-row blocks in 128-thread windows (more warps per SM).  AUTO plans
// take the float-float geometry, as they usually run in that form.
constexpr int kGenDefaultRows = 32;
constexpr int kGenDefaultRowsFF = 16;
constexpr int64_t kGenDevicePrelimMin = 1 << 15;   // default: device preliminary from this many rows

// block geometry (block size n, P blocks, the last one nlast rows); returns a status code
int gen_geometry(dich_gen_s* g, double b0) {
  const int64_t N = g->N;
  SysPlan& r = g->rec;
  std::memset(&r, 0, sizeof(r));
  r.N = N;
  r.t0 = b0;
  if (N == 1) return DICH_OK;
  const int NT = g->NT;
  const size_t budget = g->opts.n_req > 0 ? kSmemMax : kSmemBudget;
  int nmax = 2;
  while (window_gen_smem_bytes(NT, nmax + 1) <= budget) ++nmax;
  const int n = choose_n(N, NT, nmax, g->opts.n_req, g->opts.prec == DICH_PREC_F64 ? kGenDefaultRows : kGenDefaultRowsFF);
  const int64_t P = ceil_div(N, n);
  r.n = n;
  r.P = P;
  r.nlast = (int)(N - (P - 1) * (int64_t)n);
  if (r.nlast < 2) return DICH_ERR_ARG;
  r.kl = (int32_t)std::min<int64_t>(P, INT32_MAX);
  r.kr = 0;
  r.form = FORM_F64;
  r.own = NT;
  g->path = (P <= NT) ? PATH_SINGLE : PATH_GENERAL;   // final once the largest map factors are known
  g->tiles = ceil_div(P, (int64_t)NT);
  const int64_t Ppad = (P + 31) / 32 * 32;
  g->stride = Ppad * n;
  return DICH_OK;
}

// windows: one window, halo windows (coupling beyond the halo below eps), or the general path,
// from the largest |a| over blocks 0..P-2 and |c| over blocks 1..P-1 of the block maps
void gen_decide(dich_gen_s* g, double amax, double cmax) {
  g->gamma = std::max({1.0, amax, cmax});
  SysPlan& r = g->rec;
  const int64_t P = r.P;
  const int NT = g->NT;
  const double eps = g->opts.eps;
  auto halo_of = [&](double mx) -> int64_t {
    if (mx == 0.0) return 1;
    if (mx >= 1.0) return P;
    return (int64_t)std::ceil(std::log(eps) / std::log(mx)) + 1;
  };
  const int64_t hl = halo_of(amax), hr = halo_of(cmax);
  r.hl = r.hr = 0;
  if (P <= NT) {
    g->path = PATH_SINGLE;
    r.own = (int32_t)P;
  } else if (!(g->opts.flags & DICH_FLAG_FORCE_GENERAL) && hl + hr <= NT / 2) {
    g->path = PATH_HALO;
    r.hl = (int32_t)hl;
    r.hr = (int32_t)hr;
    r.own = (int32_t)(NT - hl - hr);
  } else {
    g->path = PATH_GENERAL;
    r.own = NT;
  }
  g->tiles = ceil_div(P, (int64_t)r.own);
}

// precision form.  MIXED needs the factors within 2^-40..2^40 for its float range; its error grows
// with the error gains of the two recurrences, gf (largest 1 + |a_i rd_i| gf_{i-1} over the rows
// of a block) and gb (largest 1 + |cp_i| gb_{i+1}), which for a Toeplitz matrix are 1/(1 - |rs|)
// and 1/(1 - |ib|): AUTO takes MIXED while gf + gb <= 24, as the Toeplitz policy does.
int gen_choose_form(dich_gen_s* g, double gf, double gb, double rmax, double rmin, double omax) {
  const double big = 1099511627776.0;   // 2^40
  const bool range = rmax <= big && rmin >= 1.0 / big && omax <= big;
  g->form = FORM_F64;
  if (g->opts.prec == DICH_PREC_MIXED) {
    if (!range) return DICH_ERR_UNSUPPORTED;
    g->form = FORM_MIXED;
  } else if (g->opts.prec == DICH_PREC_AUTO && range && gf + gb <= 24.0) {
    g->form = FORM_MIXED;
  }
  return DICH_OK;
}

// the O(N) preliminary step on the host; returns a status code
int gen_host_tables(dich_gen_s* g, const double* a, const double* b, const double* c) {
  const int64_t N = g->N;
  const SysPlan& r = g->rec;
  const int n = r.n;
  const int64_t P = r.P;

  // whole-system elimination factors
  std::vector<double> cp((size_t)N), cq((size_t)N);
  double prev = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const double den = b[i] - (i > 0 ? a[i] * prev : 0.0);
    if (den == 0.0 || !std::isfinite(den)) return DICH_ERR_SINGULAR;
    prev = (i < N - 1 ? c[i] : 0.0) / den;
    cp[(size_t)i] = prev;
  }
  prev = 0.0;
  for (int64_t i = N - 1; i >= 0; --i) {
    const double den = b[i] - (i < N - 1 ? c[i] * prev : 0.0);
    if (den == 0.0 || !std::isfinite(den)) return DICH_ERR_SINGULAR;
    prev = (i > 0 ? a[i] : 0.0) / den;
    cq[(size_t)i] = prev;
  }

  g->rows.assign((size_t)(kGenFields * g->stride), 0.0);
  g->recs.assign((size_t)(P * kBC), 0.0);
  double* fa = g->rows.data() + GF_A * g->stride;
  double* frd = g->rows.data() + GF_RD * g->stride;
  double* fcp = g->rows.data() + GF_CP * g->stride;
  double* fv = g->rows.data() + GF_V * g->stride;
  double* fw = g->rows.data() + GF_W * g->stride;
  std::vector<double> lcp((size_t)n), lrd((size_t)n), z((size_t)n);
  double amax = 0.0, cmax = 0.0;
  for (int64_t m = 0; m < P; ++m) {
    const int64_t s = m * n;
    const int nb = (m == P - 1) ? r.nlast : n;
    const int64_t e = s + nb - 1;
    // the block's own Thomas factors (zero values outside the block)
    for (int i = 0; i < nb; ++i) {
      const int64_t row = s + i;
      const double den = b[row] - (i > 0 ? a[row] * lcp[(size_t)i - 1] : 0.0);
      if (den == 0.0 || !std::isfinite(den)) return DICH_ERR_SINGULAR;
      lrd[(size_t)i] = 1.0 / den;
      lcp[(size_t)i] = (i < nb - 1 ? c[row] : 0.0) / den;
      const int64_t k = gen_index(m, i, n);
      fa[k] = (i > 0) ? a[row] : 0.0;
      frd[k] = lrd[(size_t)i];
      fcp[k] = lcp[(size_t)i];
    }
    // spikes v = T_m^-1 (-a_s e_0), w = T_m^-1 (-c_e e_{nb-1})
    const double as = (s > 0) ? a[s] : 0.0, ce = (e < N - 1) ? c[e] : 0.0;
    z[0] = -as * lrd[0];
    for (int i = 1; i < nb; ++i) z[(size_t)i] = -a[s + i] * z[(size_t)i - 1] * lrd[(size_t)i];
    double vn = z[(size_t)nb - 1];
    fv[gen_index(m, nb - 1, n)] = vn;
    for (int i = nb - 2; i >= 0; --i) {
      vn = z[(size_t)i] - lcp[(size_t)i] * vn;
      fv[gen_index(m, i, n)] = vn;
    }
    double wn = -ce * lrd[(size_t)nb - 1];
    fw[gen_index(m, nb - 1, n)] = wn;
    for (int i = nb - 2; i >= 0; --i) {
      wn = -lcp[(size_t)i] * wn;
      fw[gen_index(m, i, n)] = wn;
    }
    const double v0 = fv[gen_index(m, 0, n)], vend = fv[gen_index(m, nb - 1, n)];
    const double w0 = fw[gen_index(m, 0, n)], wend = fw[gen_index(m, nb - 1, n)];
    // exterior ratios and block maps
    const double kL = (m > 0) ? -cp[(size_t)s - 1] : 0.0;
    const double kR = (m < P - 1) ? -cq[(size_t)e + 1] : 0.0;
    double pa = 0.0, pc = 0.0, tL = 1.0, tR = 1.0;
    if (m < P - 1) {
      pa = 1.0;
      for (int64_t i = s + 1; i <= e + 1; ++i) pa *= -cq[(size_t)i];
    }
    if (m > 0) {
      pc = 1.0;
      for (int64_t i = s - 1; i <= e - 1; ++i) pc *= -cp[(size_t)i];
    }
    for (int64_t i = s; i <= e - 1; ++i) tL *= -cp[(size_t)i];
    for (int64_t i = s + 1; i <= e; ++i) tR *= -cq[(size_t)i];
    const double p00 = 1.0 - kL * v0, p01 = -kR * w0, p10 = -kL * vend, p11 = 1.0 - kR * wend;
    const double det = p00 * p11 - p01 * p10;
    if (det == 0.0 || !std::isfinite(det)) return DICH_ERR_SINGULAR;
    double* rc = g->recs.data() + m * kBC;
    rc[BC_A] = pa;
    rc[BC_B] = kR;
    rc[BC_C] = pc;
    rc[BC_D] = kL;
    rc[BC_TL] = tL;
    rc[BC_TR] = tR;
    rc[BC_M00] = p11 / det;
    rc[BC_M01] = -p01 / det;
    rc[BC_M10] = -p10 / det;
    rc[BC_M11] = p00 / det;
    if (m < P - 1) amax = std::max(amax, std::fabs(pa));
    if (m > 0) cmax = std::max(cmax, std::fabs(pc));
  }

  gen_decide(g, amax, cmax);
  // precision form from the tables, then (MIXED) the tables as float-float pairs in place
  double fm = 1.0, bm = 1.0, rmax = 0.0, rmin = INFINITY, omax = 0.0;
  for (int64_t m = 0; m < P; ++m) {   // error gains of the two recurrences, block by block
    const int nb = (m == P - 1) ? r.nlast : n;
    double gfi = 1.0, gbi = 1.0;
    for (int i = 1; i < nb; ++i) {
      const int64_t k = gen_index(m, i, n);
      gfi = 1.0 + std::fabs(fa[k] * frd[k]) * gfi;
      fm = std::max(fm, gfi);
    }
    for (int i = nb - 2; i >= 0; --i) {
      gbi = 1.0 + std::fabs(fcp[gen_index(m, i, n)]) * gbi;
      bm = std::max(bm, gbi);
    }
  }
  for (int64_t k = 0; k < g->stride; ++k) {
    if (frd[k] != 0.0) {
      rmax = std::max(rmax, std::fabs(frd[k]));
      rmin = std::min(rmin, std::fabs(frd[k]));
    }
    omax = std::max({omax, std::fabs(fa[k]), std::fabs(fcp[k]), std::fabs(fv[k]), std::fabs(fw[k])});
  }
  const int rc = gen_choose_form(g, fm, bm, rmax, rmin, omax);
  if (rc) return rc;
  if (g->form == FORM_MIXED) {
    for (double& d : g->rows) {
      const float hl2[2] = {(float)d, (float)(d - (double)(float)d)};
      std::memcpy(&d, hl2, sizeof(double));
    }
  }
  return DICH_OK;
}

void gen_layout(dich_gen_s* g) {
  size_t o = 0;
  g->off_plan = o;
  o += align_up(sizeof(SysPlan));
  g->off_status = o;
  o += kAlign;
  g->off_recs = o;
  o += align_up(sizeof(double) * kBC * (size_t)g->rec.P);
  g->off_rows = o;
  if (g->N > 1) o += align_up(sizeof(double) * (size_t)(kGenFields * g->stride));
  g->off_raw = o;   // the matrix
  o += align_up(sizeof(double) * 3 * (size_t)g->N);
  g->off_res = o;
  o += kAlign;
  if (g->device_prelim) {   // block composites, chunk products, largest map factors
    const int64_t nch = ceil_div(g->rec.P, (int64_t)kPreChunk);
    g->off_comp = o;
    o += align_up(sizeof(Mat2) * 2 * (size_t)g->rec.P);
    g->off_chunk = o;
    o += align_up(sizeof(Mat2) * 2 * (size_t)nch);
    g->off_max = o;
    o += kAlign;
  }
  if (g->path == PATH_GENERAL) {   // always reserved with the device preliminary (path known at bind)
    const int64_t P = g->rec.P;
    g->off_beta = o;
    o += align_up(sizeof(double) * 2 * P);
    g->off_iface = o;
    o += align_up(sizeof(double) * 2 * P);
    g->off_scan = o;
    o += align_up(sizeof(double) * 6 * (size_t)ceil_div(P, kScanChunk));
  }
  g->ws_bytes = o;
}

// the O(N) preliminary step on the device (gen_prelim.cuh), into the workspace at `base`; reads
// back the largest map factors and decides the path; returns a status code
int gen_device_tables(dich_gen_s* g, char* base, cudaStream_t st) {
  const SysPlan& r = g->rec;
  const int64_t N = g->N, P = r.P;
  const int64_t nch = ceil_div(P, (int64_t)kPreChunk);
  PreArgs A{};
  A.N = N;
  A.P = P;
  A.n = r.n;
  A.nlast = r.nlast;
  double* raw = (double*)(base + g->off_raw);
  A.a = raw;
  A.b = raw + N;
  A.c = raw + 2 * N;
  A.rows = (double*)(base + g->off_rows);
  A.stride = g->stride;
  A.recs = (double*)(base + g->off_recs);
  A.fwd = (Mat2*)(base + g->off_comp);
  A.bwd = A.fwd + P;
  A.chunk = (Mat2*)(base + g->off_chunk);
  A.maxes = (unsigned long long*)(base + g->off_max);
  const size_t nb = sizeof(double) * (size_t)N;
  cudaError_t e = cudaMemcpyAsync(raw, g->ha.data(), nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(raw + N, g->hb.data(), nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(raw + 2 * N, g->hc.data(), nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.rows, 0, sizeof(double) * (size_t)(kGenFields * g->stride), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.maxes, 0, 8 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e);
  k_pre_blocks<<<(unsigned)nch, kPreThreads, 0, st>>>(A);
  k_pre_chunk<<<(unsigned)nch, kPreThreads, 0, st>>>(A);
  k_pre_top<<<1, 32, 0, st>>>(A, nch);
  k_pre_records<<<(unsigned)nch, kPreThreads, 0, st>>>(A);
  e = cudaGetLastError();
  unsigned long long mx[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(mx, A.maxes, sizeof(mx), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (mx[2]) return DICH_ERR_SINGULAR;
  double amax, cmax;
  std::memcpy(&amax, &mx[0], sizeof(double));
  std::memcpy(&cmax, &mx[1], sizeof(double));
  gen_decide(g, amax, cmax);
  double q[5];   // forward and backward error gains, max |rd|, min |rd|, max of the other factors
  mx[6] = ~mx[6];
  for (int j = 0; j < 5; ++j) std::memcpy(&q[j], &mx[3 + j], sizeof(double));
  const int rc = gen_choose_form(g, q[0], q[1], q[2], q[3], q[4]);
  if (rc) return rc;
  if (g->form == FORM_MIXED) {
    k_pre_to_ff<<<(unsigned)std::min<int64_t>(ceil_div(kGenFields * g->stride, (int64_t)256), (int64_t)4096), 256, 0,
                  st>>>(A.rows, kGenFields * g->stride);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return DICH_OK;
}

int gen_launch(dich_gen_s* g, const double* F, double* x, cudaStream_t st, int64_t M, int64_t ldf, int64_t ldx) {
  const SysPlan* d_plan = (const SysPlan*)(g->d_ws + g->off_plan);
  const double* d_recs = (const double*)(g->d_ws + g->off_recs);
  unsigned* d_status = (unsigned*)(g->d_ws + g->off_status);
  if (g->N == 1) {
    for (int64_t k = 0; k < M; ++k) {
      cudaError_t e = launch_trivial(d_plan, nullptr, 1, F + k * ldf, x + k * ldx, nullptr, nullptr, nullptr, 0, st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    return DICH_OK;
  }
  GenArgs ga{};
  ga.w.plans = d_plan;
  ga.w.tabs = d_recs;
  ga.w.status = d_status;
  ga.w.check_finite = (g->opts.flags & DICH_FLAG_CHECK_FINITE) ? 1 : 0;
  ga.w.n_smem = g->rec.n;
  ga.rows = (const double*)(g->d_ws + g->off_rows);
  ga.stride = g->stride;
  const size_t smem = window_gen_smem_bytes(g->NT, g->rec.n);
  cudaError_t e;
  if (g->path != PATH_GENERAL) {
    ga.w.mode = MODE_FULL;
    ga.w.ldf = ldf;
    ga.w.ldx = ldx;
    for (int64_t k0 = 0; k0 < M; k0 += 65535) {
      GenArgs w = ga;
      w.w.F = F + k0 * ldf;
      w.w.x = x + k0 * ldx;
      e = launch_window_gen(g->NT, (int)g->tiles, smem, st, w, (int)std::min<int64_t>(65535, M - k0), g->form);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    return DICH_OK;
  }
  double* beta = (double*)(g->d_ws + g->off_beta);
  double* iface = (double*)(g->d_ws + g->off_iface);
  double* scan = (double*)(g->d_ws + g->off_scan);
  for (int64_t k = 0; k < M; ++k) {
    GenArgs w = ga;
    w.w.F = F + k * ldf;
    w.w.x = x + k * ldx;
    w.w.mode = MODE_BETA;
    w.w.beta = beta;
    e = launch_window_gen(g->NT, (int)g->tiles, smem, st, w, 1, g->form);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_block_scan(d_plan, d_recs, g->rec.P, beta, iface, scan, st);
    if (e != cudaSuccess) return cuda_fail(e);
    w.w.mode = MODE_APPLY;
    w.w.iface = iface;
    e = launch_window_gen(g->NT, (int)g->tiles, smem, st, w, 1, g->form);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return DICH_OK;
}

}  // namespace

extern "C" {

int dichotomy_gen_plan(int64_t N, const double* h_a, const double* h_b, const double* h_c, const dich_opts* opts,
                       dich_gen_t* out) {
  if (!out) return DICH_ERR_ARG;
  *out = nullptr;
  if (N < 0 || (N > 0 && (!h_a || !h_b || !h_c))) return DICH_ERR_ARG;
  Opts o;
  int rc = read_opts(opts, o);
  if (rc) return rc;
  // eq. 32-33 row by row (a_0 and c_{N-1} lie outside the matrix), unless waived; ||A||_inf
  const bool waive = (o.flags & DICH_FLAG_ALLOW_NOT_DOMINANT) != 0;
  double norm_inf = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const double ai = (i > 0) ? h_a[i] : 0.0, ci = (i < N - 1) ? h_c[i] : 0.0;
    if (!std::isfinite(ai) || !std::isfinite(h_b[i]) || !std::isfinite(ci)) return DICH_ERR_ARG;
    if (h_b[i] == 0.0 && ai == 0.0 && ci == 0.0) return DICH_ERR_SINGULAR;
    if (!waive && (h_b[i] == 0.0 || std::fabs(h_b[i]) < (std::fabs(ai) + std::fabs(ci)) * (1.0 - 4.0 * DBL_EPSILON)))
      return DICH_ERR_NOT_DOMINANT;
    norm_inf = std::max(norm_inf, std::fabs(ai) + std::fabs(h_b[i]) + std::fabs(ci));
  }
  dich_gen_s* g = new (std::nothrow) dich_gen_s();
  if (!g) return DICH_ERR_ARG;
  g->N = N;
  g->opts = o;
  g->NT = o.NT ? o.NT : (o.prec == DICH_PREC_F64 ? 64 : 128);
  g->norm_inf = norm_inf;
  if (N >= 1) {
    rc = gen_geometry(g, h_b[0]);
    // the matrix is kept (on the device too) for the a posteriori residual and the device preliminary
    try {
      g->ha.assign(h_a, h_a + N);
      g->hb.assign(h_b, h_b + N);
      g->hc.assign(h_c, h_c + N);
      g->ha[0] = 0.0;
      g->hc[(size_t)N - 1] = 0.0;
    } catch (...) {
      rc = DICH_ERR_ARG;
    }
    if (rc == DICH_OK && N > 1) {
      g->device_prelim = (o.flags & DICH_FLAG_DEVICE_PRELIM) ||
                         (!(o.flags & DICH_FLAG_HOST_PRELIM) && N >= kGenDevicePrelimMin);
      if (!g->device_prelim) rc = gen_host_tables(g, h_a, h_b, h_c);
    }
    if (rc) {
      delete g;
      return rc;
    }
  }
  gen_layout(g);
  *out = g;
  return DICH_OK;
}

int dichotomy_gen_info(dich_gen_t g, dich_plan_info* info) {
  if (!g || !info) return DICH_ERR_ARG;
  std::memset(info, 0, sizeof(*info));
  info->N = g->N;
  info->P = g->rec.P;
  info->n = g->rec.n;
  info->n_last = g->rec.nlast;
  info->threads = g->NT;
  info->halo_l = g->rec.hl;
  info->halo_r = g->rec.hr;
  info->path = g->path;
  info->precision = (g->form == FORM_MIXED) ? DICH_PREC_MIXED : DICH_PREC_F64;
  info->tiles = g->tiles;
  info->workspace_bytes = g->ws_bytes;
  {
    const int64_t P = std::max<int64_t>(1, g->rec.P);
    int levels = 0;
    while (((int64_t)1 << levels) < P) ++levels;
    info->growth = std::min(std::pow(g->gamma, (double)levels), 1e300);
  }
  if (g->path == PATH_GENERAL) {
    info->beta_offset = g->off_beta;
    info->iface_offset = g->off_iface;
  }
  return DICH_OK;
}

int dichotomy_gen_workspace_bytes(dich_gen_t g, size_t* bytes) {
  if (!g || !bytes) return DICH_ERR_ARG;
  *bytes = g->ws_bytes;
  return DICH_OK;
}

int dichotomy_gen_bind(dich_gen_t g, void* d_ws, size_t bytes, void* stream) {
  if (!g || !d_ws) return DICH_ERR_ARG;
  if (((uintptr_t)d_ws & (kAlign - 1)) != 0 || bytes < g->ws_bytes) return DICH_ERR_WORKSPACE;
  if (!is_device_ptr(d_ws)) return DICH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)d_ws;
  if (g->device_prelim) {
    const int rc = gen_device_tables(g, base, st);
    if (rc) return rc;
  }
  cudaError_t e = cudaMemcpyAsync(base + g->off_plan, &g->rec, sizeof(SysPlan), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + g->off_status, 0, kAlign, st);
  if (e == cudaSuccess && !g->recs.empty())
    e = cudaMemcpyAsync(base + g->off_recs, g->recs.data(), sizeof(double) * g->recs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !g->rows.empty())
    e = cudaMemcpyAsync(base + g->off_rows, g->rows.data(), sizeof(double) * g->rows.size(), cudaMemcpyHostToDevice, st);
  if (!g->device_prelim && g->N > 0) {   // the matrix, for the residual check
    double* raw = (double*)(base + g->off_raw);
    const size_t nb = sizeof(double) * (size_t)g->N;
    if (e == cudaSuccess) e = cudaMemcpyAsync(raw, g->ha.data(), nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(raw + g->N, g->hb.data(), nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(raw + 2 * g->N, g->hc.data(), nb, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host tables may be freed or reused after bind
  if (e != cudaSuccess) return cuda_fail(e);
  g->d_ws = base;
  return DICH_OK;
}

int dichotomy_gen_solve_series(dich_gen_t g, int64_t M, const double* d_F, int64_t ldf, double* d_x, int64_t ldx,
                               void* stream) {
  if (!g || M < 0) return DICH_ERR_ARG;
  if (!g->d_ws) return DICH_ERR_UNBOUND;
  if (g->N == 0 || M == 0) return DICH_OK;
  if (!d_F || !d_x || !aligned8(d_F) || !aligned8(d_x)) return DICH_ERR_ARG;
  if (M > 1 && (ldf < g->N || ldx < g->N)) return DICH_ERR_ARG;
  if (M > 1 && (ldf > INT64_MAX / M || ldx > INT64_MAX / M)) return DICH_ERR_ARG;
  const int64_t sf = (M > 1) ? ldf : 0, sx = (M > 1) ? ldx : 0;
  const size_t nf = sizeof(double) * (size_t)((M - 1) * sf + g->N);
  const size_t nx = sizeof(double) * (size_t)((M - 1) * sx + g->N);
  if (overlap(d_F, nf, d_x, nx)) return DICH_ERR_ALIAS;
  if (!is_device_ptr(d_F) || !is_device_ptr(d_x)) return DICH_ERR_ARG;
  return gen_launch(g, d_F, d_x, (cudaStream_t)stream, M, sf, sx);
}

int dichotomy_gen_solve(dich_gen_t g, const double* d_F, double* d_x, void* stream) {
  return dichotomy_gen_solve_series(g, 1, d_F, 0, d_x, 0, stream);
}

int dichotomy_gen_residual(dich_gen_t g, const double* d_F, const double* d_x, double* h_out, void* stream) {
  if (!g || !h_out) return DICH_ERR_ARG;
  if (!g->d_ws) return DICH_ERR_UNBOUND;
  h_out[0] = h_out[1] = 0.0;
  if (g->N == 0) return DICH_OK;
  if (!d_F || !d_x || !aligned8(d_F) || !aligned8(d_x) || !is_device_ptr(d_F) || !is_device_ptr(d_x))
    return DICH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const double* raw = (const double*)(g->d_ws + g->off_raw);
  unsigned long long* res = (unsigned long long*)(g->d_ws + g->off_res);
  cudaError_t e = cudaMemsetAsync(res, 0, 3 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g->N, (int64_t)256), 4 * 1184));
    k_gen_residual<<<grid, 256, 0, st>>>(g->N, raw, raw + g->N, raw + 2 * g->N, d_F, d_x, res);
    e = cudaGetLastError();
  }
  unsigned long long m[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(m, res, sizeof(m), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  double r, xm, fm;
  std::memcpy(&r, &m[0], sizeof(double));
  std::memcpy(&xm, &m[1], sizeof(double));
  std::memcpy(&fm, &m[2], sizeof(double));
  const double den = g->norm_inf * xm + fm;
  h_out[0] = r;
  h_out[1] = (den > 0.0) ? r / den : 0.0;
  return DICH_OK;
}

int dichotomy_gen_status(dich_gen_t g, void* stream, int* device_status) {
  if (!g || !device_status) return DICH_ERR_ARG;
  if (!g->d_ws) return DICH_ERR_UNBOUND;
  unsigned s = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&s, g->d_ws + g->off_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(g->d_ws + g->off_status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e);
  *device_status = map_status(s);
  return DICH_OK;
}

void dichotomy_gen_destroy(dich_gen_t g) { delete g; }

}  // extern "C"
