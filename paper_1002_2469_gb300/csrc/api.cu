// api.cu -- host planner and the C ABI of include/dichotomy.h.
//
// The planner is the paper's preliminary step for Toeplitz matrices (Sec. 3.1-3.3): for a
// system (t, N) and a block size n it computes the recurrence roots (Theorem 1), the two
// block spikes of T_n (eq. 25 in factored form), the end-dependent exterior ratios of the
// first and last few blocks (eq. 24) and the constant ratios of all other blocks -- an
// O(n + log P) amount of work instead of the O(N) general preliminary step (eq. 9-12).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dichotomy.h"
#include "launch.cuh"
#include "planner.cuh"

using namespace dich;
using namespace dich::plan;

namespace dich {
namespace plan {

thread_local std::string g_cuda_err;

int cuda_fail(cudaError_t e) {
  g_cuda_err = cudaGetErrorString(e);
  return DICH_ERR_CUDA;
}

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// window width in blocks: the MIXED kernel gives every thread two blocks
int window_blocks(int NT, int form) { return form == FORM_MIXED ? 2 * NT : NT; }

size_t smem_bytes(int NT, int n, int form) {
  return form == FORM_MIXED ? window2_smem_bytes(NT, n) : window_smem_bytes(NT, n);
}

int max_rows(int NT, int form, size_t budget) {
  // smem_bytes(NT, n, form) <= budget
  int n = 2;
  while (smem_bytes(NT, n + 1, form) <= budget) ++n;
  return n;
}

int default_threads(int form) { return form == FORM_F64 ? 64 : 128; }

// rows per block for multi-window systems (measured on GB300 at N = 2^26: small windows let
// several CTAs share an SM so loads, sweeps, tree and stores of different windows overlap)
int default_rows(int form) { return form == FORM_F64 ? 64 : 16; }

int validate_t(double tm1, double t0, double tp1, int flags) {
  if (!std::isfinite(tm1) || !std::isfinite(t0) || !std::isfinite(tp1)) return DICH_ERR_ARG;
  if (t0 == 0.0 && tm1 == 0.0 && tp1 == 0.0) return DICH_ERR_SINGULAR;
  const double off = std::fabs(tm1) + std::fabs(tp1);
  // eq. 32-33: |b| >= |a| + |c| (equality accepted: the end rows are then strict)
  if (t0 != 0.0 && std::fabs(t0) >= off * (1.0 - 4.0 * DBL_EPSILON)) return DICH_OK;
  // without dominance, on request: what the two recurrences need is real roots of
  // t_1 r^2 + t_0 r + t_-1 = 0 separated by the unit circle (|rs| < 1 < |1/ib|)
  if (!(flags & DICH_FLAG_ALLOW_NOT_DOMINANT)) return DICH_ERR_NOT_DOMINANT;
  if (t0 * t0 - 4.0 * tm1 * tp1 <= 0.0) return DICH_ERR_NOT_DOMINANT;
  const Roots r = toeplitz_roots(tm1, t0, tp1);
  const double lim = 1.0 - 1e-12;
  return (r.ok && std::fabs(r.rs) < lim && std::fabs(r.ib) < lim) ? DICH_OK : DICH_ERR_NOT_DOMINANT;
}

int read_opts(const dich_opts* o, Opts& out) {
  out = Opts();
  if (!o) return DICH_OK;
  if (o->block_size < 0 || o->block_size == 1) return DICH_ERR_ARG;
  if (o->precision < 0 || o->precision > 2) return DICH_ERR_ARG;
  if (o->threads != 0 && o->threads != 64 && o->threads != 128 && o->threads != 256) return DICH_ERR_ARG;
  if (!(o->trunc_eps >= 0.0) || o->trunc_eps >= 1e-3) return DICH_ERR_ARG;
  if ((o->flags & DICH_FLAG_REG_PATH) && (o->flags & DICH_FLAG_SMEM_PATH)) return DICH_ERR_ARG;
  out.n_req = o->block_size;
  out.prec = o->precision;
  out.NT = o->threads;
  out.flags = o->flags;
  if (o->trunc_eps > 0.0) {
    out.eps = o->trunc_eps;
    out.eps_given = true;
  }
  return DICH_OK;
}

// amplification of rounding errors through the two recurrences
double recurrence_gain(const Roots& r) {
  const double a = std::fabs(r.rs), b = std::fabs(r.ib);
  if (a >= 1.0 || b >= 1.0) return INFINITY;
  return 1.0 / (1.0 - a) + 1.0 / (1.0 - b);
}

// MIXED (compensated FP32) is used under AUTO when the recurrences amplify rounding
// errors by at most this factor.
constexpr double kMixedGainLimit = 24.0;

// MIXED holds xp = g X at the window scale of F in float-float, so the scale factor g = -1/q
// of T = -q (1 - rs E^-1)(1 - ib E) must keep the scaled solution and its low parts inside the
// float range: |g| within 2^-60..2^60 (|t| roughly within the same range).
bool mixed_scale_ok(const Roots& r) {
  const double a = std::fabs(r.g);
  return a >= 0x1p-60 && a <= 0x1p60;
}

// the form of a system; -1: MIXED requested where its scale range does not hold
int pick_form(int prec, const Roots& r) {
  if (prec == DICH_PREC_F64) return FORM_F64;
  if (prec == DICH_PREC_MIXED) return mixed_scale_ok(r) ? FORM_MIXED : -1;
  return (recurrence_gain(r) <= kMixedGainLimit && mixed_scale_ok(r)) ? FORM_MIXED : FORM_F64;
}

void split_ff(double d, float& h, float& l) {
  h = (float)d;
  l = (float)(d - (double)h);
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Choose the block size: one window when the system fits in one window of default-size
// blocks (n = ceil(N / window blocks) <= n_def), else n_def rows per block.  Longer blocks
// would fit one window up to nmax rows, but they serialise the sweeps and enlarge the shared
// memory of every CTA of a batched launch (measured: a batch with some one-window systems of
// 50-row blocks ran at half speed).  A last block of a single row is not allowed (Sec. 2.1
// asks for sub-vectors of >= 2 rows), so n moves to the nearest size with N mod n != 1:
// upwards when the system fits in one window (every larger n still does), else downwards first.
int choose_n(int64_t N, int NT, int nmax, int n_req, int n_def) {
  auto ok = [&](int64_t c) { return c >= 2 && (c >= N || N % c != 1); };
  const bool one_window = (n_req <= 0) && (N <= (int64_t)NT * std::min(nmax, n_def));
  int n;
  if (n_req > 0)
    n = std::min(n_req, nmax);
  else if (one_window)
    n = (int)std::max<int64_t>(2, ceil_div(N, NT));
  else
    n = std::min(nmax, n_def);
  if (n >= N) return (int)N;
  if (ok(n)) return n;
  if (one_window) {
    for (int c = n + 1; c <= nmax; ++c)
      if (ok(c)) return (c >= N) ? (int)N : c;
  }
  for (int d = 1; d < nmax; ++d) {
    if (n - d >= 2 && ok(n - d)) return n - d;
    if (n + d <= nmax && ok(n + d)) return (n + d >= N) ? (int)N : n + d;
  }
  return (int)std::min<int64_t>(N, nmax);
}

int build_system(double tm1, double t0, double tp1, int64_t N, int NT, int form, int n, const Opts& o,
                 bool allow_general, SysBuild& sb) {
  SysPlan& p = sb.rec;
  std::memset(&p, 0, sizeof(p));
  const Roots r = toeplitz_roots(tm1, t0, tp1);
  if (!r.ok) return DICH_ERR_SINGULAR;
  p.N = N;
  p.n = n;
  p.P = ceil_div(N, n);
  p.nlast = (int)(N - (p.P - 1) * (int64_t)n);
  if (p.nlast < 2) return DICH_ERR_ARG;  // guarded by choose_n
  p.form = form;
  p.tm1 = tm1;
  p.t0 = t0;
  p.tp1 = tp1;
  p.rs = r.rs;
  p.ib = r.ib;
  p.g = r.g;
  split_ff(r.rs, p.rs_h, p.rs_l);
  split_ff(r.ib, p.ib_h, p.ib_l);
  split_ff(r.g, p.g_h, p.g_l);

  // truncation: geometric terms below eps (relative) are dropped; for z < 0 the Q ratios can
  // exceed 1 by up to 2/(1-|z|), which the threshold absorbs
  double eps = (form == FORM_MIXED && !o.eps_given) ? kEpsMixed : o.eps;
  if (r.z < 0.0) eps *= 0.5 * r.omz;
  const int64_t BIG = (int64_t)1 << 62;
  const int64_t Ls = decay_len(std::fabs(r.rs), eps, BIG);
  const int64_t Lb = decay_len(std::fabs(r.ib), eps, BIG);
  const int64_t Lz = (r.omz == 0.0) ? BIG : decay_len(std::fabs(r.z), eps, BIG);
  p.Lv = (int)std::min<int64_t>(n, Ls);
  p.Lw = (int)std::min<int64_t>(n, Lb);

  // path and halos
  const int64_t P = p.P;
  const int WB = window_blocks(NT, form);
  if (P <= WB && !(o.flags & DICH_FLAG_FORCE_GENERAL)) {
    sb.path = PATH_SINGLE;
    p.hl = p.hr = 0;
    p.own = (int)P;
  } else {
    // the neighbour's first/last value must carry decayed coupling too: +1 row of margin
    const int64_t hl = (std::fabs(r.rs) == 0.0) ? 1 : (Ls >= BIG ? BIG : std::max<int64_t>(1, ceil_div(Ls + 1, n)));
    const int64_t hr = (std::fabs(r.ib) == 0.0) ? 1 : (Lb >= BIG ? BIG : std::max<int64_t>(1, ceil_div(Lb + 1, n)));
    if (!(o.flags & DICH_FLAG_FORCE_GENERAL) && hl + hr <= WB / 2) {
      sb.path = PATH_HALO;
      p.hl = (int)hl;
      p.hr = (int)hr;
      p.own = WB - (int)hl - (int)hr;
    } else {
      if (!allow_general) return DICH_ERR_UNSUPPORTED;
      sb.path = PATH_GENERAL;
      p.hl = p.hr = 0;
      p.own = WB;
    }
  }

  // end tables
  int64_t kl, kr;
  if (Lz >= BIG) {
    kl = P;
    kr = 0;
  } else {
    kl = std::min<int64_t>(P, ceil_div(Lz + 1, n) + 1);
    kr = std::min<int64_t>(P, ceil_div(Lz + 1, n) + 2);
    if (kl + kr >= P) {
      kl = P;
      kr = 0;
    }
  }
  if (kl * kBC > ((int64_t)1 << 30)) return DICH_ERR_UNSUPPORTED;
  p.kl = (int)kl;
  p.kr = (int)kr;

  // spikes of the block operator, full blocks (eq. 25 restated: v_i = rs^{i+1} Q(n-i)/Q(n+1))
  auto vspike = [&](int64_t nb, int64_t i) { return ipow(r.rs, i + 1) * spike_ratio(nb, i, r); };
  auto wspike_rev = [&](int64_t nb, int64_t i) { return ipow(r.ib, i + 1) * spike_ratio(nb, i, r); };
  p.v0 = vspike(n, 0);
  p.vend = vspike(n, n - 1);
  p.w0 = wspike_rev(n, n - 1);
  p.wend = wspike_rev(n, 0);
  const int nl = p.nlast;
  p.v0l = vspike(nl, 0);
  p.vendl = vspike(nl, nl - 1);
  p.w0l = wspike_rev(nl, nl - 1);
  p.wendl = wspike_rev(nl, 0);

  // table layout
  int64_t o_ = 0;
  auto take = [&](int64_t cnt) {
    const int64_t at = o_;
    o_ += cnt;
    return (int32_t)at;
  };
  p.o_v = take(p.Lv);
  p.o_w = take(p.Lw);
  p.o_vl = take(nl);
  p.o_wl = take(nl);
  p.o_vf = take(p.Lv);
  p.o_wf = take(p.Lw);
  p.o_vlf = take(nl);
  p.o_wlf = take(nl);
  p.o_bcm = take(kBC);
  p.o_bcl = take(kl * kBC);
  p.o_bcr = take(kr * kBC);
  p.o_bcmf = take(kBC);
  p.o_bclf = take(kl * kBC);
  p.o_bcrf = take(kr * kBC);
  p.o_kmf = take(4);
  p.o_klf = take(kl * 4);
  p.o_krf = take(kr * 4);
  p.o_midf = take(66);
  // warp-scan levels of the MIXED tree: a contribution from 2^(lev+1) or more blocks away carries a
  // product of ratios below |rs|^(n 2^(lev+1)) (prefix) or |ib|^(n 2^(lev+1)) (suffix): below eps
  auto levels = [&](int64_t Lrows) {
    if (Lrows >= BIG) return 5;
    const int64_t kb = ceil_div(Lrows, n);
    int lev = 0;
    while (lev < 5 && ((int64_t)2 << lev) < kb) ++lev;
    return lev;
  };
  p.lev = std::max(levels(Ls), levels(Lb));
  split_ff(r.g * r.ib, p.gib_h, p.gib_l);
  split_ff(p.v0, p.v0_h, p.v0_l);
  split_ff(p.vend, p.vend_h, p.vend_l);
  split_ff(p.v0l, p.v0l_h, p.v0l_l);
  split_ff(p.vendl, p.vendl_h, p.vendl_l);
  double* T;
  if (sb.ext) {  // caller-provided table storage (no allocation)
    if ((size_t)o_ > sb.ext_cap) return DICH_ERR_WORKSPACE;
    std::memset(sb.ext, 0, sizeof(double) * (size_t)o_);
    T = sb.ext;
    sb.ext_used = (size_t)o_;
  } else {
    sb.tab.assign((size_t)o_, 0.0);
    T = sb.tab.data();
  }
  auto put_ff = [&](int32_t at, double d) {
    float h, l;
    split_ff(d, h, l);
    float2 f2 = make_float2(h, l);
    std::memcpy(&T[at], &f2, sizeof(double));
  };
  for (int i = 0; i < p.Lv; ++i) {
    T[p.o_v + i] = vspike(n, i);
    put_ff(p.o_vf + i, T[p.o_v + i]);
  }
  for (int i = 0; i < p.Lw; ++i) {
    T[p.o_w + i] = wspike_rev(n, i);
    put_ff(p.o_wf + i, T[p.o_w + i]);
  }
  for (int i = 0; i < nl; ++i) {
    T[p.o_vl + i] = vspike(nl, i);
    T[p.o_wl + i] = wspike_rev(nl, i);
    put_ff(p.o_vlf + i, T[p.o_vl + i]);
    put_ff(p.o_wlf + i, T[p.o_wl + i]);
  }
  block_coeffs(N, (int64_t)1 << 40, ((int64_t)1 << 40) + n - 1, r, p.v0, p.vend, p.w0, p.wend, true, true,
               &T[p.o_bcm]);
  auto coeffs_of = [&](int64_t m, double* out) {
    const int64_t s = m * (int64_t)n;
    const int64_t e = (m == P - 1) ? N - 1 : s + n - 1;
    const bool lb = (m == P - 1);
    block_coeffs(N, s, e, r, lb ? p.v0l : p.v0, lb ? p.vendl : p.vend, lb ? p.w0l : p.w0, lb ? p.wendl : p.wend,
                 false, false, out);
  };
  for (int64_t m = 0; m < kl; ++m) coeffs_of(m, &T[p.o_bcl + m * kBC]);
  for (int64_t k = 0; k < kr; ++k) coeffs_of(P - kr + k, &T[p.o_bcr + k * kBC]);
  for (int j = 0; j < kBC; ++j) put_ff(p.o_bcmf + j, T[p.o_bcm + j]);
  for (int64_t j = 0; j < kl * kBC; ++j) put_ff(p.o_bclf + (int32_t)j, T[p.o_bcl + j]);
  for (int64_t j = 0; j < kr * kBC; ++j) put_ff(p.o_bcrf + (int32_t)j, T[p.o_bcr + j]);
  // beta records (K1..K4, units of X) of the middle record and of the end tables, float-float
  {
    double k4[4];
    beta_coeffs(&T[p.o_bcm], r.ib, p.v0, p.vend, k4);
    for (int j = 0; j < 4; ++j) put_ff(p.o_kmf + j, k4[j]);
    for (int64_t m = 0; m < kl; ++m) {
      const bool lb = (m == P - 1);
      beta_coeffs(&T[p.o_bcl + m * kBC], r.ib, lb ? p.v0l : p.v0, lb ? p.vendl : p.vend, k4);
      for (int j = 0; j < 4; ++j) put_ff(p.o_klf + (int32_t)(m * 4 + j), k4[j]);
    }
    for (int64_t k = 0; k < kr; ++k) {
      const bool lb = (P - kr + k == P - 1);
      beta_coeffs(&T[p.o_bcr + k * kBC], r.ib, lb ? p.v0l : p.v0, lb ? p.vendl : p.vend, k4);
      for (int j = 0; j < 4; ++j) put_ff(p.o_krf + (int32_t)(k * 4 + j), k4[j]);
    }
    // powers of the middle record's pair maps: (a^2)^t and (c^2)^t, t = 0..32
    const double a2 = T[p.o_bcm + BC_A] * T[p.o_bcm + BC_A], c2 = T[p.o_bcm + BC_C] * T[p.o_bcm + BC_C];
    p.tcheap = (a2 <= 0x1p-24 && c2 <= 0x1p-24) ? 1 : 0;
    double pa = 1.0, pc = 1.0;
    for (int t = 0; t <= 32; ++t) {
      put_ff(p.o_midf + t, pa);
      put_ff(p.o_midf + 33 + t, pc);
      pa *= a2;
      pc *= c2;
    }
  }
  return DICH_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  // device memory of another GPU would be read by kernels launched on this one
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.device == dev;
}

bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

int map_status(unsigned s) {
  if (s & ST_NONFINITE) return DICH_ERR_NONFINITE;
  if (s & ST_SCHEDULE) return DICH_ERR_SCHEDULE;
  if (s & ST_TIMEOUT) return DICH_ERR_TIMEOUT;
  return DICH_OK;
}

}  // namespace plan
}  // namespace dich

// ================================================================== quasi-Toeplitz corners (eq. 21)
// Corner data of A = T + psi e_0 e_0^T + chi e_{N-1} e_{N-1}^T, N >= 2: g = T^-1 e_0 and
// h = T^-1 e_{N-1} in closed form (the block spikes of a block of N rows), kept to Lg and Lh
// rows (g_i = -(1/q) rs^i Q(N-i)/Q(N+1); h at row N-1-k = -(1/q) ib^k Q(N-k)/Q(N+1)), stored as
// g[Lg] then h[Lh]; W = (I + K)^-1 of the Sherman-Morrison-Woodbury step and Wt the same for A^T
// (Toeplitz inverses are persymmetric, so A^T's corner vectors are h and g read backwards and its
// 2x2 system has the same determinant).  Returns DICH_ERR_SINGULAR when the 2x2 system is.
struct Corners {
  int64_t Lg = 0, Lh = 0;
  std::vector<double> gh;
  double W[4] = {1.0, 0.0, 0.0, 1.0}, Wt[4] = {1.0, 0.0, 0.0, 1.0};
};

static int corner_build(double t_m1, double t_0, double t_1, double psi, double chi, int64_t N, double eps,
                        Corners& c) {
  const Roots r = toeplitz_roots(t_m1, t_0, t_1);
  c.Lg = decay_len(std::fabs(r.rs), eps, N);
  c.Lh = decay_len(std::fabs(r.ib), eps, N);
  c.gh.resize((size_t)(c.Lg + c.Lh));
  for (int64_t i = 0; i < c.Lg; ++i) c.gh[(size_t)i] = r.g * ipow(r.rs, i) * spike_ratio(N, i, r);
  for (int64_t k = 0; k < c.Lh; ++k) c.gh[(size_t)(c.Lg + k)] = r.g * ipow(r.ib, k) * spike_ratio(N, k, r);
  const double qN1 = qnum(N + 1, r), qN = qnum(N, r);
  const double g0 = r.g * qN / qN1, gN = r.g * ipow(r.rs, N - 1) / qN1;   // (T^-1)_{0,0}, (T^-1)_{N-1,0}
  const double h0 = r.g * ipow(r.ib, N - 1) / qN1, hN = r.g * qN / qN1;   // (T^-1)_{0,N-1}, (T^-1)_{N-1,N-1}
  const double k00 = 1.0 + psi * g0, k01 = psi * h0, k10 = chi * gN, k11 = 1.0 + chi * hN;
  const double det = k00 * k11 - k01 * k10;
  if (!std::isfinite(det) || std::fabs(det) <= 64.0 * DBL_EPSILON * (std::fabs(k00 * k11) + std::fabs(k01 * k10)))
    return DICH_ERR_SINGULAR;
  c.W[0] = k11 / det;
  c.W[1] = -k01 / det;
  c.W[2] = -k10 / det;
  c.W[3] = k00 / det;
  c.Wt[0] = k11 / det;
  c.Wt[1] = -psi * gN / det;
  c.Wt[2] = -chi * h0 / det;
  c.Wt[3] = k00 / det;
  return DICH_OK;
}

// the end rows of eq. 21 must keep dominance (eq. 32-33; the interior rows are T's)
static int corner_check(double t_m1, double t_0, double t_1, double psi, double chi, int64_t N, int flags) {
  if (!std::isfinite(psi) || !std::isfinite(chi)) return DICH_ERR_ARG;
  if (N >= 2 && (flags & DICH_FLAG_ALLOW_NOT_DOMINANT)) {   // only a zero corner pivot is refused here
    if (t_0 + psi == 0.0 || t_0 + chi == 0.0) return DICH_ERR_SINGULAR;
  } else if (N >= 2) {
    const double tol = 1.0 - 4.0 * DBL_EPSILON;
    if (std::fabs(t_0 + psi) < std::fabs(t_1) * tol || std::fabs(t_0 + chi) < std::fabs(t_m1) * tol)
      return DICH_ERR_NOT_DOMINANT;
    if (t_0 + psi == 0.0 || t_0 + chi == 0.0) return DICH_ERR_SINGULAR;
  } else if (N == 1 && t_0 + psi + chi == 0.0) {
    return DICH_ERR_SINGULAR;
  }
  return DICH_OK;
}

// ================================================================== single-system plan
struct dich_plan_s {
  int64_t N = 0;
  double tm1 = 0, t0 = 0, tp1 = 0;
  Opts opts;
  int NT = 64;
  int form = FORM_F64;
  int path = PATH_SINGLE;
  int n_smem = 2;
  int64_t tiles = 0;
  SysBuild fwd, adj;
  // quasi-Toeplitz corners (eq. 21): t_0 + psi in row 0, t_0 + chi in row N-1
  bool quasi = false;
  bool corners = false;                // psi or chi nonzero: the adjoint also returns dL/dpsi, dL/dchi
  double psi = 0.0, chi = 0.0;
  int64_t Lg = 0, Lh = 0;              // kept rows of g = T^-1 e_0 and h = T^-1 e_{N-1}
  double W[4] = {1.0, 0.0, 0.0, 1.0};  // (I + K)^-1 of the Sherman-Morrison-Woodbury step
  double Wt[4] = {1.0, 0.0, 0.0, 1.0}; // the same for A^T (its corner vectors are h and g reversed)
  std::vector<double> corner;          // g[Lg], then h[Lh] (h[k] is row N-1-k)
  // workspace layout (bytes)
  size_t ws_bytes = 0, off_plans = 0, off_status = 0, off_tabs = 0, off_beta = 0, off_iface = 0,
         off_scan = 0, off_part = 0;
  std::vector<unsigned char> staging;  // [plans | status | tables]
  char* d_ws = nullptr;
  size_t d_ws_bytes = 0;
  // host-memory solves: copy-in and copy-out streams and the pipeline's events (created on first use)
  cudaStream_t hs[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> hev;
  ~dich_plan_s() {
    for (cudaEvent_t ev : hev) cudaEventDestroy(ev);
    for (cudaStream_t h : hs)
      if (h) cudaStreamDestroy(h);
  }
};

extern "C" {

const char* dichotomy_version(void) { return "0.1.0"; }

const char* dichotomy_last_cuda_error(void) { return g_cuda_err.c_str(); }

const char* dichotomy_strerror(int s) {
  switch (s) {
    case DICH_OK: return "ok";
    case DICH_ERR_ARG: return "invalid argument";
    case DICH_ERR_NOT_DOMINANT: return "matrix is not diagonally dominant (eq. 32-33)";
    case DICH_ERR_SINGULAR: return "matrix is singular";
    case DICH_ERR_TIMEOUT: return "device wait timed out";
    case DICH_ERR_NONFINITE: return "non-finite value produced on the device";
    case DICH_ERR_CUDA: return "CUDA runtime error";
    case DICH_ERR_ALIAS: return "output aliases an input";
    case DICH_ERR_UNBOUND: return "plan is not bound to a device workspace";
    case DICH_ERR_WORKSPACE: return "workspace too small or misaligned";
    case DICH_ERR_SCHEDULE: return "coefficients need a larger schedule than prepared";
    case DICH_ERR_UNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
  }
}

// Workspace layout and the staging copy of a plan: records, status word, tables (forward,
// transposed, quasi-Toeplitz corners), general-path scratch, adjoint partials.
static void plan_layout(dich_plan_s* p) {
  // workspace layout
  size_t o_ = 0;
  p->off_plans = o_;
  o_ += align_up(2 * sizeof(SysPlan));
  p->off_status = o_;
  o_ += kAlign;
  p->off_tabs = o_;
  o_ += align_up(sizeof(double) * (p->fwd.tab.size() + p->adj.tab.size() + p->corner.size()));
  const int64_t P = (p->N >= 2) ? p->fwd.rec.P : 0;
  if (p->path == PATH_GENERAL) {
    p->off_beta = o_;
    o_ += align_up(sizeof(double) * 2 * P);
    p->off_iface = o_;
    o_ += align_up(sizeof(double) * 2 * P);
    p->off_scan = o_;
    o_ += align_up(sizeof(double) * 6 * (size_t)ceil_div(P, kScanChunk));
  }
  p->off_part = o_;
  o_ += align_up(sizeof(double) * 3 * (size_t)std::max<int64_t>(1, p->tiles));
  p->ws_bytes = o_;
  // staging copy: records, zero status, tables
  p->staging.assign(p->off_tabs + sizeof(double) * (p->fwd.tab.size() + p->adj.tab.size() + p->corner.size()), 0);
  SysPlan recs[2] = {p->fwd.rec, p->adj.rec};
  recs[0].tab = 0;
  recs[1].tab = (int64_t)p->fwd.tab.size();
  std::memcpy(p->staging.data() + p->off_plans, recs, sizeof(recs));
  if (!p->fwd.tab.empty())
    std::memcpy(p->staging.data() + p->off_tabs, p->fwd.tab.data(), sizeof(double) * p->fwd.tab.size());
  if (!p->adj.tab.empty())
    std::memcpy(p->staging.data() + p->off_tabs + sizeof(double) * p->fwd.tab.size(), p->adj.tab.data(),
                sizeof(double) * p->adj.tab.size());
  if (!p->corner.empty())
    std::memcpy(p->staging.data() + p->off_tabs + sizeof(double) * (p->fwd.tab.size() + p->adj.tab.size()),
                p->corner.data(), sizeof(double) * p->corner.size());
}

// Blocks, halo/general path and windows of a single-system plan for window width NT and block
// size n (fills p->NT, fwd, adj, path, n_smem, tiles).
static int plan_geometry(dich_plan_s* p, const Opts& o, int NT, int n) {
  const int WB = window_blocks(NT, p->form);
  p->NT = NT;
  int rc = build_system(p->tm1, p->t0, p->tp1, p->N, NT, p->form, n, o, true, p->fwd);
  if (!rc) rc = build_system(p->tp1, p->t0, p->tm1, p->N, NT, p->form, n, o, true, p->adj);
  if (rc) return rc;
  // both solves must take the same path; the transposed system swaps the halos
  p->path = std::max(p->fwd.path, p->adj.path);
  if (p->path == PATH_GENERAL && (p->fwd.path != PATH_GENERAL || p->adj.path != PATH_GENERAL)) {
    Opts og = o;
    og.flags |= DICH_FLAG_FORCE_GENERAL;
    build_system(p->tm1, p->t0, p->tp1, p->N, NT, p->form, n, og, true, p->fwd);
    build_system(p->tp1, p->t0, p->tm1, p->N, NT, p->form, n, og, true, p->adj);
  }
  // the transposed system swaps the decay lengths, so its halos are the forward ones mirrored and
  // both directions own the same blocks per window (the same tiles); otherwise one geometry for both
  const bool mirrored = p->fwd.rec.hl == p->adj.rec.hr && p->fwd.rec.hr == p->adj.rec.hl;
  if (p->path == PATH_HALO && !mirrored) {
    const int hl = std::max(p->fwd.rec.hl, p->adj.rec.hl), hr = std::max(p->fwd.rec.hr, p->adj.rec.hr);
    for (SysBuild* sb : {&p->fwd, &p->adj}) {
      sb->rec.hl = hl;
      sb->rec.hr = hr;
      sb->rec.own = WB - hl - hr;
    }
    if (WB - hl - hr < WB / 2) {
      Opts og = o;
      og.flags |= DICH_FLAG_FORCE_GENERAL;
      build_system(p->tm1, p->t0, p->tp1, p->N, NT, p->form, n, og, true, p->fwd);
      build_system(p->tp1, p->t0, p->tm1, p->N, NT, p->form, n, og, true, p->adj);
      p->path = PATH_GENERAL;
    }
  }
  p->n_smem = n;
  p->tiles = ceil_div(p->fwd.rec.P, p->fwd.rec.own);
  return DICH_OK;
}

// SMs of the current device (0 when no device is visible: plans are then built for the defaults)
static int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

int dichotomy_plan_ex(double t_m1, double t_0, double t_1, int64_t N, const dich_opts* opts, dich_plan_t* out) {
  if (!out) return DICH_ERR_ARG;
  *out = nullptr;
  if (N < 0) return DICH_ERR_ARG;
  Opts o;
  int rc = read_opts(opts, o);
  if (rc) return rc;
  rc = validate_t(t_m1, t_0, t_1, o.flags);
  if (rc) return rc;
  dich_plan_s* p = new (std::nothrow) dich_plan_s();
  if (!p) return DICH_ERR_ARG;
  p->N = N;
  p->tm1 = t_m1;
  p->t0 = t_0;
  p->tp1 = t_1;
  p->opts = o;
  const Roots r = toeplitz_roots(t_m1, t_0, t_1);
  p->form = pick_form(o.prec, r);
  if (p->form < 0) {
    delete p;
    return DICH_ERR_UNSUPPORTED;
  }
  p->NT = o.NT ? o.NT : default_threads(p->form);
  if (N >= 2) {
    const int n0 = choose_n(N, window_blocks(p->NT, p->form),
                            max_rows(p->NT, p->form, o.n_req > 0 ? kSmemMax : kSmemBudget), o.n_req,
                            default_rows(p->form));
    rc = plan_geometry(p, o, p->NT, n0);
    if (rc) {
      delete p;
      return rc;
    }
    // A multi-window system with fewer windows than twice the GPU's SMs is latency-bound: unless
    // the caller fixed the geometry, take narrower windows, then shorter blocks, while the system
    // stays on the halo path (halo at most half the window).  Measured on GB300: N = 65536 solves
    // 2x faster with 64-thread windows of 2-row blocks than with the large-N default.
    const int sms = device_sms();
    if (o.NT == 0 && o.n_req == 0 && p->path == PATH_HALO && p->tiles < 2 * (int64_t)sms) {
      const int nmin = (p->form == FORM_MIXED) ? 2 : 4;
      int NT = p->NT, n = n0;
      while (p->tiles < 2 * (int64_t)sms) {
        if (NT > 64)
          NT = 64;
        else if (n / 2 >= nmin)
          n /= 2;
        else
          break;
        dich_plan_s q;
        q.N = N;
        q.tm1 = t_m1;
        q.t0 = t_0;
        q.tp1 = t_1;
        q.opts = o;
        q.form = p->form;
        const int nc = choose_n(N, window_blocks(NT, p->form), max_rows(NT, p->form, kSmemBudget), n, n);
        if (plan_geometry(&q, o, NT, nc) != DICH_OK || q.path != PATH_HALO) break;
        p->NT = NT;
        p->fwd = std::move(q.fwd);
        p->adj = std::move(q.adj);
        p->path = q.path;
        p->n_smem = q.n_smem;
        p->tiles = q.tiles;
      }
    }
  } else {
    // N = 0 or 1: trivial; keep a minimal record for the N = 1 kernel
    std::memset(&p->fwd.rec, 0, sizeof(SysPlan));
    p->fwd.rec.N = N;
    p->fwd.rec.t0 = t_0;
    p->adj.rec = p->fwd.rec;
    p->tiles = 0;
  }
  plan_layout(p);
  *out = p;
  return DICH_OK;
}

int dichotomy_plan(double t_m1, double t_0, double t_1, int64_t N, dich_plan_t* out) {
  return dichotomy_plan_ex(t_m1, t_0, t_1, N, nullptr, out);
}

int dichotomy_plan_quasi(double t_m1, double t_0, double t_1, double psi, double chi, int64_t N,
                         const dich_opts* opts, dich_plan_t* out) {
  if (!out) return DICH_ERR_ARG;
  *out = nullptr;
  int rc = corner_check(t_m1, t_0, t_1, psi, chi, N, opts ? opts->flags : 0);
  if (rc) return rc;
  dich_plan_t p = nullptr;
  rc = dichotomy_plan_ex(t_m1, t_0, t_1, N, opts, &p);
  if (rc) return rc;
  p->quasi = (psi != 0.0 || chi != 0.0);
  p->corners = true;   // a corner plan reports dL/dpsi and dL/dchi, zero corners included
  p->psi = psi;
  p->chi = chi;
  if (p->quasi && N == 1) {
    // one row: t_0 + psi + chi
    p->fwd.rec.t0 = p->adj.rec.t0 = t_0 + psi + chi;
    p->quasi = false;
    plan_layout(p);
  } else if (p->quasi && N >= 2) {
    Corners c;
    rc = corner_build(t_m1, t_0, t_1, psi, chi, N, p->opts.eps, c);
    if (rc) {
      dichotomy_destroy(p);
      return rc;
    }
    p->Lg = c.Lg;
    p->Lh = c.Lh;
    p->corner = std::move(c.gh);
    std::memcpy(p->W, c.W, sizeof(p->W));
    std::memcpy(p->Wt, c.Wt, sizeof(p->Wt));
    plan_layout(p);
  }
  *out = p;
  return DICH_OK;
}

int dichotomy_plan_info(dich_plan_t p, dich_plan_info* info) {
  if (!p || !info) return DICH_ERR_ARG;
  std::memset(info, 0, sizeof(*info));
  const SysPlan& r = p->fwd.rec;
  info->N = p->N;
  info->P = (p->N >= 2) ? r.P : 0;
  info->n = r.n;
  info->n_last = r.nlast;
  info->threads = p->NT;
  info->halo_l = r.hl;
  info->halo_r = r.hr;
  info->path = p->path;
  info->precision = p->form == FORM_F64 ? DICH_PREC_F64 : DICH_PREC_MIXED;
  info->tiles = p->tiles;
  info->Lv = r.Lv;
  info->Lw = r.Lw;
  info->kl = r.kl;
  info->kr = r.kr;
  const Roots rt = toeplitz_roots(p->tm1, p->t0, p->tp1);
  info->rs = rt.rs;
  info->ib = rt.ib;
  info->z = rt.z;
  info->workspace_bytes = p->ws_bytes;
  info->growth = 1.0;   // dominant Toeplitz matrices: every block map contracts
  if (p->path == PATH_GENERAL) {
    info->beta_offset = p->off_beta;
    info->iface_offset = p->off_iface;
  }
  return DICH_OK;
}

int dichotomy_plan_workspace_bytes(dich_plan_t p, size_t* bytes) {
  if (!p || !bytes) return DICH_ERR_ARG;
  *bytes = p->ws_bytes;
  return DICH_OK;
}

int dichotomy_plan_bind(dich_plan_t p, void* d_ws, size_t bytes, void* stream) {
  if (!p || !d_ws) return DICH_ERR_ARG;
  if (((uintptr_t)d_ws & (kAlign - 1)) != 0 || bytes < p->ws_bytes) return DICH_ERR_WORKSPACE;
  if (!is_device_ptr(d_ws)) return DICH_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(d_ws, p->staging.data(), p->staging.size(), cudaMemcpyHostToDevice,
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  p->d_ws = (char*)d_ws;
  p->d_ws_bytes = bytes;
  return DICH_OK;
}

// device_mem: F and x are device memory (false: mapped host memory, read and written by the kernels
// over the host link), which lets aligned windows use bulk copies
static int plan_launch(dich_plan_t p, const double* F, double* x, const double* xf, double* gt, bool adjoint,
                       cudaStream_t st, int64_t M = 1, int64_t ldf = 0, int64_t ldx = 0, int64_t win0 = 0,
                       int64_t nwin = -1, bool device_mem = true) {
  const SysPlan* d_plans = (const SysPlan*)(p->d_ws + p->off_plans);
  const double* d_tabs = (const double*)(p->d_ws + p->off_tabs);
  unsigned* d_status = (unsigned*)(p->d_ws + p->off_status);
  const int sys_offset = adjoint ? 1 : 0;
  if (p->N == 0) return DICH_OK;
  if (p->N == 1) {
    for (int64_t k = 0; k < M; ++k) {
      cudaError_t e = launch_trivial(d_plans, nullptr, 1, adjoint ? nullptr : F + k * ldf, x + k * ldx, xf,
                                     adjoint ? F : nullptr, gt, sys_offset, st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    return DICH_OK;
  }
  WinArgs a{};
  a.plans = d_plans;
  a.tabs = d_tabs;
  a.items = nullptr;
  a.F = F;
  a.x = x;
  a.status = d_status;
  a.xf = adjoint ? xf : nullptr;
  a.part = adjoint ? (double*)(p->d_ws + p->off_part) : nullptr;
  a.check_finite = (p->opts.flags & DICH_FLAG_CHECK_FINITE) ? 1 : 0;
  a.n_smem = p->n_smem;
  a.sys_offset = sys_offset;
  a.ldf = ldf;
  a.ldx = ldx;
  // the register path (bulk copies) only for full solves of device memory, unless the plan asks
  // for the shared-memory path (the general path's passes always take that one)
  a.bulk = (device_mem && p->path != PATH_GENERAL && !(p->opts.flags & DICH_FLAG_SMEM_PATH)) ? 1 : 0;
  const size_t smem = smem_bytes(p->NT, p->n_smem, p->form);
  // windows [win0, win0 + grid) of the single and halo paths (all of them unless a range is given)
  const int grid = (int)((nwin < 0) ? p->tiles : nwin);
  auto launch = [&](const WinArgs& w, int gy) {
    return p->form == FORM_F64 ? launch_window_f64(p->NT, grid, smem, st, w, gy)
                               : launch_window_mixed(p->NT, grid, smem, st, w, gy);
  };
  cudaError_t e;
  if (p->path != PATH_GENERAL) {
    // every right-hand side of a series in one launch (grid.y), at most 65535 per launch
    a.mode = MODE_FULL;
    a.win0 = win0;
    for (int64_t k0 = 0; k0 < M; k0 += 65535) {
      WinArgs w = a;
      w.F = F + k0 * ldf;
      w.x = x + k0 * ldx;
      e = launch(w, (int)std::min<int64_t>(65535, M - k0));
      if (e != cudaSuccess) return cuda_fail(e);
    }
  } else if (M > 1) {
    // general path: the per-block scratch serves one right-hand side at a time (stream order)
    for (int64_t k = 0; k < M; ++k) {
      const int rc = plan_launch(p, F + k * ldf, x + k * ldx, nullptr, nullptr, false, st);
      if (rc != DICH_OK) return rc;
    }
  } else {
    double* beta = (double*)(p->d_ws + p->off_beta);
    double* iface = (double*)(p->d_ws + p->off_iface);
    double* scan = (double*)(p->d_ws + p->off_scan);
    WinArgs b = a;
    b.mode = MODE_BETA;
    b.beta = beta;
    b.xf = nullptr;
    b.part = nullptr;
    e = launch(b, 1);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_block_scan(d_plans + sys_offset, d_tabs, p->fwd.rec.P, beta, iface, scan, st);
    if (e != cudaSuccess) return cuda_fail(e);
    a.mode = MODE_APPLY;
    a.iface = iface;
    e = launch(a, 1);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (adjoint) {
    e = launch_adj_finalize(a.part, nullptr, nullptr, nullptr, p->tiles, 1, gt, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (p->quasi && adjoint) {
    // lambda = A^-T w from T^-T w: the corner correction with the transposed corner vectors, and
    // its share of the gradient sums plus dL/dpsi, dL/dchi (read before lambda is corrected)
    const double* ctab = d_tabs + p->fwd.tab.size() + p->adj.tab.size();
    CornerArgs c{p->N, p->Lh, p->Lg, ctab + p->Lg, ctab, p->psi, p->chi, p->Wt[0], p->Wt[1], p->Wt[2], p->Wt[3]};
    e = launch_corner_adjoint(xf, x, gt, c, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (!p->quasi && p->corners && adjoint && p->N >= 2) {
    // zero corners: lambda needs no correction; dL/dpsi = -lambda_0 x_0, dL/dchi = -lambda_{N-1} x_{N-1}
    e = launch_end_gradients(xf, x, gt, p->N, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (p->quasi && !adjoint && !(p->path == PATH_GENERAL && M > 1)) {
    const double* ctab = d_tabs + p->fwd.tab.size() + p->adj.tab.size();
    CornerArgs c{p->N, p->Lg, p->Lh, ctab, ctab + p->Lg, p->psi, p->chi, p->W[0], p->W[1], p->W[2], p->W[3]};
    e = launch_corner(x, M, M > 1 ? ldx : 0, c, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return DICH_OK;
}

int dichotomy_solve(dich_plan_t p, const double* d_F, double* d_x, void* stream) {
  if (!p) return DICH_ERR_ARG;
  if (!p->d_ws) return DICH_ERR_UNBOUND;
  if (p->N == 0) return DICH_OK;
  if (!d_F || !d_x || !aligned8(d_F) || !aligned8(d_x)) return DICH_ERR_ARG;
  const size_t nb = sizeof(double) * (size_t)p->N;
  if (overlap(d_F, nb, d_x, nb)) return DICH_ERR_ALIAS;
  if (!is_device_ptr(d_F) || !is_device_ptr(d_x)) return DICH_ERR_ARG;
  return plan_launch(p, d_F, d_x, nullptr, nullptr, false, (cudaStream_t)stream);
}

int dichotomy_solve_host(dich_plan_t p, const double* h_F, double* h_x, double* d_F, double* d_x, int32_t chunks,
                         void* stream) {
  if (!p || chunks < 0) return DICH_ERR_ARG;
  if (!p->d_ws) return DICH_ERR_UNBOUND;
  if (p->N == 0) return DICH_OK;
  if (!h_F || !h_x || !aligned8(h_F) || !aligned8(h_x)) return DICH_ERR_ARG;
  const int64_t N = p->N;
  const size_t nb = sizeof(double) * (size_t)N;
  if (overlap(h_F, nb, h_x, nb)) return DICH_ERR_ALIAS;
  if (is_device_ptr(h_F) || is_device_ptr(h_x)) return DICH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  // page-locked buffers mapped into the device's address space: the kernels read F and write x
  // there directly (one pass over the host link, no staging), except on the general path, which
  // reads F twice
  if (chunks == 0 && p->path != PATH_GENERAL) {
    auto mapped = [](const void* h) -> void* {
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
    };
    const double* zF = (const double*)mapped(h_F);
    double* zx = (double*)mapped(h_x);
    if (zF && zx) return plan_launch(p, zF, zx, nullptr, nullptr, false, st, 1, 0, 0, 0, -1, false);
  }
  if (!d_F || !d_x || !aligned8(d_F) || !aligned8(d_x)) return DICH_ERR_ARG;
  if (overlap(d_F, nb, d_x, nb)) return DICH_ERR_ALIAS;
  if (!is_device_ptr(d_F) || !is_device_ptr(d_x)) return DICH_ERR_ARG;
  const int64_t T = p->tiles;
  // only independent windows pipeline: the halo path of a plain Toeplitz plan with two or more windows
  const bool pipe = p->N >= 2 && p->path == PATH_HALO && !p->quasi && T >= 2 && chunks != 1;
  if (!pipe) {
    e = cudaMemcpyAsync(d_F, h_F, nb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
    const int rc = plan_launch(p, d_F, d_x, nullptr, nullptr, false, st);
    if (rc != DICH_OK) return rc;
    e = cudaMemcpyAsync(h_x, d_x, nb, cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? DICH_OK : cuda_fail(e);
  }
  const int64_t K = std::min<int64_t>(T, chunks ? chunks : 16);   // pieces of whole windows
  // streams and 2K + 2 events, kept by the plan
  for (cudaStream_t& h : p->hs)
    if (!h && (e = cudaStreamCreateWithFlags(&h, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e);
  while ((int64_t)p->hev.size() < 2 * K + 2) {
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e);
    p->hev.push_back(ev);
  }
  cudaEvent_t* evin = p->hev.data();           // [K]: chunk k of F is on the device
  cudaEvent_t* evk = evin + K;                 // [K]: the windows of chunk k are solved
  cudaEvent_t evs = evk[K], eve = evk[K + 1];  // start (on st), end (copy-out stream)
  const SysPlan& r = p->fwd.rec;
  const int64_t rows_w = (int64_t)r.own * r.n;   // rows owned by a window
  auto row_of = [&](int64_t w) { return std::min<int64_t>(N, w * rows_w); };
  auto win_of = [&](int64_t k) { return T * k / K; };
  if ((e = cudaEventRecord(evs, st)) != cudaSuccess) return cuda_fail(e);
  for (cudaStream_t h : p->hs)
    if ((e = cudaStreamWaitEvent(h, evs, 0)) != cudaSuccess) return cuda_fail(e);
  // F in K chunks of whole windows' own rows, in order on the copy-in stream
  for (int64_t k = 0; k < K; ++k) {
    const int64_t r0 = row_of(win_of(k)), r1 = row_of(win_of(k + 1));
    e = cudaMemcpyAsync(d_F + r0, h_F + r0, sizeof(double) * (size_t)(r1 - r0), cudaMemcpyHostToDevice, p->hs[0]);
    if (e == cudaSuccess) e = cudaEventRecord(evin[k], p->hs[0]);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // chunk k's windows once every row they read (own rows plus the right halo) has arrived; its own
  // rows of x go back on the copy-out stream while later chunks are copied in and solved
  int64_t j = 0;
  for (int64_t k = 0; k < K; ++k) {
    const int64_t w0 = win_of(k), w1 = win_of(k + 1);
    const int64_t need = std::min<int64_t>(N, (w1 * (int64_t)r.own + r.hr) * r.n);
    while (row_of(win_of(j + 1)) < need) ++j;
    if ((e = cudaStreamWaitEvent(st, evin[j], 0)) != cudaSuccess) return cuda_fail(e);
    const int rc = plan_launch(p, d_F, d_x, nullptr, nullptr, false, st, 1, 0, 0, w0, w1 - w0);
    if (rc != DICH_OK) return rc;
    if ((e = cudaEventRecord(evk[k], st)) != cudaSuccess) return cuda_fail(e);
    const int64_t r0 = row_of(w0), r1 = row_of(w1);
    e = cudaStreamWaitEvent(p->hs[1], evk[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_x + r0, d_x + r0, sizeof(double) * (size_t)(r1 - r0), cudaMemcpyDeviceToHost, p->hs[1]);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  e = cudaEventRecord(eve, p->hs[1]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, eve, 0);
  return e == cudaSuccess ? DICH_OK : cuda_fail(e);
}

int dichotomy_solve_series(dich_plan_t p, int64_t M, const double* d_F, int64_t ldf, double* d_x, int64_t ldx,
                           void* stream) {
  if (!p || M < 0) return DICH_ERR_ARG;
  if (!p->d_ws) return DICH_ERR_UNBOUND;
  if (p->N == 0 || M == 0) return DICH_OK;
  if (!d_F || !d_x || !aligned8(d_F) || !aligned8(d_x)) return DICH_ERR_ARG;
  if (M > 1 && (ldf < p->N || ldx < p->N)) return DICH_ERR_ARG;
  if (M > 1 && (ldf > INT64_MAX / M || ldx > INT64_MAX / M)) return DICH_ERR_ARG;
  const int64_t sf = (M > 1) ? ldf : 0, sx = (M > 1) ? ldx : 0;
  const size_t nf = sizeof(double) * (size_t)((M - 1) * sf + p->N);
  const size_t nx = sizeof(double) * (size_t)((M - 1) * sx + p->N);
  if (overlap(d_F, nf, d_x, nx)) return DICH_ERR_ALIAS;
  if (!is_device_ptr(d_F) || !is_device_ptr(d_x)) return DICH_ERR_ARG;
  return plan_launch(p, d_F, d_x, nullptr, nullptr, false, (cudaStream_t)stream, M, sf, sx);
}

int dichotomy_adjoint(dich_plan_t p, const double* d_w, const double* d_x, double* d_gF, double* d_gt,
                      void* stream) {
  if (!p) return DICH_ERR_ARG;
  if (!p->d_ws) return DICH_ERR_UNBOUND;
  if (!d_gt || !aligned8(d_gt) || !is_device_ptr(d_gt)) return DICH_ERR_ARG;
  const size_t ngt = sizeof(double) * (p->corners ? 5 : 3);
  cudaStream_t st = (cudaStream_t)stream;
  if (p->N == 0) {
    cudaError_t e = cudaMemsetAsync(d_gt, 0, ngt, st);
    return e == cudaSuccess ? DICH_OK : cuda_fail(e);
  }
  if (!d_w || !d_x || !d_gF || !aligned8(d_w) || !aligned8(d_x) || !aligned8(d_gF)) return DICH_ERR_ARG;
  const size_t nb = sizeof(double) * (size_t)p->N;
  if (overlap(d_gF, nb, d_w, nb) || overlap(d_gF, nb, d_x, nb) || overlap(d_gt, ngt, d_gF, nb)) return DICH_ERR_ALIAS;
  if (!is_device_ptr(d_w) || !is_device_ptr(d_x) || !is_device_ptr(d_gF)) return DICH_ERR_ARG;
  const int rc = plan_launch(p, d_w, d_gF, d_x, d_gt, true, st);
  if (rc != DICH_OK || !p->corners || p->quasi || p->N != 1) return rc;
  // one row (t_0 + psi + chi): dL/dpsi = dL/dchi = dL/dt_0
  cudaError_t e = cudaMemcpyAsync(d_gt + 3, d_gt + 1, sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_gt + 4, d_gt + 1, sizeof(double), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? DICH_OK : cuda_fail(e);
}

int dichotomy_residual(dich_plan_t p, const double* d_F, const double* d_x, double* h_out, void* stream) {
  if (!p || !h_out) return DICH_ERR_ARG;
  if (!p->d_ws) return DICH_ERR_UNBOUND;
  h_out[0] = h_out[1] = 0.0;
  if (p->N == 0) return DICH_OK;
  if (!d_F || !d_x || !aligned8(d_F) || !aligned8(d_x) || !is_device_ptr(d_F) || !is_device_ptr(d_x))
    return DICH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // three maxima in the status region's spare bytes (the status word is its first 4 bytes)
  unsigned long long* res = (unsigned long long*)(p->d_ws + p->off_status + 64);
  const double t0 = (p->corners && p->N == 1) ? p->fwd.rec.t0 : p->t0;
  cudaError_t e = launch_toeplitz_residual(p->N, p->tm1, t0, p->tp1, p->quasi ? p->psi : 0.0,
                                           p->quasi ? p->chi : 0.0, d_F, d_x, res, st);
  unsigned long long m[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(m, res, sizeof(m), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  double r, xm, fm;
  std::memcpy(&r, &m[0], sizeof(double));
  std::memcpy(&xm, &m[1], sizeof(double));
  std::memcpy(&fm, &m[2], sizeof(double));
  double nA = std::fabs(p->tm1) + std::fabs(p->t0) + std::fabs(p->tp1);
  if (p->quasi) nA = std::max({nA, std::fabs(p->t0 + p->psi) + std::fabs(p->tp1), std::fabs(p->tm1) + std::fabs(p->t0 + p->chi)});
  if (p->N == 1) nA = std::fabs(t0);
  const double den = nA * xm + fm;
  h_out[0] = r;
  h_out[1] = (den > 0.0) ? r / den : 0.0;
  return DICH_OK;
}

int dichotomy_status(dich_plan_t p, void* stream, int* device_status) {
  if (!p || !device_status) return DICH_ERR_ARG;
  if (!p->d_ws) return DICH_ERR_UNBOUND;
  unsigned s = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&s, p->d_ws + p->off_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(p->d_ws + p->off_status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e);
  *device_status = map_status(s);
  return DICH_OK;
}

void dichotomy_destroy(dich_plan_t p) { delete p; }

// ================================================================== sharded solve of one system
// Shard k of nshards owns the windows [k T / S, (k + 1) T / S) of the plan (T windows of `own`
// blocks, S shards): blocks [block_lo, block_hi), rows [row_lo, row_hi).  The shard runs the beta
// pass and the block scan over its own blocks only; what crosses shards is the paper's exchange
// between processes (Sec. 2.4-2.5, eq. 17-19, collapsed by associativity to one level): the four
// numbers of each shard's composite prefix and suffix maps, then one boundary value to each
// neighbour.  Workspace of one shard (caller-owned, 256-byte aligned): totals [4], every shard's
// totals [4 S], beta [2 nb], first/last values with one neighbour entry on each side [2 (nb + 2)],
// scan scratch [6 chunks].
namespace {
struct ShardGeo {
  int64_t w_lo, w_hi, block_lo, block_hi, row_lo, row_hi, nb, nch;
  size_t off_tot, off_maps, off_beta, off_iface, off_scan, bytes;
};
int shard_geo(dich_plan_t p, int32_t nshards, int32_t k, ShardGeo& g) {
  if (!p || nshards < 1 || k < 0 || k >= nshards) return DICH_ERR_ARG;
  if (p->N < 2 || p->quasi) return DICH_ERR_UNSUPPORTED;
  const SysPlan& r = p->fwd.rec;
  const int64_t own = r.own, P = r.P, T = ceil_div(P, own);
  if (nshards > T) return DICH_ERR_ARG;
  g.w_lo = (int64_t)k * T / nshards;
  g.w_hi = (int64_t)(k + 1) * T / nshards;
  g.block_lo = g.w_lo * own;
  g.block_hi = std::min<int64_t>(P, g.w_hi * own);
  g.row_lo = g.block_lo * r.n;
  g.row_hi = std::min<int64_t>(p->N, g.block_hi * r.n);
  g.nb = g.block_hi - g.block_lo;
  g.nch = ceil_div(g.nb, kScanChunk);
  size_t o = 0;
  g.off_tot = o;
  o = align_up(o + sizeof(double) * 4);
  g.off_maps = o;
  o = align_up(o + sizeof(double) * 4 * (size_t)nshards);
  g.off_beta = o;
  o = align_up(o + sizeof(double) * 2 * (size_t)g.nb);
  g.off_iface = o;
  o = align_up(o + sizeof(double) * 2 * (size_t)(g.nb + 2));
  g.off_scan = o;
  o = align_up(o + sizeof(double) * 6 * (size_t)g.nch);
  g.bytes = o;
  return DICH_OK;
}
int shard_check(dich_plan_t p, const ShardGeo& g, const void* d_ws, size_t ws_bytes) {
  if (!p->d_ws) return DICH_ERR_UNBOUND;
  if (!d_ws || ((uintptr_t)d_ws & (kAlign - 1)) != 0 || ws_bytes < g.bytes) return DICH_ERR_WORKSPACE;
  if (!is_device_ptr(d_ws)) return DICH_ERR_ARG;
  return DICH_OK;
}
// the shard's windows in one mode (beta pass or apply pass); F and x hold the shard's rows only
cudaError_t shard_windows(dich_plan_t p, const ShardGeo& g, int mode, const double* d_F, double* d_x, double* beta,
                          const double* iface, cudaStream_t st) {
  WinArgs a{};
  a.plans = (const SysPlan*)(p->d_ws + p->off_plans);
  a.tabs = (const double*)(p->d_ws + p->off_tabs);
  a.F = d_F - g.row_lo;   // the kernels index rows of the whole system
  a.x = d_x - g.row_lo;
  a.status = (unsigned*)(p->d_ws + p->off_status);
  a.mode = mode;
  a.beta = beta;
  a.iface = iface;
  a.check_finite = (p->opts.flags & DICH_FLAG_CHECK_FINITE) ? 1 : 0;
  a.n_smem = p->n_smem;
  a.win0 = g.w_lo;
  const int grid = (int)(g.w_hi - g.w_lo);
  const size_t smem = smem_bytes(p->NT, p->n_smem, p->form);
  return p->form == FORM_F64 ? launch_window_f64(p->NT, grid, smem, st, a, 1)
                             : launch_window_mixed(p->NT, grid, smem, st, a, 1);
}
}  // namespace

int dichotomy_shard_info(dich_plan_t p, int32_t nshards, int32_t k, dich_shard_info* info) {
  if (!info) return DICH_ERR_ARG;
  ShardGeo g;
  const int rc = shard_geo(p, nshards, k, g);
  if (rc) return rc;
  info->row_lo = g.row_lo;
  info->row_hi = g.row_hi;
  info->block_lo = g.block_lo;
  info->block_hi = g.block_hi;
  info->workspace_bytes = g.bytes;
  return DICH_OK;
}

int dichotomy_shard_reduce(dich_plan_t p, int32_t nshards, int32_t k, const double* d_F, double* d_x, void* d_ws,
                           size_t ws_bytes, double* h_maps, void* stream) {
  ShardGeo g;
  int rc = shard_geo(p, nshards, k, g);
  if (rc) return rc;
  if ((rc = shard_check(p, g, d_ws, ws_bytes))) return rc;
  if (!h_maps || !d_F || !d_x || !aligned8(d_F) || !aligned8(d_x)) return DICH_ERR_ARG;
  const size_t nr = sizeof(double) * (size_t)(g.row_hi - g.row_lo);
  if (overlap(d_F, nr, d_x, nr)) return DICH_ERR_ALIAS;
  if (!is_device_ptr(d_F) || !is_device_ptr(d_x)) return DICH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)d_ws;
  double* beta = (double*)(w + g.off_beta);
  // beta of the shard's blocks (eq. 16); the kernels index blocks of the whole system
  cudaError_t e = shard_windows(p, g, MODE_BETA, d_F, d_x, beta - 2 * g.block_lo, nullptr, st);
  ScanMap m{};
  m.mbase = g.block_lo;
  m.mend = g.block_hi;
  m.shard = k;
  m.nshards = nshards;
  m.tot = (double*)(w + g.off_tot);
  if (e == cudaSuccess)
    e = launch_shard_scan_reduce((const SysPlan*)(p->d_ws + p->off_plans), (const double*)(p->d_ws + p->off_tabs), m,
                                 beta - 2 * g.block_lo, (double*)(w + g.off_scan), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_maps, w + g.off_tot, sizeof(double) * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? DICH_OK : cuda_fail(e);
}

int dichotomy_shard_bounds(dich_plan_t p, int32_t nshards, int32_t k, const double* h_all_maps, void* d_ws,
                           size_t ws_bytes, double* h_ends, void* stream) {
  ShardGeo g;
  int rc = shard_geo(p, nshards, k, g);
  if (rc) return rc;
  if ((rc = shard_check(p, g, d_ws, ws_bytes))) return rc;
  if (!h_all_maps || !h_ends) return DICH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)d_ws;
  double* maps = (double*)(w + g.off_maps);
  double* iface = (double*)(w + g.off_iface);
  cudaError_t e = cudaMemcpyAsync(maps, h_all_maps, sizeof(double) * 4 * (size_t)nshards, cudaMemcpyHostToDevice, st);
  ScanMap m{};
  m.mbase = g.block_lo;
  m.mend = g.block_hi;
  m.maps = maps;
  m.shard = k;
  m.nshards = nshards;
  double* beta = (double*)(w + g.off_beta);
  if (e == cudaSuccess)
    e = launch_shard_scan_apply((const SysPlan*)(p->d_ws + p->off_plans), (const double*)(p->d_ws + p->off_tabs), m,
                                beta - 2 * g.block_lo, iface - 2 * (g.block_lo - 1), (double*)(w + g.off_scan), st);
  // x at the shard's first row (x_s of its first block) and last row (x_e of its last block)
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_ends, iface + 2, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_ends + 1, iface + 2 * g.nb + 1, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? DICH_OK : cuda_fail(e);
}

int dichotomy_shard_finish(dich_plan_t p, int32_t nshards, int32_t k, const double* d_F, double* d_x,
                           const double* h_nbr, void* d_ws, size_t ws_bytes, void* stream) {
  ShardGeo g;
  int rc = shard_geo(p, nshards, k, g);
  if (rc) return rc;
  if ((rc = shard_check(p, g, d_ws, ws_bytes))) return rc;
  if (!h_nbr || !d_F || !d_x || !aligned8(d_F) || !aligned8(d_x)) return DICH_ERR_ARG;
  const size_t nr = sizeof(double) * (size_t)(g.row_hi - g.row_lo);
  if (overlap(d_F, nr, d_x, nr)) return DICH_ERR_ALIAS;
  if (!is_device_ptr(d_F) || !is_device_ptr(d_x)) return DICH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)d_ws;
  double* iface = (double*)(w + g.off_iface);
  // the neighbours' boundary values: x_e of the block before the shard, x_s of the block after it
  cudaError_t e = cudaMemcpyAsync(iface + 1, h_nbr, sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(iface + 2 * (g.nb + 1), h_nbr + 1, sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = shard_windows(p, g, MODE_APPLY, d_F, d_x, nullptr, iface - 2 * (g.block_lo - 1), st);
  return e == cudaSuccess ? DICH_OK : cuda_fail(e);
}

}  // extern "C"

// ================================================================== batches
struct dich_batch_s {
  ~dich_batch_s() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (aux) cudaStreamDestroy(aux);
  }
  int64_t nsys = 0;
  Opts opts;
  bool reg_path = true;                   // MIXED windows on the register path (else shared memory)
  // a second stream for the FP64-form windows when a batch has both forms: the two launches
  // overlap (fork/join through events on the caller's stream; CUDA-graph capture follows them)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int NT[2] = {64, 128};                  // window width per form
  std::vector<SysBuild> fwd, adj;          // per system (N >= 2); empty records for N < 2
  std::vector<int32_t> form;               // per system
  std::vector<int32_t> trivial;            // systems with N == 1
  std::vector<int32_t> general;            // systems on the general path
  // general-path systems per form: windows, scan chunk map, their systems and first chunks,
  // gradient ranges; beta and first/last values of all of them in two shared buffers
  std::vector<Item> gitems[2];
  std::vector<int32_t> gcmap[2], gsys[2];
  std::vector<int64_t> gc0[2], gfirst[2], gcount[2];
  int64_t gblocks = 0;
  int n_smem_g[2] = {2, 2};
  size_t off_gitems[2] = {0, 0}, off_gcmap[2] = {0, 0}, off_gsys[2] = {0, 0}, off_gc0[2] = {0, 0},
         off_gfirst[2] = {0, 0}, off_gcount[2] = {0, 0}, off_gscan[2] = {0, 0}, off_gpart[2] = {0, 0},
         off_gbeta = 0, off_giface = 0;
  std::vector<Item> items[2];              // per form
  std::vector<int32_t> sys_ids[2];         // per form: its systems, in item order
  std::vector<int64_t> first[2], count[2]; // per form, parallel to sys_ids: CTA range of each system
  int n_smem[2] = {2, 2};
  size_t ws_bytes = 0, off_plans = 0, off_status = 0, off_tabs = 0, off_items[2] = {0, 0},
         off_ids[2] = {0, 0}, off_first[2] = {0, 0}, off_count[2] = {0, 0}, off_trivial = 0,
         off_part[2] = {0, 0};
  std::vector<unsigned char> staging;
  char* d_ws = nullptr;
  size_t d_ws_bytes = 0;
  // quasi-Toeplitz systems (eq. 21): their corner records and corner vectors, after the rest
  std::vector<CornerRec> crec;
  std::vector<double> ctab;
  std::vector<CornerRec> crec_adj;         // every system: its transposed corner record (adjoint)
  size_t off_crec = 0, off_ctab = 0, off_crec_adj = 0, off_gt3 = 0;
};

extern "C" {

int dichotomy_batch_prepare(int64_t nsys, const int64_t* h_N, const int64_t* h_offset, const double* h_tm1,
                            const double* h_t0, const double* h_tp1, const dich_opts* opts, dich_batch_t* out) {
  if (!out) return DICH_ERR_ARG;
  *out = nullptr;
  if (nsys < 0 || (nsys > 0 && (!h_N || !h_offset || !h_tm1 || !h_t0 || !h_tp1))) return DICH_ERR_ARG;
  if (nsys > ((int64_t)1 << 30)) return DICH_ERR_ARG;
  Opts o;
  int rc = read_opts(opts, o);
  if (rc) return rc;
  dich_batch_s* b = new (std::nothrow) dich_batch_s();
  if (!b) return DICH_ERR_ARG;
  b->nsys = nsys;
  b->opts = o;
  for (int f = 0; f < 2; ++f) b->NT[f] = o.NT ? o.NT : default_threads(f);
  if (!o.NT && o.n_req == 0) {
    // few FP64-form windows (a handful of ill-conditioned systems beside many MIXED ones, such as
    // the lowest Poisson modes) are latency-bound: 256-thread windows of shorter blocks
    int64_t w64 = 0;
    for (int64_t s = 0; s < nsys; ++s) {
      if (h_N[s] < 2 || !std::isfinite(h_tm1[s]) || !std::isfinite(h_t0[s]) || !std::isfinite(h_tp1[s])) continue;
      const Roots r = toeplitz_roots(h_tm1[s], h_t0[s], h_tp1[s]);
      if (r.ok && pick_form(o.prec, r) == FORM_F64)
        w64 += ceil_div(h_N[s], (int64_t)default_threads(FORM_F64) * default_rows(FORM_F64));
    }
    const int sms = device_sms();
    if (w64 > 0 && w64 < 2 * (int64_t)sms) b->NT[FORM_F64] = 256;
  }
  b->fwd.resize((size_t)nsys);
  b->adj.resize((size_t)nsys);
  b->form.assign((size_t)nsys, FORM_F64);
  for (int64_t s = 0; s < nsys; ++s) {
    if (h_N[s] < 0 || h_offset[s] < 0) {
      delete b;
      return DICH_ERR_ARG;
    }
    rc = validate_t(h_tm1[s], h_t0[s], h_tp1[s], o.flags);
    if (rc) {
      delete b;
      return rc;
    }
    const Roots r = toeplitz_roots(h_tm1[s], h_t0[s], h_tp1[s]);
    b->form[s] = pick_form(o.prec, r);
    if (b->form[s] < 0) {
      delete b;
      return DICH_ERR_UNSUPPORTED;
    }
    if (h_N[s] < 2) {
      SysPlan& q = b->fwd[s].rec;
      std::memset(&q, 0, sizeof(q));
      q.N = h_N[s];
      q.off = h_offset[s];
      q.t0 = h_t0[s];
      b->adj[s].rec = q;
      if (h_N[s] == 1) b->trivial.push_back((int32_t)s);
      continue;
    }
    const int NTs = b->NT[b->form[s]];
    const int nmax = max_rows(NTs, b->form[s], o.n_req > 0 ? kSmemMax : kSmemBudget);
    const int n = choose_n(h_N[s], window_blocks(NTs, b->form[s]), nmax, o.n_req, default_rows(b->form[s]));
    Opts oh = o;
    oh.flags &= ~DICH_FLAG_FORCE_GENERAL;
    rc = build_system(h_tm1[s], h_t0[s], h_tp1[s], h_N[s], NTs, b->form[s], n, oh, true, b->fwd[s]);
    if (!rc) rc = build_system(h_tp1[s], h_t0[s], h_tm1[s], h_N[s], NTs, b->form[s], n, oh, true, b->adj[s]);
    if (rc) {
      delete b;
      return rc;
    }
    const int WBs = window_blocks(NTs, b->form[s]);
    bool general = (b->fwd[s].path == PATH_GENERAL || b->adj[s].path == PATH_GENERAL);
    const bool mirrored = b->fwd[s].path == PATH_HALO && b->adj[s].path == PATH_HALO &&
                          b->fwd[s].rec.hl == b->adj[s].rec.hr && b->fwd[s].rec.hr == b->adj[s].rec.hl;
    if (!general && !mirrored && (b->fwd[s].path == PATH_HALO || b->adj[s].path == PATH_HALO)) {
      const int hl = std::max(b->fwd[s].rec.hl, b->adj[s].rec.hl);
      const int hr = std::max(b->fwd[s].rec.hr, b->adj[s].rec.hr);
      if (hl + hr > WBs / 2) {
        general = true;
      } else {
        for (SysBuild* sb : {&b->fwd[s], &b->adj[s]}) {
          sb->rec.hl = hl;
          sb->rec.hr = hr;
          sb->rec.own = WBs - hl - hr;
          sb->path = PATH_HALO;
        }
      }
    }
    if (general) {
      // coupling longer than half a window: this system takes the general path (its own beta
      // pass, block scan and apply pass) after the windowed launches
      Opts og = oh;
      og.flags |= DICH_FLAG_FORCE_GENERAL;
      build_system(h_tm1[s], h_t0[s], h_tp1[s], h_N[s], NTs, b->form[s], n, og, true, b->fwd[s]);
      build_system(h_tp1[s], h_t0[s], h_tm1[s], h_N[s], NTs, b->form[s], n, og, true, b->adj[s]);
      b->general.push_back((int32_t)s);
    }
    for (SysBuild* sb : {&b->fwd[s], &b->adj[s]}) sb->rec.off = h_offset[s];
  }
  // windows, longest systems first (LPT); windows of one system stay contiguous
  std::vector<int64_t> order;
  std::vector<char> is_general((size_t)nsys, 0);
  for (int32_t s : b->general) is_general[(size_t)s] = 1;
  for (int64_t s = 0; s < nsys; ++s)
    if (h_N[s] >= 2 && !is_general[(size_t)s]) order.push_back(s);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t c) { return h_N[a] > h_N[c]; });
  for (int64_t s : order) {
    const SysPlan& q = b->fwd[s].rec;
    const int f = b->form[s];
    const int64_t first = (int64_t)b->items[f].size();
    for (int64_t m0 = 0; m0 < q.P; m0 += q.own) {
      Item it;
      it.m0 = m0;
      it.sys = (int32_t)s;
      it.n_own = (int32_t)std::min<int64_t>(q.own, q.P - m0);
      b->items[f].push_back(it);
    }
    b->sys_ids[f].push_back((int32_t)s);
    b->first[f].push_back(first);
    b->count[f].push_back((int64_t)b->items[f].size() - first);
    b->n_smem[f] = std::max(b->n_smem[f], q.n);
  }
  // MIXED windows: the register path unless most of them are whole one-window systems, whose
  // windows are latency-bound (their own tables, no halo to amortise the set-up): there the
  // shared-memory path's six CTAs per SM win (4096 Poisson modes of 4096 rows: 101 us against
  // 106-110 us); explicit flags decide otherwise
  {
    int64_t whole = 0;
    for (int64_t s : order)
      if (b->form[s] == FORM_MIXED && b->fwd[s].rec.P <= window_blocks(b->NT[FORM_MIXED], FORM_MIXED)) ++whole;
    const int64_t nmix = (int64_t)b->items[FORM_MIXED].size();
    b->reg_path = (o.flags & DICH_FLAG_REG_PATH) ? true
                  : (o.flags & DICH_FLAG_SMEM_PATH) ? false
                                                    : (2 * whole <= nmix);
  }
  // general-path systems: block offsets in the shared buffers, windows without halo, scan chunks
  for (int32_t s : b->general) {
    SysPlan& rf = b->fwd[(size_t)s].rec;
    rf.gboff = b->gblocks;
    b->adj[(size_t)s].rec.gboff = b->gblocks;
    b->gblocks += rf.P;
    const int f = b->form[(size_t)s];
    const int64_t first = (int64_t)b->gitems[f].size();
    for (int64_t m0 = 0; m0 < rf.P; m0 += rf.own) {
      Item it;
      it.m0 = m0;
      it.sys = s;
      it.n_own = (int32_t)std::min<int64_t>(rf.own, rf.P - m0);
      b->gitems[f].push_back(it);
    }
    b->gfirst[f].push_back(first);
    b->gcount[f].push_back((int64_t)b->gitems[f].size() - first);
    const int64_t nch = ceil_div(rf.P, kScanChunk);
    b->gc0[f].push_back((int64_t)b->gcmap[f].size());
    for (int64_t c = 0; c < nch; ++c) b->gcmap[f].push_back((int32_t)b->gsys[f].size());
    b->gsys[f].push_back(s);
    b->n_smem_g[f] = std::max(b->n_smem_g[f], rf.n);
  }
  // tables
  int64_t tabsz = 0;
  for (int64_t s = 0; s < nsys; ++s) {
    b->fwd[s].rec.tab = tabsz;
    tabsz += (int64_t)b->fwd[s].tab.size();
    b->adj[s].rec.tab = tabsz;
    tabsz += (int64_t)b->adj[s].tab.size();
  }
  size_t o_ = 0;
  b->off_plans = o_;
  o_ += align_up(sizeof(SysPlan) * 2 * (size_t)std::max<int64_t>(1, nsys));
  b->off_status = o_;
  o_ += kAlign;
  for (int f = 0; f < 2; ++f) {
    b->off_items[f] = o_;
    o_ += align_up(sizeof(Item) * std::max<size_t>(1, b->items[f].size()));
    b->off_ids[f] = o_;
    o_ += align_up(sizeof(int32_t) * std::max<size_t>(1, b->sys_ids[f].size()));
    b->off_first[f] = o_;
    o_ += align_up(sizeof(int64_t) * std::max<size_t>(1, b->first[f].size()));
    b->off_count[f] = o_;
    o_ += align_up(sizeof(int64_t) * std::max<size_t>(1, b->count[f].size()));
  }
  b->off_trivial = o_;
  o_ += align_up(sizeof(int32_t) * std::max<size_t>(1, b->trivial.size()));
  for (int f = 0; f < 2; ++f) {
    b->off_gitems[f] = o_;
    o_ += align_up(sizeof(Item) * std::max<size_t>(1, b->gitems[f].size()));
    b->off_gcmap[f] = o_;
    o_ += align_up(sizeof(int32_t) * std::max<size_t>(1, b->gcmap[f].size()));
    b->off_gsys[f] = o_;
    o_ += align_up(sizeof(int32_t) * std::max<size_t>(1, b->gsys[f].size()));
    b->off_gc0[f] = o_;
    o_ += align_up(sizeof(int64_t) * std::max<size_t>(1, b->gc0[f].size()));
    b->off_gfirst[f] = o_;
    o_ += align_up(sizeof(int64_t) * std::max<size_t>(1, b->gfirst[f].size()));
    b->off_gcount[f] = o_;
    o_ += align_up(sizeof(int64_t) * std::max<size_t>(1, b->gcount[f].size()));
  }
  b->off_tabs = o_;
  o_ += align_up(sizeof(double) * (size_t)std::max<int64_t>(1, tabsz));
  const size_t staged = o_;
  for (int f = 0; f < 2; ++f) {
    b->off_part[f] = o_;
    o_ += align_up(sizeof(double) * 3 * std::max<size_t>(1, b->items[f].size()));
  }
  b->off_gbeta = o_;
  o_ += align_up(sizeof(double) * 2 * (size_t)std::max<int64_t>(1, b->gblocks));
  b->off_giface = o_;
  o_ += align_up(sizeof(double) * 2 * (size_t)std::max<int64_t>(1, b->gblocks));
  for (int f = 0; f < 2; ++f) {
    b->off_gscan[f] = o_;
    o_ += align_up(sizeof(double) * 6 * std::max<size_t>(1, b->gcmap[f].size()));
    b->off_gpart[f] = o_;
    o_ += align_up(sizeof(double) * 3 * std::max<size_t>(1, b->gitems[f].size()));
  }
  b->ws_bytes = o_;
  b->staging.assign(staged, 0);
  unsigned char* S = b->staging.data();
  for (int64_t s = 0; s < nsys; ++s) {
    std::memcpy(S + b->off_plans + sizeof(SysPlan) * s, &b->fwd[s].rec, sizeof(SysPlan));
    std::memcpy(S + b->off_plans + sizeof(SysPlan) * (nsys + s), &b->adj[s].rec, sizeof(SysPlan));
    if (!b->fwd[s].tab.empty())
      std::memcpy(S + b->off_tabs + sizeof(double) * b->fwd[s].rec.tab, b->fwd[s].tab.data(),
                  sizeof(double) * b->fwd[s].tab.size());
    if (!b->adj[s].tab.empty())
      std::memcpy(S + b->off_tabs + sizeof(double) * b->adj[s].rec.tab, b->adj[s].tab.data(),
                  sizeof(double) * b->adj[s].tab.size());
  }
  for (int f = 0; f < 2; ++f) {
    if (!b->items[f].empty()) std::memcpy(S + b->off_items[f], b->items[f].data(), sizeof(Item) * b->items[f].size());
    if (!b->sys_ids[f].empty()) {
      std::memcpy(S + b->off_ids[f], b->sys_ids[f].data(), sizeof(int32_t) * b->sys_ids[f].size());
      std::memcpy(S + b->off_first[f], b->first[f].data(), sizeof(int64_t) * b->first[f].size());
      std::memcpy(S + b->off_count[f], b->count[f].data(), sizeof(int64_t) * b->count[f].size());
    }
  }
  if (!b->trivial.empty())
    std::memcpy(S + b->off_trivial, b->trivial.data(), sizeof(int32_t) * b->trivial.size());
  for (int f = 0; f < 2; ++f) {
    if (b->gitems[f].empty()) continue;
    std::memcpy(S + b->off_gitems[f], b->gitems[f].data(), sizeof(Item) * b->gitems[f].size());
    std::memcpy(S + b->off_gcmap[f], b->gcmap[f].data(), sizeof(int32_t) * b->gcmap[f].size());
    std::memcpy(S + b->off_gsys[f], b->gsys[f].data(), sizeof(int32_t) * b->gsys[f].size());
    std::memcpy(S + b->off_gc0[f], b->gc0[f].data(), sizeof(int64_t) * b->gc0[f].size());
    std::memcpy(S + b->off_gfirst[f], b->gfirst[f].data(), sizeof(int64_t) * b->gfirst[f].size());
    std::memcpy(S + b->off_gcount[f], b->gcount[f].data(), sizeof(int64_t) * b->gcount[f].size());
  }
  *out = b;
  return DICH_OK;
}

int dichotomy_batch_prepare_quasi(int64_t nsys, const int64_t* h_N, const int64_t* h_offset, const double* h_tm1,
                                  const double* h_t0, const double* h_tp1, const double* h_psi, const double* h_chi,
                                  const dich_opts* opts, dich_batch_t* out) {
  if (!out) return DICH_ERR_ARG;
  *out = nullptr;
  if (nsys < 0 || (nsys > 0 && (!h_N || !h_offset || !h_tm1 || !h_t0 || !h_tp1 || !h_psi || !h_chi)))
    return DICH_ERR_ARG;
  // one-row systems read t_0 + psi + chi (and have no off-diagonal entries)
  std::vector<double> tm1e(h_tm1, h_tm1 + nsys), t0e(h_t0, h_t0 + nsys), tp1e(h_tp1, h_tp1 + nsys);
  for (int64_t s = 0; s < nsys; ++s) {
    const int rc = corner_check(h_tm1[s], h_t0[s], h_tp1[s], h_psi[s], h_chi[s], h_N[s], opts ? opts->flags : 0);
    if (rc) return rc;
    if (h_N[s] == 1) {
      t0e[(size_t)s] = h_t0[s] + h_psi[s] + h_chi[s];
      tm1e[(size_t)s] = tp1e[(size_t)s] = 0.0;
    }
  }
  dich_batch_t b = nullptr;
  int rc = dichotomy_batch_prepare(nsys, h_N, h_offset, tm1e.data(), t0e.data(), tp1e.data(), opts, &b);
  if (rc) return rc;
  b->crec_adj.reserve((size_t)nsys);
  for (int64_t s = 0; s < nsys; ++s) {
    // the adjoint's record: plain systems keep empty corner vectors (their dL/dpsi, dL/dchi are
    // still -lambda_0 x_0 and -lambda_{N-1} x_{N-1})
    CornerRec adj{h_N[s], h_offset[s], 0, 0, 0, 0, h_psi[s], h_chi[s], 1.0, 0.0, 0.0, 1.0};
    if (h_N[s] >= 2 && (h_psi[s] != 0.0 || h_chi[s] != 0.0)) {
      Corners c;
      rc = corner_build(h_tm1[s], h_t0[s], h_tp1[s], h_psi[s], h_chi[s], h_N[s], b->opts.eps, c);
      if (rc) {
        dichotomy_batch_destroy(b);
        return rc;
      }
      const int64_t og = (int64_t)b->ctab.size();
      b->ctab.insert(b->ctab.end(), c.gh.begin(), c.gh.end());
      b->crec.push_back(CornerRec{h_N[s], h_offset[s], c.Lg, c.Lh, og, og + c.Lg, h_psi[s], h_chi[s], c.W[0], c.W[1],
                                  c.W[2], c.W[3]});
      // A^T: corner vectors h and g read backwards (persymmetry), the transposed 2x2 inverse
      adj = CornerRec{h_N[s], h_offset[s], c.Lh, c.Lg, og + c.Lg, og, h_psi[s], h_chi[s], c.Wt[0], c.Wt[1], c.Wt[2],
                      c.Wt[3]};
    }
    b->crec_adj.push_back(adj);
  }
  {
    // appended after the workspace (and staged whole: the scratch in between is uploaded as zeros)
    size_t o_ = b->ws_bytes;
    b->off_crec = o_;
    o_ += align_up(sizeof(CornerRec) * std::max<size_t>(1, b->crec.size()));
    b->off_ctab = o_;
    o_ += align_up(sizeof(double) * std::max<size_t>(1, b->ctab.size()));
    b->off_crec_adj = o_;
    o_ += align_up(sizeof(CornerRec) * std::max<size_t>(1, b->crec_adj.size()));
    const size_t staged = o_;
    b->off_gt3 = o_;   // the Toeplitz gradients of the adjoint, 3 per system (scratch)
    o_ += align_up(sizeof(double) * 3 * (size_t)std::max<int64_t>(1, nsys));
    b->ws_bytes = o_;
    b->staging.resize(staged, 0);
    if (!b->crec.empty()) std::memcpy(b->staging.data() + b->off_crec, b->crec.data(), sizeof(CornerRec) * b->crec.size());
    if (!b->ctab.empty()) std::memcpy(b->staging.data() + b->off_ctab, b->ctab.data(), sizeof(double) * b->ctab.size());
    if (!b->crec_adj.empty())
      std::memcpy(b->staging.data() + b->off_crec_adj, b->crec_adj.data(), sizeof(CornerRec) * b->crec_adj.size());
  }
  *out = b;
  return DICH_OK;
}

int dichotomy_batch_workspace_bytes(dich_batch_t b, size_t* bytes) {
  if (!b || !bytes) return DICH_ERR_ARG;
  *bytes = b->ws_bytes;
  return DICH_OK;
}

int dichotomy_batch_bind(dich_batch_t b, void* d_ws, size_t bytes, void* stream) {
  if (!b || !d_ws) return DICH_ERR_ARG;
  if (((uintptr_t)d_ws & (kAlign - 1)) != 0 || bytes < b->ws_bytes) return DICH_ERR_WORKSPACE;
  if (!is_device_ptr(d_ws)) return DICH_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(d_ws, b->staging.data(), b->staging.size(), cudaMemcpyHostToDevice,
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  b->d_ws = (char*)d_ws;
  b->d_ws_bytes = bytes;
  if (!b->items[0].empty() && !b->items[1].empty() && !b->aux) {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess) {
      // both forms overlap from now on
    } else {
      cudaGetLastError();   // no second stream: the two forms run one after the other
    }
  }
  return DICH_OK;
}

static int batch_launch(dich_batch_t b, const double* F, double* x, const double* xf, double* gt, bool adjoint,
                        cudaStream_t st) {
  const SysPlan* d_plans = (const SysPlan*)(b->d_ws + b->off_plans);
  const double* d_tabs = (const double*)(b->d_ws + b->off_tabs);
  unsigned* d_status = (unsigned*)(b->d_ws + b->off_status);
  const int sys_offset = adjoint ? (int)b->nsys : 0;
  // both forms present: the FP64-form windows go to the second stream after a fork event
  const bool fork = b->aux && b->ev_fork && b->ev_join && !b->items[0].empty() && !b->items[1].empty();
  if (fork) {
    cudaError_t e = cudaEventRecord(b->ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->aux, b->ev_fork, 0);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // FP64-form windows first: with a fork their long CTAs then start beside the MIXED waves
  // instead of after them
  for (int f : {FORM_F64, FORM_MIXED}) {
    const int64_t nitems = (int64_t)b->items[f].size();
    if (nitems == 0) continue;
    const cudaStream_t sf = (fork && f == FORM_F64) ? b->aux : st;
    WinArgs a{};
    a.plans = d_plans;
    a.tabs = d_tabs;
    a.items = (const Item*)(b->d_ws + b->off_items[f]);
    a.F = F;
    a.x = x;
    a.status = d_status;
    a.xf = adjoint ? xf : nullptr;
    a.part = adjoint ? (double*)(b->d_ws + b->off_part[f]) : nullptr;
    a.mode = MODE_FULL;
    a.check_finite = (b->opts.flags & DICH_FLAG_CHECK_FINITE) ? 1 : 0;
    a.n_smem = b->n_smem[f];
    a.sys_offset = sys_offset;
    a.bulk = b->reg_path ? 1 : 0;   // batch vectors are device memory
    const size_t smem = smem_bytes(b->NT[f], a.n_smem, f);
    cudaError_t e = (f == FORM_F64) ? launch_window_f64(b->NT[f], (int)nitems, smem, sf, a)
                                    : launch_window_mixed(b->NT[f], (int)nitems, smem, sf, a);
    if (e != cudaSuccess) return cuda_fail(e);
    if (adjoint) {
      e = launch_adj_finalize(a.part, (const int32_t*)(b->d_ws + b->off_ids[f]),
                              (const int64_t*)(b->d_ws + b->off_first[f]),
                              (const int64_t*)(b->d_ws + b->off_count[f]), 0, (int64_t)b->sys_ids[f].size(), gt, sf);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  if (fork) {
    cudaError_t e = cudaEventRecord(b->ev_join, b->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_join, 0);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (!b->trivial.empty()) {
    cudaError_t e = launch_trivial(d_plans, (const int32_t*)(b->d_ws + b->off_trivial), (int64_t)b->trivial.size(),
                                   adjoint ? nullptr : F, x, xf, adjoint ? F : nullptr, gt, sys_offset, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // systems on the general path, per form: one beta pass over all their windows, one block scan
  // over all their blocks, one apply pass (with the gradient sums for the adjoint)
  for (int f = 0; f < 2; ++f) {
    const int64_t ng = (int64_t)b->gitems[f].size();
    if (ng == 0) continue;
    WinArgs a{};
    a.plans = d_plans;
    a.tabs = d_tabs;
    a.items = (const Item*)(b->d_ws + b->off_gitems[f]);
    a.F = F;
    a.x = x;
    a.status = d_status;
    a.check_finite = (b->opts.flags & DICH_FLAG_CHECK_FINITE) ? 1 : 0;
    a.n_smem = b->n_smem_g[f];
    a.sys_offset = sys_offset;
    double* beta = (double*)(b->d_ws + b->off_gbeta);
    double* iface = (double*)(b->d_ws + b->off_giface);
    const size_t smem = smem_bytes(b->NT[f], a.n_smem, f);
    auto launch = [&](const WinArgs& w) {
      return f == FORM_F64 ? launch_window_f64(b->NT[f], (int)ng, smem, st, w)
                           : launch_window_mixed(b->NT[f], (int)ng, smem, st, w);
    };
    WinArgs wb = a;
    wb.mode = MODE_BETA;
    wb.beta = beta;
    cudaError_t e = launch(wb);
    if (e == cudaSuccess) {
      ScanMap map{(const int32_t*)(b->d_ws + b->off_gcmap[f]), (const int32_t*)(b->d_ws + b->off_gsys[f]),
                  (const int64_t*)(b->d_ws + b->off_gc0[f])};
      e = launch_block_scan_batched(d_plans + sys_offset, d_tabs, map, (int64_t)b->gcmap[f].size(),
                                    (int64_t)b->gsys[f].size(), beta, iface, (double*)(b->d_ws + b->off_gscan[f]),
                                    st);
    }
    if (e == cudaSuccess) {
      a.mode = MODE_APPLY;
      a.iface = iface;
      a.xf = adjoint ? xf : nullptr;
      a.part = adjoint ? (double*)(b->d_ws + b->off_gpart[f]) : nullptr;
      e = launch(a);
    }
    if (e == cudaSuccess && adjoint)
      e = launch_adj_finalize(a.part, (const int32_t*)(b->d_ws + b->off_gsys[f]),
                              (const int64_t*)(b->d_ws + b->off_gfirst[f]),
                              (const int64_t*)(b->d_ws + b->off_gcount[f]), 0, (int64_t)b->gsys[f].size(), gt, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // quasi-Toeplitz systems: the corner correction on the Toeplitz solutions (all streams joined)
  if (!adjoint && !b->crec.empty()) {
    cudaError_t e = launch_corner_batch((const CornerRec*)(b->d_ws + b->off_crec), (int64_t)b->crec.size(),
                                        (const double*)(b->d_ws + b->off_ctab), x, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return DICH_OK;
}

int dichotomy_solve_batched(dich_batch_t b, const double* d_F, double* d_x, void* stream) {
  if (!b) return DICH_ERR_ARG;
  if (!b->d_ws) return DICH_ERR_UNBOUND;
  if (b->nsys == 0) return DICH_OK;
  if (!d_F || !d_x || !aligned8(d_F) || !aligned8(d_x)) return DICH_ERR_ARG;
  if (!is_device_ptr(d_F) || !is_device_ptr(d_x)) return DICH_ERR_ARG;
  if (d_F == d_x) return DICH_ERR_ALIAS;
  return batch_launch(b, d_F, d_x, nullptr, nullptr, false, (cudaStream_t)stream);
}

int dichotomy_adjoint_batched(dich_batch_t b, const double* d_w, const double* d_x, double* d_gF, double* d_gt,
                              void* stream) {
  if (!b) return DICH_ERR_ARG;
  if (!b->d_ws) return DICH_ERR_UNBOUND;
  if (b->nsys == 0) return DICH_OK;
  if (!d_w || !d_x || !d_gF || !d_gt) return DICH_ERR_ARG;
  if (!aligned8(d_w) || !aligned8(d_x) || !aligned8(d_gF) || !aligned8(d_gt)) return DICH_ERR_ARG;
  if (!is_device_ptr(d_w) || !is_device_ptr(d_x) || !is_device_ptr(d_gF) || !is_device_ptr(d_gt)) return DICH_ERR_ARG;
  if (d_gF == d_w || d_gF == d_x) return DICH_ERR_ALIAS;
  cudaStream_t st = (cudaStream_t)stream;
  if (b->crec_adj.empty()) {
    cudaError_t e = cudaMemsetAsync(d_gt, 0, sizeof(double) * 3 * (size_t)b->nsys, st);
    if (e != cudaSuccess) return cuda_fail(e);
    return batch_launch(b, d_w, d_gF, d_x, d_gt, true, st);
  }
  // a batch prepared with corners: the Toeplitz adjoint into scratch, then per system the corner
  // terms, dL/dpsi, dL/dchi (5 gradients per system in d_gt) and the correction of lambda
  double* gt3 = (double*)(b->d_ws + b->off_gt3);
  cudaError_t e = cudaMemsetAsync(gt3, 0, sizeof(double) * 3 * (size_t)b->nsys, st);
  if (e != cudaSuccess) return cuda_fail(e);
  const int rc = batch_launch(b, d_w, d_gF, d_x, gt3, true, st);
  if (rc != DICH_OK) return rc;
  e = launch_corner_adjoint_batch((const CornerRec*)(b->d_ws + b->off_crec_adj), b->nsys,
                                  (const double*)(b->d_ws + b->off_ctab), d_x, d_gF, gt3, d_gt, st);
  return e == cudaSuccess ? DICH_OK : cuda_fail(e);
}

int dichotomy_batch_status(dich_batch_t b, void* stream, int* device_status) {
  if (!b || !device_status) return DICH_ERR_ARG;
  if (!b->d_ws) return DICH_ERR_UNBOUND;
  unsigned s = 0;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(&s, b->d_ws + b->off_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(b->d_ws + b->off_status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e);
  *device_status = map_status(s);
  return DICH_OK;
}

int dichotomy_batch_info(dich_batch_t b, int64_t* nsys, int64_t* windows, int32_t* h_form) {
  if (!b) return DICH_ERR_ARG;
  if (nsys) *nsys = b->nsys;
  if (windows) *windows = (int64_t)(b->items[0].size() + b->items[1].size());
  if (h_form)
    for (int64_t s = 0; s < b->nsys; ++s) h_form[s] = b->form[s];
  return DICH_OK;
}

void dichotomy_batch_destroy(dich_batch_t b) { delete b; }

}  // extern "C"
