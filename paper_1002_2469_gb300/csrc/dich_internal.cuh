// dich_internal.cuh -- data layout and Toeplitz math shared by the host planner and the
// sm_103a kernels of the Dichotomy solver (arXiv 1002.2469).
//
// Notation (0-based rows; the paper is 1-based):
//   row i:  t_-1 x[i-1] + t_0 x[i] + t_1 x[i+1] = F[i],  x[-1] = x[N] = 0.
//   Roots of t_1 r^2 + t_0 r + t_-1 = 0 (the q_1, q_2 of Theorem 1, eq. 20):
//     rs = the root of modulus <= 1, ib = 1 / (the other root).  With
//     q = -(t_0 + sgn(t_0) sqrt(t_0^2 - 4 t_1 t_-1)) / 2:  rs = t_-1 / q,  ib = t_1 / q,
//     and T = -q (1 - rs E^-1)(1 - ib E) on bi-infinite sequences (E = shift).
//   z = rs * ib (= q_small / q_big),  Q(k) = (1 - z^k)/(1 - z)  (Q(k) = k when z = 1).
//   Homogeneous solutions: phi(i) ~ ib^{-(i+1)} Q(i+1) vanishes at i = -1 (left end),
//   psi(i) ~ rs^i Q(N - i) vanishes at i = N (right end).  Every exterior ratio the paper
//   needs (Z of eq. 10-12, the "transfer" ratios of the remark after eq. 18) is a ratio
//   of these, i.e. a power of rs or ib times a ratio of Q's: the exact, overflow-free
//   counterpart of eq. 24-25 / eq. 29-31 (all exponents <= 0).
//
// Block m covers rows [s, e], size n_m = e - s + 1 (n for all blocks but the last).
// Per block the kernels compute the local particular solution xp (two first-order
// recurrences with constant coefficients rs and ib and the scale g = -1/q), its
// virtual end values xp(-1), xp(n) = 0, the zero-Dirichlet block solution ends
//   alpha = y_0, omega = y_{n-1},  y = T_n^-1 F_m = xp - xp(-1) v
// (v = -t_-1 T_n^-1 e_1 and w = -t_1 T_n^-1 e_n are the block spikes), and
//   (beta^L, beta^R) = M (alpha, omega),  M = (I - [[kL v_0, kR w_0],[kL v_{n-1}, kR w_{n-1}]])^-1
// which is the paper's beta of eq. 16 (global Green rows dotted with F_m), kL = phi(s-1)/phi(s),
// kR = psi(e+1)/psi(e).  eq. 15 then becomes two affine scans over blocks:
//   A_{m+1} = a_m A_m + b_m beta^R_m       a = psi(s_{m+1})/psi(s_m), b = psi(s_{m+1})/psi(e_m)
//   B_{m-1} = c_m B_m + d_m beta^L_m       c = phi(e_{m-1})/phi(e_m), d = phi(e_{m-1})/phi(s_m)
//   x_s = A_m + beta^L_m + tL_m B_m,  x_e = tR_m A_m + beta^R_m + B_m
//   tL = phi(s)/phi(e), tR = psi(e)/psi(s)            (eq. 18 and its remark)
// and the block interior (eq. 7) is  x = xp + (x_{s-1} - xp(-1)) v + x_{e+1} w.
#pragma once
#include <cstdint>
#include <cmath>

#if defined(__CUDACC__)
#define DICH_HD __host__ __device__ inline
#define DICH_DEV __device__ __forceinline__
#else
#define DICH_HD inline
#define DICH_DEV inline
#endif

namespace dich {

// ---------------------------------------------------------------- layout constants
constexpr int kBC = 10;  // doubles per block-coefficient record
enum BCIdx { BC_A = 0, BC_B, BC_C, BC_D, BC_TL, BC_TR, BC_M00, BC_M01, BC_M10, BC_M11 };

enum Form : int32_t { FORM_F64 = 0, FORM_MIXED = 1 };
enum Path : int32_t { PATH_SINGLE = 0, PATH_HALO = 1, PATH_GENERAL = 2 };

// kernel modes of the window kernel
enum Mode : int32_t {
  MODE_FULL = 0,    // sweeps, beta, in-window scans, interface values, correction, store x
  MODE_BETA = 1,    // sweeps and beta only: store (beta^L, beta^R) per block (general path)
  MODE_APPLY = 2,   // sweeps, neighbour interface values from global, correction, store x
};

// status bits latched by kernels
enum StatusBits : uint32_t {
  ST_NONFINITE = 1u,
  ST_SCHEDULE = 2u,
  ST_TIMEOUT = 4u,    // a bounded wait for the CTA's own bulk copies ran out (the CTA stored nothing)
};

// Device-side plan record of one system (256 bytes, 8-byte fields first).
struct SysPlan {
  int64_t N;        // rows
  int64_t off;      // offset of row 0 in F / x
  int64_t P;        // blocks
  int64_t tab;      // offset (in doubles) of this system's tables in the table buffer
  int32_t n, nlast; // block size, last block size
  int32_t Lv, Lw;   // truncated spike lengths (full-size blocks)
  int32_t kl, kr;   // blocks with end-dependent coefficients (left table / right table)
  int32_t hl, hr;   // halo blocks per window (left / right)
  int32_t form;     // Form
  int32_t own;      // own blocks per window (single system)
  double tm1, t0, tp1;
  double rs, ib, g; // forward / backward recurrence coefficients, output scale -1/q
  float rs_h, rs_l, ib_h, ib_l, g_h, g_l;   // float-float splits of rs, ib, g
  double v0, vend, w0, wend;                // corner spikes, full-size blocks
  double v0l, vendl, w0l, wendl;            // corner spikes, last block
  int64_t gboff;    // general path in a batch: first block of this system in the beta / first-last buffers
  double pad_;
  // table sub-offsets (in doubles, relative to `tab`)
  int32_t o_v, o_w, o_vl, o_wl;             // v[Lv], w_rev[Lw], v_last[nlast], w_last_rev[nlast]
  int32_t o_vf, o_wf, o_vlf, o_wlf;         // float-float copies (float2 per entry)
  int32_t o_bcm, o_bcl, o_bcr, pad2_;       // middle record, left table [kl], right table [kr]
  int32_t o_bcmf, o_bclf, o_bcrf, pad3_;    // the same records as float-float (float2 per entry)
  // float-float copies of g * ib and of the corner spikes (MIXED form)
  float gib_h, gib_l;
  float v0_h, v0_l, vend_h, vend_l, v0l_h, v0l_l, vendl_h, vendl_l;
  // MIXED form: warp-scan levels of the tree (couplings beyond 2^(lev+1) blocks are below the
  // truncation threshold), beta records from the block-end values (4 float-float entries per
  // record: middle, left table [kl], right table [kr]) and the middle record's map powers
  // ((a^2)^t, t = 0..32, then (c^2)^t); tcheap: both pair-map factors a^2, c^2 are at most 2^-24,
  // so that every level of the middle-window scan multiplies by at most 2^-24 (its products need
  // only their leading parts)
  int32_t lev, o_kmf, o_klf, o_krf, o_midf, tcheap;
};
static_assert(sizeof(SysPlan) % 8 == 0, "SysPlan must be 8-byte granular");

// One window of a batched launch: own blocks [m0, m0 + n_own) of system `sys`.
struct Item {
  int64_t m0;
  int32_t sys;
  int32_t n_own;
};

// ---------------------------------------------------------------- Toeplitz math (host + device)
struct Roots {
  double rs, ib, z, omz, g, q;
  bool ok;
};

// Roots of t_1 r^2 + t_0 r + t_-1 = 0 in the cancellation-free form.  The discriminant
// is evaluated with a compensated product (Kahan's trick) so that nearly double roots
// (weak dominance) keep full relative accuracy in 1 - z.
DICH_HD Roots toeplitz_roots(double tm1, double t0, double tp1) {
  Roots r{};
  double p = tp1 * tm1;
  double pe = fma(tp1, tm1, -p);
  double disc = fma(t0, t0, -4.0 * p) - 4.0 * pe;
  if (disc < 0.0) disc = 0.0;                // only reachable without dominance (rejected)
  double sd = sqrt(disc);
  double q = -0.5 * (t0 + copysign(sd, t0));
  r.q = q;
  r.ok = (q != 0.0);
  if (!r.ok) return r;
  r.rs = tm1 / q;
  r.ib = tp1 / q;
  r.z = r.rs * r.ib;
  // 1 - z = sqrt(disc) (sqrt(disc) + |t_0|) / (2 q^2), free of cancellation
  r.omz = sd * (sd + fabs(t0)) / (2.0 * q * q);
  r.g = -1.0 / q;
  return r;
}

// x^k for k >= 0 by binary powering
DICH_HD double ipow(double x, int64_t k) {
  double r = 1.0;
  while (k > 0) {
    if (k & 1) r *= x;
    x *= x;
    k >>= 1;
  }
  return r;
}

// Q(k) = (1 - z^k) / (1 - z) = sum_{j<k} z^j, accurate for z -> 1 (weak dominance).
DICH_HD double qnum(int64_t k, const Roots& r) {
  if (k <= 0) return 0.0;
  if (r.omz == 0.0) return (double)k;
  if (r.z == 0.0) return 1.0;
  if (r.z > 0.0) {
    double lz = log1p(-r.omz);
    return -expm1((double)k * lz) / r.omz;
  }
  double lz = log(-r.z);
  if ((k & 1) == 0) return -expm1((double)k * lz) / r.omz;
  return (1.0 + exp((double)k * lz)) / r.omz;
}

// Block spike entries for a block of size nb:
//   v_i = rs^{i+1} Q(nb-i)/Q(nb+1),   w_{nb-1-i} = ib^{i+1} Q(nb-i)/Q(nb+1).
DICH_HD double spike_ratio(int64_t nb, int64_t i, const Roots& r) {
  return qnum(nb - i, r) / qnum(nb + 1, r);
}

// Number of leading terms of |r|^{k} that exceed eps (at least 1, at most cap).
DICH_HD int64_t decay_len(double absr, double eps, int64_t cap) {
  if (absr == 0.0) return 1;
  if (absr >= 1.0) return cap;
  double L = ceil(log(eps) / log(absr)) + 1.0;
  if (L > (double)cap) return cap;
  return L < 1.0 ? 1 : (int64_t)L;
}

// beta of a block (eq. 16) in units of X from the ends X_0, X_{n-1} of its local backward
// recurrence (the particular solution is xp = g X):  alpha = g (X_0 - ib v_0 X_0),
// omega = g (X_{n-1} - ib v_{n-1} X_0), (beta^L, beta^R) = M (alpha, omega); so beta / g is
//   beta^L / g = K1 X_0 + K2 X_{n-1},  beta^R / g = K3 X_0 + K4 X_{n-1}
// with K1 = M00 (1 - ib v_0) - M01 ib v_{n-1}, K2 = M01, K3 = M10 (1 - ib v_0) - M11 ib v_{n-1}, K4 = M11.
// bc: the block's record (BC_*), v0 / vend: its corner spikes; out[0..3] = K1..K4.
DICH_HD void beta_coeffs(const double* bc, double ib, double v0, double vend, double* out) {
  const double ca = 1.0 - ib * v0, cw = -ib * vend;
  out[0] = bc[BC_M00] * ca + bc[BC_M01] * cw;
  out[1] = bc[BC_M01];
  out[2] = bc[BC_M10] * ca + bc[BC_M11] * cw;
  out[3] = bc[BC_M11];
}

// Block coefficients of block [s, e] of a system of N rows (eq. 15-18 restated):
// out[BC_*].  v0, vend, w0, wend are the corner spikes for this block's size.
DICH_HD void block_coeffs(int64_t N, int64_t s, int64_t e, const Roots& r, double v0, double vend,
                          double w0, double wend, bool far_left, bool far_right, double* out) {
  const int64_t nb = e - s + 1;
  double kL, kR, a, b, c, d, tL, tR;
  double rsn = ipow(r.rs, nb), rsn1 = ipow(r.rs, nb - 1);
  double ibn = ipow(r.ib, nb), ibn1 = ipow(r.ib, nb - 1);
  if (far_left) {
    kL = r.ib;
    c = ibn;
    tL = ibn1;
  } else {
    double qs = qnum(s, r), qs1 = qnum(s + 1, r), qe1 = qnum(e + 1, r);
    kL = r.ib * qs / qs1;
    c = ibn * qs / qe1;
    tL = ibn1 * qs1 / qe1;
  }
  d = kL;
  if (far_right) {
    kR = r.rs;
    a = rsn;
    tR = rsn1;
  } else {
    double qNe = qnum(N - e, r), qNe1 = qnum(N - e - 1, r), qNs = qnum(N - s, r);
    kR = r.rs * qNe1 / qNe;
    a = rsn * qNe1 / qNs;
    tR = rsn1 * qNe / qNs;
  }
  b = kR;
  // M = (I - Pm)^-1, Pm = [[kL v0, kR w0], [kL vend, kR wend]]
  double p00 = 1.0 - kL * v0, p01 = -kR * w0, p10 = -kL * vend, p11 = 1.0 - kR * wend;
  double det = p00 * p11 - p01 * p10;
  out[BC_A] = a;
  out[BC_B] = b;
  out[BC_C] = c;
  out[BC_D] = d;
  out[BC_TL] = tL;
  out[BC_TR] = tR;
  out[BC_M00] = p11 / det;
  out[BC_M01] = -p01 / det;
  out[BC_M10] = -p10 / det;
  out[BC_M11] = p00 / det;
}

}  // namespace dich
