// window_gen.cuh -- the window kernel for a general (non-Toeplitz) tridiagonal matrix, FP64.
//
// Row i reads a_i x_{i-1} + b_i x_i + c_i x_{i+1} = F_i.  The Dichotomy steps are those of the
// Toeplitz kernel (window.cuh) with the preliminary quantities taken from the plan instead of
// closed forms (Sec. 2.3, the general preliminary step):
//   - local solve of each block m (rows s..e) with zero outside values, y = T_m^-1 F_m, by the
//     block's own Thomas factors (forward z_i = (F_i - a_i z_{i-1}) rd_i, backward
//     y_i = z_i - cp_i y_{i+1}; rd_i, cp_i precomputed per row);
//   - alpha = y_s, omega = y_e, beta = M (alpha, omega) with the block's record (eq. 16);
//   - the dichotomy tree over the window's blocks (tree_f64, eq. 15, 18);
//   - interiors (eq. 7): x = y + x_{s-1} v + x_{e+1} w with the block spikes
//     v = T_m^-1 (-a_s e_0), w = T_m^-1 (-c_e e_{n-1}) stored per row.
// Per-row tables are interleaved by groups of 32 blocks (gen_index), so that the threads of a
// warp -- consecutive blocks, one per thread -- read row i of their blocks contiguously.
// General path: the beta pass (MODE_BETA) leaves the local solutions y in x, and the apply
// pass (MODE_APPLY) reads them back instead of F, so the local solve runs once.
#pragma once
#include <type_traits>
#include "ff.cuh"
#include "window.cuh"

namespace dich {

// per-row table fields of a general plan
enum GenField : int { GF_A = 0, GF_RD = 1, GF_CP = 2, GF_V = 3, GF_W = 4, kGenFields = 5 };

// element (block m, row i) of one field; n = rows per block
__host__ __device__ inline int64_t gen_index(int64_t m, int i, int n) {
  return ((m >> 5) * (int64_t)n + i) * 32 + (m & 31);
}

struct GenArgs {
  WinArgs w;            // one plan record (plans[0]), block records in tabs, F, x, status, mode
  const double* rows;   // per-row tables: field f at rows + f * stride
  int64_t stride;       // doubles per field
};

// shared memory of the general window kernel: NT threads, n_smem rows
__host__ __device__ inline size_t window_gen_smem_bytes(int NT, int n_smem) {
  const size_t nw = (size_t)(NT / 32);
  return sizeof(double) * ((size_t)n_smem * (size_t)(NT + 1) + 4 * (size_t)NT + 4 * nw + 8);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_window_gen(const GenArgs G) {
  constexpr int LD = NT + 1;
  const WinArgs& A = G.w;
  extern __shared__ __align__(16) double sm[];
  // launched with programmatic stream serialization: nothing is read or written before the
  // previous kernel of the stream has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int tid = threadIdx.x;
  const int ns = A.n_smem;
  double* S = sm;
  double* sxs = S + (size_t)ns * LD;
  double* sxe = sxs + NT;
  double* scl = sxe + NT;
  double* scr = scl + NT;
  double* swa = scr + NT;                          // 4 * NW scan scratch

  // ---------------------------------------------------------------- the window
  const SysPlan* pp = A.plans;
  const int64_t P = pp->P;
  const int nown0 = pp->own;
  const int64_t m0 = (int64_t)blockIdx.x * nown0;
  const int nown = (int)min((int64_t)nown0, P - m0);
  int hl = 0, hr = 0;
  if (A.mode == MODE_FULL) {
    hl = (int)min((int64_t)pp->hl, m0);
    hr = (int)min((int64_t)pp->hr, P - m0 - nown);
  }
  const int64_t wlo = m0 - hl;
  const int nwin = hl + nown + hr;
  const int n = pp->n, nlast = pp->nlast;
  const bool has_last = (wlo + nwin == P);
  const int64_t row_lo = wlo * (int64_t)n;
  const int len = nwin * n - (has_last ? (n - nlast) : 0);
  const double* Fw = A.F + (int64_t)blockIdx.y * A.ldf;
  double* xw = A.x + (int64_t)blockIdx.y * A.ldx;

  // ---------------------------------------------------------------- F -> smem (transposed, async)
  // (MODE_APPLY: the block solutions y the beta pass left in x, instead of F)
  {
    const double* src = ((A.mode == MODE_APPLY) ? xw : Fw) + row_lo;
    int b = tid / n, i = tid - (tid / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = tid; j < len; j += NT) {
      cp_async8(&S[i * LD + b], src + j);
      i += di;
      b += db;
      if (i >= n) {
        i -= n;
        ++b;
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // ---------------------------------------------------------------- local solves (a1)
  const bool act = tid < nwin;
  const int64_t mb = wlo + tid;
  const int nbk = (act && mb == P - 1) ? nlast : n;
  const double* ra = G.rows + GF_A * G.stride;
  const double* rd = G.rows + GF_RD * G.stride;
  const double* rc = G.rows + GF_CP * G.stride;
  const double* rv = G.rows + GF_V * G.stride;
  const double* rw = G.rows + GF_W * G.stride;
  double alpha = 0.0, omega = 0.0;
  double* col = S + tid;
  const int64_t k0 = gen_index(act ? mb : 0, 0, n);   // row i of the block at k0 + 32 i
  if (act && A.mode != MODE_APPLY) {
    // the per-row factors of four rows are loaded ahead of their dependent recurrence steps
    double z = 0.0;
    int i = 0;
    for (; i + 4 <= nbk; i += 4) {
      const int64_t k = k0 + 32 * i;
      const double a0 = ra[k], a1 = ra[k + 32], a2 = ra[k + 64], a3 = ra[k + 96];
      const double d0 = rd[k], d1 = rd[k + 32], d2 = rd[k + 64], d3 = rd[k + 96];
      z = fma(-a0, z, col[i * LD]) * d0;
      col[i * LD] = z;
      z = fma(-a1, z, col[(i + 1) * LD]) * d1;
      col[(i + 1) * LD] = z;
      z = fma(-a2, z, col[(i + 2) * LD]) * d2;
      col[(i + 2) * LD] = z;
      z = fma(-a3, z, col[(i + 3) * LD]) * d3;
      col[(i + 3) * LD] = z;
    }
    for (; i < nbk; ++i) {
      const int64_t k = k0 + 32 * i;
      z = fma(-ra[k], z, col[i * LD]) * rd[k];
      col[i * LD] = z;
    }
    double y = 0.0;
    i = nbk - 1;
    for (; i - 3 >= 0; i -= 4) {
      const int64_t k = k0 + 32 * i;
      const double c0 = rc[k], c1 = rc[k - 32], c2 = rc[k - 64], c3 = rc[k - 96];
      y = fma(-c0, y, col[i * LD]);
      col[i * LD] = y;
      y = fma(-c1, y, col[(i - 1) * LD]);
      col[(i - 1) * LD] = y;
      y = fma(-c2, y, col[(i - 2) * LD]);
      col[(i - 2) * LD] = y;
      y = fma(-c3, y, col[(i - 3) * LD]);
      col[(i - 3) * LD] = y;
    }
    for (; i >= 0; --i) {
      y = fma(-rc[k0 + 32 * i], y, col[i * LD]);
      col[i * LD] = y;
    }
    alpha = col[0];
    omega = col[(nbk - 1) * LD];
  }

  // ---------------------------------------------------------------- beta (eq. 16)
  const double* bc = A.tabs + pp->o_bcl + (act ? mb : 0) * kBC;
  const double bL = act ? fma(bc[BC_M00], alpha, bc[BC_M01] * omega) : 0.0;
  const double bR = act ? fma(bc[BC_M10], alpha, bc[BC_M11] * omega) : 0.0;
  if (A.mode == MODE_BETA) {   // beta and the block solutions y leave the window
    if (act) {
      A.beta[2 * (pp->gboff + mb)] = bL;
      A.beta[2 * (pp->gboff + mb) + 1] = bR;
    }
    __syncthreads();
    int b = tid / n, i = tid - (tid / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = tid; j < len; j += NT) {
      xw[row_lo + j] = S[i * LD + b];
      i += di;
      b += db;
      if (i >= n) {
        i -= n;
        ++b;
      }
    }
    return;
  }

  double XL = 0.0, XR = 0.0;
  if (A.mode == MODE_FULL) {
    tree_f64<NT>(bc, act, bL, bR, mb, P, nwin, tid, swa, sxs, sxe, XL, XR);
  } else if (act) {  // MODE_APPLY: neighbours' first/last values from the global scan
    XL = (mb == 0) ? 0.0 : A.iface[2 * (pp->gboff + mb - 1) + 1];
    XR = (mb == P - 1) ? 0.0 : A.iface[2 * (pp->gboff + mb + 1)];
  }

  // ---------------------------------------------------------------- interiors (eq. 7), per column
  if (act) {
#pragma unroll 4
    for (int i = 0; i < nbk; ++i) {
      const int64_t k = k0 + 32 * i;
      col[i * LD] = fma(XR, rw[k], fma(XL, rv[k], col[i * LD]));
    }
  }
  __syncthreads();

  asm volatile("griddepcontrol.launch_dependents;");   // the next kernel may begin its launch
  // ---------------------------------------------------------------- coalesced store of the own rows
  unsigned bad = 0u;
  {
    const int jlo = hl * n;
    const int jhi = min(len, (hl + nown) * n);
    double* dst = xw + row_lo;
    int b = (jlo + tid) / n, i = (jlo + tid) - ((jlo + tid) / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = jlo + tid; j < jhi; j += NT) {
      const double dv = S[i * LD + b];
      __stcs(dst + j, dv);
      if (A.check_finite && !isfinite(dv)) bad = 1u;
      i += di;
      b += db;
      if (i >= n) {
        i -= n;
        ++b;
      }
    }
  }
  if (bad) atomicOr(A.status, (unsigned)ST_NONFINITE);
}

// ---------------------------------------------------------------- MIXED form
// The same steps with the per-row work in float-float arithmetic (ff.cuh) on values scaled per
// window by one exact power of two (largest |F| of the window near 2^16): the per-row tables
// hold float-float pairs (hi, lo) in the 8-byte slots of the FP64 tables, the local solve runs
// z_i = (F_i - a_i z_{i-1}) rd_i and y_i = z_i - cp_i y_{i+1} in float-float; in a window that
// runs the tree (MODE_FULL) beta and the tree are float-float too (tree_gen_ff: the block records
// split once per block, so no FP64 work per block), on the general path beta leaves as FP64 for
// the FP64 block scan; the correction x = y + x_{s-1} v + x_{e+1} w runs in float-float before
// one join to FP64 per row.  Tiles of narrow exponent range take the fast split and join.
// block record entry j as a float-float pair (the records are ratios of order one on the paths
// that run the tree in the window; the general split flushes what lies below the float range)
__device__ __forceinline__ ffv gen_rec_ff(const double* bc, int j) {
  float h, l;
  split_sc(bc[j], 0, h, l);
  return ffv{h, l};
}

// the dichotomy tree of one window (eq. 15, 17-19) in float-float, one block per thread: the
// steps of tree_f64 with the block's beta and the returned first/last values of the neighbours
// in window units (XL = x_{s-1}, XR = x_{e+1}; left untouched at the ends of the system)
template <int NT>
__device__ __forceinline__ void tree_gen_ff(const double* bc, bool act, ffv bL, ffv bR, int64_t mb, int64_t P,
                                            int nwin, int tid, double* swa, double* sxs, double* sxe, ffv& XL,
                                            ffv& XR) {
  constexpr int NW = NT / 32;
  const int lane = tid & 31, wid = tid >> 5;
  ffv pa = act ? gen_rec_ff(bc, BC_A) : ff_one();
  ffv pb = act ? ff_mul(gen_rec_ff(bc, BC_B), bR) : ff_zero();
  ffv qa = act ? gen_rec_ff(bc, BC_C) : ff_one();
  ffv qb = act ? ff_mul(gen_rec_ff(bc, BC_D), bL) : ff_zero();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const ffv ya = ff_shfl_up(pa, d), yb = ff_shfl_up(pb, d);
    const ffv za = ff_shfl_down(qa, d), zb = ff_shfl_down(qb, d);
    if (lane >= d) {
      pb = ff_fma(pa, yb, pb);
      pa = ff_mul(pa, ya);
    }
    if (lane + d < 32) {
      qb = ff_fma(qa, zb, qb);
      qa = ff_mul(qa, za);
    }
  }
  ffv* sw = reinterpret_cast<ffv*>(swa);   // 4 NW pairs in the 4 NW doubles of the scratch
  if (lane == 31) {
    sw[wid] = pa;
    sw[NW + wid] = pb;
  }
  if (lane == 0) {
    sw[2 * NW + wid] = qa;
    sw[3 * NW + wid] = qb;
  }
  // previous lane's inclusive prefix, next lane's inclusive suffix
  ffv ea = ff_shfl_up(pa, 1), eb = ff_shfl_up(pb, 1);
  ffv fa = ff_shfl_down(qa, 1), fb = ff_shfl_down(qb, 1);
  if (lane == 0) {
    ea = ff_one();
    eb = ff_zero();
  }
  if (lane == 31) {
    fa = ff_one();
    fb = ff_zero();
  }
  __syncthreads();
  ffv Aw = ff_zero(), Bw = ff_zero();   // zero coupling enters at both window ends
  for (int w = 0; w < wid; ++w) Aw = ff_fma(sw[w], Aw, sw[NW + w]);
  for (int w = NW - 1; w > wid; --w) Bw = ff_fma(sw[2 * NW + w], Bw, sw[3 * NW + w]);
  const ffv Am = ff_fma(ea, Aw, eb), Bm = ff_fma(fa, Bw, fb);
  ffv* fs = reinterpret_cast<ffv*>(sxs);
  ffv* fe = reinterpret_cast<ffv*>(sxe);
  fs[tid] = ff_add(ff_fma(gen_rec_ff(bc, BC_TL), Bm, bL), Am);   // x_s (eq. 18)
  fe[tid] = ff_fma(gen_rec_ff(bc, BC_TR), Am, ff_add(bR, Bm));   // x_e
  __syncthreads();
  if (act) {
    if (!(mb == 0 || tid == 0)) XL = fe[tid - 1];
    if (!(mb == P - 1 || tid + 1 >= nwin)) XR = fs[tid + 1];
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_window_gen_ff(const GenArgs G) {
  constexpr int LD = NT + 1;
  constexpr int NW = NT / 32;
  const WinArgs& A = G.w;
  extern __shared__ __align__(16) double sm[];
  // launched with programmatic stream serialization: nothing is read or written before the
  // previous kernel of the stream has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int tid = threadIdx.x;
  const int ns = A.n_smem;
  double* S = sm;
  double* sxs = S + (size_t)ns * LD;
  double* sxe = sxs + NT;
  double* scl = sxe + NT;
  double* scr = scl + NT;
  double* swa = scr + NT;                          // 4 * NW scan scratch (also the exponent maxima)

  const SysPlan* pp = A.plans;
  const int64_t P = pp->P;
  const int nown0 = pp->own;
  const int64_t m0 = (int64_t)blockIdx.x * nown0;
  const int nown = (int)min((int64_t)nown0, P - m0);
  int hl = 0, hr = 0;
  if (A.mode == MODE_FULL) {
    hl = (int)min((int64_t)pp->hl, m0);
    hr = (int)min((int64_t)pp->hr, P - m0 - nown);
  }
  const int64_t wlo = m0 - hl;
  const int nwin = hl + nown + hr;
  const int n = pp->n, nlast = pp->nlast;
  const bool has_last = (wlo + nwin == P);
  const int64_t row_lo = wlo * (int64_t)n;
  const int len = nwin * n - (has_last ? (n - nlast) : 0);
  const double* Fw = A.F + (int64_t)blockIdx.y * A.ldf;
  double* xw = A.x + (int64_t)blockIdx.y * A.ldx;

  // ---------------------------------------------------------------- F (or y) -> smem (transposed)
  {
    const double* src = ((A.mode == MODE_APPLY) ? xw : Fw) + row_lo;
    int b = tid / n, i = tid - (tid / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = tid; j < len; j += NT) {
      cp_async8(&S[i * LD + b], src + j);
      i += di;
      b += db;
      if (i >= n) {
        i -= n;
        ++b;
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  const bool act = tid < nwin;
  const int64_t mb = wlo + tid;
  const int nbk = (act && mb == P - 1) ? nlast : n;
  double* col = S + tid;

  // ---------------------------------------------------------------- window scale
  // largest |value| of the tile near 2^16; a tile of normal values within 2^119 of each other
  // (not near the ends of the FP64 range) takes the fast split and join of ff.cuh
  int wscale;
  bool fast;
  {
    unsigned hmax = 0u, hmin = 0xFFFFFFFFu;
    if (act)
      for (int i = 0; i < nbk; ++i) {
        const unsigned h = (unsigned)__double2hiint(col[i * LD]) & 0x7FFFFFFFu;
        hmax = max(hmax, h);
        hmin = min(hmin, h);
      }
    hmax = __reduce_max_sync(0xffffffffu, hmax);
    hmin = __reduce_min_sync(0xffffffffu, hmin);
    unsigned* sexp = reinterpret_cast<unsigned*>(swa);
    if ((tid & 31) == 0) {
      sexp[tid >> 5] = hmax;
      sexp[NW + (tid >> 5)] = hmin;
    }
    __syncthreads();
    hmax = 0u;
    hmin = 0xFFFFFFFFu;
    for (int w = 0; w < NW; ++w) {
      hmax = max(hmax, sexp[w]);
      hmin = min(hmin, sexp[NW + w]);
    }
    __syncthreads();
    const int emax = (int)(hmax >> 20), emin = (int)(hmin >> 20);
    wscale = (emax == 2047) ? 0 : ((emax == 0) ? 1000 : max(-1000, min(1000, (1023 + 16) - emax)));
    fast = (emin >= 1) && (emax >= 239) && (emax <= 1935) && (emax - emin <= 119);
  }
  const FastK fk = fast_k(wscale);
  // the tile's FP64 value -> (h, l) at the window scale; FASTC: std::true_type in a fast tile
  auto split_t = [&](double d, float& h, float& l, auto fastc) {
    if constexpr (decltype(fastc)::value)
      split_fast(d, fk, h, l);
    else
      split_sc(d, wscale, h, l);
  };

  const float2* ra = reinterpret_cast<const float2*>(G.rows + GF_A * G.stride);
  const float2* rd = reinterpret_cast<const float2*>(G.rows + GF_RD * G.stride);
  const float2* rc = reinterpret_cast<const float2*>(G.rows + GF_CP * G.stride);
  const float2* rv = reinterpret_cast<const float2*>(G.rows + GF_V * G.stride);
  const float2* rw = reinterpret_cast<const float2*>(G.rows + GF_W * G.stride);
  const int64_t k0 = gen_index(act ? mb : 0, 0, n);   // row i of the block at k0 + 32 i
  float2* colf = reinterpret_cast<float2*>(col);     // the same slots, as float-float pairs (stride LD)
  auto ldff = [](const float2* t, int64_t k) {
    const float2 v = t[k];
    return ffv{v.x, v.y};
  };

  // ---------------------------------------------------------------- local solves (a1), float-float
  if (act && A.mode != MODE_APPLY) {
    // the factors of four rows are loaded ahead of their dependent steps (the per-row global
    // loads would otherwise sit on the recurrence's critical path)
    auto sweeps = [&](auto fastc) {
      ffv z = ff_zero();
      int i = 0;
      for (; i + 4 <= nbk; i += 4) {
        const int64_t k = k0 + 32 * i;
        ffv a4[4], d4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a4[u] = ldff(ra, k + 32 * u);
          d4[u] = ldff(rd, k + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float fh, fl;
          split_t(col[(i + u) * LD], fh, fl, fastc);
          z = ff_mul(ff_fma(ff_neg(a4[u]), z, ffv{fh, fl}), d4[u]);
          colf[(i + u) * LD] = make_float2(z.h, z.l);
        }
      }
      for (; i < nbk; ++i) {
        const int64_t k = k0 + 32 * i;
        float fh, fl;
        split_t(col[i * LD], fh, fl, fastc);
        z = ff_mul(ff_fma(ff_neg(ldff(ra, k)), z, ffv{fh, fl}), ldff(rd, k));
        colf[i * LD] = make_float2(z.h, z.l);
      }
      ffv y = ff_zero();
      i = nbk - 1;
      for (; i - 3 >= 0; i -= 4) {
        ffv c4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c4[u] = ldff(rc, k0 + 32 * (i - u));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 zz = colf[(i - u) * LD];
          y = ff_fma(ff_neg(c4[u]), y, ffv{zz.x, zz.y});
          colf[(i - u) * LD] = make_float2(y.h, y.l);
        }
      }
      for (; i >= 0; --i) {
        const float2 zz = colf[i * LD];
        y = ff_fma(ff_neg(ldff(rc, k0 + 32 * i)), y, ffv{zz.x, zz.y});
        colf[i * LD] = make_float2(y.h, y.l);
      }
    };
    if (fast)
      sweeps(std::true_type());
    else
      sweeps(std::false_type());
  }

  // ---------------------------------------------------------------- beta (eq. 16)
  const double* bc = A.tabs + pp->o_bcl + (act ? mb : 0) * kBC;
  if (A.mode == MODE_BETA) {   // beta (FP64) and the block solutions y (joined) leave the window
    if (act) {
      const float2 y0 = colf[0], ye = colf[(nbk - 1) * LD];
      const double alpha = join_dadd(y0.x, y0.y, wscale), omega = join_dadd(ye.x, ye.y, wscale);
      A.beta[2 * (pp->gboff + mb)] = fma(bc[BC_M00], alpha, bc[BC_M01] * omega);
      A.beta[2 * (pp->gboff + mb) + 1] = fma(bc[BC_M10], alpha, bc[BC_M11] * omega);
      for (int i = 0; i < nbk; ++i) {
        const float2 yy = colf[i * LD];
        col[i * LD] = join_dadd(yy.x, yy.y, wscale);
      }
    }
    __syncthreads();
    int b = tid / n, i = tid - (tid / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = tid; j < len; j += NT) {
      xw[row_lo + j] = S[i * LD + b];
      i += di;
      b += db;
      if (i >= n) {
        i -= n;
        ++b;
      }
    }
    return;
  }

  // the neighbours' end values x_{s-1}, x_{e+1} in window units
  ffv cL = ff_zero(), cR = ff_zero();
  if (A.mode == MODE_FULL) {   // beta and the tree in float-float (window units)
    ffv bL = ff_zero(), bR = ff_zero();
    if (act) {
      const float2 y0 = colf[0], ye = colf[(nbk - 1) * LD];
      const ffv al{y0.x, y0.y}, om{ye.x, ye.y};
      bL = ff_fma(gen_rec_ff(bc, BC_M00), al, ff_mul(gen_rec_ff(bc, BC_M01), om));
      bR = ff_fma(gen_rec_ff(bc, BC_M10), al, ff_mul(gen_rec_ff(bc, BC_M11), om));
    }
    tree_gen_ff<NT>(bc, act, bL, bR, mb, P, nwin, tid, swa, sxs, sxe, cL, cR);
  } else if (act) {
    const double XL = (mb == 0) ? 0.0 : A.iface[2 * (pp->gboff + mb - 1) + 1];
    const double XR = (mb == P - 1) ? 0.0 : A.iface[2 * (pp->gboff + mb + 1)];
    float ch, cl, dh, dl;
    split_sc(XL, wscale, ch, cl);
    split_sc(XR, wscale, dh, dl);
    cL = ffv{ch, cl};
    cR = ffv{dh, dl};
  }

  // ---------------------------------------------------------------- interiors (eq. 7), float-float
  if (act) {
    auto interiors = [&](auto fastc) {
#pragma unroll 4
      for (int i = 0; i < nbk; ++i) {
        const int64_t k = k0 + 32 * i;
        ffv y;
        if (A.mode == MODE_APPLY) {
          float yh, yl;
          split_t(col[i * LD], yh, yl, fastc);
          y = ffv{yh, yl};
        } else {
          const float2 yy = colf[i * LD];
          y = ffv{yy.x, yy.y};
        }
        const ffv xv = ff_fma(cR, ldff(rw, k), ff_fma(cL, ldff(rv, k), y));
        if constexpr (decltype(fastc)::value)
          col[i * LD] = join_fast(xv.h, xv.l, fk);
        else
          col[i * LD] = join_dadd(xv.h, xv.l, wscale);
      }
    };
    if (fast)
      interiors(std::true_type());
    else
      interiors(std::false_type());
  }
  __syncthreads();

  asm volatile("griddepcontrol.launch_dependents;");   // the next kernel may begin its launch
  // ---------------------------------------------------------------- coalesced store of the own rows
  unsigned bad = 0u;
  {
    const int jlo = hl * n;
    const int jhi = min(len, (hl + nown) * n);
    double* dst = xw + row_lo;
    int b = (jlo + tid) / n, i = (jlo + tid) - ((jlo + tid) / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = jlo + tid; j < jhi; j += NT) {
      const double dv = S[i * LD + b];
      __stcs(dst + j, dv);
      if (A.check_finite && !isfinite(dv)) bad = 1u;
      i += di;
      b += db;
      if (i >= n) {
        i -= n;
        ++b;
      }
    }
  }
  if (bad) atomicOr(A.status, (unsigned)ST_NONFINITE);
}

}  // namespace dich
