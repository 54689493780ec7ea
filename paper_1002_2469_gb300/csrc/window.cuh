// window.cuh -- the Dichotomy window kernel (sm_103a).
//
// One CTA of NT threads handles a window of up to NT consecutive blocks of one system;
// thread b owns window block b.  Per window:
//   1. the window's rows of F (contiguous in HBM) are copied into shared memory with
//      8-byte cp.async copies, every thread issuing all of its copies before waiting, into
//      a transposed layout (row i of all blocks side by side, stride NT+1 doubles, so the
//      per-thread sweeps below read conflict-free);
//   2. local sweeps (a1): every thread runs the two first-order recurrences of its block
//      (u_i = f_i + rs u_{i-1}, X_i = u_i + ib X_{i+1}, xp_i = g X_i) in place, giving the
//      block ends alpha, omega of T_n^-1 F_m and then beta^{L,R}_m of eq. 16 through the
//      2x2 map M;
//   3. the dichotomy tree (a2): eq. 15 as two affine scans (prefix A, suffix B) -- five
//      warp-shuffle levels, then one shared-memory level across warps -- and the
//      first/last values x_s, x_e of every block (eq. 18);
//   4. the basis correction (a3): x = xp + (x_{s-1} - xp(-1)) v + x_{e+1} w, applied only
//      where the spikes v, w exceed the truncation threshold, and a contiguous,
//      coalesced store of the own rows.
// Windows of a long system overlap by halo blocks on each side whose coupling into the
// own blocks has decayed below the truncation threshold (2^-64 for FP64 plans, 2^-56 for
// MIXED ones, whose float-float values hold about 48 bits); on the
// general path the window instead takes the first/last values from a global scan (the FP64
// form's beta pass leaves xp in x and its apply pass starts from there, without new sweeps).
//
// This file holds the FP64 form (one block per thread) and what both window kernels share;
// the MIXED form's kernel is in window_mixed.cuh.
#pragma once

#include "dich_internal.cuh"

namespace dich {

struct WinArgs {
  const SysPlan* plans;   // plan records (device)
  const double* tabs;     // table buffer (device)
  const Item* items;      // batched: one item per CTA; nullptr: single system, window = blockIdx
  const double* F;        // right-hand sides
  double* x;              // solutions
  unsigned* status;       // device status word
  const double* iface;    // MODE_APPLY: (x_s, x_e) per block
  double* beta;           // MODE_BETA: (beta^L, beta^R) per block
  const double* xf;       // adjoint: forward solution (gradient sums), else nullptr
  double* part;           // adjoint: per-CTA partial sums [3 per CTA]
  int32_t mode;
  int32_t check_finite;
  int32_t n_smem;         // shared-memory rows (>= largest block size in the launch)
  int32_t sys_offset;     // added to the item's system index (adjoint twin records)
  int64_t ldf, ldx;       // series: right-hand side blockIdx.y starts at F + y ldf, its solution at x + y ldx
  int64_t win0;           // single system: window of CTA blockIdx.x is win0 + blockIdx.x
  int32_t bulk;           // F and x are device memory: 16-byte aligned windows may use bulk copies
};

// shared memory bytes for a window kernel of width NT and n_smem rows
__host__ __device__ inline size_t window_smem_bytes(int NT, int n_smem) {
  const size_t nw = (size_t)(NT / 32);
  return sizeof(double) * ((size_t)n_smem * (size_t)(NT + 1) + 4 * (size_t)n_smem + 5 * (size_t)NT + 4 * nw + 8);
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// 2^k as a double for |k| <= 1000 (bit construction)
__device__ __forceinline__ double pow2i(int k) { return __hiloint2double((1023 + k) << 20, 0); }

// The dichotomy tree of one FP64 window (a2): eq. 15 as two affine scans over the window's blocks
// (prefix maps A -> a A + b beta^R left to right, suffix maps B -> c B + d beta^L right to left),
// five warp-shuffle levels and one shared-memory level, then the first/last values of every
// block (eq. 18) in sxs/sxe and the neighbours' values each block needs: XL = x_{s-1}, XR = x_{e+1}.
// bc: the block's coefficient record; zero coupling enters at both window ends.
template <int NT>
__device__ __forceinline__ void tree_f64(const double* bc, bool act, double bL, double bR, int64_t mb, int64_t P,
                                         int nwin, int tid, double* swa, double* sxs, double* sxe, double& XL,
                                         double& XR) {
  constexpr int NW = NT / 32;
  const int lane = tid & 31, wid = tid >> 5;
  double pa = act ? bc[BC_A] : 1.0;
  double pb = act ? bc[BC_B] * bR : 0.0;
  double qa = act ? bc[BC_C] : 1.0;
  double qb = act ? bc[BC_D] * bL : 0.0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double ya = __shfl_up_sync(0xffffffffu, pa, d), yb = __shfl_up_sync(0xffffffffu, pb, d);
    const double za = __shfl_down_sync(0xffffffffu, qa, d), zb = __shfl_down_sync(0xffffffffu, qb, d);
    if (lane >= d) {
      pb = fma(pa, yb, pb);
      pa = pa * ya;
    }
    if (lane + d < 32) {
      qb = fma(qa, zb, qb);
      qa = qa * za;
    }
  }
  if (lane == 31) {
    swa[wid] = pa;
    swa[NW + wid] = pb;
  }
  if (lane == 0) {
    swa[2 * NW + wid] = qa;
    swa[3 * NW + wid] = qb;
  }
  // previous lane's inclusive prefix, next lane's inclusive suffix
  double ea = __shfl_up_sync(0xffffffffu, pa, 1), eb = __shfl_up_sync(0xffffffffu, pb, 1);
  double fa = __shfl_down_sync(0xffffffffu, qa, 1), fb = __shfl_down_sync(0xffffffffu, qb, 1);
  if (lane == 0) {
    ea = 1.0;
    eb = 0.0;
  }
  if (lane == 31) {
    fa = 1.0;
    fb = 0.0;
  }
  __syncthreads();
  double Aw = 0.0, Bw = 0.0;  // zero coupling enters at both window ends
  for (int w = 0; w < wid; ++w) Aw = fma(swa[w], Aw, swa[NW + w]);
  for (int w = NW - 1; w > wid; --w) Bw = fma(swa[2 * NW + w], Bw, swa[3 * NW + w]);
  const double Am = fma(ea, Aw, eb);
  const double Bm = fma(fa, Bw, fb);
  sxs[tid] = fma(bc[BC_TL], Bm, bL) + Am;            // x_s (eq. 18)
  sxe[tid] = fma(bc[BC_TR], Am, bR + Bm);            // x_e
  __syncthreads();
  if (act) {
    if (!(mb == 0 || tid == 0)) XL = sxe[tid - 1];
    if (!(mb == P - 1 || tid + 1 >= nwin)) XR = sxs[tid + 1];
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_window(const WinArgs A) {
  constexpr int NW = NT / 32;
  constexpr int LD = NT + 1;
  extern __shared__ __align__(16) double sm[];
  // launched with programmatic stream serialization: this grid may start while the previous
  // kernel of the stream finishes; nothing is read or written before that kernel has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ns = A.n_smem;
  double* S = sm;
  double* tv = S + (size_t)ns * LD;
  double* tw = tv + ns;
  double* tvl = tw + ns;
  double* twl = tvl + ns;
  double* sxs = twl + ns;
  double* sxe = sxs + NT;
  double* scl = sxe + NT;
  double* scr = scl + NT;
  double* swa = scr + 2 * NT;                     // 4 * NW scan scratch

  // ---------------------------------------------------------------- the window
  int sys;
  int64_t m0;
  int nown;
  if (A.items) {
    const Item it = A.items[blockIdx.x];
    sys = it.sys;
    m0 = it.m0;
    nown = it.n_own;
  } else {
    sys = 0;
    m0 = 0;
    nown = 0;
  }
  sys += A.sys_offset;
  const SysPlan* pp = A.plans + sys;
  const int64_t P = pp->P;
  if (!A.items) {
    nown = pp->own;
    m0 = ((int64_t)blockIdx.x + A.win0) * nown;
    if (m0 + nown > P) nown = (int)(P - m0);
  }
  int hl = 0, hr = 0;
  if (A.mode == MODE_FULL) {
    hl = (int)min((int64_t)pp->hl, m0);
    hr = (int)min((int64_t)pp->hr, P - m0 - nown);
  }
  const int64_t wlo = m0 - hl;
  const int nwin = hl + nown + hr;
  const int n = pp->n, nlast = pp->nlast;
  const int Lv = pp->Lv, Lw = pp->Lw;
  const int64_t off = pp->off;
  const double* tab = A.tabs + pp->tab;
  const bool has_last = (wlo + nwin == P);
  const int64_t row_lo = wlo * (int64_t)n;                   // first row of the window
  const int len = nwin * n - (has_last ? (n - nlast) : 0);  // rows in the window

  // ---------------------------------------------------------------- F -> smem (transposed, async)
  // (MODE_APPLY: the block solutions y the beta pass left in x, instead of F)
  {
    const double* src = (A.mode == MODE_APPLY) ? (A.x + (int64_t)blockIdx.y * A.ldx + off + row_lo)
                                               : (A.F + (int64_t)blockIdx.y * A.ldf + off + row_lo);
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
  // tables -> smem (overlaps the copies in flight)
  for (int i = tid; i < Lv; i += NT) tv[i] = tab[pp->o_v + i];
  for (int i = tid; i < Lw; i += NT) tw[i] = tab[pp->o_w + i];
  if (has_last)
    for (int i = tid; i < nlast; i += NT) {
      tvl[i] = tab[pp->o_vl + i];
      twl[i] = tab[pp->o_wl + i];
    }
  cp_async_wait_all();
  __syncthreads();

  // ---------------------------------------------------------------- local sweeps (a1)
  const bool act = tid < nwin;
  const int64_t mb = wlo + tid;
  const bool lastb = act && (mb == P - 1);
  const int nbk = lastb ? nlast : n;
  double xm1 = 0.0, alpha = 0.0, omega = 0.0;
  if (act && A.mode == MODE_APPLY) {
    xm1 = pp->ib * S[tid];   // xp(-1) = g ib X_0 = ib y_0
  } else if (act) {
    const double rs = pp->rs, ib = pp->ib, g = pp->g;
    double* col = S + tid;
    double u = 0.0;
    int i = 0;
    for (; i + 4 <= nbk; i += 4) {
      const double f0 = col[(i)*LD], f1 = col[(i + 1) * LD], f2 = col[(i + 2) * LD], f3 = col[(i + 3) * LD];
      const double u0 = fma(rs, u, f0);
      const double u1 = fma(rs, u0, f1);
      const double u2 = fma(rs, u1, f2);
      const double u3 = fma(rs, u2, f3);
      col[(i)*LD] = u0;
      col[(i + 1) * LD] = u1;
      col[(i + 2) * LD] = u2;
      col[(i + 3) * LD] = u3;
      u = u3;
    }
    for (; i < nbk; ++i) {
      u = fma(rs, u, col[i * LD]);
      col[i * LD] = u;
    }
    double X = 0.0;
    i = nbk - 1;
    for (; i - 3 >= 0; i -= 4) {
      const double a0 = col[(i)*LD], a1 = col[(i - 1) * LD], a2 = col[(i - 2) * LD], a3 = col[(i - 3) * LD];
      const double X0 = fma(ib, X, a0);
      const double X1 = fma(ib, X0, a1);
      const double X2 = fma(ib, X1, a2);
      const double X3 = fma(ib, X2, a3);
      col[(i)*LD] = g * X0;
      col[(i - 1) * LD] = g * X1;
      col[(i - 2) * LD] = g * X2;
      col[(i - 3) * LD] = g * X3;
      X = X3;
    }
    for (; i >= 0; --i) {
      X = fma(ib, X, col[i * LD]);
      col[i * LD] = g * X;
    }
    const double v0 = lastb ? pp->v0l : pp->v0;
    const double vend = lastb ? pp->vendl : pp->vend;
    const double xm = g * ib * X;
    xm1 = xm;
    alpha = col[0] - xm * v0;
    omega = col[(nbk - 1) * LD] - xm * vend;
  }

  // ---------------------------------------------------------------- beta (eq. 16)
  int64_t rec = pp->o_bcm;
  if (act) {
    if (mb < pp->kl)
      rec = pp->o_bcl + mb * kBC;
    else if (mb >= P - pp->kr)
      rec = pp->o_bcr + (mb - (P - pp->kr)) * kBC;
  }
  const double* bc = tab + rec;
  const double bL = act ? fma(bc[BC_M00], alpha, bc[BC_M01] * omega) : 0.0;
  const double bR = act ? fma(bc[BC_M10], alpha, bc[BC_M11] * omega) : 0.0;

  if (A.mode == MODE_BETA) {  // general path: beta and the block solutions y leave the window
    if (act) {
      A.beta[2 * (pp->gboff + mb)] = bL;
      A.beta[2 * (pp->gboff + mb) + 1] = bR;
    }
    __syncthreads();
    double* dst = A.x + (int64_t)blockIdx.y * A.ldx + off + row_lo;
    int b = tid / n, i = tid - (tid / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = tid; j < len; j += NT) {
      dst[j] = S[i * LD + b];
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
  } else {  // MODE_APPLY: first/last values of the neighbours from the global scan
    if (act) {
      XL = (mb == 0) ? 0.0 : A.iface[2 * (pp->gboff + mb - 1) + 1];
      XR = (mb == P - 1) ? 0.0 : A.iface[2 * (pp->gboff + mb + 1)];
    }
  }
  // correction coefficients of the block spikes (a3): x = xp + cL v + cR w
  scl[tid] = XL - xm1;
  scr[tid] = XR;
  __syncthreads();

  // the next kernel of the stream may begin its launch (it waits for this grid to complete)
  asm volatile("griddepcontrol.launch_dependents;");
  // ---------------------------------------------------------------- correction + store (a3)
  const bool adj = (A.xf != nullptr);
  double g0 = 0.0, gm = 0.0, gp = 0.0;
  unsigned bad = 0u;
  const int64_t N = pp->N;
  {
    const int jlo = hl * n;
    const int jhi = min(len, (hl + nown) * n);
    double* dst = A.x + (int64_t)blockIdx.y * A.ldx + off + row_lo;
    int b = (jlo + tid) / n, i = (jlo + tid) - ((jlo + tid) / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = jlo + tid; j < jhi; j += NT) {
      const bool lb = has_last && (b == nwin - 1);
      const int nb = lb ? nlast : n;
      const int lv = lb ? nlast : Lv, lw = lb ? nlast : Lw;
      const int jr = nb - 1 - i;
      double dv = S[i * LD + b];
      if (i < lv) dv = fma(scl[b], (lb ? tvl : tv)[i], dv);
      if (jr < lw) dv = fma(scr[b], (lb ? twl : tw)[jr], dv);
      __stcs(dst + j, dv);
      if (A.check_finite && !isfinite(dv)) bad = 1u;
      if (adj) {
        const int64_t r = row_lo + j;
        const double* xr = A.xf + off + r;
        g0 = fma(dv, xr[0], g0);
        if (r > 0) gm = fma(dv, xr[-1], gm);
        if (r + 1 < N) gp = fma(dv, xr[1], gp);
      }
      i += di;
      b += db;
      if (i >= n) {
        i -= n;
        ++b;
      }
    }
  }
  if (bad) atomicOr(A.status, (unsigned)ST_NONFINITE);
  if (adj) {
    // CTA sum of the three gradient partials in a fixed order
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      g0 += __shfl_down_sync(0xffffffffu, g0, d);
      gm += __shfl_down_sync(0xffffffffu, gm, d);
      gp += __shfl_down_sync(0xffffffffu, gp, d);
    }
    __syncthreads();
    if (lane == 0) {
      swa[wid] = gm;
      swa[NW + wid] = g0;
      swa[2 * NW + wid] = gp;
    }
    __syncthreads();
    if (tid < 3) {
      double s = 0.0;
      for (int w = 0; w < NW; ++w) s += swa[tid * NW + w];
      A.part[3 * (size_t)blockIdx.x + tid] = s;
    }
  }
}

}  // namespace dich
