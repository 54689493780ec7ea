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
// own blocks has decayed below 2^-64 (the truncation is exact to that level); on the
// general path the window instead takes the first/last values from a global scan.
//
// MIXED form: the sweeps run in compensated FP32 (ff.cuh) and the per-block quantities and the
// tree in float-float, all on values scaled per window by an exact power of two (largest |F|
// of the window near 2^16); only the general path's beta and first/last values cross the
// window boundary, as unscaled FP64.
#pragma once
#include <type_traits>

#include "dich_internal.cuh"
#include "ff.cuh"

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

// Arithmetic of the per-block quantities and of the dichotomy tree: FP64 in the FP64 form,
// float-float on the FP32 pipe in the MIXED form (GB300's FP64 pipe is ~70x slower).
struct OpsF64 {
  using V = double;
  static __device__ __forceinline__ V zero() { return 0.0; }
  static __device__ __forceinline__ V one() { return 1.0; }
  static __device__ __forceinline__ V add(V a, V b) { return a + b; }
  static __device__ __forceinline__ V sub(V a, V b) { return a - b; }
  static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ V up(V a, int d) { return __shfl_up_sync(0xffffffffu, a, d); }
  static __device__ __forceinline__ V down(V a, int d) { return __shfl_down_sync(0xffffffffu, a, d); }
  // block coefficient record j (BC_*) of the record at table offset `rec` (plan offsets in doubles)
  static __device__ __forceinline__ V bc(const double* tab, int64_t rec, int j) { return tab[rec + j]; }
};
struct OpsFF {
  using V = ffv;
  static __device__ __forceinline__ V zero() { return ff_zero(); }
  static __device__ __forceinline__ V one() { return ff_one(); }
  static __device__ __forceinline__ V add(V a, V b) { return ff_add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return ff_sub(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return ff_mul(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return ff_fma(a, b, c); }
  static __device__ __forceinline__ V up(V a, int d) { return ff_shfl_up(a, d); }
  static __device__ __forceinline__ V down(V a, int d) { return ff_shfl_down(a, d); }
  static __device__ __forceinline__ V bc(const double* tab, int64_t rec, int j) {
    return ff_of(reinterpret_cast<const float2*>(tab)[rec + j]);
  }
};

template <int NT, int FORM>
__global__ void __launch_bounds__(NT) k_window(const WinArgs A) {
  constexpr int NW = NT / 32;
  constexpr int LD = NT + 1;
  extern __shared__ __align__(16) double sm[];
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
  float2* S2 = reinterpret_cast<float2*>(S);

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
    m0 = (int64_t)blockIdx.x * nown;
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
  {
    const double* src = A.F + off + row_lo;
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
  if constexpr (FORM == FORM_F64) {
    for (int i = tid; i < Lv; i += NT) tv[i] = tab[pp->o_v + i];
    for (int i = tid; i < Lw; i += NT) tw[i] = tab[pp->o_w + i];
    if (has_last)
      for (int i = tid; i < nlast; i += NT) {
        tvl[i] = tab[pp->o_vl + i];
        twl[i] = tab[pp->o_wl + i];
      }
  } else {
    for (int i = tid; i < Lv; i += NT) tv[i] = tab[pp->o_vf + i];
    for (int i = tid; i < Lw; i += NT) tw[i] = tab[pp->o_wf + i];
    if (has_last)
      for (int i = tid; i < nlast; i += NT) {
        tvl[i] = tab[pp->o_vlf + i];
        twl[i] = tab[pp->o_wlf + i];
      }
  }
  cp_async_wait_all();
  __syncthreads();

  // ---------------------------------------------------------------- local sweeps (a1)
  const bool act = tid < nwin;
  const int64_t mb = wlo + tid;
  const bool lastb = act && (mb == P - 1);
  const int nbk = lastb ? nlast : n;
  using O = typename std::conditional<FORM == FORM_F64, OpsF64, OpsFF>::type;
  using V = typename O::V;
  V xm1 = O::zero(), alpha = O::zero(), omega = O::zero();

  // MIXED: one exact power-of-two scale per window puts its largest |F| near 2^16, so the
  // float-float sweeps and tree keep full relative precision at any magnitude of F
  int wscale = 0;
  if constexpr (FORM == FORM_MIXED) {
    unsigned e = 0u;
    if (act) {
      const unsigned* colw = reinterpret_cast<const unsigned*>(S + tid);
      for (int i = 0; i < nbk; ++i) e = max(e, (colw[2 * i * LD + 1] >> 20) & 0x7FFu);
    }
    e = __reduce_max_sync(0xffffffffu, e);
    unsigned* sexp = reinterpret_cast<unsigned*>(swa);
    if (lane == 0) sexp[wid] = e;
    __syncthreads();
    e = 0u;
    for (int w = 0; w < NW; ++w) e = max(e, sexp[w]);
    __syncthreads();
    // e == 0: zeros or subnormals only -> the largest scale; e == 2047: Inf/NaN -> none
    wscale = (e == 2047u) ? 0 : ((e == 0u) ? 1000 : max(-1000, min(1000, (1023 + 16) - (int)e)));
  }

  if (act) {
    if constexpr (FORM == FORM_F64) {
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
    } else {
      const float rh = pp->rs_h, rl = pp->rs_l, bh = pp->ib_h, bl = pp->ib_l, gh = pp->g_h, gl = pp->g_l;
      const double* cold = S + tid;
      float2* col = S2 + tid;
      float uh = 0.f, ul = 0.f;
      int i = 0;
      for (; i + 4 <= nbk; i += 4) {
        const float2 f0 = f64_to_ff_sc(cold[(i)*LD], wscale), f1 = f64_to_ff_sc(cold[(i + 1) * LD], wscale),
                     f2 = f64_to_ff_sc(cold[(i + 2) * LD], wscale), f3 = f64_to_ff_sc(cold[(i + 3) * LD], wscale);
        float2 o0, o1, o2, o3;
        ff_axpy(f0.x, f0.y, rh, rl, uh, ul, o0.x, o0.y);
        ff_axpy(f1.x, f1.y, rh, rl, o0.x, o0.y, o1.x, o1.y);
        ff_axpy(f2.x, f2.y, rh, rl, o1.x, o1.y, o2.x, o2.y);
        ff_axpy(f3.x, f3.y, rh, rl, o2.x, o2.y, o3.x, o3.y);
        col[(i)*LD] = o0;
        col[(i + 1) * LD] = o1;
        col[(i + 2) * LD] = o2;
        col[(i + 3) * LD] = o3;
        uh = o3.x;
        ul = o3.y;
      }
      for (; i < nbk; ++i) {
        const float2 f0 = f64_to_ff_sc(cold[i * LD], wscale);
        ff_axpy(f0.x, f0.y, rh, rl, uh, ul, uh, ul);
        col[i * LD] = make_float2(uh, ul);
      }
      float Xh = 0.f, Xl = 0.f;
      i = nbk - 1;
      for (; i - 3 >= 0; i -= 4) {
        const float2 a0 = col[(i)*LD], a1 = col[(i - 1) * LD], a2 = col[(i - 2) * LD], a3 = col[(i - 3) * LD];
        float2 X0, X1, X2, X3, y0, y1, y2, y3;
        ff_axpy(a0.x, a0.y, bh, bl, Xh, Xl, X0.x, X0.y);
        ff_axpy(a1.x, a1.y, bh, bl, X0.x, X0.y, X1.x, X1.y);
        ff_axpy(a2.x, a2.y, bh, bl, X1.x, X1.y, X2.x, X2.y);
        ff_axpy(a3.x, a3.y, bh, bl, X2.x, X2.y, X3.x, X3.y);
        ff_mul(gh, gl, X0.x, X0.y, y0.x, y0.y);
        ff_mul(gh, gl, X1.x, X1.y, y1.x, y1.y);
        ff_mul(gh, gl, X2.x, X2.y, y2.x, y2.y);
        ff_mul(gh, gl, X3.x, X3.y, y3.x, y3.y);
        col[(i)*LD] = y0;
        col[(i - 1) * LD] = y1;
        col[(i - 2) * LD] = y2;
        col[(i - 3) * LD] = y3;
        Xh = X3.x;
        Xl = X3.y;
      }
      for (; i >= 0; --i) {
        const float2 a0 = col[i * LD];
        ff_axpy(a0.x, a0.y, bh, bl, Xh, Xl, Xh, Xl);
        float2 y0;
        ff_mul(gh, gl, Xh, Xl, y0.x, y0.y);
        col[i * LD] = y0;
      }
      // block-end quantities (float-float, window-scaled units)
      const ffv gib = ffv{pp->gib_h, pp->gib_l};
      const ffv v0 = lastb ? ffv{pp->v0l_h, pp->v0l_l} : ffv{pp->v0_h, pp->v0_l};
      const ffv vend = lastb ? ffv{pp->vendl_h, pp->vendl_l} : ffv{pp->vend_h, pp->vend_l};
      const ffv xm = ff_mul(gib, ff_make(Xh, Xl));
      xm1 = xm;
      alpha = ff_sub(ff_of(col[0]), ff_mul(xm, v0));
      omega = ff_sub(ff_of(col[(nbk - 1) * LD]), ff_mul(xm, vend));
    }
  }

  // ---------------------------------------------------------------- beta (eq. 16)
  int64_t rec = (FORM == FORM_F64) ? pp->o_bcm : pp->o_bcmf;
  if (act) {
    if (mb < pp->kl)
      rec = ((FORM == FORM_F64) ? pp->o_bcl : pp->o_bclf) + mb * kBC;
    else if (mb >= P - pp->kr)
      rec = ((FORM == FORM_F64) ? pp->o_bcr : pp->o_bcrf) + (mb - (P - pp->kr)) * kBC;
  }
  const V bL = act ? O::fma(O::bc(tab, rec, BC_M00), alpha, O::mul(O::bc(tab, rec, BC_M01), omega)) : O::zero();
  const V bR = act ? O::fma(O::bc(tab, rec, BC_M10), alpha, O::mul(O::bc(tab, rec, BC_M11), omega)) : O::zero();

  if (A.mode == MODE_BETA) {  // general path: beta leaves the window as unscaled FP64
    if (act) {
      if constexpr (FORM == FORM_F64) {
        A.beta[2 * mb] = *reinterpret_cast<const double*>(&bL);
        A.beta[2 * mb + 1] = *reinterpret_cast<const double*>(&bR);
      } else {
        const double dn = pow2i(-wscale);
        A.beta[2 * mb] = ff_to_double(*reinterpret_cast<const ffv*>(&bL)) * dn;
        A.beta[2 * mb + 1] = ff_to_double(*reinterpret_cast<const ffv*>(&bR)) * dn;
      }
    }
    return;
  }

  V XL = O::zero(), XR = O::zero();
  V* swv = reinterpret_cast<V*>(swa);
  V* sxsv = reinterpret_cast<V*>(sxs);
  V* sxev = reinterpret_cast<V*>(sxe);
  if (A.mode == MODE_FULL) {
    // ------------------------------------------------------------ dichotomy tree (a2)
    // prefix maps A -> a A + b beta^R (left to right), suffix maps B -> c B + d beta^L
    V pa = act ? O::bc(tab, rec, BC_A) : O::one();
    V pb = act ? O::mul(O::bc(tab, rec, BC_B), bR) : O::zero();
    V qa = act ? O::bc(tab, rec, BC_C) : O::one();
    V qb = act ? O::mul(O::bc(tab, rec, BC_D), bL) : O::zero();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const V ya = O::up(pa, d), yb = O::up(pb, d);
      const V za = O::down(qa, d), zb = O::down(qb, d);
      if (lane >= d) {
        pb = O::fma(pa, yb, pb);
        pa = O::mul(pa, ya);
      }
      if (lane + d < 32) {
        qb = O::fma(qa, zb, qb);
        qa = O::mul(qa, za);
      }
    }
    if (lane == 31) {
      swv[wid] = pa;
      swv[NW + wid] = pb;
    }
    if (lane == 0) {
      swv[2 * NW + wid] = qa;
      swv[3 * NW + wid] = qb;
    }
    // previous lane's inclusive prefix, next lane's inclusive suffix
    V ea = O::up(pa, 1), eb = O::up(pb, 1);
    V fa = O::down(qa, 1), fb = O::down(qb, 1);
    if (lane == 0) {
      ea = O::one();
      eb = O::zero();
    }
    if (lane == 31) {
      fa = O::one();
      fb = O::zero();
    }
    __syncthreads();
    V Aw = O::zero(), Bw = O::zero();  // zero coupling enters at both window ends
    for (int w = 0; w < wid; ++w) Aw = O::fma(swv[w], Aw, swv[NW + w]);
    for (int w = NW - 1; w > wid; --w) Bw = O::fma(swv[2 * NW + w], Bw, swv[3 * NW + w]);
    const V Am = O::fma(ea, Aw, eb);
    const V Bm = O::fma(fa, Bw, fb);
    sxsv[tid] = O::add(O::fma(O::bc(tab, rec, BC_TL), Bm, bL), Am);            // x_s (eq. 18)
    sxev[tid] = O::fma(O::bc(tab, rec, BC_TR), Am, O::add(bR, Bm));           // x_e
    __syncthreads();
    if (act) {
      if (!(mb == 0 || tid == 0)) XL = sxev[tid - 1];
      if (!(mb == P - 1 || tid + 1 >= nwin)) XR = sxsv[tid + 1];
    }
  } else {  // MODE_APPLY: first/last values of the neighbours from the global scan
    if (act) {
      const double dl = (mb == 0) ? 0.0 : A.iface[2 * (mb - 1) + 1];
      const double dr = (mb == P - 1) ? 0.0 : A.iface[2 * (mb + 1)];
      if constexpr (FORM == FORM_F64) {
        *reinterpret_cast<double*>(&XL) = dl;
        *reinterpret_cast<double*>(&XR) = dr;
      } else {
        const double upw = pow2i(wscale);
        const float2 a2 = f64_to_ff_rn(dl * upw), b2 = f64_to_ff_rn(dr * upw);
        *reinterpret_cast<ffv*>(&XL) = ffv{a2.x, a2.y};
        *reinterpret_cast<ffv*>(&XR) = ffv{b2.x, b2.y};
      }
    }
  }
  // correction coefficients of the block spikes (a3): x = xp + cL v + cR w
  reinterpret_cast<V*>(scl)[tid] = O::sub(XL, xm1);
  reinterpret_cast<V*>(scr)[tid] = XR;
  __syncthreads();

  // ---------------------------------------------------------------- correction + store (a3)
  const bool adj = (A.xf != nullptr);
  double g0 = 0.0, gm = 0.0, gp = 0.0;
  unsigned bad = 0u;
  const int64_t N = pp->N;
  {
    const int jlo = hl * n;
    const int jhi = min(len, (hl + nown) * n);
    double* dst = A.x + off + row_lo;
    int b = (jlo + tid) / n, i = (jlo + tid) - ((jlo + tid) / n) * n;
    const int db = NT / n, di = NT - (NT / n) * n;
    for (int j = jlo + tid; j < jhi; j += NT) {
      const bool lb = has_last && (b == nwin - 1);
      const int nb = lb ? nlast : n;
      const int lv = lb ? nlast : Lv, lw = lb ? nlast : Lw;
      const int jr = nb - 1 - i;
      double dv;
      if constexpr (FORM == FORM_F64) {
        double val = S[i * LD + b];
        if (i < lv) val = fma(scl[b], (lb ? tvl : tv)[i], val);
        if (jr < lw) val = fma(scr[b], (lb ? twl : tw)[jr], val);
        dv = val;
      } else {
        float2 val = S2[i * LD + b];
        if (i < lv) {
          const float2 c = reinterpret_cast<const float2*>(scl)[b];
          const float2 vv = reinterpret_cast<const float2*>(lb ? tvl : tv)[i];
          ff_fma_acc(c.x, c.y, vv.x, vv.y, val.x, val.y);
        }
        if (jr < lw) {
          const float2 c = reinterpret_cast<const float2*>(scr)[b];
          const float2 ww = reinterpret_cast<const float2*>(lb ? twl : tw)[jr];
          ff_fma_acc(c.x, c.y, ww.x, ww.y, val.x, val.y);
        }
        dv = ff_to_f64_int(val.x, val.y, wscale);
      }
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
