// window_mixed.cuh -- the MIXED-form window kernel: two blocks per thread, packed FP32x2.
//
// Same steps as the FP64 form's k_window (window.cuh): load the window transposed, local sweeps (a1), beta,
// the dichotomy tree (a2), the spike correction and store (a3).  Differences:
//   - thread t owns the adjacent window blocks 2t and 2t+1; shared-memory rows hold a
//     thread's pair in one 16-byte slot, and both recurrences advance through one f32x2
//     instruction (sm_100+ FFMA2/FADD2/FMUL2), halving the issue slots of the sweeps and
//     doubling the independent work per thread;
//   - the per-row layout of a pair is [hi(2t), hi(2t+1), lo(2t), lo(2t+1)] during the
//     sweeps and [x(2t), x(2t+1)] as FP64 after the correction;
//   - the thread composes its two blocks' affine maps before the warp/CTA scans;
//   - the correction and the FP64 join run per thread along its own columns (no per-element
//     index bookkeeping), then the CTA stores its own rows with contiguous coalesced writes.
// Arithmetic: compensated FP32 sweeps, float-float block quantities and tree, one exact
// power-of-two scale per window (see ff.cuh).
#pragma once
#include <type_traits>
#include "ff.cuh"
#include "window.cuh"

namespace dich {

// float-float arithmetic of the per-block quantities and of the dichotomy tree
struct OpsFF {
  using V = ffv;
  static __device__ __forceinline__ V add(V a, V b) { return ff_add(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return ff_mul(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return ff_fma(a, b, c); }
  static __device__ __forceinline__ V up(V a, int d) { return ff_shfl_up(a, d); }
  static __device__ __forceinline__ V down(V a, int d) { return ff_shfl_down(a, d); }
  // block coefficient record j (BC_*) of the record at float-pair offset `rec`
  static __device__ __forceinline__ V bc(const double* tab, int64_t rec, int j) {
    return ff_of(reinterpret_cast<const float2*>(tab)[rec + j]);
  }
};


// forward and backward sweeps of a thread's pair of blocks, in place.  GUARD: the two blocks
// may differ in size (the system's last block) or be inactive (nb = 0): rows at or beyond a
// block's size enter as zero, which keeps its backward recurrence exact.
template <int LD, bool GUARD, bool FAST, int NR = 0>
__device__ __forceinline__ void sweep_pair(double* S, int tid, int nrow_, int nb0, int nb1, int wscale,
                                           const SysPlan* pp, float2& Xh, float2& Xl) {
  const int nrow = NR ? NR : nrow_;
  const FastK fk = fast_k(wscale);
  const float2 rh = f2(pp->rs_h), rl = f2(pp->rs_l), bh = f2(pp->ib_h), bl = f2(pp->ib_l);
  const float2 gh = f2(pp->g_h), gl = f2(pp->g_l);
  float2 uh = f2(0.f), ul = f2(0.f);
#pragma unroll 4
  for (int i = 0; i < nrow; ++i) {
    double* row = S + (size_t)i * LD + 2 * tid;
    const double2 fd = *reinterpret_cast<const double2*>(row);
    float2 fh, fl;
    if (FAST) {
      split_fast(fd.x, fk, fh.x, fl.x);
      split_fast(fd.y, fk, fh.y, fl.y);
    } else {
      split_sc(fd.x, wscale, fh.x, fl.x);
      split_sc(fd.y, wscale, fh.y, fl.y);
    }
    if (GUARD) {
      if (i >= nb0) fh.x = fl.x = 0.f;
      if (i >= nb1) fh.y = fl.y = 0.f;
    }
    ff_axpy2(fh, fl, rh, rl, uh, ul, uh, ul);
    *reinterpret_cast<float4*>(row) = make_float4(uh.x, uh.y, ul.x, ul.y);
  }
  float2 xh = f2(0.f), xl = f2(0.f);
#pragma unroll 4
  for (int i = nrow - 1; i >= 0; --i) {
    double* row = S + (size_t)i * LD + 2 * tid;
    float4 q = *reinterpret_cast<const float4*>(row);
    if (GUARD) {
      if (i >= nb0) q.x = q.z = 0.f;
      if (i >= nb1) q.y = q.w = 0.f;
    }
    ff_axpy2(make_float2(q.x, q.y), make_float2(q.z, q.w), bh, bl, xh, xl, xh, xl);
    float2 yh, yl;
    ff_mul2(gh, gl, xh, xl, yh, yl);
    *reinterpret_cast<float4*>(row) = make_float4(yh.x, yh.y, yl.x, yl.y);
  }
  Xh = xh;
  Xl = xl;
}

// correction x = xp + cL v + cR w along the thread's pair of columns and the FP64 join, in place.
// tv4[i] = (v_h, v_h, v_l, v_l) and tw4[j] = (w_h, w_h, w_l, w_l) hold the full-size blocks' spikes
// (w reversed) with both lanes filled and zeros past their truncation lengths, so the full-block
// loop needs neither bounds nor lane moves.  The system's last block (size nlast) reads its own
// spikes from global memory (tvl, twl: float-float pairs).  KEEP: no join; each block's corrected
// value stays a float-float pair (h, l) in its FP64 slot of the row (the adjoint's store loop
// joins it and also forms the gradient products from it).
template <int LD, bool GUARD, bool FAST, int NR = 0, bool KEEP = false>
__device__ __forceinline__ void correct_pair(double* S, int tid, int nrow_, int nb0, int nb1, bool last0,
                                             bool last1, int n, const float4* tv4, const float4* tw4,
                                             const float2* tvl, const float2* twl, const ff2& cL, const ff2& cR,
                                             int wscale) {
  const int nrow = NR ? NR : nrow_;
  const float2 clh = cL.h, cll = cL.l, crh = cR.h, crl = cR.l;
  const FastK fk = fast_k(wscale);
  if (!GUARD) {
    // both blocks full size: one spike table, one row index for both
#pragma unroll 2
    for (int i = 0; i < nrow; ++i) {
      double* row = S + (size_t)i * LD + 2 * tid;
      const float4 q = *reinterpret_cast<const float4*>(row);
      float2 xh = make_float2(q.x, q.y), xl = make_float2(q.z, q.w);
      const float4 v = tv4[i], w = tw4[n - 1 - i];
      ff_fma_acc2(clh, cll, make_float2(v.x, v.y), make_float2(v.z, v.w), xh, xl);
      ff_fma_acc2(crh, crl, make_float2(w.x, w.y), make_float2(w.z, w.w), xh, xl);
      if (KEEP)
        *reinterpret_cast<float4*>(row) = make_float4(xh.x, xl.x, xh.y, xl.y);
      else if (FAST)
        *reinterpret_cast<double2*>(row) =
            make_double2(join_fast(xh.x, xl.x, fk), join_fast(xh.y, xl.y, fk));
      else
        *reinterpret_cast<double2*>(row) =
            make_double2(join_dadd(xh.x, xl.x, wscale), join_dadd(xh.y, xl.y, wscale));
    }
  } else {
    for (int i = 0; i < nrow; ++i) {
      double* row = S + (size_t)i * LD + 2 * tid;
      const float4 q = *reinterpret_cast<const float4*>(row);
      float2 xh = make_float2(q.x, q.y), xl = make_float2(q.z, q.w);
      float2 vh = f2(0.f), vl = f2(0.f), wh = f2(0.f), wl = f2(0.f);
      const int j0 = nb0 - 1 - i, j1 = nb1 - 1 - i;
      if (i < nb0) {
        const float2 v = last0 ? tvl[i] : make_float2(tv4[i].x, tv4[i].z);
        const float2 w = last0 ? twl[j0] : make_float2(tw4[j0].x, tw4[j0].z);
        vh.x = v.x;
        vl.x = v.y;
        wh.x = w.x;
        wl.x = w.y;
      }
      if (i < nb1) {
        const float2 v = last1 ? tvl[i] : make_float2(tv4[i].x, tv4[i].z);
        const float2 w = last1 ? twl[j1] : make_float2(tw4[j1].x, tw4[j1].z);
        vh.y = v.x;
        vl.y = v.y;
        wh.y = w.x;
        wl.y = w.y;
      }
      ff_fma_acc2(clh, cll, vh, vl, xh, xl);
      ff_fma_acc2(crh, crl, wh, wl, xh, xl);
      if (KEEP) {
        *reinterpret_cast<float4*>(row) = make_float4(i < nb0 ? xh.x : 0.f, i < nb0 ? xl.x : 0.f,
                                                      i < nb1 ? xh.y : 0.f, i < nb1 ? xl.y : 0.f);
      } else {
        double d0 = (i < nb0) ? join_dadd(xh.x, xl.x, wscale) : 0.0;
        double d1 = (i < nb1) ? join_dadd(xh.y, xl.y, wscale) : 0.0;
        *reinterpret_cast<double2*>(row) = make_double2(d0, d1);
      }
    }
  }
}

// After the tree: the values of the neighbouring blocks a thread's pair needs -- x_e of block 2t-1
// (the previous thread's second block) and x_s of block 2t+2 (the next thread's first block) -- by
// warp shuffles, across warp boundaries through sbd (2 NW entries: each warp's last x_e, first x_s).
// Zeros beyond the window's ends; the caller masks the system's ends and inactive blocks.
template <int NT>
__device__ __forceinline__ void pair_neighbours(const ff2& xs, const ff2& xe, int tid, ffv* sbd, ffv& xe_prev,
                                                ffv& xs_next) {
  constexpr int NW = NT / 32;
  const int lane = tid & 31, wid = tid >> 5;
  ffv up{__shfl_up_sync(0xffffffffu, xe.h.y, 1), __shfl_up_sync(0xffffffffu, xe.l.y, 1)};
  ffv dn{__shfl_down_sync(0xffffffffu, xs.h.x, 1), __shfl_down_sync(0xffffffffu, xs.l.x, 1)};
  if (lane == 31) sbd[wid] = ff2_y(xe);
  if (lane == 0) sbd[NW + wid] = ff2_x(xs);
  __syncthreads();
  if (lane == 0) up = (wid > 0) ? sbd[wid - 1] : ff_zero();
  if (lane == 31) dn = (wid < NW - 1) ? sbd[NW + wid + 1] : ff_zero();
  xe_prev = up;
  xs_next = dn;
}

// The dichotomy tree of one MIXED window (a2): the prefix and suffix affine scans of eq. 15 over the
// window's blocks in packed float-float (five warp-shuffle levels, one shared-memory level), the
// first/last values of every block (eq. 18), and the neighbours' values the correction of the
// thread's two blocks needs: XL = x_{s-1}, XR = x_{e+1} (zero coupling enters at both window ends).
// bc2(j): coefficient j of both blocks' records; bL, bR: beta (eq. 16) of both blocks; sbd: 2 NW
// entries of shared memory for the exchange across warps.
// lev: warp-scan levels that run (the plan's; contributions from 2^(lev+1) or more blocks away are
// below its truncation threshold, 5 = the whole warp).
template <int NT, class BC>
__device__ __forceinline__ void tree2(const BC& bc2, bool act0, bool act1, int64_t mb0, int64_t mb1, int64_t P,
                                      int nwin, int tid, const ff2& bL, const ff2& bR, ffv* swv, ffv* sbd,
                                      ffv& XL0, ffv& XR0, ffv& XL1, ffv& XR1, int lev = 5) {
  using O = OpsFF;
  constexpr int NW = NT / 32;
  const int lane = tid & 31, wid = tid >> 5;
  const int b0 = 2 * tid, b1 = 2 * tid + 1;
  const ff2 one2{f2(1.f), f2(0.f)};
  // ------------------------------------------------------------ dichotomy tree (a2)
  // block maps: prefix A -> a A + b beta^R, suffix B -> c B + d beta^L
  const ff2 av = ff2_sel(act0, act1, bc2(BC_A), one2), cv = ff2_sel(act0, act1, bc2(BC_C), one2);
  const ff2 pbv = ff2_mul(bc2(BC_B), bR), qbv = ff2_mul(bc2(BC_D), bL);
  // the thread's composite maps, lane x the prefix (block 1 after block 0), lane y the suffix
  // (block 0 after block 1): (a1 a0, c0 c1) and (a1 pb0 + pb1, c0 qb1 + qb0)
  const ff2 m1{make_float2(av.h.y, cv.h.x), make_float2(av.l.y, cv.l.x)};
  ff2 Sv = ff2_mul(m1, ff2{make_float2(av.h.x, cv.h.y), make_float2(av.l.x, cv.l.y)});
  ff2 Tv = ff2_fma(m1, ff2{make_float2(pbv.h.x, qbv.h.y), make_float2(pbv.l.x, qbv.l.y)},
                   ff2{make_float2(pbv.h.y, qbv.h.x), make_float2(pbv.l.y, qbv.l.x)});
  // warp scans: the prefix from lane - d, the suffix from lane + d; identity maps past the ends
  const int dlim = 1 << lev;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    if (d >= dlim) break;
    const float yah = __shfl_up_sync(0xffffffffu, Sv.h.x, d), yal = __shfl_up_sync(0xffffffffu, Sv.l.x, d);
    const float ybh = __shfl_up_sync(0xffffffffu, Tv.h.x, d), ybl = __shfl_up_sync(0xffffffffu, Tv.l.x, d);
    const float zah = __shfl_down_sync(0xffffffffu, Sv.h.y, d), zal = __shfl_down_sync(0xffffffffu, Sv.l.y, d);
    const float zbh = __shfl_down_sync(0xffffffffu, Tv.h.y, d), zbl = __shfl_down_sync(0xffffffffu, Tv.l.y, d);
    const bool up = lane >= d, dn = lane + d < 32;
    const ff2 Ya{make_float2(up ? yah : 1.f, dn ? zah : 1.f), make_float2(up ? yal : 0.f, dn ? zal : 0.f)};
    const ff2 Yb{make_float2(up ? ybh : 0.f, dn ? zbh : 0.f), make_float2(up ? ybl : 0.f, dn ? zbl : 0.f)};
    Tv = ff2_fma(Sv, Yb, Tv);
    Sv = ff2_mul(Sv, Ya);
  }
  const ffv pa = ff2_x(Sv), pb = ff2_x(Tv), qa = ff2_y(Sv), qb = ff2_y(Tv);
  if (lane == 31) {
    swv[wid] = pa;
    swv[NW + wid] = pb;
  }
  if (lane == 0) {
    swv[2 * NW + wid] = qa;
    swv[3 * NW + wid] = qb;
  }
  ffv ea = O::up(pa, 1), eb = O::up(pb, 1);
  ffv fa = O::down(qa, 1), fb = O::down(qb, 1);
  if (lane == 0) {
    ea = ff_one();
    eb = ff_zero();
  }
  if (lane == 31) {
    fa = ff_one();
    fb = ff_zero();
  }
  __syncthreads();
  ffv Aw = ff_zero(), Bw = ff_zero();  // zero coupling enters at both window ends
  for (int w = 0; w < wid; ++w) Aw = O::fma(swv[w], Aw, swv[NW + w]);
  for (int w = NW - 1; w > wid; --w) Bw = O::fma(swv[2 * NW + w], Bw, swv[3 * NW + w]);
  // (A entering block 0, B beyond block 1), then (A entering block 1, B beyond block 0)
  const ff2 E = ff2_fma(ff2_pair(ea, fa), ff2_pair(Aw, Bw), ff2_pair(eb, fb));
  const ff2 G = ff2_fma(ff2_pair(ff2_x(av), ff2_y(cv)), E, ff2_pair(ff2_x(pbv), ff2_y(qbv)));
  const ff2 Av{make_float2(E.h.x, G.h.x), make_float2(E.l.x, G.l.x)};   // (A_0, A_1)
  const ff2 Bv{make_float2(G.h.y, E.h.y), make_float2(G.l.y, E.l.y)};   // (B_0, B_1)
  // first/last values of both blocks (eq. 18)
  const ff2 xs = ff2_add(ff2_fma(bc2(BC_TL), Bv, bL), Av);
  const ff2 xe = ff2_fma(bc2(BC_TR), Av, ff2_add(bR, Bv));
  ffv xe_prev, xs_next;
  pair_neighbours<NT>(xs, xe, tid, sbd, xe_prev, xs_next);
  if (act0) {
    if (!(mb0 == 0 || b0 == 0)) XL0 = xe_prev;
    if (!(mb0 == P - 1 || b0 + 1 >= nwin)) XR0 = ff2_y(xs);
  }
  if (act1) {
    XL1 = ff2_x(xe);
    if (!(mb1 == P - 1 || b1 + 1 >= nwin)) XR1 = xs_next;
  }
}

// coefficient records of a thread's two blocks (the float-float copies of the plan tables) and
// their beta records (K1..K4 of beta_coeffs)
struct Recs2 {
  const float2* tf;
  int64_t r0, r1, k0, k1;
  __device__ __forceinline__ ff2 operator()(int j) const {  // coefficient j of both blocks' records
    const float2 c0 = tf[r0 + j], c1 = tf[r1 + j];
    return ff2_make(make_float2(c0.x, c1.x), make_float2(c0.y, c1.y));
  }
  __device__ __forceinline__ ff2 k(int j) const {           // beta coefficient K_{j+1} of both blocks
    const float2 c0 = tf[k0 + j], c1 = tf[k1 + j];
    return ff2_make(make_float2(c0.x, c1.x), make_float2(c0.y, c1.y));
  }
};
__device__ __forceinline__ Recs2 recs2(const SysPlan* pp, const double* tab, int64_t P, bool act0, bool act1,
                                       int64_t mb0, int64_t mb1) {
  auto rec_of = [&](int64_t m) -> int64_t {
    if (m < pp->kl) return pp->o_bclf + m * kBC;
    if (m >= P - pp->kr) return pp->o_bcrf + (m - (P - pp->kr)) * kBC;
    return pp->o_bcmf;
  };
  auto krec_of = [&](int64_t m) -> int64_t {
    if (m < pp->kl) return pp->o_klf + m * 4;
    if (m >= P - pp->kr) return pp->o_krf + (m - (P - pp->kr)) * 4;
    return pp->o_kmf;
  };
  return Recs2{reinterpret_cast<const float2*>(tab), act0 ? rec_of(mb0) : pp->o_bcmf,
               act1 ? rec_of(mb1) : pp->o_bcmf, act0 ? krec_of(mb0) : pp->o_kmf, act1 ? krec_of(mb1) : pp->o_kmf};
}

}  // namespace dich
#include "window_reg.cuh"
namespace dich {

// shared memory of the MIXED window kernel: NT threads, 2 NT window blocks, n_smem rows (at least
// what the register path needs when blocks of its size may occur)
__host__ __device__ inline size_t window2_smem_bytes(int NT, int n_smem) {
  const size_t nw = (size_t)(NT / 32);
  const size_t LD = 2 * (size_t)NT + 2;
  const size_t tile = sizeof(double) * ((size_t)n_smem * LD + 4 * (size_t)n_smem + 2 * nw + 4 * nw + 8);
  if (n_smem < kRegRows) return tile;
  const size_t reg = window_reg_smem_bytes(NT);
  return tile > reg ? tile : reg;
}

// Instantiations: KIND_REG -- the forward solve with the register path for windows it serves (up to
// 80 registers: six CTAs of 128 threads per SM); KIND_SMEM -- the forward solve on the shared-memory
// path only (80 registers: six CTAs per SM, for launches of many short, latency-bound windows);
// KIND_ADJ -- the adjoint (shared-memory path, gradient sums in the store loop, six CTAs per SM).
// KIND_REGADJ -- the adjoint with the register path for the windows it serves (up to 128 registers:
// four CTAs per SM; its slots hold x during the tree).
enum WinKind : int { KIND_REG = 0, KIND_ADJ = 1, KIND_SMEM = 2, KIND_REGADJ = 3 };

template <int NT, int KIND>
__global__ void __launch_bounds__(NT, (KIND == KIND_REGADJ ? 512 : 768) / NT)
    k_window2(const WinArgs A) {
  constexpr bool ADJ = (KIND == KIND_ADJ || KIND == KIND_REGADJ);
  constexpr int NW = NT / 32;
  constexpr int WB = 2 * NT;       // window blocks
  constexpr int LD = 2 * NT + 2;   // shared row stride in doubles (even: 16-byte pairs)
  using O = OpsFF;
  extern __shared__ __align__(16) double sm[];
  // launched with programmatic stream serialization: this grid may start while the previous
  // kernel of the stream finishes; nothing is read or written before that kernel has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ns = A.n_smem;
  double* S = sm;
  float4* tv4 = reinterpret_cast<float4*>(S + (size_t)ns * LD);   // spikes, both lanes, zero-padded
  float4* tw4 = tv4 + ns;
  ffv* sbd = reinterpret_cast<ffv*>(tw4 + ns);   // 2 * NW warp-boundary first/last values
  ffv* swv = sbd + 2 * NW;                       // 4 * NW scan scratch (also the exponent maxima)

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
  const int64_t row_lo = wlo * (int64_t)n;
  const int len = nwin * n - (has_last ? (n - nlast) : 0);

  if constexpr (KIND == KIND_REG || KIND == KIND_REGADJ) {
    // 16-row blocks, all of full size, 16-byte aligned device memory: the register path
    if (A.bulk && A.mode == MODE_FULL && n == kRegRows && (!has_last || nlast == kRegRows) && !A.check_finite &&
        ((reinterpret_cast<uintptr_t>(A.F + (int64_t)blockIdx.y * A.ldf + off + row_lo) |
          reinterpret_cast<uintptr_t>(A.x + (int64_t)blockIdx.y * A.ldx + off + row_lo) |
          (ADJ ? reinterpret_cast<uintptr_t>(A.xf + off + row_lo) : (uintptr_t)0)) & 15u) == 0u) {
      window_reg<NT, ADJ>(A, pp, tab, P, wlo, nwin, hl, nown, row_lo, reinterpret_cast<unsigned char*>(sm));
      return;
    }
  }

  // ---------------------------------------------------------------- F -> smem (transposed, async)
  {
    const double* src = A.F + (int64_t)blockIdx.y * A.ldf + off + row_lo;
    if (n == 16) {
      // element j = tid + k NT sits in row tid % 16 of block tid / 16 + k NT / 16: fixed strides
      double* d = S + (size_t)(tid & 15) * LD + (tid >> 4);
      const int cnt = (len - tid + NT - 1) / NT;
#pragma unroll 4
      for (int k = 0; k < cnt; ++k) cp_async8(d + k * (NT / 16), src + tid + k * NT);
    } else {
      int b = tid / n, i = tid - (tid / n) * n;
      const int db = NT / n, di = NT - (NT / n) * n;
      for (int j = tid; j < len; j += NT) {
        cp_async8(&S[(size_t)i * LD + b], src + j);
        i += di;
        b += db;
        if (i >= n) {
          i -= n;
          ++b;
        }
      }
    }
  }
  {
    const float2* tf = reinterpret_cast<const float2*>(tab);
    for (int i = tid; i < ns; i += NT) {
      const float2 v = (i < Lv) ? tf[pp->o_vf + i] : make_float2(0.f, 0.f);
      const float2 w = (i < Lw) ? tf[pp->o_wf + i] : make_float2(0.f, 0.f);
      tv4[i] = make_float4(v.x, v.x, v.y, v.y);
      tw4[i] = make_float4(w.x, w.x, w.y, w.y);
    }
  }
  // the adjoint: exponent range of the forward solution over the rows its gradient sums read
  // (the own rows and one beyond each end), loaded while the right-hand side streams in
  unsigned xhmax = 0u, xhmin = 0xFFFFFFFFu;
  if constexpr (ADJ) {
    const int jlo = hl * n, jhi = min(len, (hl + nown) * n);
    const unsigned* xw = reinterpret_cast<const unsigned*>(A.xf + off + row_lo) + 1;   // high words
    const int klo = (row_lo + jlo > 0) ? jlo - 1 : jlo;
    const int khi = (row_lo + jhi < pp->N) ? jhi + 1 : jhi;
#pragma unroll 16
    for (int k = klo + tid; k < khi; k += NT) {
      const unsigned h = __ldg(xw + 2 * k) & 0x7FFFFFFFu;
      xhmax = max(xhmax, h);
      xhmin = min(xhmin, h);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // ---------------------------------------------------------------- the thread's two blocks
  const int b0 = 2 * tid, b1 = 2 * tid + 1;
  const bool act0 = b0 < nwin, act1 = b1 < nwin;
  const int64_t mb0 = wlo + b0, mb1 = wlo + b1;
  const bool last0 = act0 && (mb0 == P - 1), last1 = act1 && (mb1 == P - 1);
  const int nb0 = act0 ? (last0 ? nlast : n) : 0;
  const int nb1 = act1 ? (last1 ? nlast : n) : 0;
  const int nrow = max(nb0, nb1);
  const bool full = (nb0 == n) && (nb1 == n);

  // window scale: largest |F| of the window near 2^16 (exact power of two).  The largest and
  // smallest FP64 high words (sign cleared) give the exponent range of the window: a window of
  // normal values within 2^119 of each other, not too close to the ends of the FP64 range,
  // takes the fast split and join (ff.cuh).
  int wscale, xscale = 0;
  bool fast, xfast = false;   // x: the adjoint's forward solution (gradient sums)
  {
    unsigned hmax = 0u, hmin = 0xFFFFFFFFu;
    if (full) {
#pragma unroll 4
      for (int i = 0; i < nrow; ++i) {
        const uint4 q = *reinterpret_cast<const uint4*>(S + (size_t)i * LD + 2 * tid);
        const unsigned a = q.y & 0x7FFFFFFFu, c = q.w & 0x7FFFFFFFu;
        hmax = __vimax3_u32(hmax, a, c);
        hmin = __vimin3_u32(hmin, a, c);
      }
    } else {
      for (int i = 0; i < nrow; ++i) {
        const uint4 q = *reinterpret_cast<const uint4*>(S + (size_t)i * LD + 2 * tid);
        if (i < nb0) {
          hmax = max(hmax, q.y & 0x7FFFFFFFu);
          hmin = min(hmin, q.y & 0x7FFFFFFFu);
        }
        if (i < nb1) {
          hmax = max(hmax, q.w & 0x7FFFFFFFu);
          hmin = min(hmin, q.w & 0x7FFFFFFFu);
        }
      }
    }
    hmax = __reduce_max_sync(0xffffffffu, hmax);
    hmin = __reduce_min_sync(0xffffffffu, hmin);
    if (ADJ) {
      xhmax = __reduce_max_sync(0xffffffffu, xhmax);
      xhmin = __reduce_min_sync(0xffffffffu, xhmin);
    }
    unsigned* sexp = reinterpret_cast<unsigned*>(swv);
    if (lane == 0) {
      sexp[wid] = hmax;
      sexp[NW + wid] = hmin;
      if (ADJ) {
        sexp[2 * NW + wid] = xhmax;
        sexp[3 * NW + wid] = xhmin;
      }
    }
    __syncthreads();
    hmax = 0u;
    hmin = 0xFFFFFFFFu;
    for (int w = 0; w < NW; ++w) {
      hmax = max(hmax, sexp[w]);
      hmin = min(hmin, sexp[NW + w]);
      if (ADJ) {
        xhmax = max(xhmax, sexp[2 * NW + w]);
        xhmin = min(xhmin, sexp[3 * NW + w]);
      }
    }
    __syncthreads();
    auto scale_of = [](unsigned hmx, unsigned hmn, int& sc, bool& fs) {
      const int emax = (int)(hmx >> 20), emin = (int)(hmn >> 20);
      sc = (emax == 2047) ? 0 : ((emax == 0) ? 1000 : max(-1000, min(1000, (1023 + 16) - emax)));
      fs = (emin >= 1) && (emax >= 239) && (emax <= 1935) && (emax - emin <= 119);
    };
    scale_of(hmax, hmin, wscale, fast);
    if (ADJ) scale_of(xhmax, xhmin, xscale, xfast);
  }

  // ---------------------------------------------------------------- local sweeps (a1)
  float2 Xh, Xl;
  if (full && fast && n == 16)
    sweep_pair<LD, false, true, 16>(S, tid, nrow, nb0, nb1, wscale, pp, Xh, Xl);
  else if (full && fast)
    sweep_pair<LD, false, true>(S, tid, nrow, nb0, nb1, wscale, pp, Xh, Xl);
  else if (full)
    sweep_pair<LD, false, false>(S, tid, nrow, nb0, nb1, wscale, pp, Xh, Xl);
  else
    sweep_pair<LD, true, false>(S, tid, nrow, nb0, nb1, wscale, pp, Xh, Xl);

  // Per-block quantities and the tree advance the thread's two blocks (or the prefix and the
  // suffix scan) together in packed float-float pairs (ff2: lane x = block 2t, lane y = block
  // 2t+1); inactive blocks enter as zero values and identity maps.
  const ff2 zero2{f2(0.f), f2(0.f)}, one2{f2(1.f), f2(0.f)};

  // block-end quantities: xp(-1) = g ib X_0, alpha = xp_0 - xp(-1) v_0, omega = xp_{n-1} - xp(-1) v_{n-1}
  ff2 xm, al, om;
  {
    const ffv v0f{pp->v0_h, pp->v0_l}, v0l{pp->v0l_h, pp->v0l_l}, vef{pp->vend_h, pp->vend_l},
        vel{pp->vendl_h, pp->vendl_l};
    const ff2 v0 = ff2_pair(last0 ? v0l : v0f, last1 ? v0l : v0f);
    const ff2 ve = ff2_pair(last0 ? vel : vef, last1 ? vel : vef);
    xm = ff2_mul(ff2_bcast(ffv{pp->gib_h, pp->gib_l}), ff2_make(Xh, Xl));
    const float4 q0 = *reinterpret_cast<const float4*>(S + 2 * tid);
    const float4 qe0 = *reinterpret_cast<const float4*>(S + (size_t)max(nb0 - 1, 0) * LD + 2 * tid);
    const float4 qe1 = *reinterpret_cast<const float4*>(S + (size_t)max(nb1 - 1, 0) * LD + 2 * tid);
    al = ff2_sub(ff2_make(make_float2(q0.x, q0.y), make_float2(q0.z, q0.w)), ff2_mul(xm, v0));
    om = ff2_sub(ff2_make(make_float2(qe0.x, qe1.y), make_float2(qe0.z, qe1.w)), ff2_mul(xm, ve));
  }

  // ---------------------------------------------------------------- beta (eq. 16)
  const Recs2 bc2 = recs2(pp, tab, P, act0, act1, mb0, mb1);
  const ff2 bL = ff2_sel(act0, act1, ff2_fma(bc2(BC_M00), al, ff2_mul(bc2(BC_M01), om)), zero2);
  const ff2 bR = ff2_sel(act0, act1, ff2_fma(bc2(BC_M10), al, ff2_mul(bc2(BC_M11), om)), zero2);

  if (A.mode == MODE_BETA) {  // general path: beta leaves the window as unscaled FP64
    const double dn = pow2i(-wscale);
    if (act0) {
      A.beta[2 * (pp->gboff + mb0)] = ff_to_double(ff2_x(bL)) * dn;
      A.beta[2 * (pp->gboff + mb0) + 1] = ff_to_double(ff2_x(bR)) * dn;
    }
    if (act1) {
      A.beta[2 * (pp->gboff + mb1)] = ff_to_double(ff2_y(bL)) * dn;
      A.beta[2 * (pp->gboff + mb1) + 1] = ff_to_double(ff2_y(bR)) * dn;
    }
    return;
  }

  ffv XL0 = ff_zero(), XR0 = ff_zero(), XL1 = ff_zero(), XR1 = ff_zero();
  if (A.mode == MODE_FULL) {
    tree2<NT>(bc2, act0, act1, mb0, mb1, P, nwin, tid, bL, bR, swv, sbd, XL0, XR0, XL1, XR1, pp->lev);
  } else {  // MODE_APPLY: neighbours' first/last values from the global scan (unscaled FP64)
    const double upw = pow2i(wscale);
    auto to_ff = [&](double d) {
      const float2 t = f64_to_ff_rn(d * upw);
      return ffv{t.x, t.y};
    };
    if (act0) {
      if (mb0 > 0) XL0 = to_ff(A.iface[2 * (pp->gboff + mb0 - 1) + 1]);
      if (mb0 < P - 1) XR0 = to_ff(A.iface[2 * (pp->gboff + mb0 + 1)]);
    }
    if (act1) {
      if (mb1 > 0) XL1 = to_ff(A.iface[2 * (pp->gboff + mb1 - 1) + 1]);
      if (mb1 < P - 1) XR1 = to_ff(A.iface[2 * (pp->gboff + mb1 + 1)]);
    }
  }

  // ---------------------------------------------------------------- correction (a3), per column
  const ff2 cL = ff2_sub(ff2_pair(XL0, XL1), xm), cR = ff2_pair(XR0, XR1);
  const float2* tvl_g = reinterpret_cast<const float2*>(tab) + pp->o_vlf;    // last block's spikes
  const float2* twl_g = reinterpret_cast<const float2*>(tab) + pp->o_wlf;
  // blocks of the halo are not stored: a thread whose two blocks both lie in it skips the correction
  const bool owns = (b1 >= hl) && (b0 < hl + nown);
  if (!owns) {
  } else if (full && fast && n == 16)
    correct_pair<LD, false, true, 16, ADJ>(S, tid, nrow, nb0, nb1, last0, last1, n, tv4, tw4, tvl_g, twl_g, cL, cR,
                                  wscale);
  else if (full && fast)
    correct_pair<LD, false, true, 0, ADJ>(S, tid, nrow, nb0, nb1, last0, last1, n, tv4, tw4, tvl_g, twl_g, cL, cR,
                                  wscale);
  else if (full)
    correct_pair<LD, false, false, 0, ADJ>(S, tid, nrow, nb0, nb1, last0, last1, n, tv4, tw4, tvl_g, twl_g, cL, cR,
                                  wscale);
  else if (nrow > 0)
    correct_pair<LD, true, false, 0, ADJ>(S, tid, nrow, nb0, nb1, last0, last1, n, tv4, tw4, tvl_g, twl_g, cL, cR,
                                  wscale);
  __syncthreads();

  // the next kernel of the stream may begin its launch (it waits for this grid to complete)
  asm volatile("griddepcontrol.launch_dependents;");
  // ---------------------------------------------------------------- coalesced store of the own rows
  unsigned bad = 0u;
  const int64_t N = pp->N;
  const int jlo = hl * n;
  const int jhi = min(len, (hl + nown) * n);
  double* dst = A.x + (int64_t)blockIdx.y * A.ldx + off + row_lo;
  auto nonfinite = [](double d) { return ((__double2hiint(d) >> 20) & 0x7FF) == 0x7FF; };
  if constexpr (!ADJ) {
    // rows j, j + 1 (j even) of one block (column b, rows i, i + 1 of the tile): one 16-byte store
    auto put2 = [&](int j, const double* col) {
      const double d0 = col[0];
      if (j + 1 < jhi) {
        const double d1 = col[LD];
        __stcs(reinterpret_cast<double2*>(dst + j), make_double2(d0, d1));
        if (A.check_finite && (nonfinite(d0) || nonfinite(d1))) bad = 1u;
      } else {
        __stcs(dst + j, d0);
        if (A.check_finite && nonfinite(d0)) bad = 1u;
      }
    };
    if (n == 16 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0u) {
      // jlo is a multiple of 16: row 2 (tid % 8) of block hl + tid / 8 + k NT / 8, fixed strides
      const double* col = S + (size_t)(2 * (tid & 7)) * LD + hl + (tid >> 3);
#pragma unroll 2
      for (int j = jlo + 2 * tid; j < jhi; j += 2 * NT, col += NT / 8) put2(j, col);
    } else if ((n & 1) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0u) {
      int b = (jlo + 2 * tid) / n, i = (jlo + 2 * tid) - ((jlo + 2 * tid) / n) * n;
      const int db = (2 * NT) / n, di = (2 * NT) - ((2 * NT) / n) * n;
      for (int j = jlo + 2 * tid; j < jhi; j += 2 * NT) {
        put2(j, S + (size_t)i * LD + b);
        i += di;
        b += db;
        if (i >= n) {
          i -= n;
          ++b;
        }
      }
    } else {
      int b = (jlo + tid) / n, i = (jlo + tid) - ((jlo + tid) / n) * n;
      const int db = NT / n, di = NT - (NT / n) * n;
      for (int j = jlo + tid; j < jhi; j += NT) {
        const double dv = S[(size_t)i * LD + b];
        __stcs(dst + j, dv);
        if (A.check_finite && nonfinite(dv)) bad = 1u;
        i += di;
        b += db;
        if (i >= n) {
          i -= n;
          ++b;
        }
      }
    }
    if (bad) atomicOr(A.status, (unsigned)ST_NONFINITE);
  } else {
    // The adjoint: the tile holds lambda as float-float pairs (window scale 2^wscale); the store
    // joins them, and the gradient sums (a5) -- sum_r lambda_r x_{r-1}, x_r, x_{r+1} over the own
    // rows -- are accumulated from the same pairs.  Where the forward solution x qualifies for the
    // fast split with its own power-of-two scale (all rows the sums read normal and within 2^119
    // of each other), each product is formed error-free in FP32 (FMA) and summed with TwoSum into
    // packed float-float accumulators (units 2^(wscale + xscale)); otherwise the FP64 pipe takes
    // the products.
    const FastK fk = fast_k(wscale), fkx = fast_k(xscale);
    float2 s0h = f2(0.f), s0l = f2(0.f), smh = f2(0.f), sml = f2(0.f), sph = f2(0.f), spl = f2(0.f);
    double g0 = 0.0, gm = 0.0, gp = 0.0;
    double g0b = 0.0, gmb = 0.0, gpb = 0.0;   // second FP64 set: independent chains
    struct X4 {
      double a, b, c, d;   // x_{r-1}, x_r, x_{r+1}, x_{r+2}
    };
    // x rows of the pair at row r; rows outside the system read row r instead (masked later)
    auto loadx = [&](int j) {
      const int64_t r = row_lo + j;
      const double* xr = A.xf + off + r;
      return X4{__ldg(xr + ((r > 0) ? -1 : 0)), __ldg(xr), __ldg(xr + ((r + 1 < N) ? 1 : 0)),
                __ldg(xr + ((r + 2 < N) ? 2 : 0))};
    };
    // one instantiation per (join form, product form): no FP64 work of the other form is
    // if-converted into the loop
    auto body = [&](auto fj_, auto xf_) {
      constexpr bool FJ = decltype(fj_)::value, XF = decltype(xf_)::value;
      auto join = [&](float2 v) {
        if constexpr (FJ)
          return join_fast(v.x, v.y, fk);
        else
          return join_dadd(v.x, v.y, wscale);
      };
      auto take = [&](double dv, int j) {
        if (A.check_finite && nonfinite(dv)) bad = 1u;
        const int64_t r = row_lo + j;
        const double* xr = A.xf + off + r;
        g0 = fma(dv, xr[0], g0);
        if (r > 0) gm = fma(dv, xr[-1], gm);
        if (r + 1 < N) gp = fma(dv, xr[1], gp);
      };
      // float-float products of rows r (lane x) and r + 1 (lane y; v1 = 0 for a lone row)
      auto ffrow = [&](int64_t r, float2 v0, float2 v1, const X4& xq) {
        float ha, la, h0, l0, h1, l1, hb, lb;
        split_fast(xq.a, fkx, ha, la);
        split_fast(xq.b, fkx, h0, l0);
        split_fast(xq.c, fkx, h1, l1);
        split_fast(xq.d, fkx, hb, lb);
        if (r == 0) ha = la = 0.f;
        if (r + 1 >= N) h1 = l1 = 0.f;
        if (r + 2 >= N) hb = lb = 0.f;
        const float2 ah = make_float2(v0.x, v1.x), al = make_float2(v0.y, v1.y);
        ff_fma_acc2(ah, al, make_float2(h0, h1), make_float2(l0, l1), s0h, s0l);
        ff_fma_acc2(ah, al, make_float2(ha, h0), make_float2(la, l0), smh, sml);
        ff_fma_acc2(ah, al, make_float2(h1, hb), make_float2(l1, lb), sph, spl);
      };
      // rows j, j + 1 (j even) of one block: col[0], col[LD] hold their (h, l) pairs
      auto put2 = [&](int j, const double* col, const X4& xq) {
        const float2 v0 = *reinterpret_cast<const float2*>(col);
        if (j + 1 < jhi) {
          const float2 v1 = *reinterpret_cast<const float2*>(col + LD);
          const double d0 = join(v0), d1 = join(v1);
          __stcs(reinterpret_cast<double2*>(dst + j), make_double2(d0, d1));
          if (A.check_finite && (nonfinite(d0) || nonfinite(d1))) bad = 1u;
          const int64_t r = row_lo + j;
          if constexpr (XF) {
            ffrow(r, v0, v1, xq);
          } else {
            g0 = fma(d0, xq.b, g0);
            gm = fma(d0, (r > 0) ? xq.a : 0.0, gm);
            gp = fma(d0, xq.c, gp);
            g0b = fma(d1, xq.c, g0b);
            gmb = fma(d1, xq.b, gmb);
            gpb = fma(d1, (r + 2 < N) ? xq.d : 0.0, gpb);
          }
        } else {
          const double d0 = join(v0);
          __stcs(dst + j, d0);
          if constexpr (XF) {
            if (A.check_finite && nonfinite(d0)) bad = 1u;
            ffrow(row_lo + j, v0, make_float2(0.f, 0.f), xq);
          } else {
            take(d0, j);
          }
        }
      };
      if (n == 16 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0u) {
        // the x rows of the next pair are loaded one step ahead
        const double* col = S + (size_t)(2 * (tid & 7)) * LD + hl + (tid >> 3);
        int j = jlo + 2 * tid;
        X4 xq{0.0, 0.0, 0.0, 0.0};
        if (j < jhi) xq = loadx(j);
#pragma unroll 1
        for (; j < jhi; j += 2 * NT, col += NT / 8) {
          const X4 cur = xq;
          if (j + 2 * NT < jhi) xq = loadx(j + 2 * NT);
          put2(j, col, cur);
        }
      } else if ((n & 1) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0u) {
        int b = (jlo + 2 * tid) / n, i = (jlo + 2 * tid) - ((jlo + 2 * tid) / n) * n;
        const int db = (2 * NT) / n, di = (2 * NT) - ((2 * NT) / n) * n;
        for (int j = jlo + 2 * tid; j < jhi; j += 2 * NT) {
          put2(j, S + (size_t)i * LD + b, loadx(j));
          i += di;
          b += db;
          if (i >= n) {
            i -= n;
            ++b;
          }
        }
      } else {
        int b = (jlo + tid) / n, i = (jlo + tid) - ((jlo + tid) / n) * n;
        const int db = NT / n, di = NT - (NT / n) * n;
        for (int j = jlo + tid; j < jhi; j += NT) {
          const float2 v = *reinterpret_cast<const float2*>(S + (size_t)i * LD + b);
          const double dv = join(v);
          __stcs(dst + j, dv);
          if constexpr (XF) {
            if (A.check_finite && nonfinite(dv)) bad = 1u;
            ffrow(row_lo + j, v, make_float2(0.f, 0.f), loadx(j));
          } else {
            take(dv, j);
          }
          i += di;
          b += db;
          if (i >= n) {
            i -= n;
            ++b;
          }
        }
      }
    };
    if (fast) {
      if (xfast)
        body(std::true_type(), std::true_type());
      else
        body(std::true_type(), std::false_type());
    } else {
      if (xfast)
        body(std::false_type(), std::true_type());
      else
        body(std::false_type(), std::false_type());
    }
    if (bad) atomicOr(A.status, (unsigned)ST_NONFINITE);
    __syncthreads();   // the scan scratch takes the per-warp sums
    if (xfast) {
      // float-float sums (FP32 pipes): the thread's two lanes, the warp, the CTA; one join to
      // FP64 per sum, in units 2^wscale, then the exact power of two 2^-wscale
      ffv a[3] = {ff_add(ffv{smh.x, sml.x}, ffv{smh.y, sml.y}), ff_add(ffv{s0h.x, s0l.x}, ffv{s0h.y, s0l.y}),
                  ff_add(ffv{sph.x, spl.x}, ffv{sph.y, spl.y})};
#pragma unroll
      for (int d = 16; d > 0; d >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] = ff_add(a[k], ff_shfl_down(a[k], d));
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) swv[k * NW + wid] = a[k];
      __syncthreads();
      if (tid < 3) {
        ffv sum = ff_zero();
        for (int w = 0; w < NW; ++w) sum = ff_add(sum, swv[tid * NW + w]);
        A.part[3 * (size_t)blockIdx.x + tid] = join_dadd(sum.h, sum.l, xscale) * pow2i(-wscale);
      }
    } else {
      g0 += g0b;
      gm += gmb;
      gp += gpb;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        g0 += __shfl_down_sync(0xffffffffu, g0, d);
        gm += __shfl_down_sync(0xffffffffu, gm, d);
        gp += __shfl_down_sync(0xffffffffu, gp, d);
      }
      double* sred = reinterpret_cast<double*>(swv);
      if (lane == 0) {
        sred[wid] = gm;
        sred[NW + wid] = g0;
        sred[2 * NW + wid] = gp;
      }
      __syncthreads();
      if (tid < 3) {
        double sum = 0.0;
        for (int w = 0; w < NW; ++w) sum += sred[tid * NW + w];
        A.part[3 * (size_t)blockIdx.x + tid] = sum;
      }
    }
  }
}

}  // namespace dich
