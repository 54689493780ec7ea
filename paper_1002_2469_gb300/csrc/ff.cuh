// ff.cuh -- float-float (double-FP32) helpers for the MIXED form of the Dichotomy sweeps.
//
// On GB300 the FP64 pipe issues about 1.6 operations per clock per SM (and FP64<->FP32
// conversions run on it too), against about 110 FP32 FMAs.  The MIXED form therefore
// keeps every per-element operation on the FP32/INT pipes:
//   - FP64 input -> (hi, lo) floats with integer bit operations (no conversion unit),
//   - the first-order recurrences in compensated FP32 arithmetic (error-free product
//     by FMA, Knuth's TwoSum, the rounding errors carried in a second float),
//   - (hi, lo) -> FP64 output: exact float->double by bit operations plus one FP64 add.
// All arithmetic uses the explicit __f*_rn intrinsics so the compiler can neither fuse
// nor reassociate the error-free transformations.
#pragma once
#include <cstdint>

namespace dich {

// p + e = a * b exactly
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// s + e = a + b exactly (Knuth; no ordering assumption)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// FP64 -> float-float with correct rounding of hi (FP64 pipe; used once per block only)
__device__ __forceinline__ float2 f64_to_ff_rn(double d) {
  const float h = __double2float_rn(d);
  const float l = __double2float_rn(__dsub_rn(d, (double)h));
  return make_float2(h, l);
}

// ---------------------------------------------------------------- float-float values for the
// per-block quantities and the dichotomy tree of the MIXED form (normalised: |l| <= ulp(h)/2)
struct ffv {
  float h, l;
};

__device__ __forceinline__ ffv ff_make(float h, float l) {  // FastTwoSum renormalisation
  const float s = __fadd_rn(h, l);
  return ffv{s, __fsub_rn(l, __fsub_rn(s, h))};
}
// a (hi, lo) pair of the plan's float tables: the host splits each FP64 entry as hi = float(d),
// lo = float(d - hi), already normalised, so the pair is taken as it is
__device__ __forceinline__ ffv ff_of(float2 v) { return ffv{v.x, v.y}; }
__device__ __forceinline__ ffv ff_zero() { return ffv{0.f, 0.f}; }
__device__ __forceinline__ ffv ff_one() { return ffv{1.f, 0.f}; }
__device__ __forceinline__ ffv ff_neg(ffv a) { return ffv{-a.h, -a.l}; }

__device__ __forceinline__ ffv ff_add(ffv a, ffv b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return ff_make(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ffv ff_sub(ffv a, ffv b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ffv ff_mul(ffv a, ffv b) {
  float p, e;
  two_prod(a.h, b.h, p, e);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return ff_make(p, e);
}

// a * b + c
__device__ __forceinline__ ffv ff_fma(ffv a, ffv b, ffv c) {
  float p, e, s, f;
  two_prod(a.h, b.h, p, e);
  two_sum(p, c.h, s, f);
  float lo = __fadd_rn(__fadd_rn(e, f), c.l);
  lo = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, lo));
  return ff_make(s, lo);
}

__device__ __forceinline__ ffv ff_shfl_up(ffv a, int d) {
  return ffv{__shfl_up_sync(0xffffffffu, a.h, d), __shfl_up_sync(0xffffffffu, a.l, d)};
}
__device__ __forceinline__ ffv ff_shfl_down(ffv a, int d) {
  return ffv{__shfl_down_sync(0xffffffffu, a.h, d), __shfl_down_sync(0xffffffffu, a.l, d)};
}
__device__ __forceinline__ double ff_to_double(ffv a) { return (double)a.h + (double)a.l; }

// ---------------------------------------------------------------- packed (two-chain) helpers
// The MIXED window kernel advances two blocks per thread; both chains go through one
// f32x2 instruction (sm_100+ FFMA2/FADD2/FMUL2: half the issue slots of scalar FP32).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// two chains of y ~= f + r * x, with f, x, y as (hi pair, lo pair) and r a float-float scalar:
// the rounding errors of the leading product (FMA) and sum (TwoSum) are kept exactly and
// accumulated, with the cross terms, in the unnormalised low part
__device__ __forceinline__ void ff_axpy2(float2 fh, float2 fl, float2 rh, float2 rl, float2 xh, float2 xl,
                                         float2& yh, float2& yl) {
  const float2 pn = mul2(make_float2(-rh.x, -rh.y), xh);
  const float2 pe = fma2(rh, xh, pn);
  const float2 s = sub2(fh, pn);
  const float2 bb = sub2(s, fh);
  const float2 se = sub2(sub2(fh, sub2(s, bb)), add2(pn, bb));
  float2 c = add2(fl, add2(pe, se));
  c = fma2(rl, xh, c);
  c = fma2(rh, xl, c);
  yh = s;
  yl = c;
}

// two chains of y ~= g * x (error-free leading product plus cross terms)
__device__ __forceinline__ void ff_mul2(float2 gh, float2 gl, float2 xh, float2 xl, float2& yh, float2& yl) {
  const float2 p = mul2(gh, xh);
  float2 c = fma2(gh, xh, mul2(make_float2(-gh.x, -gh.y), xh));
  c = fma2(gl, xh, c);
  c = fma2(gh, xl, c);
  yh = p;
  yl = c;
}

// two chains of x += c * v, c and v float-float (per chain)
__device__ __forceinline__ void ff_fma_acc2(float2 ch, float2 cl, float2 vh, float2 vl, float2& xh, float2& xl) {
  const float2 pn = mul2(make_float2(-ch.x, -ch.y), vh);
  const float2 pe = fma2(ch, vh, pn);
  const float2 pc = fma2(cl, vh, fma2(ch, vl, pe));
  const float2 s = sub2(xh, pn);
  const float2 bb = sub2(s, xh);
  const float2 se = sub2(sub2(xh, sub2(s, bb)), add2(pn, bb));
  xl = add2(xl, add2(pc, se));
  xh = s;
}

// ---------------------------------------------------------------- packed float-float pairs
// ff2 holds two float-float values, one per block of a thread's pair (lane x: block 2t, lane y:
// block 2t+1), so the per-block quantities and the tree advance both blocks -- or the prefix
// and the suffix scan -- with one f32x2 instruction per step.  Same arithmetic as ffv.
struct ff2 {
  float2 h, l;
};
__device__ __forceinline__ ff2 ff2_make(float2 h, float2 l) {  // FastTwoSum renormalisation
  const float2 s = add2(h, l);
  return ff2{s, sub2(l, sub2(s, h))};
}
__device__ __forceinline__ ff2 ff2_pair(ffv a, ffv b) { return ff2{make_float2(a.h, b.h), make_float2(a.l, b.l)}; }
__device__ __forceinline__ ffv ff2_x(const ff2& a) { return ffv{a.h.x, a.l.x}; }
__device__ __forceinline__ ffv ff2_y(const ff2& a) { return ffv{a.h.y, a.l.y}; }
__device__ __forceinline__ ff2 ff2_bcast(ffv a) { return ff2{f2(a.h), f2(a.l)}; }
__device__ __forceinline__ ff2 ff2_add(const ff2& a, const ff2& b) {
  const float2 s = add2(a.h, b.h);
  const float2 bb = sub2(s, a.h);
  const float2 e = add2(sub2(a.h, sub2(s, bb)), sub2(b.h, bb));
  return ff2_make(s, add2(e, add2(a.l, b.l)));
}
__device__ __forceinline__ ff2 ff2_sub(const ff2& a, const ff2& b) {
  const float2 s = sub2(a.h, b.h);
  const float2 bb = sub2(s, a.h);
  const float2 e = sub2(sub2(a.h, sub2(s, bb)), add2(b.h, bb));
  return ff2_make(s, add2(e, sub2(a.l, b.l)));
}
__device__ __forceinline__ ff2 ff2_mul(const ff2& a, const ff2& b) {
  const float2 p = mul2(a.h, b.h);
  float2 e = fma2(a.h, b.h, make_float2(-p.x, -p.y));
  e = fma2(a.h, b.l, fma2(a.l, b.h, e));
  return ff2_make(p, e);
}
// a * b + c
__device__ __forceinline__ ff2 ff2_fma(const ff2& a, const ff2& b, const ff2& c) {
  const float2 p = mul2(a.h, b.h);
  const float2 e = fma2(a.h, b.h, make_float2(-p.x, -p.y));
  const float2 s = add2(p, c.h);
  const float2 bb = sub2(s, p);
  const float2 f = add2(sub2(p, sub2(s, bb)), sub2(c.h, bb));
  float2 lo = add2(add2(e, f), c.l);
  lo = fma2(a.h, b.l, fma2(a.l, b.h, lo));
  return ff2_make(s, lo);
}
// error-free renormalisation of a pair whose low part may exceed half an ulp of its high part
// (TwoSum: no ordering of |h| and |l| assumed)
__device__ __forceinline__ ff2 ff2_renorm(const ff2& a) {
  const float2 s = add2(a.h, a.l);
  const float2 bb = sub2(s, a.h);
  return ff2{s, add2(sub2(a.h, sub2(s, bb)), sub2(a.l, bb))};
}
// per-lane choice: lane x from a if px else from b, lane y likewise
__device__ __forceinline__ ff2 ff2_sel(bool px, bool py, const ff2& a, const ff2& b) {
  return ff2{make_float2(px ? a.h.x : b.h.x, py ? a.h.y : b.h.y), make_float2(px ? a.l.x : b.l.x, py ? a.l.y : b.l.y)};
}

// rare paths kept out of line so that their FP64 operations are not if-converted into the
// per-element code (GB300's FP64 pipe is ~70x slower than FP32)
static __device__ __noinline__ double rescale_subnormal(double d) { return d * 18446744073709551616.0; }  // * 2^64

// FP64 -> (hi, lo) floats of d * 2^s with integer operations.
// hi = leading 24 bits (truncated), lo = next 23 bits (truncated); values whose scaled
// exponent falls outside the float range flush to zero (hi) / drop lo, exponents of
// Inf/NaN give Inf/NaN.  Subnormal FP64 inputs are rescaled exactly first (rare path).
__device__ __forceinline__ void split_sc(double d, int s, float& hi, float& lo) {
  unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
  int sb = s - 896;
  if ((hw & 0x7FF00000u) == 0u && ((hw & 0x000FFFFFu) | lw) != 0u) {   // FP64 subnormal
    const double d2 = rescale_subnormal(d);                            // * 2^64, exact
    hw = (unsigned)__double2hiint(d2);
    lw = (unsigned)__double2loint(d2);
    sb -= 64;
  }
  const unsigned sgn = hw & 0x80000000u;
  const int E0 = (int)((hw >> 20) & 0x7FFu);
  const int ef = E0 + sb;                                             // float exponent of hi
  const unsigned m23 = __funnelshift_l(lw, hw, 3) & 0x7FFFFFu;        // 23 fraction bits
  unsigned hib = sgn | ((unsigned)ef << 23) | m23;
  const bool in_range = ((unsigned)(ef - 1) < 254u) && (E0 != 0);
  if (!in_range) hib = (E0 == 2047) ? (sgn | 0x7F800000u | (m23 ? 0x400000u : 0u)) :
                                      ((ef > 254 && E0 != 0) ? (sgn | 0x7F800000u) : sgn);
  const float rf = __fsub_rn(__uint_as_float(0x4B000000u | ((lw >> 6) & 0x7FFFFFu)), 8388608.0f);
  const int es = ef - 46;                                             // exponent of the lo scale
  const float sc = __uint_as_float((unsigned)es << 23);
  float l = __fmul_rn(rf, sc);
  l = ((unsigned)(es - 1) < 254u && in_range) ? l : 0.0f;
  hi = __uint_as_float(hib);
  lo = __uint_as_float(__float_as_uint(l) | sgn);
}

// exact (h, l) * 2^-s on the FP64 pipe, out of line (rare cases of the joins below); the FP64
// unit rounds into the subnormal range correctly
static __device__ __noinline__ double join_slow(float h, float l, int s) {
  const double sc = __hiloint2double((1023 - s) << 20, 0);
  return (double)h * sc + (double)l * sc;
}

// ---------------------------------------------------------------- fast windows
// A window is "fast" when every |F| of it is a normal FP64 number whose exponent lies within
// 119 of the window's largest (emax) and emax is in [239, 1935] (the window scale is then
// s = 1039 - emax, inside [-896, 800]).  In such a window the split and the join below need
// no range handling: every scaled float exponent and every rebuilt FP64 exponent is in range.

// constants of a fast window with scale s
struct FastK {
  unsigned split;   // added to the funnel-shifted FP64 bits: float exponent of hi, minus 23
  unsigned join;    // added to a float's shifted bits: FP64 exponent rebias (896 - s) << 20
};
__device__ __forceinline__ FastK fast_k(int s) {
  return FastK{(unsigned)(s - 896 - 23) << 23, (unsigned)(896 - s) << 20};
}

// d * 2^s -> (hi, lo) in a fast window: hi = leading 24 significant bits, lo = next 23 (both
// truncated).  The float exponent of hi, ef = 143 - (emax - E), is in [24, 143]:
//   T  = sign | (ef - 23) << 23 | m23    (nine low exponent bits of d shifted in, rebiased mod 2^8)
//   hi = T + 23 << 23
//   lo = (T's sign/exponent | next 23 fraction bits) - (T's sign/exponent), exact (Sterbenz).
__device__ __forceinline__ void split_fast(double d, const FastK& k, float& hi, float& lo) {
  const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
  const unsigned x = __funnelshift_l(lw, hw, 3);
  const unsigned t = ((x + k.split) & 0x7FFFFFFFu) | (hw & 0x80000000u);
  const unsigned b = t & 0xFF800000u;
  hi = __uint_as_float(t + (23u << 23));
  lo = __fsub_rn(__uint_as_float(b | ((lw >> 6) & 0x7FFFFFu)), __uint_as_float(b));
}

// split_fast in a window whose largest |F| qualifies (emax in [239, 1935], no Inf/NaN) while some of
// its values lie further than 2^119 below it (zeros and subnormals included -- the usual shape of a
// spectrum that decays over hundreds of decades): those values, whose FP64 high word (sign cleared)
// is below hlo = (emax - 119) << 20, become (0, 0).  They are below 2^-103 of the window's largest
// |F| in window units -- under the floor the conversions already put under the error (values below
// 2^-126 window units are not resolved) -- so the window keeps the fast conversions.
__device__ __forceinline__ void split_fast_flush(double d, const FastK& k, unsigned hlo, float& hi, float& lo) {
  split_fast(d, k, hi, lo);
  if (((unsigned)__double2hiint(d) & 0x7FFFFFFFu) < hlo) hi = lo = 0.f;
}

// (h, l) * 2^-s -> FP64 in a fast window: both floats rebuilt as exact FP64 bit patterns and
// added once on the FP64 pipe.  A float's bits shifted right by 3 (sign kept) give the FP64
// fraction and exponent fields; adding (896 - s) << 20 rebiases and unscales the exponent,
// which stays inside [1, 2046] for every normal float because s is in [-896, 800].  No part is
// tested: a zero or subnormal part is rebuilt as if its exponent field were that of a normal
// float, i.e. as a value of magnitude below 2^-126 in window units -- at most 2^-141 of the
// window's largest |F| for both parts together, far inside the form's norm-wise error -- so the
// per-row loops carry neither branches nor selects.
__device__ __forceinline__ double join_fast(float h, float l, const FastK& k) {
  const unsigned bh = __float_as_uint(h), bl = __float_as_uint(l);
  const unsigned hh = ((unsigned)((int)bh >> 3) & 0x8FFFFFFFu) + k.join;
  const unsigned lh = ((unsigned)((int)bl >> 3) & 0x8FFFFFFFu) + k.join;
  return __dadd_rn(__hiloint2double((int)hh, (int)(bh << 29)), __hiloint2double((int)lh, (int)(bl << 29)));
}

// (h, l) * 2^-s -> FP64 in any window: both parts converted exactly by integer operations and
// one FP64 addition.  Anything outside the plain case -- a zero or subnormal leading part,
// a part whose unscaled exponent leaves the FP64 normal range, Inf/NaN -- takes the
// out-of-line FP64 path, which rounds into the subnormal range correctly.
__device__ __forceinline__ double join_dadd(float h, float l, int s) {
  const unsigned bh = __float_as_uint(h), bl = __float_as_uint(l);
  const int eh = (int)((bh >> 23) & 0xFFu), el = (int)((bl >> 23) & 0xFFu);
  const int edh = eh + 896 - s, edl = el + 896 - s;
  const bool okh = ((unsigned)(edh - 1) < 2046u) && ((unsigned)(eh - 1) < 254u);
  const bool okl = (el == 0) || (((unsigned)(edl - 1) < 2046u) && (el != 255));
  if (!(okh && okl)) return join_slow(h, l, s);
  const unsigned mh = bh & 0x7FFFFFu, ml = bl & 0x7FFFFFu;
  const double hd = __hiloint2double((int)((bh & 0x80000000u) | ((unsigned)edh << 20) | (mh >> 3)), (int)(mh << 29));
  const double ld = (el == 0) ? 0.0
                              : __hiloint2double((int)((bl & 0x80000000u) | ((unsigned)edl << 20) | (ml >> 3)),
                                                 (int)(ml << 29));
  return __dadd_rn(hd, ld);
}

}  // namespace dich
