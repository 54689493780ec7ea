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

// (yh, yl) ~= (fh + fl) + (rh + rl) * (xh + xl), rounding errors of the leading terms kept
// exactly and accumulated in yl (unnormalised float-float).
__device__ __forceinline__ void ff_axpy(float fh, float fl, float rh, float rl, float xh, float xl,
                                        float& yh, float& yl) {
  float p, pe, s, se;
  two_prod(rh, xh, p, pe);
  two_sum(fh, p, s, se);
  float c = __fadd_rn(fl, __fadd_rn(pe, se));
  c = __fmaf_rn(rl, xh, c);
  c = __fmaf_rn(rh, xl, c);
  yh = s;
  yl = c;
}

// (yh, yl) ~= (gh + gl) * (xh + xl)
__device__ __forceinline__ void ff_mul(float gh, float gl, float xh, float xl, float& yh, float& yl) {
  float p, pe;
  two_prod(gh, xh, p, pe);
  float c = __fmaf_rn(gl, xh, pe);
  c = __fmaf_rn(gh, xl, c);
  yh = p;
  yl = c;
}

// (xh, xl) += (ch + cl) * (vh + vl)
__device__ __forceinline__ void ff_fma_acc(float ch, float cl, float vh, float vl, float& xh, float& xl) {
  float p, pe, s, se;
  two_prod(ch, vh, p, pe);
  float pc = __fmaf_rn(cl, vh, __fmaf_rn(ch, vl, pe));
  two_sum(xh, p, s, se);
  xl = __fadd_rn(xl, __fadd_rn(pc, se));
  xh = s;
}

// FP64 -> (hi, lo) by integer operations.  hi keeps the leading 24 significant bits
// (truncated), lo the next 23 (truncated), so |d - hi - lo| < 2^-46 |d|.  Valid for
// 2^-80 <= |d| < 2^127; below 2^-80 lo is dropped, below 2^-126 the value flushes to 0,
// above 2^127 (and Inf/NaN) hi becomes Inf/NaN so the output is flagged non-finite.
__device__ __forceinline__ float2 f64_to_ff(double d) {
  const unsigned hw = (unsigned)__double2hiint(d);
  const unsigned lw = (unsigned)__double2loint(d);
  const unsigned sgn = hw & 0x80000000u;
  const int E = (int)((hw >> 20) & 0x7FFu);
  const unsigned m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const int ef = E - 896;
  unsigned hib = sgn | ((unsigned)ef << 23) | m23;
  if (ef < 1) hib = sgn;
  if (ef > 254) hib = sgn | 0x7F800000u | ((E == 2047 && ((hw & 0xFFFFFu) | lw)) ? 0x400000u : 0u);
  const unsigned r = lw & 0x1FFFFFFFu;
  const float rf = __fsub_rn(__uint_as_float(0x4B000000u | (r >> 6)), 8388608.0f);
  const int es = E - 942;
  float lo = (es >= 1 && ef <= 254) ? __fmul_rn(rf, __uint_as_float((unsigned)es << 23)) : 0.0f;
  lo = __uint_as_float(__float_as_uint(lo) | sgn);
  return make_float2(__uint_as_float(hib), lo);
}

// Scaled split: the same as f64_to_ff for d * 2^s (s chosen per window so that the largest
// |F| of the window sits near 2^16); exact in the scaling, no FP64 operation.
__device__ __forceinline__ float2 f64_to_ff_sc(double d, int s) {
  const unsigned hw0 = (unsigned)__double2hiint(d);
  if (((hw0 >> 20) & 0x7FFu) == 0u && ((hw0 & 0x7FFFFFFFu) | (unsigned)__double2loint(d)) != 0u) {  // subnormal
    d = d * 18446744073709551616.0;   // * 2^64, exact
    s -= 64;
  }
  const unsigned hw = (unsigned)__double2hiint(d);
  const unsigned lw = (unsigned)__double2loint(d);
  const unsigned sgn = hw & 0x80000000u;
  const int E0 = (int)((hw >> 20) & 0x7FFu);
  const int E = E0 + s;
  const unsigned m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const int ef = E - 896;
  const bool special = (E0 == 2047);
  unsigned hib = sgn | ((unsigned)ef << 23) | m23;
  if (ef < 1 || E0 == 0) hib = sgn;
  if (ef > 254 || special) hib = sgn | 0x7F800000u | ((special && ((hw & 0xFFFFFu) | lw)) ? 0x400000u : 0u);
  const unsigned r = lw & 0x1FFFFFFFu;
  const float rf = __fsub_rn(__uint_as_float(0x4B000000u | (r >> 6)), 8388608.0f);
  const int es = E - 942;
  float lo = (es >= 1 && ef <= 254 && E0 != 0 && !special) ? __fmul_rn(rf, __uint_as_float((unsigned)es << 23))
                                                          : 0.0f;
  lo = __uint_as_float(__float_as_uint(lo) | sgn);
  return make_float2(__uint_as_float(hib), lo);
}

// exact float -> double by integer operations (denormal floats flush to signed zero)
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned m = b & 0x7FFFFFu;
  const unsigned ed = (e == 0u) ? 0u : ((e == 255u) ? 0x7FFu : e + 896u);
  const unsigned md = (e == 0u) ? 0u : m;
  const unsigned hi = s | (ed << 20) | (md >> 3);
  const unsigned lo = md << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// float * 2^-s -> double by integer operations (the window scale removed exactly; results
// below the FP64 normal range flush to signed zero)
__device__ __forceinline__ double f32_to_f64_bits_sc(float f, int s) {
  const unsigned b = __float_as_uint(f);
  const unsigned sg = b & 0x80000000u;
  const int e = (int)((b >> 23) & 0xFFu);
  const unsigned m = b & 0x7FFFFFu;
  int ed = e + 896 - s;
  unsigned md = m;
  if (e == 255 || ed >= 2047) {
    ed = 2047;
    md = (e == 255) ? m : 0u;
  }
  if (e == 0 || ed <= 0) {
    ed = 0;
    md = 0u;
  }
  const unsigned hi = sg | ((unsigned)ed << 20) | (md >> 3);
  const unsigned lo = md << 29;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double ff_to_f64_sc(float h, float l, int s) {
  return __dadd_rn(f32_to_f64_bits_sc(h, s), f32_to_f64_bits_sc(l, s));
}

// (h, l) -> FP64: both parts converted exactly, one FP64 addition.
__device__ __forceinline__ double ff_to_f64(float h, float l) {
  return __dadd_rn(f32_to_f64_bits(h), f32_to_f64_bits(l));
}

// (h, l) * 2^-s -> FP64 with integer operations only (no FP64 pipe).  (h, l) is first
// renormalised with TwoSum so |e| <= ulp(s1)/2; s1 gives the leading 24 bits of the double,
// e is aligned to the double's last bit and added to the 53-bit significand as an integer
// (bits of e below the double's ulp are truncated: error < 2 ulp of the result).
__device__ __forceinline__ double ff_to_f64_int(float h, float l, int s) {
  float s1, e1;
  two_sum(h, l, s1, e1);
  const unsigned b1 = __float_as_uint(s1);
  const unsigned sg = b1 & 0x80000000u;
  const int E1 = (int)((b1 >> 23) & 0xFFu);
  if (E1 == 0) return __hiloint2double((int)sg, 0);                 // zero (or float denormal)
  if (E1 == 255) return __hiloint2double((int)(sg | 0x7FF00000u | ((b1 & 0x7FFFFFu) ? 0x80000u : 0u)), 0);
  unsigned long long M = (1ull << 52) | ((unsigned long long)(b1 & 0x7FFFFFu) << 29);
  const unsigned be = __float_as_uint(e1);
  const int Ee = (int)((be >> 23) & 0xFFu);
  if (Ee != 0) {
    const unsigned long long Me = (unsigned long long)((be & 0x7FFFFFu) | 0x800000u);
    const int sh = Ee - E1 + 29;      // <= 5 because |e1| <= ulp(s1)/2
    unsigned long long K = 0ull;
    if (sh >= 0)
      K = Me << sh;
    else if (sh > -24)
      K = Me >> (-sh);
    M = ((be ^ b1) & 0x80000000u) ? M - K : M + K;
  }
  int Ed = E1 + 896 - s;
  if (M < (1ull << 52)) {             // borrow from an exact power of two: renormalise
    M <<= 1;
    Ed -= 1;
  }
  if (Ed <= 0) {                      // below the normal range: FP64 subnormal (truncated)
    const int sh = 1 - Ed;
    M = (sh < 64) ? (M >> sh) : 0ull;
    return __hiloint2double((int)(sg | ((unsigned)(M >> 32) & 0xFFFFFu)), (int)(unsigned)M);
  }
  if (Ed >= 2047) return __hiloint2double((int)(sg | 0x7FF00000u), 0);
  const unsigned hi = sg | ((unsigned)Ed << 20) | ((unsigned)(M >> 32) & 0xFFFFFu);
  return __hiloint2double((int)hi, (int)(unsigned)M);
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
__device__ __forceinline__ ffv ff_of(float2 v) { return ff_make(v.x, v.y); }
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
__device__ __forceinline__ float2 ff_f2(ffv a) { return make_float2(a.h, a.l); }

// ---------------------------------------------------------------- packed (two-chain) helpers
// The MIXED window kernel advances two blocks per thread; both chains go through one
// f32x2 instruction (sm_100+ FFMA2/FADD2/FMUL2: half the issue slots of scalar FP32).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// two chains of ff_axpy: y = f + r * x with f, x, y as (hi pair, lo pair), r a float-float scalar
__device__ __forceinline__ void ff_axpy2(float2 fh, float2 fl, float2 rh, float2 rl, float2 xh, float2 xl,
                                         float2& yh, float2& yl) {
  const float2 p = mul2(rh, xh);
  const float2 pe = fma2(rh, xh, make_float2(-p.x, -p.y));
  const float2 s = add2(fh, p);
  const float2 bb = sub2(s, fh);
  const float2 se = add2(sub2(fh, sub2(s, bb)), sub2(p, bb));
  float2 c = add2(fl, add2(pe, se));
  c = fma2(rl, xh, c);
  c = fma2(rh, xl, c);
  yh = s;
  yl = c;
}

// two chains of ff_mul: y = g * x
__device__ __forceinline__ void ff_mul2(float2 gh, float2 gl, float2 xh, float2 xl, float2& yh, float2& yl) {
  const float2 p = mul2(gh, xh);
  float2 c = fma2(gh, xh, make_float2(-p.x, -p.y));
  c = fma2(gl, xh, c);
  c = fma2(gh, xl, c);
  yh = p;
  yl = c;
}

// two chains of x += c * v, c and v float-float (per chain)
__device__ __forceinline__ void ff_fma_acc2(float2 ch, float2 cl, float2 vh, float2 vl, float2& xh, float2& xl) {
  const float2 p = mul2(ch, vh);
  const float2 pe = fma2(ch, vh, make_float2(-p.x, -p.y));
  const float2 pc = fma2(cl, vh, fma2(ch, vl, pe));
  const float2 s = add2(xh, p);
  const float2 bb = sub2(s, xh);
  const float2 se = add2(sub2(xh, sub2(s, bb)), sub2(p, bb));
  xl = add2(xl, add2(pc, se));
  xh = s;
}

// rare paths kept out of line so that their FP64 operations are not if-converted into the
// per-element code (GB300's FP64 pipe is ~70x slower than FP32)
static __device__ __noinline__ double rescale_subnormal(double d) { return d * 18446744073709551616.0; }  // * 2^64
static __device__ __noinline__ double join_rare(float s1, float e1, int s) {
  const unsigned b1 = __float_as_uint(s1);
  const unsigned sg = b1 & 0x80000000u;
  const int E1 = (int)((b1 >> 23) & 0xFFu);
  const unsigned f1 = b1 & 0x7FFFFFu;
  if (E1 == 0) return __hiloint2double((int)sg, 0);
  if (E1 == 255 || E1 + 896 - s >= 2047)
    return __hiloint2double((int)(sg | 0x7FF00000u | (E1 == 255 && f1 ? 0x80000u : 0u)), 0);
  const double sc = __hiloint2double((1023 - s) << 20, 0);
  return (double)s1 * sc + (double)e1 * sc;   // the FP64 unit rounds into the subnormal range
}

// FP64 -> (hi, lo) floats of d * 2^s with integer operations; `sb` = s - 896 is precomputed.
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

// (h, l) * 2^-s -> FP64 with 32-bit integer operations only.  FastTwoSum renormalises
// (|e| <= ulp(s1)/2 when |l| <= |h|); e is turned into an integer count K of the double's
// last place (bits below it truncated) and added to the 64-bit pattern of s1 with one
// carry-propagating add.  Results below the FP64 normal range become subnormal or zero.
__device__ __forceinline__ double join_sc(float h, float l, int s) {
  const float s1 = __fadd_rn(h, l);
  const float e1 = __fsub_rn(l, __fsub_rn(s1, h));
  const unsigned b1 = __float_as_uint(s1), be = __float_as_uint(e1);
  const unsigned sg = b1 & 0x80000000u;
  const int E1 = (int)((b1 >> 23) & 0xFFu);
  const unsigned f1 = b1 & 0x7FFFFFu;
  const int Ed = E1 + 896 - s;
  const int Ee = (int)((be >> 23) & 0xFFu);
  const unsigned Me = (be & 0x7FFFFFu) | 0x800000u;
  const int sh = Ee - E1 + 29;                 // <= 5
  unsigned K = (sh >= 0) ? (Me << sh) : ((sh > -32) ? (Me >> (-sh)) : 0u);
  if (Ee == 0) K = 0u;
  if (f1 == 0u && ((be ^ b1) & 0x80000000u)) K <<= 1;   // below an exact power of two
  const int Ks = ((be ^ b1) & 0x80000000u) ? -(int)K : (int)K;
  unsigned lo = f1 << 29;
  unsigned hi = sg | ((unsigned)Ed << 20) | (f1 >> 3);
  // 64-bit add of the signed count to (hi:lo), magnitude direction (sign bit untouched)
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+r"(lo), "+r"(hi) : "r"((unsigned)Ks),
      "r"((unsigned)(Ks >> 31)));
  if ((unsigned)(Ed - 1) >= 2046u || (unsigned)(E1 - 1) >= 254u) return join_rare(s1, e1, s);
  return __hiloint2double((int)hi, (int)lo);
}

// (h, l) * 2^-s -> FP64 with both parts converted exactly by integer operations and one FP64
// addition (the FP64 pipe does one operation per element; the integer-only join_sc needs about
// twice the issue slots).  Anything outside the plain case -- a zero or subnormal leading part,
// a part whose unscaled exponent leaves the FP64 normal range, Inf/NaN -- takes the
// out-of-line FP64 path, which rounds into the subnormal range correctly.
static __device__ __noinline__ double join_slow(float h, float l, int s) {
  const double sc = __hiloint2double((1023 - s) << 20, 0);
  return (double)h * sc + (double)l * sc;
}
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
