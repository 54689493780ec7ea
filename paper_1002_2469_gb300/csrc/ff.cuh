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

}  // namespace dich
