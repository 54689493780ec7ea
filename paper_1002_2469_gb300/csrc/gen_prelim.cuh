// gen_prelim.cuh -- the general O(N) preliminary step of the Dichotomy Algorithm (Sec. 2.3) on
// the device, for general tridiagonal matrices (general.cu).
//
// The host version walks the rows once; here the work is parallel over blocks:
//   1. per block (one thread per block): its own Thomas factors and spikes into the per-row tables,
//      and the block's composite of the whole-system elimination steps as 2x2 matrices -- the
//      forward factors cp_i = c_i / (b_i - a_i cp_{i-1}) are ratios p_i / q_i of
//      (p_i, q_i) = [[0, c_i], [-a_i, b_i]] (p_{i-1}, q_{i-1}), the backward factors
//      cq_i = a_i / (b_i - c_i cq_{i+1}) likewise with [[0, a_i], [-c_i, b_i]];
//   2. prefix (forward) and suffix (backward) products of the block composites, in chunks of
//      kPreChunk blocks (chunk products, a one-CTA pass over the chunks, chunk-local scans), every
//      partial product rescaled by a power of two (ratios are unchanged, nothing overflows);
//   3. per block: from the incoming cp_{s-1} and cq_{e+1}, the block's exterior ratios, block maps
//      and 2x2 beta map (the record of the dichotomy tree), and the largest |a|, |c| map factors;
//      step 1 also records what the precision choice needs (the error gains of the two local
//      recurrences, the range of the factors), and for the float-float form the tables are then
//      rewritten as (hi, lo) pairs in place (k_pre_to_ff).
#pragma once
#include "window_gen.cuh"

namespace dich {

constexpr int kPreThreads = 256;
constexpr int kPreChunk = kPreThreads;   // blocks per scan chunk (one per thread)

struct Mat2 {
  double a, b, c, d;   // [[a, b], [c, d]]
};

__host__ __device__ inline Mat2 mat_mul(const Mat2& x, const Mat2& y) {   // x * y
  return Mat2{fma(x.a, y.a, x.b * y.c), fma(x.a, y.b, x.b * y.d), fma(x.c, y.a, x.d * y.c),
              fma(x.c, y.b, x.d * y.d)};
}

// rescale by a power of two so that the largest entry lies in [1, 2) (exact; ratios unchanged)
__device__ __forceinline__ Mat2 mat_norm(Mat2 m) {
  const double mx = fmax(fmax(fabs(m.a), fabs(m.b)), fmax(fabs(m.c), fabs(m.d)));
  if (mx == 0.0 || !isfinite(mx)) return m;
  int e;
  frexp(mx, &e);
  return Mat2{ldexp(m.a, 1 - e), ldexp(m.b, 1 - e), ldexp(m.c, 1 - e), ldexp(m.d, 1 - e)};
}

struct PreArgs {
  int64_t N, P;
  int n, nlast;
  const double* a;      // raw sub-diagonal, diagonal, super-diagonal (N each)
  const double* b;
  const double* c;
  double* rows;         // per-row tables (window_gen.cuh layout), field stride `stride`
  int64_t stride;
  double* recs;         // block records, kBC per block
  Mat2* fwd;            // per block: forward composite (rows s..e)
  Mat2* bwd;            // per block: backward composite (rows e..s)
  Mat2* chunk;          // 2 per chunk: forward, backward chunk products, then the incoming products
  unsigned long long* maxes;   // [8]: bits of max |a_m| (m < P-1), max |c_m| (m > 0); a failure flag;
                               // then for the precision choice: the largest forward and backward error
                               // gains, max |rd_i|, ~bits of min |rd_i|, max |a_i|, |cp_i|, |v_i|, |w_i|
};

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(fabs(v)); }

// 1. per block: local factors, spikes, composites
__global__ void __launch_bounds__(kPreThreads) k_pre_blocks(const PreArgs A) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= A.P) return;
  const int n = A.n, nb = (m == A.P - 1) ? A.nlast : n;
  const int64_t s = m * n, e = s + nb - 1, N = A.N;
  double* fa = A.rows + GF_A * A.stride;
  double* frd = A.rows + GF_RD * A.stride;
  double* fcp = A.rows + GF_CP * A.stride;
  double* fv = A.rows + GF_V * A.stride;
  double* fw = A.rows + GF_W * A.stride;
  // local Thomas factors; z of the spike v = T_m^-1 (-a_s e_0) in the V field for now
  double lcp = 0.0, z = 0.0;
  // for the precision choice: the error gains of the two local recurrences (gf_i = 1 + |a_i rd_i|
  // gf_{i-1}, gb_i = 1 + |cp_i| gb_{i+1}), the range of rd and the largest other factor
  double fm = 0.0, bm = 0.0, rmax = 0.0, rmin = INFINITY, omax = 0.0, gf = 1.0;
  Mat2 F{1.0, 0.0, 0.0, 1.0};
  for (int i = 0; i < nb; ++i) {
    const int64_t r = s + i;
    const double ar = (r > 0) ? A.a[r] : 0.0, br = A.b[r], cr = (r < N - 1) ? A.c[r] : 0.0;
    const double den = br - ((i > 0) ? ar * lcp : 0.0);
    if (den == 0.0 || !isfinite(den)) atomicOr(&A.maxes[2], 1ull);   // a zero pivot: singular
    const double rd = 1.0 / den;
    lcp = (i < nb - 1 ? cr : 0.0) * rd;
    const int64_t k = gen_index(m, i, n);
    fa[k] = (i > 0) ? ar : 0.0;
    frd[k] = rd;
    fcp[k] = lcp;
    z = (i == 0) ? -ar * rd : -ar * z * rd;
    fv[k] = z;
    F = mat_norm(mat_mul(Mat2{0.0, cr, -ar, br}, F));
    gf = (i > 0) ? fma(fabs(ar * rd), gf, 1.0) : 1.0;
    fm = fmax(fm, gf);
    rmax = fmax(rmax, fabs(rd));
    rmin = fmin(rmin, fabs(rd));
    omax = fmax(omax, fmax(fabs(fa[k]), fabs(lcp)));
  }
  // backward: v_i = z_i - lcp_i v_{i+1}; w_i = -lcp_i w_{i+1} from w_e = -c_e rd_e
  const double ce = (e < N - 1) ? A.c[e] : 0.0;
  double v = fv[gen_index(m, nb - 1, n)];
  double w = -ce * frd[gen_index(m, nb - 1, n)];
  fw[gen_index(m, nb - 1, n)] = w;
  omax = fmax(omax, fmax(fabs(v), fabs(w)));
  double gb = 1.0;
  bm = 1.0;
  Mat2 B{1.0, 0.0, 0.0, 1.0};
  {
    const int64_t r = e;
    const double ar = (r > 0) ? A.a[r] : 0.0, br = A.b[r], cr = (r < N - 1) ? A.c[r] : 0.0;
    B = mat_norm(mat_mul(Mat2{0.0, ar, -cr, br}, B));
  }
  for (int i = nb - 2; i >= 0; --i) {
    const int64_t k = gen_index(m, i, n);
    v = fv[k] - fcp[k] * v;
    fv[k] = v;
    w = -fcp[k] * w;
    fw[k] = w;
    omax = fmax(omax, fmax(fabs(v), fabs(w)));
    gb = fma(fabs(fcp[k]), gb, 1.0);
    bm = fmax(bm, gb);
    const int64_t r = s + i;
    const double ar = (r > 0) ? A.a[r] : 0.0, br = A.b[r], cr = (r < N - 1) ? A.c[r] : 0.0;
    B = mat_norm(mat_mul(Mat2{0.0, ar, -cr, br}, B));
  }
  A.fwd[m] = F;
  A.bwd[m] = B;
  atomicMax(&A.maxes[3], dbits(fm));
  atomicMax(&A.maxes[4], dbits(bm));
  atomicMax(&A.maxes[5], dbits(rmax));
  atomicMax(&A.maxes[6], ~dbits(rmin));
  atomicMax(&A.maxes[7], dbits(omax));
}

// the per-row tables as float-float pairs (hi, lo) in their own 8-byte slots (MIXED form)
__global__ void k_pre_to_ff(double* rows, int64_t count) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x) {
    const double d = rows[j];
    const float h = __double2float_rn(d);
    const float l = __double2float_rn(d - (double)h);
    reinterpret_cast<float2*>(rows)[j] = make_float2(h, l);
  }
}

// CTA-wide inclusive scan of 2x2 matrices: forward (later blocks multiply on the left) or
// backward (earlier blocks multiply on the left); sh holds 4 * kPreThreads doubles
template <bool FWD>
__device__ Mat2 cta_mat_scan(Mat2 x, Mat2* sh) {
  const int t = threadIdx.x;
  sh[t] = x;
  __syncthreads();
  for (int d = 1; d < kPreThreads; d <<= 1) {
    Mat2 y = x;
    if (FWD && t >= d) y = mat_norm(mat_mul(x, sh[t - d]));
    if (!FWD && t + d < kPreThreads) y = mat_norm(mat_mul(x, sh[t + d]));
    __syncthreads();
    sh[t] = y;
    x = y;
    __syncthreads();
  }
  return x;
}

// 2a. chunk products (forward: M_last ... M_first; backward: M_first ... M_last)
__global__ void __launch_bounds__(kPreThreads) k_pre_chunk(const PreArgs A) {
  __shared__ Mat2 sh[kPreThreads];
  const int64_t m = blockIdx.x * (int64_t)kPreChunk + threadIdx.x;
  const Mat2 I{1.0, 0.0, 0.0, 1.0};
  const Mat2 f = cta_mat_scan<true>(m < A.P ? A.fwd[m] : I, sh);
  if (threadIdx.x == kPreThreads - 1) A.chunk[2 * blockIdx.x] = f;
  __syncthreads();
  const Mat2 b = cta_mat_scan<false>(m < A.P ? A.bwd[m] : I, sh);
  if (threadIdx.x == 0) A.chunk[2 * blockIdx.x + 1] = b;
}

// 2b. one thread: the product entering every chunk, forward from the left, backward from the right
__global__ void k_pre_top(const PreArgs A, int64_t nchunks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Mat2 run{1.0, 0.0, 0.0, 1.0};
  for (int64_t k = 0; k < nchunks; ++k) {
    const Mat2 own = A.chunk[2 * k];
    A.chunk[2 * k] = run;
    run = mat_norm(mat_mul(own, run));
  }
  run = Mat2{1.0, 0.0, 0.0, 1.0};
  for (int64_t k = nchunks - 1; k >= 0; --k) {
    const Mat2 own = A.chunk[2 * k + 1];
    A.chunk[2 * k + 1] = run;
    run = mat_norm(mat_mul(own, run));
  }
}

// 2c + 3. per block: incoming products, then the block's record
__global__ void __launch_bounds__(kPreThreads) k_pre_records(const PreArgs A) {
  __shared__ Mat2 sh[kPreThreads];
  const int64_t m = blockIdx.x * (int64_t)kPreChunk + threadIdx.x;
  const Mat2 I{1.0, 0.0, 0.0, 1.0};
  // exclusive chunk-local prefix / suffix, then the chunk's incoming product
  cta_mat_scan<true>(m < A.P ? A.fwd[m] : I, sh);            // sh[t]: inclusive prefix
  Mat2 fex = (threadIdx.x > 0) ? sh[threadIdx.x - 1] : I;
  __syncthreads();
  cta_mat_scan<false>(m < A.P ? A.bwd[m] : I, sh);           // sh[t]: inclusive suffix
  Mat2 bex = (threadIdx.x + 1 < kPreThreads) ? sh[threadIdx.x + 1] : I;
  if (m >= A.P) return;
  fex = mat_norm(mat_mul(fex, A.chunk[2 * blockIdx.x]));
  bex = mat_norm(mat_mul(bex, A.chunk[2 * blockIdx.x + 1]));
  // state entering the block: forward (p, q) at row s - 1 from (0, 1) at row -1; backward at
  // row e + 1 from (0, 1) at row N
  const int n = A.n, nb = (m == A.P - 1) ? A.nlast : n;
  const int64_t s = m * n, N = A.N, P = A.P;
  const double cp_in = (m > 0) ? fex.b / fex.d : 0.0;   // (p, q) = fex (0, 1)
  const double cq_in = (m < P - 1) ? bex.b / bex.d : 0.0;
  // whole-system factors over the block's rows: products of -cp_i and -cq_i
  bool pivots = true;   // every whole-system pivot nonzero and finite
  double cp = cp_in, tL = 1.0, pc = (m > 0) ? -cp_in : 0.0;
  for (int i = 0; i < nb; ++i) {
    const int64_t r = s + i;
    const double ar = (r > 0) ? A.a[r] : 0.0, br = A.b[r], cr = (r < N - 1) ? A.c[r] : 0.0;
    const double den = br - ar * cp;
    pivots = pivots && den != 0.0 && isfinite(den);
    cp = cr / den;
    if (i < nb - 1) {
      tL *= -cp;
      if (m > 0) pc *= -cp;
    }
  }
  double cq = cq_in, tR = 1.0, pa = (m < P - 1) ? -cq_in : 0.0;
  for (int i = nb - 1; i >= 0; --i) {
    const int64_t r = s + i;
    const double ar = (r > 0) ? A.a[r] : 0.0, br = A.b[r], cr = (r < N - 1) ? A.c[r] : 0.0;
    const double den = br - cr * cq;
    pivots = pivots && den != 0.0 && isfinite(den);
    cq = ar / den;
    if (i > 0) {
      tR *= -cq;
      if (m < P - 1) pa *= -cq;
    }
  }
  const double kL = (m > 0) ? -cp_in : 0.0, kR = (m < P - 1) ? -cq_in : 0.0;
  const double* fv = A.rows + GF_V * A.stride;
  const double* fw = A.rows + GF_W * A.stride;
  const double v0 = fv[gen_index(m, 0, n)], vend = fv[gen_index(m, nb - 1, n)];
  const double w0 = fw[gen_index(m, 0, n)], wend = fw[gen_index(m, nb - 1, n)];
  const double p00 = 1.0 - kL * v0, p01 = -kR * w0, p10 = -kL * vend, p11 = 1.0 - kR * wend;
  const double det = p00 * p11 - p01 * p10;
  double* rc = A.recs + m * kBC;
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
  const bool finite = pivots && isfinite(det) && det != 0.0 && isfinite(pa) && isfinite(pc) && isfinite(tL) && isfinite(tR) &&
                      isfinite(kL) && isfinite(kR);
  if (!finite) atomicOr(&A.maxes[2], 1ull);     // a zero pivot: the plan is refused as singular
  if (m < P - 1 && finite) atomicMax(&A.maxes[0], (unsigned long long)__double_as_longlong(fabs(pa)));
  if (m > 0 && finite) atomicMax(&A.maxes[1], (unsigned long long)__double_as_longlong(fabs(pc)));
}

}  // namespace dich
