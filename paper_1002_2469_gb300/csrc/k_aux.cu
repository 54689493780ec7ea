// k_aux.cu -- general-path block scan, adjoint gradient finalisation, one-row systems,
// quasi-Toeplitz corner corrections (single plans and batches, forward and adjoint), and the
// residual check of Toeplitz plans.
#include "launch.cuh"

namespace dich {

__device__ __forceinline__ const double* bc_of(const SysPlan* pp, const double* tab, int64_t m) {
  if (m < pp->kl) return tab + pp->o_bcl + m * kBC;
  if (m >= pp->P - pp->kr) return tab + pp->o_bcr + (m - (pp->P - pp->kr)) * kBC;
  return tab + pp->o_bcm;
}

// CTA scans of affine maps t -> a t + b.  Prefix: maps of threads 0..tid composed left to
// right (lower index applied first).  Suffix: maps of threads tid..NTH-1 composed right to
// left (higher index applied first).  (ia, ib): inclusive composite; (ea, eb): exclusive.
// `sh` holds 4 * NTH/32 doubles; the CTA must call these uniformly.
template <int NTH>
__device__ __forceinline__ void cta_prefix(double& ia, double& ib, double& ea, double& eb, double* sh) {
  constexpr int NW = NTH / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double ya = __shfl_up_sync(0xffffffffu, ia, d), yb = __shfl_up_sync(0xffffffffu, ib, d);
    if (lane >= d) {
      ib = fma(ia, yb, ib);
      ia = ia * ya;
    }
  }
  if (lane == 31) {
    sh[wid] = ia;
    sh[NW + wid] = ib;
  }
  double pa = __shfl_up_sync(0xffffffffu, ia, 1), pb = __shfl_up_sync(0xffffffffu, ib, 1);
  if (lane == 0) {
    pa = 1.0;
    pb = 0.0;
  }
  __syncthreads();
  double ma = 1.0, mb = 0.0;  // composite of the previous warps
  for (int w = 0; w < wid; ++w) {
    mb = fma(sh[w], mb, sh[NW + w]);
    ma = sh[w] * ma;
  }
  __syncthreads();
  ea = pa * ma;
  eb = fma(pa, mb, pb);
  ib = fma(ia, mb, ib);
  ia = ia * ma;
}

template <int NTH>
__device__ __forceinline__ void cta_suffix(double& ia, double& ib, double& ea, double& eb, double* sh) {
  constexpr int NW = NTH / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double ya = __shfl_down_sync(0xffffffffu, ia, d), yb = __shfl_down_sync(0xffffffffu, ib, d);
    if (lane + d < 32) {
      ib = fma(ia, yb, ib);
      ia = ia * ya;
    }
  }
  if (lane == 0) {
    sh[2 * NW + wid] = ia;
    sh[3 * NW + wid] = ib;
  }
  double pa = __shfl_down_sync(0xffffffffu, ia, 1), pb = __shfl_down_sync(0xffffffffu, ib, 1);
  if (lane == 31) {
    pa = 1.0;
    pb = 0.0;
  }
  __syncthreads();
  double ma = 1.0, mb = 0.0;  // composite of the following warps
  for (int w = NW - 1; w > wid; --w) {
    mb = fma(sh[2 * NW + w], mb, sh[3 * NW + w]);
    ma = sh[2 * NW + w] * ma;
  }
  __syncthreads();
  ea = pa * ma;
  eb = fma(pa, mb, pb);
  ib = fma(ia, mb, ib);
  ia = ia * ma;
}

// per-thread composite of its kScanPer blocks
__device__ __forceinline__ void thread_maps(const SysPlan* pp, const double* tab, int64_t P, const double* beta,
                                            int64_t m_first, double& pa, double& pb, double& sa, double& sb) {
  pa = 1.0; pb = 0.0; sa = 1.0; sb = 0.0;
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t m = m_first + k;
    if (m >= P) break;
    const double* bc = bc_of(pp, tab, m);
    const double bR = beta[2 * m + 1];
    pb = fma(bc[BC_A], pb, bc[BC_B] * bR);
    pa = bc[BC_A] * pa;
  }
  for (int k = kScanPer - 1; k >= 0; --k) {
    const int64_t m = m_first + k;
    if (m >= P) continue;
    const double* bc = bc_of(pp, tab, m);
    const double bL = beta[2 * m];
    sb = fma(bc[BC_C], sb, bc[BC_D] * bL);
    sa = bc[BC_C] * sa;
  }
}

// Chunk c of a scan: its system (the single system of `plans` when map.cmap is null, else the
// general-path system map.sys[map.cmap[c]] of a batch) and its chunk index within that system.
__device__ __forceinline__ const SysPlan* chunk_system(const SysPlan* plans, const ScanMap& map, int64_t c,
                                                      int64_t& lc) {
  if (!map.cmap) {
    lc = c;
    return plans;
  }
  const int j = map.cmap[c];
  lc = c - map.c0[j];
  return plans + map.sys[j];
}

__global__ void __launch_bounds__(kScanThreads) k_bscan_reduce(const SysPlan* plans, const double* tabs, ScanMap map,
                                                               const double* beta_base, double* agg) {
  __shared__ double sh[4 * kScanThreads / 32];
  int64_t lc;
  const SysPlan* pp = chunk_system(plans, map, blockIdx.x, lc);
  const double* tab = tabs + pp->tab;
  const double* beta = beta_base + 2 * pp->gboff;
  const int64_t mb = map.cmap ? 0 : map.mbase, me = (map.cmap || map.mend == 0) ? pp->P : map.mend;
  const int64_t m_first = mb + lc * kScanChunk + (int64_t)threadIdx.x * kScanPer;
  double pa, pb, sa, sb, ea, eb;
  thread_maps(pp, tab, me, beta, m_first, pa, pb, sa, sb);
  cta_prefix<kScanThreads>(pa, pb, ea, eb, sh);
  cta_suffix<kScanThreads>(sa, sb, ea, eb, sh);
  if (threadIdx.x == kScanThreads - 1) {
    agg[4 * (size_t)blockIdx.x + 0] = pa;
    agg[4 * (size_t)blockIdx.x + 1] = pb;
  }
  if (threadIdx.x == 0) {
    agg[4 * (size_t)blockIdx.x + 2] = sa;
    agg[4 * (size_t)blockIdx.x + 3] = sb;
  }
}

// One CTA per system: over the system's chunks c0 .. c0 + nchunks - 1,
// carry[2 c] = A entering chunk c, carry[2 c + 1] = B at the end of chunk c.
__global__ void __launch_bounds__(1024) k_bscan_top(const SysPlan* plans, ScanMap map, const double* agg,
                                                    double* carry) {
  __shared__ double sh[4 * 1024 / 32];
  __shared__ double run;
  __shared__ double cin[2], runa;
  const SysPlan* pp = map.cmap ? plans + map.sys[blockIdx.x] : plans;
  const int64_t cbase = map.cmap ? map.c0[blockIdx.x] : 0;
  const int64_t nb = (map.cmap || map.mend == 0) ? pp->P : map.mend - map.mbase;
  const int64_t nchunks = (nb + kScanChunk - 1) / kScanChunk;
  const double* ag = agg + 4 * cbase;
  double* ca = carry + 2 * cbase;
  if (threadIdx.x == 0) {
    // a shard: the prefix entering it composes the totals of the shards before it (the paper's
    // dichotomy levels across processes, eq. 17-19, in one fold), the suffix those after it
    double A = 0.0, B = 0.0;
    if (!map.cmap && map.maps) {
      for (int j = 0; j < map.shard; ++j) A = fma(map.maps[4 * j], A, map.maps[4 * j + 1]);
      for (int j = map.nshards - 1; j > map.shard; --j) B = fma(map.maps[4 * j + 2], B, map.maps[4 * j + 3]);
    }
    cin[0] = A;
    cin[1] = B;
    run = A;
    runa = 1.0;
  }
  __syncthreads();
  for (int64_t g0 = 0; g0 < nchunks; g0 += 1024) {
    const int64_t c = g0 + threadIdx.x;
    double ia = 1.0, ib = 0.0, ea, eb;
    if (c < nchunks) {
      ia = ag[4 * c];
      ib = ag[4 * c + 1];
    }
    cta_prefix<1024>(ia, ib, ea, eb, sh);
    const double r = run;
    if (c < nchunks) ca[2 * c] = fma(ea, r, eb);
    __syncthreads();
    if (threadIdx.x == 1023) {
      run = fma(ia, r, ib);
      runa *= ia;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (!map.cmap && map.tot) {   // the shard's prefix total map (zero carry-in: run is its b part)
      map.tot[0] = runa;
      map.tot[1] = run;
    }
    run = cin[1];
    runa = 1.0;
  }
  __syncthreads();
  const int64_t ngroups = (nchunks + 1023) / 1024;
  for (int64_t g = ngroups - 1; g >= 0; --g) {
    const int64_t c = g * 1024 + threadIdx.x;
    double ia = 1.0, ib = 0.0, ea, eb;
    if (c < nchunks) {
      ia = ag[4 * c + 2];
      ib = ag[4 * c + 3];
    }
    cta_suffix<1024>(ia, ib, ea, eb, sh);
    const double r = run;
    if (c < nchunks) ca[2 * c + 1] = fma(ea, r, eb);
    __syncthreads();
    if (threadIdx.x == 0) {
      run = fma(ia, r, ib);
      runa *= ia;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && !map.cmap && map.tot) {
    map.tot[2] = runa;
    map.tot[3] = run;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_bscan_apply(const SysPlan* plans, const double* tabs, ScanMap map,
                                                              const double* beta_base, const double* carry,
                                                              double* iface_base) {
  __shared__ double sh[4 * kScanThreads / 32];
  int64_t lc;
  const SysPlan* pp = chunk_system(plans, map, blockIdx.x, lc);
  const int64_t P = (map.cmap || map.mend == 0) ? pp->P : map.mend;   // end of the scanned blocks
  const double* tab = tabs + pp->tab;
  const double* beta = beta_base + 2 * pp->gboff;
  double* iface = iface_base + 2 * pp->gboff;
  const int64_t m_first = (map.cmap ? 0 : map.mbase) + lc * kScanChunk + (int64_t)threadIdx.x * kScanPer;
  double pa, pb, sa, sb, ea, eb, fa, fb;
  thread_maps(pp, tab, P, beta, m_first, pa, pb, sa, sb);
  cta_prefix<kScanThreads>(pa, pb, ea, eb, sh);
  cta_suffix<kScanThreads>(sa, sb, fa, fb, sh);
  double Acur = fma(ea, carry[2 * (size_t)blockIdx.x], eb);
  const double Bend = fma(fa, carry[2 * (size_t)blockIdx.x + 1], fb);
  double Am[kScanPer], Bm[kScanPer];
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t m = m_first + k;
    Am[k] = Acur;
    if (m < P) {
      const double* bc = bc_of(pp, tab, m);
      Acur = fma(bc[BC_A], Acur, bc[BC_B] * beta[2 * m + 1]);
    }
  }
  double Bcur = Bend;
  for (int k = kScanPer - 1; k >= 0; --k) {
    const int64_t m = m_first + k;
    Bm[k] = Bcur;
    if (m < P) {
      const double* bc = bc_of(pp, tab, m);
      Bcur = fma(bc[BC_C], Bcur, bc[BC_D] * beta[2 * m]);
    }
  }
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t m = m_first + k;
    if (m >= P) break;
    const double* bc = bc_of(pp, tab, m);
    const double bL = beta[2 * m], bR = beta[2 * m + 1];
    iface[2 * m] = Am[k] + bL + bc[BC_TL] * Bm[k];
    iface[2 * m + 1] = fma(bc[BC_TR], Am[k], bR + Bm[k]);
  }
}

cudaError_t launch_block_scan(const SysPlan* plan, const double* tabs, int64_t P, const double* beta,
                              double* iface, double* scratch, cudaStream_t st) {
  const int64_t nchunks = (P + kScanChunk - 1) / kScanChunk;
  return launch_block_scan_batched(plan, tabs, ScanMap{}, nchunks, 1, beta, iface, scratch, st);
}

cudaError_t launch_shard_scan_reduce(const SysPlan* plan, const double* tabs, const ScanMap& map, const double* beta,
                                     double* scratch, cudaStream_t st) {
  const int64_t nchunks = (map.mend - map.mbase + kScanChunk - 1) / kScanChunk;
  if (nchunks <= 0) return cudaErrorInvalidValue;
  ScanMap m = map;
  m.maps = nullptr;   // totals with zero carry-ins
  k_bscan_reduce<<<(unsigned)nchunks, kScanThreads, 0, st>>>(plan, tabs, m, beta, scratch);
  k_bscan_top<<<1, 1024, 0, st>>>(plan, m, scratch, scratch + 4 * nchunks);
  return cudaGetLastError();
}

cudaError_t launch_shard_scan_apply(const SysPlan* plan, const double* tabs, const ScanMap& map, const double* beta,
                                    double* iface, double* scratch, cudaStream_t st) {
  const int64_t nchunks = (map.mend - map.mbase + kScanChunk - 1) / kScanChunk;
  if (nchunks <= 0) return cudaErrorInvalidValue;
  ScanMap m = map;
  m.tot = nullptr;
  k_bscan_top<<<1, 1024, 0, st>>>(plan, m, scratch, scratch + 4 * nchunks);
  k_bscan_apply<<<(unsigned)nchunks, kScanThreads, 0, st>>>(plan, tabs, m, beta, scratch + 4 * nchunks, iface);
  return cudaGetLastError();
}

cudaError_t launch_block_scan_batched(const SysPlan* plans, const double* tabs, const ScanMap& map, int64_t nchunks,
                                      int64_t nsys, const double* beta, double* iface, double* scratch,
                                      cudaStream_t st) {
  if (nchunks <= 0) return cudaSuccess;
  double* agg = scratch;
  double* carry = scratch + 4 * nchunks;
  k_bscan_reduce<<<(unsigned)nchunks, kScanThreads, 0, st>>>(plans, tabs, map, beta, agg);
  k_bscan_top<<<(unsigned)nsys, 1024, 0, st>>>(plans, map, agg, carry);
  k_bscan_apply<<<(unsigned)nchunks, kScanThreads, 0, st>>>(plans, tabs, map, beta, carry, iface);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_adj_finalize(const double* part, const int32_t* sys_ids,
                                                      const int64_t* first, const int64_t* count, int64_t count0,
                                                      double* gt) {
  __shared__ double sh[3 * 256];
  const int64_t k = blockIdx.x;
  const int64_t s = sys_ids ? sys_ids[k] : k;
  const int64_t f = first ? first[k] : 0;
  const int64_t c = count ? count[k] : count0;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int64_t i = threadIdx.x; i < c; i += 256) {
    a0 += part[3 * (f + i)];
    a1 += part[3 * (f + i) + 1];
    a2 += part[3 * (f + i) + 2];
  }
  sh[threadIdx.x] = a0;
  sh[256 + threadIdx.x] = a1;
  sh[512 + threadIdx.x] = a2;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) {
      sh[threadIdx.x] += sh[threadIdx.x + d];
      sh[256 + threadIdx.x] += sh[256 + threadIdx.x + d];
      sh[512 + threadIdx.x] += sh[512 + threadIdx.x + d];
    }
    __syncthreads();
  }
  if (threadIdx.x < 3) gt[3 * s + threadIdx.x] = -sh[256 * threadIdx.x];
}

cudaError_t launch_adj_finalize(const double* part, const int32_t* sys_ids, const int64_t* first,
                                const int64_t* count, int64_t count0, int64_t nsys, double* gt, cudaStream_t st) {
  if (nsys <= 0) return cudaSuccess;
  k_adj_finalize<<<(unsigned)nsys, 256, 0, st>>>(part, sys_ids, first, count, count0, gt);
  return cudaGetLastError();
}

// x = F / t_0 for one-row systems; adjoint form when w != nullptr:
//   gF = w / t_0, dL/dt_0 = -gF * xf, dL/dt_-1 = dL/dt_1 = 0.
__global__ void k_trivial(const SysPlan* plans, const int32_t* idx, int64_t nidx, const double* F, double* x,
                          const double* xf, const double* w, double* gt, int sys_offset) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nidx) return;
  const int s = idx ? idx[k] : 0;
  const SysPlan* pp = plans + s + sys_offset;
  const int64_t o = pp->off;
  if (w == nullptr) {
    x[o] = F[o] / pp->t0;
  } else {
    const double lam = w[o] / pp->t0;
    x[o] = lam;
    gt[3 * s + 0] = 0.0;
    gt[3 * s + 1] = -lam * xf[o];
    gt[3 * s + 2] = 0.0;
  }
}

cudaError_t launch_trivial(const SysPlan* plans, const int32_t* idx, int64_t nidx, const double* F, double* x,
                           const double* xf, const double* w, double* gt, int sys_offset, cudaStream_t st) {
  if (nidx <= 0) return cudaSuccess;
  k_trivial<<<(unsigned)((nidx + 127) / 128), 128, 0, st>>>(plans, idx, nidx, F, x, xf, w, gt, sys_offset);
  return cudaGetLastError();
}


// ---------------------------------------------------------------- quasi-Toeplitz corners (eq. 21)
// A = T + psi e_0 e_0^T + chi e_{N-1} e_{N-1}^T.  With y = T^-1 F (the Toeplitz solve, already in
// x), g = T^-1 e_0, h = T^-1 e_{N-1}, the Sherman-Morrison-Woodbury identity gives
//   A^-1 F = y - c_0 g - c_1 h,   (c_0, c_1) = W (psi y_0, chi y_{N-1}),
//   W = (I + [[psi g_0, psi h_0], [chi g_{N-1}, chi h_{N-1}]])^-1.
// g is kept for its first Lg rows and h (indexed from the end) for its last Lh rows, where they
// exceed the truncation threshold.  Pass 1 (ends = false) corrects rows 1..N-2 and leaves
// rows 0 and N-1 -- which every CTA reads for c -- untouched; pass 2 (ends = true, one thread
// per right-hand side) then corrects those two.  grid.y runs over the right-hand sides of a
// series (x + y ldx).
__global__ void k_corner(double* x, int64_t ldx, CornerArgs c, bool ends) {
  double* xr = x + (int64_t)blockIdx.y * ldx;
  const int64_t N = c.N;
  const double y0 = xr[0], yn = xr[N - 1];
  const double a = c.psi * y0, b = c.chi * yn;
  const double c0 = fma(c.w00, a, c.w01 * b), c1 = fma(c.w10, a, c.w11 * b);
  auto corr = [&](int64_t i) {
    double v = xr[i];
    if (i < c.Lg) v = fma(-c0, c.g[i], v);
    const int64_t k = N - 1 - i;
    if (k < c.Lh) v = fma(-c1, c.h[k], v);
    return v;
  };
  if (ends) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const double v0 = corr(0), vn = (N > 1) ? corr(N - 1) : v0;
      xr[0] = v0;
      if (N > 1) xr[N - 1] = vn;
    }
    return;
  }
  // rows 1..N-2 inside [0, Lg) or [N - Lh, N): one range when the two meet
  const int64_t lo1 = 1, hi1 = min(c.Lg, N - 1);
  const int64_t lo2 = max(N - c.Lh, (int64_t)1), hi2 = N - 1;
  const bool merged = lo2 <= hi1;
  const int64_t n1 = merged ? (hi2 - lo1) : max(hi1 - lo1, (int64_t)0);
  const int64_t n2 = merged ? 0 : max(hi2 - lo2, (int64_t)0);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n1 + n2; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (j < n1) ? lo1 + j : lo2 + (j - n1);
    xr[i] = corr(i);
  }
}

cudaError_t launch_corner(double* x, int64_t M, int64_t ldx, const CornerArgs& c, cudaStream_t st) {
  if (c.N <= 0 || M <= 0) return cudaSuccess;
  const int64_t rows = min(c.N, c.Lg + c.Lh);
  const unsigned gx = (unsigned)max((int64_t)1, min((rows + 255) / 256, (int64_t)1184));
  for (int64_t k0 = 0; k0 < M; k0 += 65535) {
    const unsigned gy = (unsigned)min((int64_t)65535, M - k0);
    k_corner<<<dim3(gx, gy), 256, 0, st>>>(x + k0 * ldx, ldx, c, false);
    k_corner<<<dim3(1, gy), 32, 0, st>>>(x + k0 * ldx, ldx, c, true);
  }
  return cudaGetLastError();
}

// Adjoint of a quasi-Toeplitz plan, before the corner correction of lambda (launched after the
// adjoint window kernels and k_adj_finalize): with lambda_T = T^-T w in lam and the transposed
// corner vectors in c, lambda = lambda_T - c0 g - c1 h changes the gradient sums by
// + c0 sum_i g_i x_{i+s} + c1 sum_i h_i x_{i+s} (s = -1, 0, 1; gt holds -sum lambda x), and
// dL/dpsi = -lambda_0 x_0, dL/dchi = -lambda_{N-1} x_{N-1} come from the corrected end values.
__global__ void __launch_bounds__(256) k_corner_adj(const double* xf, const double* lam, CornerArgs c, double* gt) {
  __shared__ double sh[6 * 256];
  const int64_t N = c.N;
  const double y0 = lam[0], yn = lam[N - 1];
  const double a = c.psi * y0, b = c.chi * yn;
  const double c0 = fma(c.w00, a, c.w01 * b), c1 = fma(c.w10, a, c.w11 * b);
  auto xv = [&](int64_t i) { return (i >= 0 && i < N) ? xf[i] : 0.0; };
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // sum g x_{i-1}, g x_i, g x_{i+1}, then h
  for (int64_t i = threadIdx.x; i < c.Lg; i += 256) {
    const double gi = c.g[i];
    acc[0] = fma(gi, xv(i - 1), acc[0]);
    acc[1] = fma(gi, xv(i), acc[1]);
    acc[2] = fma(gi, xv(i + 1), acc[2]);
  }
  for (int64_t k = threadIdx.x; k < c.Lh; k += 256) {
    const int64_t i = N - 1 - k;
    const double hk = c.h[k];
    acc[3] = fma(hk, xv(i - 1), acc[3]);
    acc[4] = fma(hk, xv(i), acc[4]);
    acc[5] = fma(hk, xv(i + 1), acc[5]);
  }
  for (int j = 0; j < 6; ++j) sh[j * 256 + threadIdx.x] = acc[j];
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d)
      for (int j = 0; j < 6; ++j) sh[j * 256 + threadIdx.x] += sh[j * 256 + threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < 3; ++s) gt[s] += fma(c0, sh[s * 256], c1 * sh[(3 + s) * 256]);
    // the corrected end values, in the corner kernel's order of operations
    double l0 = y0, ln = yn;
    if (0 < c.Lg) l0 = fma(-c0, c.g[0], l0);
    if (N - 1 < c.Lh) l0 = fma(-c1, c.h[N - 1], l0);
    if (N - 1 < c.Lg) ln = fma(-c0, c.g[N - 1], ln);
    if (0 < c.Lh) ln = fma(-c1, c.h[0], ln);
    gt[3] = -l0 * xf[0];
    gt[4] = -ln * xf[N - 1];
  }
}

// Batched corner correction: every thread reads both end values of its system before any row
// is corrected (one barrier), then rows [0, Lg) and [N - Lh, N) are corrected once each, with the
// single-system kernel's order of operations.
__global__ void __launch_bounds__(256) k_corner_batch(const CornerRec* recs, const double* tab, double* x) {
  const CornerRec c = recs[blockIdx.x];
  double* xr = x + c.off;
  const int64_t N = c.N;
  const double y0 = xr[0], yn = xr[N - 1];
  __syncthreads();
  const double a = c.psi * y0, b = c.chi * yn;
  const double c0 = fma(c.w00, a, c.w01 * b), c1 = fma(c.w10, a, c.w11 * b);
  const double* g = tab + c.og;
  const double* h = tab + c.oh;
  auto corr = [&](int64_t i) {
    double v = xr[i];
    if (i < c.Lg) v = fma(-c0, g[i], v);
    const int64_t k = N - 1 - i;
    if (k < c.Lh) v = fma(-c1, h[k], v);
    xr[i] = v;
  };
  const int64_t hi1 = min(c.Lg, N), lo2 = max(N - c.Lh, hi1);
  for (int64_t i = threadIdx.x; i < hi1; i += 256) corr(i);
  for (int64_t i = lo2 + threadIdx.x; i < N; i += 256) corr(i);
}

cudaError_t launch_corner_batch(const CornerRec* recs, int64_t n, const double* tab, double* x, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_corner_batch<<<(unsigned)n, 256, 0, st>>>(recs, tab, x);
  return cudaGetLastError();
}

// Batched adjoint with corners: one CTA per system (every system of the batch).  gt3 holds the
// Toeplitz adjoint's -sum lambda_T x products (3 per system); gt5 receives the five gradients
// (t_-1, t_0, t_1, psi, chi).  A system with corners (Lg or Lh nonzero in its transposed record)
// adds its corner correction's share to the sums and has lambda corrected in place; one-row
// systems (psi and chi folded into t_0) repeat dL/dt_0.
__global__ void __launch_bounds__(256) k_corner_adj_batch(const CornerRec* recs, const double* tab, const double* xf,
                                                          double* lam, const double* gt3, double* gt5) {
  __shared__ double sh[6 * 256];
  const int64_t s = blockIdx.x;
  const CornerRec c = recs[s];
  const int64_t N = c.N;
  double* out = gt5 + 5 * s;
  if (N <= 1) {
    if (threadIdx.x < 5) out[threadIdx.x] = (N == 0) ? 0.0 : gt3[3 * s + ((threadIdx.x < 3) ? threadIdx.x : 1)];
    return;
  }
  const double* x = xf + c.off;
  double* l = lam + c.off;
  const double y0 = l[0], yn = l[N - 1];
  const double a = c.psi * y0, b = c.chi * yn;
  const double c0 = fma(c.w00, a, c.w01 * b), c1 = fma(c.w10, a, c.w11 * b);
  const double* g = tab + c.og;
  const double* h = tab + c.oh;
  auto xv = [&](int64_t i) { return (i >= 0 && i < N) ? x[i] : 0.0; };
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < c.Lg; i += 256) {
    acc[0] = fma(g[i], xv(i - 1), acc[0]);
    acc[1] = fma(g[i], xv(i), acc[1]);
    acc[2] = fma(g[i], xv(i + 1), acc[2]);
  }
  for (int64_t k = threadIdx.x; k < c.Lh; k += 256) {
    const int64_t i = N - 1 - k;
    acc[3] = fma(h[k], xv(i - 1), acc[3]);
    acc[4] = fma(h[k], xv(i), acc[4]);
    acc[5] = fma(h[k], xv(i + 1), acc[5]);
  }
  for (int j = 0; j < 6; ++j) sh[j * 256 + threadIdx.x] = acc[j];
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d)
      for (int j = 0; j < 6; ++j) sh[j * 256 + threadIdx.x] += sh[j * 256 + threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int j = 0; j < 3; ++j) out[j] = gt3[3 * s + j] + fma(c0, sh[j * 256], c1 * sh[(3 + j) * 256]);
    double l0 = y0, ln = yn;
    if (0 < c.Lg) l0 = fma(-c0, g[0], l0);
    if (N - 1 < c.Lh) l0 = fma(-c1, h[N - 1], l0);
    if (N - 1 < c.Lg) ln = fma(-c0, g[N - 1], ln);
    if (0 < c.Lh) ln = fma(-c1, h[0], ln);
    out[3] = -l0 * x[0];
    out[4] = -ln * x[N - 1];
  }
  // lambda = lambda_T - c0 g - c1 h on the corner rows (both end values were read above)
  const int64_t hi1 = min(c.Lg, N), lo2 = max(N - c.Lh, hi1);
  auto corr = [&](int64_t i) {
    double v = l[i];
    if (i < c.Lg) v = fma(-c0, g[i], v);
    const int64_t k = N - 1 - i;
    if (k < c.Lh) v = fma(-c1, h[k], v);
    l[i] = v;
  };
  for (int64_t i = threadIdx.x; i < hi1; i += 256) corr(i);
  for (int64_t i = lo2 + threadIdx.x; i < N; i += 256) corr(i);
}

cudaError_t launch_corner_adjoint_batch(const CornerRec* recs, int64_t nsys, const double* tab, const double* xf,
                                        double* lam, const double* gt3, double* gt5, cudaStream_t st) {
  if (nsys <= 0) return cudaSuccess;
  k_corner_adj_batch<<<(unsigned)nsys, 256, 0, st>>>(recs, tab, xf, lam, gt3, gt5);
  return cudaGetLastError();
}

// residual check of a (quasi-)Toeplitz system: max |F - A x|, max |x|, max |F| as bits of
// non-negative doubles in res[0..2] (zeroed here first)
__global__ void __launch_bounds__(256) k_toeplitz_residual(int64_t N, double tm1, double t0, double tp1, double psi,
                                                           double chi, const double* F, const double* x,
                                                           unsigned long long* res) {
  double r = 0.0, xm = 0.0, fm = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double d = t0;
    if (i == 0) d += psi;
    if (i == N - 1) d += chi;
    double ax = d * x[i];
    if (i > 0) ax = fma(tm1, x[i - 1], ax);
    if (i + 1 < N) ax = fma(tp1, x[i + 1], ax);
    r = fmax(r, fabs(F[i] - ax));
    xm = fmax(xm, fabs(x[i]));
    fm = fmax(fm, fabs(F[i]));
  }
  for (int d = 16; d > 0; d >>= 1) {
    r = fmax(r, __shfl_xor_sync(0xffffffffu, r, d));
    xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, d));
    fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, d));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&res[0], (unsigned long long)__double_as_longlong(r));
    atomicMax(&res[1], (unsigned long long)__double_as_longlong(xm));
    atomicMax(&res[2], (unsigned long long)__double_as_longlong(fm));
  }
}

cudaError_t launch_toeplitz_residual(int64_t N, double tm1, double t0, double tp1, double psi, double chi,
                                     const double* F, const double* x, unsigned long long* res, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(res, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)max((int64_t)1, min((N + 255) / 256, (int64_t)4 * 1184));
  k_toeplitz_residual<<<grid, 256, 0, st>>>(N, tm1, t0, tp1, psi, chi, F, x, res);
  return cudaGetLastError();
}

cudaError_t launch_end_gradients(const double* xf, const double* lam, double* gt, int64_t N, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  // empty corner vectors and zero corners: the kernel adds nothing to the three sums and writes
  // gt[3] = -lambda_0 x_0, gt[4] = -lambda_{N-1} x_{N-1}
  const CornerArgs c{N, 0, 0, nullptr, nullptr, 0.0, 0.0, 1.0, 0.0, 0.0, 1.0};
  k_corner_adj<<<1, 256, 0, st>>>(xf, lam, c, gt);
  return cudaGetLastError();
}

cudaError_t launch_corner_adjoint(const double* xf, double* lam, double* gt, const CornerArgs& c, cudaStream_t st) {
  if (c.N <= 0) return cudaSuccess;
  k_corner_adj<<<1, 256, 0, st>>>(xf, lam, c, gt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_corner(lam, 1, 0, c, st);
}

}  // namespace dich
