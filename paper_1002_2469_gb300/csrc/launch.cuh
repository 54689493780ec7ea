// launch.cuh -- internal launch entry points shared by the kernel translation units and the
// host API (C++ linkage, not exported).
#pragma once
#include <cuda_runtime.h>
#include "window.cuh"
#include "window_mixed.cuh"

namespace dich {

// window kernel of width NT (64, 128 or 256) in the given form, grid (grid, grid_y): grid_y
// right-hand sides of a series (WinArgs::ldf, ldx); returns the launch error
cudaError_t launch_window_f64(int NT, int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y = 1);
cudaError_t launch_window_mixed(int NT, int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y = 1);

// general path: first/last values of every block from per-block beta (global block scan)
//   beta [2P] -> iface [2P]; scratch needs 6 * ceil(P / kScanChunk) doubles.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanThreads * kScanPer;
cudaError_t launch_block_scan(const SysPlan* plan, const double* tabs, int64_t P, const double* beta,
                              double* iface, double* scratch, cudaStream_t st);

// the general-path systems of a batch in one scan: chunk c (kScanChunk blocks) belongs to system
// plans[sys[cmap[c]]], whose chunks start at c0[cmap[c]]; a system's beta and first/last values
// start at block SysPlan::gboff of the shared buffers.  A null cmap is the single-system scan.
struct ScanMap {
  const int32_t* cmap;
  const int32_t* sys;
  const int64_t* c0;
  // single system (cmap null): the scan covers blocks [mbase, mend) (mend 0: the whole system).
  // A shard of a sharded solve passes its block range, `maps` = every shard's totals (4 doubles per
  // shard: prefix a, b, suffix a, b) with its index `shard` (the carry-ins are folded from them), and
  // or `tot` = where its own totals go (4 doubles); null maps: zero coupling enters at both ends.
  int64_t mbase, mend;
  const double* maps;
  int32_t shard, nshards;
  double* tot;
};
//   scratch: 6 doubles per chunk; nsys systems, nchunks chunks in all
cudaError_t launch_block_scan_batched(const SysPlan* plans, const double* tabs, const ScanMap& map, int64_t nchunks,
                                      int64_t nsys, const double* beta, double* iface, double* scratch,
                                      cudaStream_t st);
// a shard's block scan in two halves: reduce (chunk aggregates and the shard's totals into map.tot,
// zero carry-ins), then apply (carry-ins folded from map.maps, first/last values into iface)
cudaError_t launch_shard_scan_reduce(const SysPlan* plan, const double* tabs, const ScanMap& map, const double* beta,
                                     double* scratch, cudaStream_t st);
cudaError_t launch_shard_scan_apply(const SysPlan* plan, const double* tabs, const ScanMap& map, const double* beta,
                                    double* iface, double* scratch, cudaStream_t st);

// adjoint: gt[3 s + j] = -(sum of part[3 i + j] over the CTAs i of system s), fixed order.
//   For k = 0..nsys-1: s = sys_ids[k], CTAs first[k] .. first[k] + count[k] - 1 (device
//   arrays), or (nullptr) one system s = k = 0 covering CTAs 0 .. count0 - 1.
cudaError_t launch_adj_finalize(const double* part, const int32_t* sys_ids, const int64_t* first,
                                const int64_t* count, int64_t count0, int64_t nsys, double* gt, cudaStream_t st);

// systems of one row: x = F / t_0.  idx: device list of system indices (nullptr: the single
// system of `plans`).
cudaError_t launch_trivial(const SysPlan* plans, const int32_t* idx, int64_t nidx, const double* F,
                           double* x, const double* xf, const double* w, double* gt, int sys_offset,
                           cudaStream_t st);

// quasi-Toeplitz corner data of a plan (eq. 21): g[Lg] = T^-1 e_0 (leading rows), h[Lh] = T^-1 e_{N-1}
// (trailing rows, h[k] is row N-1-k), W = (I + K)^-1 of the Sherman-Morrison-Woodbury step
struct CornerArgs {
  int64_t N, Lg, Lh;
  const double* g;
  const double* h;
  double psi, chi;
  double w00, w01, w10, w11;
};

// x_k <- A^-1 F_k from y_k = T^-1 F_k (already in x_k = x + k ldx), k = 0..M-1: two kernels
cudaError_t launch_corner(double* x, int64_t M, int64_t ldx, const CornerArgs& c, cudaStream_t st);
// one quasi-Toeplitz system of a batch: rows [off, off + N), corner vectors at tab + og (Lg
// entries) and tab + oh (Lh entries), corners psi, chi, (I + K)^-1 = [[w00, w01], [w10, w11]]
struct CornerRec {
  int64_t N, off, Lg, Lh, og, oh;
  double psi, chi, w00, w01, w10, w11;
};
// x <- A_s^-1 F_s from y_s = T_s^-1 F_s (already in x) for every listed system: one CTA each
cudaError_t launch_corner_batch(const CornerRec* recs, int64_t n, const double* tab, double* x, cudaStream_t st);

// residual check of one (quasi-)Toeplitz system (res: 3 maxima, zeroed first)
cudaError_t launch_toeplitz_residual(int64_t N, double tm1, double t0, double tp1, double psi, double chi,
                                     const double* F, const double* x, unsigned long long* res, cudaStream_t st);
// adjoint of a batch with quasi-Toeplitz systems: recs are the transposed corner records of every
// system; gt3 the Toeplitz gradients (3 per system), gt5 the result (5 per system)
cudaError_t launch_corner_adjoint_batch(const CornerRec* recs, int64_t nsys, const double* tab, const double* xf,
                                        double* lam, const double* gt3, double* gt5, cudaStream_t st);
// adjoint of a quasi-Toeplitz plan: gradient terms of the corner correction, dL/dpsi, dL/dchi
// (gt[0..4]), then the corner correction of lambda (c: the transposed corner vectors)
cudaError_t launch_corner_adjoint(const double* xf, double* lam, double* gt, const CornerArgs& c, cudaStream_t st);
// dL/dpsi = -lambda_0 x_0 and dL/dchi = -lambda_{N-1} x_{N-1} (gt[3], gt[4]) of a corner plan whose
// corners are zero (lambda needs no correction there)
cudaError_t launch_end_gradients(const double* xf, const double* lam, double* gt, int64_t N, cudaStream_t st);

}  // namespace dich
