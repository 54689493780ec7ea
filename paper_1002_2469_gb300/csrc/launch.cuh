// launch.cuh -- internal launch entry points shared by the kernel translation units and the
// host API (C++ linkage, not exported).
#pragma once
#include <cuda_runtime.h>
#include "window.cuh"
#include "window_mixed.cuh"

namespace dich {

// window kernel of width NT (64, 128 or 256) in the given form; returns the launch error
cudaError_t launch_window_f64(int NT, int grid, size_t smem, cudaStream_t st, const WinArgs& a);
cudaError_t launch_window_mixed(int NT, int grid, size_t smem, cudaStream_t st, const WinArgs& a);

// general path: first/last values of every block from per-block beta (global block scan)
//   beta [2P] -> iface [2P]; scratch needs 6 * ceil(P / kScanChunk) doubles.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanThreads * kScanPer;
cudaError_t launch_block_scan(const SysPlan* plan, const double* tabs, int64_t P, const double* beta,
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

}  // namespace dich
