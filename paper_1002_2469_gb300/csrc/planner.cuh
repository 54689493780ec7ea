// planner.cuh -- host-side planning internals shared by the C-ABI translation units
// (C++ linkage, not exported).  Definitions live in api.cu.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dichotomy.h"
#include "dich_internal.cuh"

namespace dich {
namespace plan {

constexpr size_t kAlign = 256;
// shared-memory budget per CTA for library-chosen block sizes (several CTAs share an SM so
// the load, sweeps, tree and store of different windows overlap)
constexpr size_t kSmemBudget = 110 * 1024;
// an explicitly requested block size may use up to the per-CTA maximum (one CTA per SM)
constexpr size_t kSmemMax = 225 * 1024;

struct Opts {
  int n_req = 0;
  int prec = DICH_PREC_F64;
  int NT = 0;
  int flags = 0;
  double eps = 0x1p-64;     // caller's threshold, or the F64 default
  bool eps_given = false;   // false: MIXED plans use kEpsMixed
};

// default truncation of the MIXED form: its float-float values carry about 48 bits, so terms
// below 2^-56 of the coupling are far inside its own rounding
constexpr double kEpsMixed = 0x1p-56;

// Host construction of one system's plan record and tables.  Tables go to `tab`, or to the
// caller's buffer `ext` of `ext_cap` doubles when it is set (no allocation in that case).
struct SysBuild {
  SysPlan rec{};
  std::vector<double> tab;
  int path = PATH_SINGLE;
  double* ext = nullptr;
  size_t ext_cap = 0;
  size_t ext_used = 0;
};

extern thread_local std::string g_cuda_err;
int cuda_fail(cudaError_t e);
size_t align_up(size_t v);
int window_blocks(int NT, int form);
size_t smem_bytes(int NT, int n, int form);
int max_rows(int NT, int form, size_t budget);
int default_threads(int form);
int default_rows(int form);
int validate_t(double tm1, double t0, double tp1, int flags = 0);
int read_opts(const dich_opts* o, Opts& out);
int pick_form(int prec, const Roots& r);
int64_t ceil_div(int64_t a, int64_t b);
int choose_n(int64_t N, int NT, int nmax, int n_req, int n_def);
int build_system(double tm1, double t0, double tp1, int64_t N, int NT, int form, int n, const Opts& o,
                 bool allow_general, SysBuild& sb);
bool is_device_ptr(const void* p);
bool aligned8(const void* p);
bool overlap(const void* a, size_t na, const void* b, size_t nb);
int map_status(unsigned s);

}  // namespace plan
}  // namespace dich
