/*
 * dichotomy.h -- C ABI of the GB300 (sm_103a) Dichotomy solver for tridiagonal
 * Toeplitz systems  T x = F,  T = tridiag{t_-1, t_0, t_1}   (arXiv 1002.2469, eq. 1).
 *
 * Conventions shared by every entry point
 *   - Rows are 0-based: row i reads t_-1 x[i-1] + t_0 x[i] + t_1 x[i+1] = F[i], with
 *     x[-1] = x[N] = 0 (the Dirichlet ends of eq. 22).  t_-1 is the sub-diagonal (the
 *     paper's c_i, eq. 2), t_1 the super-diagonal (the paper's a_i).
 *   - Pointers named d_* are CUDA device pointers; h_* are host pointers.  FP64 vectors
 *     are contiguous, 8-byte aligned, and not aliased with each other (x may not alias F:
 *     DICH_ERR_ALIAS).  Host pointers passed where device pointers are required are
 *     rejected with DICH_ERR_ARG; the library has no CPU fallback.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *     Solve/adjoint calls only enqueue work: they never synchronize, never allocate
 *     device memory and are safe to capture in a CUDA graph once the plan is bound
 *     (dichotomy_solve_host creates its two copy streams and events on first use; binds,
 *     status reads and the residual checks synchronize; dichotomy_solve_noalloc stages its
 *     plan from pageable host memory and refuses capture, see there).
 *   - Plan and batch objects are not locked: calls on one object from several host threads
 *     must be serialized by the caller; distinct objects are independent.
 *   - Device memory is owned by the caller.  The library owns only host-side plan
 *     objects (freed by dichotomy_destroy / dichotomy_batch_destroy).
 *   - Every function returns a dich_status (0 = DICH_OK).  Errors detected on the GPU
 *     (non-finite output, plan/schedule mismatch) are latched in a device status word
 *     inside the workspace and read back with dichotomy_status().
 *
 * The method (what each call computes)
 *   N rows are split into P blocks of n rows (the last block takes the remainder; every
 *   block has >= 2 rows, Sec. 2.1).  The Toeplitz preliminary calculation (Sec. 3.1,
 *   Theorem 1 / eq. 20, in the exact factored form of eq. 24-25) is done once per
 *   (t, n): recurrence roots, the two boundary spikes of the block operator T_n and the
 *   O(1) per-block exterior ratios Z (eq. 10-12).  A solve then (a) sweeps every block
 *   locally, giving beta^{L,R}_m of eq. 16, (b) computes the first/last value of every
 *   block from eq. 15 as two affine scans over blocks -- the log2 P dichotomy tree of
 *   eq. 17-19, mapped onto warp shuffles, shared memory and the grid -- and (c) applies
 *   the basis correction that solves every block interior (eq. 7).  The result is
 *   x = T^-1 F up to rounding.
 */
#ifndef DICHOTOMY_H_
#define DICHOTOMY_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
typedef enum {
  DICH_OK = 0,
  DICH_ERR_ARG = 1,           /* bad size, NULL / host / misaligned pointer, bad option */
  DICH_ERR_NOT_DOMINANT = 2,  /* |t_0| < |t_-1| + |t_1|: eq. 32-33 fails (not supported) */
  DICH_ERR_SINGULAR = 3,      /* t_0 = 0 with dominance, or a zero block pivot (Theorem 1) */
  DICH_ERR_TIMEOUT = 4,       /* a bounded wait for a kernel's own bulk copies ran out (not
                                 expected; no kernel waits on another CTA or rank) */
  DICH_ERR_NONFINITE = 5,     /* a NaN/Inf was produced on the device */
  DICH_ERR_CUDA = 6,          /* a CUDA runtime call failed; see dichotomy_last_cuda_error */
  DICH_ERR_ALIAS = 7,         /* output aliases an input */
  DICH_ERR_UNBOUND = 8,       /* solve called before the plan was bound to a workspace */
  DICH_ERR_WORKSPACE = 9,     /* workspace too small or misaligned */
  DICH_ERR_SCHEDULE = 10,     /* batch coefficients at solve time need a larger schedule */
  DICH_ERR_UNSUPPORTED = 11   /* combination not supported by this build */
} dich_status;

/* ---------------------------------------------------------------- options */
typedef enum {
  DICH_PREC_F64 = 0,    /* every step in FP64 */
  DICH_PREC_MIXED = 1,  /* local sweeps and spike correction in compensated FP32 (float-float, one
                           power-of-two scale per window); block quantities and the in-window tree
                           in float-float, the general path's block scan in FP64.  Toeplitz plans
                           need the scale factor g = -1/q (T = -q (1 - rs E^-1)(1 - ib E)) within
                           2^-60..2^60 */
  DICH_PREC_AUTO = 2    /* MIXED where the two recurrences' error gain is at most 24 (error about
                           1e-14 relative) and MIXED's range conditions hold, else F64 */
} dich_precision;

enum {
  DICH_FLAG_FORCE_GENERAL = 1,  /* never truncate cross-tile coupling (3-kernel path) */
  DICH_FLAG_CHECK_FINITE = 2,   /* latch DICH_ERR_NONFINITE if any output is not finite */
  DICH_FLAG_HOST_PRELIM = 4,    /* general matrices: preliminary step on the host at plan time */
  DICH_FLAG_DEVICE_PRELIM = 8,  /* general matrices: preliminary step on the device at bind time */
  DICH_FLAG_ALLOW_NOT_DOMINANT = 16, /* accept matrices without diagonal dominance.  Toeplitz plans and
                                        batches: when the roots of t_1 r^2 + t_0 r + t_-1 are real and
                                        separated by the unit circle (what the recurrences need);
                                        general matrices: any rows, judged by dich_plan_info.growth;
                                        check results with dichotomy_residual / dichotomy_gen_residual */
  /* MIXED-form window kernel of Toeplitz plans and batches (the results agree to rounding):
   * the register path keeps a thread's two 16-row blocks in registers (bulk copies in and out,
   * four CTAs per SM); the shared-memory path sweeps the window's tile in shared memory (six CTAs
   * per SM).  Default: the register path for single plans, and for batches unless most of their
   * MIXED windows are whole one-window systems (latency-bound windows, where occupancy wins). */
  DICH_FLAG_REG_PATH = 32,           /* the register path wherever its window shape allows */
  DICH_FLAG_SMEM_PATH = 64           /* the shared-memory path for every window */
};

typedef struct {
  int32_t block_size;    /* n, rows per block; 0 = chosen by the library */
  int32_t precision;     /* dich_precision */
  int32_t threads;       /* window width in blocks (CTA size): 0 = default; 64, 128 or 256 */
  int32_t flags;         /* DICH_FLAG_* */
  double trunc_eps;      /* relative truncation of geometrically small terms; 0 = the
                            default: 2^-64 for F64 plans, 2^-56 for MIXED plans (whose
                            float-float values carry about 48 bits) */
} dich_opts;

/* Read-only description of a plan (for tests, tuning and reporting). */
typedef struct {
  int64_t N, P;            /* rows, blocks */
  int32_t n, n_last;       /* block size, size of the last block */
  int32_t threads;         /* CTA width (window blocks) */
  int32_t halo_l, halo_r;  /* halo blocks per window (0 on the general path) */
  int32_t path;            /* 0 = single window, 1 = halo windows, 2 = general 3-kernel */
  int32_t precision;       /* effective dich_precision (F64 or MIXED) */
  int64_t tiles;           /* CTAs per solve */
  int32_t Lv, Lw;          /* truncated lengths of the block spikes */
  int32_t kl, kr;          /* blocks with end-dependent coefficients at the left/right end */
  double rs, ib;           /* roots: |rs| <= 1 <= |1/ib| of t_1 r^2 + t_0 r + t_-1 = 0 */
  double z;                /* rs * ib */
  size_t workspace_bytes;
  size_t beta_offset;      /* general path: byte offsets into the workspace of the per-block */
  size_t iface_offset;     /* (beta^L, beta^R) of eq. 16 and first/last values (x_s, x_e) of
                              eq. 18 the last solve left there, 2 doubles per block; 0 otherwise */
  double growth;           /* general matrices: the a priori error growth gamma^l of the error
                              estimate after eq. 33 (gamma: the largest block map factor, at least 1;
                              l = ceil(log2 P) dichotomy levels); 1 under diagonal dominance */
} dich_plan_info;

typedef struct dich_plan_s* dich_plan_t;
typedef struct dich_batch_s* dich_batch_t;
typedef struct dich_gen_s* dich_gen_t;

/* ---------------------------------------------------------------- single system */

/* Build a plan for one N x N system (host only, no GPU work).  Performs the paper's
 * Toeplitz preliminary step (Sec. 3.1-3.3): validates diagonal dominance (eq. 32-33,
 * equality accepted), computes the recurrence roots of Theorem 1, the truncation lengths,
 * the spikes of the block operator and the per-block exterior ratios (eq. 24-25 in
 * overflow-free factored form).  N = 0 and N = 1 are accepted (trivial solves).
 * Errors: DICH_ERR_ARG (N < 0, out == NULL, bad opts), DICH_ERR_NOT_DOMINANT,
 * DICH_ERR_SINGULAR (t_0 == 0), DICH_ERR_UNSUPPORTED (DICH_PREC_MIXED requested with the scale
 * factor g outside 2^-60..2^60).  On error *out is set to NULL. */
int dichotomy_plan(double t_m1, double t_0, double t_1, int64_t N, dich_plan_t* out);
int dichotomy_plan_ex(double t_m1, double t_0, double t_1, int64_t N, const dich_opts* opts,
                      dich_plan_t* out);

/* A plan for the quasi-Toeplitz matrix of Sec. 3.1, eq. 21: tridiag{t_-1, t_0, t_1} of order N
 * with the first diagonal entry t_0 + psi and the last t_0 + chi (Neumann or Robin ends; a
 * single row reads t_0 + psi + chi).  The solve is the Toeplitz Dichotomy solve y = T^-1 F
 * followed by the rank-2 corner correction x = y - c_0 g - c_1 h (Sherman-Morrison-Woodbury:
 * g, h are the first and last columns of T^-1 in closed form, kept where they exceed the
 * truncation threshold, and (c_0, c_1) solves a 2x2 system in psi y_0, chi y_{N-1}); two extra
 * small kernels per solve.  psi = chi = 0 gives the plain Toeplitz plan.  dichotomy_solve,
 * dichotomy_solve_series and dichotomy_adjoint (with dL/dpsi, dL/dchi) serve the plan.
 * Errors: as dichotomy_plan_ex; DICH_ERR_NOT_DOMINANT when an end row loses dominance
 * (|t_0 + psi| < |t_1| or |t_0 + chi| < |t_-1|), DICH_ERR_SINGULAR when the corner system is. */
int dichotomy_plan_quasi(double t_m1, double t_0, double t_1, double psi, double chi, int64_t N,
                         const dich_opts* opts, dich_plan_t* out);

/* Describe a plan.  Errors: DICH_ERR_ARG. */
int dichotomy_plan_info(dich_plan_t plan, dich_plan_info* info);

/* Bytes of device workspace the plan needs (256-byte aligned region). */
int dichotomy_plan_workspace_bytes(dich_plan_t plan, size_t* bytes);

/* Attach a caller-owned device workspace of at least dichotomy_plan_workspace_bytes
 * bytes (256-byte aligned) and upload the plan tables into it on `stream`
 * (one cudaMemcpyAsync from a host staging copy held by the plan; the status word is
 * cleared).  Must precede solve/adjoint; may be called again to move the plan.
 * Errors: DICH_ERR_ARG, DICH_ERR_WORKSPACE, DICH_ERR_CUDA. */
int dichotomy_plan_bind(dich_plan_t plan, void* d_workspace, size_t bytes, void* stream);

/* x = T^-1 F for the bound plan.  d_F, d_x: N doubles each on the device, no aliasing.
 * Enqueues one kernel (single/halo path) or three (general path) on `stream`.
 * Errors: DICH_ERR_ARG, DICH_ERR_ALIAS, DICH_ERR_UNBOUND, DICH_ERR_CUDA (launch). */
int dichotomy_solve(dich_plan_t plan, const double* d_F, double* d_x, void* stream);

/* A series with a constant matrix (Sec. 1, eq. 2; Sec. 3.1): x_k = T^-1 F_k for the M
 * right-hand sides F_k = d_F + k ldf, x_k = d_x + k ldx (k = 0 .. M-1; row-major [M][N] when
 * ldf = ldx = N).  The plan (the preliminary step) serves every right-hand side.  The single
 * and halo paths enqueue one kernel per 65535 right-hand sides; the general path three
 * kernels per right-hand side, in order on `stream`.  M = 1 is dichotomy_solve.
 * Errors: DICH_ERR_ARG (M < 0, ld < N for M > 1, null/misaligned/host pointers),
 * DICH_ERR_ALIAS (the F and x ranges overlap), DICH_ERR_UNBOUND, DICH_ERR_CUDA (launch). */
int dichotomy_solve_series(dich_plan_t plan, int64_t M, const double* d_F, int64_t ldf, double* d_x,
                           int64_t ldx, void* stream);

/* x = T^-1 F with F and x in host memory (not in the paper: the solve of eq. 1 fed from and
 * returned to the host).  h_F, h_x: N doubles each in host memory, no aliasing; d_F, d_x: N
 * doubles each of device staging memory owned by the caller.  Two ways, chosen by `chunks`:
 *  - chunks = 0 and h_F, h_x page-locked memory mapped into the device's address space
 *    (cudaHostAlloc, cudaHostRegister, torch pin_memory): the window kernels read F and write x
 *    there directly, one pass over the host link (d_F, d_x unused, may be NULL); not on the
 *    general path (it reads F twice), which takes the copies below;
 *  - otherwise the copies: on the halo path of a Toeplitz plan the rows go to d_F in `chunks`
 *    pieces of whole windows (0 = min(16, windows); 1 = no pipeline), the windows of a piece are
 *    solved on `stream` as soon as the rows they read (their own and the right halo) have
 *    arrived, and their own rows of x go back from d_x while later pieces are still being copied
 *    in and solved (copy-in, kernels and copy-out overlap on `stream` and two copy streams the
 *    plan creates on first use; pageable host memory works, its copies serialise).  Other plans
 *    (one window, the general path, quasi-Toeplitz corners): copy in, solve, copy out.
 * Enqueues only: h_x is complete once `stream` has synchronized; h_F, h_x, d_F, d_x must not be
 * reused before.  Errors: DICH_ERR_ARG (null/misaligned pointers, h_* on the device, d_* not on
 * the device when needed, chunks < 0), DICH_ERR_ALIAS, DICH_ERR_UNBOUND, DICH_ERR_CUDA. */
int dichotomy_solve_host(dich_plan_t plan, const double* h_F, double* h_x, double* d_F, double* d_x, int32_t chunks,
                         void* stream);

/* Adjoint of L(x) with x = T^-1 F, given d_w = dL/dx and the forward solution d_x:
 *   d_gF = lambda = T^-T w   (the same Dichotomy solve for T^T = tridiag{t_1, t_0, t_-1}),
 *   d_gt[0..2] = (dL/dt_-1, dL/dt_0, dL/dt_1) = -(sum_i lambda_i x_{i-1},
 *                sum_i lambda_i x_i, sum_i lambda_i x_{i+1}).
 * Plans made by dichotomy_plan_quasi (eq. 21; zero corners included): lambda = A^-T w (the
 * transposed corner correction after T^-T w, none for zero corners) and d_gt holds 5 doubles,
 * adding dL/dpsi = -lambda_0 x_0 and dL/dchi = -lambda_{N-1} x_{N-1}, all computed on the
 * device.  Not in the paper.  d_gt is 3 (5) doubles on the device.
 * d_gF may not alias d_w or d_x. */
int dichotomy_adjoint(dich_plan_t plan, const double* d_w, const double* d_x, double* d_gF,
                      double* d_gt, void* stream);

/* A posteriori check of a solution (as dichotomy_gen_residual): h_out[0] = max_i |F_i - (T x)_i|,
 * h_out[1] = max|F - T x| / (||T||_inf max|x| + max|F|), with the corners of eq. 21 for
 * quasi-Toeplitz plans.  d_F, d_x: N doubles on the device; h_out: 2 doubles on the host.
 * Synchronizes `stream`.  Errors: DICH_ERR_ARG, DICH_ERR_UNBOUND, DICH_ERR_CUDA. */
int dichotomy_residual(dich_plan_t plan, const double* d_F, const double* d_x, double* h_out, void* stream);

/* Synchronize `stream`, read and clear the device status word of a bound plan.
 * *device_status receives DICH_OK or the first latched device error. */
int dichotomy_status(dich_plan_t plan, void* stream, int* device_status);

void dichotomy_destroy(dich_plan_t plan);

/* x = T^-1 F for one system without any allocation by the library.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory themselves (for
 * example code running under a framework whose allocator owns the device, or plugins
 * forbidden to call cudaMalloc).  It plans on the host into a static buffer and keeps the
 * plan on the device in one library-owned static array of 256 KiB per GPU, held until the
 * process exits; no cudaMalloc, cudaFree or other allocating routine is called.
 * d_F, d_x: N doubles on the device, no aliasing.  Precision policy DICH_PREC_AUTO.
 * Limit: the plan tables (and, for systems on the general path, 32 bytes per block of beta
 * and first/last values plus the block-scan scratch) must fit the array; larger needs --
 * long systems whose coupling does not decay, such as the 1-D Laplacian -- return
 * DICH_ERR_WORKSPACE (use dichotomy_plan + dichotomy_solve with a caller workspace).
 * Every call reuses the same array (its status word is cleared on each call, so these solves
 * report no device status): calls whose kernels overlap on the GPU (other streams, other host
 * threads) race; calls on one stream are ordered.  The first call on a device looks up the
 * array's device address.  Unlike the other solve calls this one may block the host: the plan
 * reaches the array by a copy from a static pageable host buffer, which waits until `stream`
 * has reached it.  It cannot be captured in a CUDA graph: a capturing stream gets
 * DICH_ERR_UNSUPPORTED (a captured copy would replay the buffer's later contents).
 * Errors: DICH_ERR_ARG (N < 0, null/misaligned pointers, pointers not on the current device),
 * DICH_ERR_NOT_DOMINANT, DICH_ERR_SINGULAR, DICH_ERR_ALIAS, DICH_ERR_WORKSPACE,
 * DICH_ERR_UNSUPPORTED, DICH_ERR_CUDA. */
int dichotomy_solve_noalloc(double t_m1, double t_0, double t_1, int64_t N, const double* d_F, double* d_x,
                            void* stream);

/* ---------------------------------------------------------------- one system in shards */

/* The paper's distributed dichotomy process (Sec. 2.4-2.5: blocks spread over p processes, the
 * interface values gathered by eq. 17-19's levels) for callers that split one system across
 * devices or processes: shard k of nshards owns a contiguous range of whole windows of the plan
 * (blocks [block_lo, block_hi), rows [row_lo, row_hi)) and holds only its own rows of F and x.
 * Because the dichotomy tree's maps compose associatively (Sec. 2.5), the levels collapse into one
 * exchange of four numbers per shard plus one value to each neighbour:
 *   1. dichotomy_shard_reduce:  beta of the shard's blocks (eq. 16) and its block scan; returns
 *      the shard's composite maps h_maps = (prefix a, b, suffix a, b) of eq. 15's two scans;
 *   2. the caller all-gathers the 4 numbers of every shard (h_all_maps[4 nshards], in shard order);
 *   3. dichotomy_shard_bounds:  folds the other shards' maps into the prefix entering the shard
 *      and the suffix beyond it (on the device) and finishes its first/last values (eq. 18);
 *      returns h_ends = (x at row_lo, x at row_hi - 1);
 *   4. the caller passes each neighbour its boundary value: shard k receives
 *      h_nbr = (h_ends[1] of shard k-1, h_ends[0] of shard k+1), zeros at the system's ends;
 *   5. dichotomy_shard_finish:  the shard's interiors (eq. 7) into d_x.
 * Any plan of N >= 2 rows without quasi-Toeplitz corners serves (its tables must be bound);
 * nshards <= the plan's windows (dich_plan_info.tiles).  d_F, d_x: the shard's rows only, device,
 * no aliasing (d_x also receives intermediate values between steps 1 and 5 in the FP64 form).
 * d_ws: the shard's own device workspace of dich_shard_info.workspace_bytes (256-byte aligned),
 * kept from step 1 to step 5.  Steps 1 and 3 synchronize `stream` (they return host values).
 * Errors: DICH_ERR_ARG, DICH_ERR_ALIAS, DICH_ERR_UNBOUND, DICH_ERR_WORKSPACE, DICH_ERR_UNSUPPORTED
 * (N < 2, corners), DICH_ERR_CUDA. */
typedef struct {
  int64_t row_lo, row_hi;      /* the shard's rows of the system */
  int64_t block_lo, block_hi;  /* its blocks */
  size_t workspace_bytes;      /* device workspace one shard needs */
} dich_shard_info;
int dichotomy_shard_info(dich_plan_t plan, int32_t nshards, int32_t k, dich_shard_info* info);
int dichotomy_shard_reduce(dich_plan_t plan, int32_t nshards, int32_t k, const double* d_F, double* d_x,
                           void* d_ws, size_t ws_bytes, double* h_maps, void* stream);
int dichotomy_shard_bounds(dich_plan_t plan, int32_t nshards, int32_t k, const double* h_all_maps, void* d_ws,
                           size_t ws_bytes, double* h_ends, void* stream);
int dichotomy_shard_finish(dich_plan_t plan, int32_t nshards, int32_t k, const double* d_F, double* d_x,
                           const double* h_nbr, void* d_ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- batches */

/* A series of independent systems (the paper's eq. 2 series, or separation-of-variables
 * modes), stored back to back: system s occupies F[offset[s] .. offset[s] + N[s]).
 * Prepare (host only) runs the preliminary step of every system, chooses block sizes,
 * the precision form per system (DICH_PREC_AUTO) and an LPT-ordered list of windows.
 * h_N, h_offset, h_tm1, h_t0, h_tp1: nsys entries each on the host.
 * Errors: DICH_ERR_ARG, DICH_ERR_NOT_DOMINANT / DICH_ERR_SINGULAR (first bad system),
 * DICH_ERR_UNSUPPORTED (DICH_PREC_MIXED with a system's scale factor outside 2^-60..2^60). */
int dichotomy_batch_prepare(int64_t nsys, const int64_t* h_N, const int64_t* h_offset,
                            const double* h_tm1, const double* h_t0, const double* h_tp1,
                            const dich_opts* opts, dich_batch_t* out);

/* A batch in which system s is the quasi-Toeplitz matrix of eq. 21: tridiag{t_-1, t_0, t_1}[s]
 * with t_0 + psi[s] in its first row and t_0 + chi[s] in its last (host arrays of nsys entries;
 * psi = chi = 0 leaves a system plain).  The Toeplitz solves run as in dichotomy_batch_prepare;
 * then one CTA per quasi system applies its rank-2 corner correction (as dichotomy_plan_quasi).
 * dichotomy_adjoint_batched on such a batch returns lambda_s = A_s^-T w_s and 5 doubles per
 * system in d_gt: dL/dt_-1, dL/dt_0, dL/dt_1, dL/dpsi, dL/dchi (as dichotomy_adjoint).
 * Errors: as dichotomy_batch_prepare and dichotomy_plan_quasi (per system). */
int dichotomy_batch_prepare_quasi(int64_t nsys, const int64_t* h_N, const int64_t* h_offset, const double* h_tm1,
                                  const double* h_t0, const double* h_tp1, const double* h_psi, const double* h_chi,
                                  const dich_opts* opts, dich_batch_t* out);
int dichotomy_batch_workspace_bytes(dich_batch_t batch, size_t* bytes);
int dichotomy_batch_bind(dich_batch_t batch, void* d_workspace, size_t bytes, void* stream);
/* Solve every system of the batch in one launch per precision form. */
int dichotomy_solve_batched(dich_batch_t batch, const double* d_F, double* d_x, void* stream);
/* Batched adjoint: d_gF like d_x; d_gt is nsys x 3 doubles (dL/dt_-1, dL/dt_0, dL/dt_1), or
 * nsys x 5 for a batch from dichotomy_batch_prepare_quasi (adding dL/dpsi, dL/dchi). */
int dichotomy_adjoint_batched(dich_batch_t batch, const double* d_w, const double* d_x,
                              double* d_gF, double* d_gt, void* stream);
int dichotomy_batch_status(dich_batch_t batch, void* stream, int* device_status);
/* Systems, windows and the precision form chosen per system (nsys int32, 0 = F64, 1 = MIXED). */
int dichotomy_batch_info(dich_batch_t batch, int64_t* nsys, int64_t* windows, int32_t* h_form);
void dichotomy_batch_destroy(dich_batch_t batch);

/* ---------------------------------------------------------------- misc */
const char* dichotomy_strerror(int status);
/* The last CUDA error string seen by this thread (empty if none). */
const char* dichotomy_last_cuda_error(void);
/* Library version, e.g. "0.1.0". */
const char* dichotomy_version(void);

/* ---------------------------------------------------------------- general tridiagonal matrices
 * The Dichotomy Algorithm for a general (non-Toeplitz) tridiagonal matrix (Sec. 2): row i reads
 * a_i x_{i-1} + b_i x_i + c_i x_{i+1} = F_i (a_0 and c_{N-1} are ignored).  The preliminary step
 * (Sec. 2.3) is the general O(N) one: the whole-system elimination factors (the homogeneous
 * solutions that give the exterior vectors of eq. 10-12 as ratios), each block's own Thomas
 * factors and spikes, and the block maps of the dichotomy tree.  It runs on the device at bind
 * time (from 2^15 rows, or with DICH_FLAG_DEVICE_PRELIM: the elimination factors as prefix and
 * suffix products of 2x2 matrices over the blocks) or on the host at plan time (below 2^15 rows,
 * or with DICH_FLAG_HOST_PRELIM).  Every solve of a series (eq. 2) reuses it.  FP64 or
 * float-float (see dichotomy_gen_plan).  The
 * plan keeps 5 doubles per row of factors and spikes and the matrix itself (for the residual
 * check) in the device workspace (64 bytes per row, plus 80 bytes per block); the device
 * preliminary adds 64 bytes per block. */

/* Plan for the N x N matrix given by the host arrays h_a (sub-diagonal), h_b (diagonal), h_c
 * (super-diagonal), N entries each (copied; the caller keeps ownership).  opts as for
 * dichotomy_plan_ex; DICH_PREC_MIXED runs the local solves and the correction in float-float
 * (factors within 2^-40..2^40, else DICH_ERR_UNSUPPORTED -- from dichotomy_gen_bind with the
 * device preliminary); DICH_PREC_AUTO takes MIXED when the local recurrences' error gains
 * stay below 24 (as for Toeplitz plans) and the factors are in range, else FP64.  Default
 * geometry: 64-thread windows of 32-row blocks for FP64 plans, 128-thread windows of 16-row
 * blocks for MIXED and AUTO plans.
 * Every row must satisfy |b_i| >= |a_i| + |c_i| (eq. 32-33) unless DICH_FLAG_ALLOW_NOT_DOMINANT
 * is set; then the block maps may grow (dich_plan_info.growth bounds the error growth a priori)
 * and dichotomy_gen_residual checks the solution a posteriori.  Errors: DICH_ERR_ARG (null, negative N, non-finite entry,
 * bad opts), DICH_ERR_NOT_DOMINANT, DICH_ERR_SINGULAR (a zero pivot; with the device preliminary
 * reported by dichotomy_gen_bind), DICH_ERR_UNSUPPORTED. */
int dichotomy_gen_plan(int64_t N, const double* h_a, const double* h_b, const double* h_c, const dich_opts* opts,
                       dich_gen_t* out);
/* Geometry of a general plan (the Toeplitz-only fields are zero).  With the device preliminary,
 * path, halo_l, halo_r, tiles and precision are provisional (general path) until dichotomy_gen_bind has
 * returned.  Errors: DICH_ERR_ARG. */
int dichotomy_gen_info(dich_gen_t plan, dich_plan_info* info);
/* Bytes of device workspace (256-byte aligned region). */
int dichotomy_gen_workspace_bytes(dich_gen_t plan, size_t* bytes);
/* Attach the caller's workspace and upload the plan on `stream` (with the device preliminary:
 * upload the matrix and run the preliminary step there); returns after all of it has completed.
 * Errors: DICH_ERR_ARG, DICH_ERR_WORKSPACE, DICH_ERR_SINGULAR, DICH_ERR_CUDA. */
int dichotomy_gen_bind(dich_gen_t plan, void* d_workspace, size_t bytes, void* stream);
/* x = A^-1 F: one kernel (one window or halo windows) or three (general path) on `stream`.
 * Errors: DICH_ERR_ARG, DICH_ERR_ALIAS, DICH_ERR_UNBOUND, DICH_ERR_CUDA. */
int dichotomy_gen_solve(dich_gen_t plan, const double* d_F, double* d_x, void* stream);
/* The series form (as dichotomy_solve_series). */
int dichotomy_gen_solve_series(dich_gen_t plan, int64_t M, const double* d_F, int64_t ldf, double* d_x,
                               int64_t ldx, void* stream);
/* The a posteriori check recommended after eq. 33: with F and x (N doubles each on the device),
 * h_out[0] = max_i |F_i - (A x)_i| and h_out[1] = the norm-wise backward error
 * max|F - A x| / (||A||_inf max|x| + max|F|) (2 doubles on the host).  Synchronizes `stream`.
 * Errors: DICH_ERR_ARG, DICH_ERR_UNBOUND, DICH_ERR_CUDA. */
int dichotomy_gen_residual(dich_gen_t plan, const double* d_F, const double* d_x, double* h_out, void* stream);
/* Synchronize, read and clear the device status word (as dichotomy_status). */
int dichotomy_gen_status(dich_gen_t plan, void* stream, int* device_status);
void dichotomy_gen_destroy(dich_gen_t plan);

#ifdef __cplusplus
}
#endif
#endif /* DICHOTOMY_H_ */
