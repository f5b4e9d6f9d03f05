/*
 * chol.h -- C ABI of the GB300 (sm_103a) tiled Cholesky library.
 *
 * The library factors a dense symmetric positive definite matrix with the right-looking
 * tile algorithm that the paper schedules (PLASMA DPOTRF: POTRF, TRSM, SYRK and GEMM tile
 * tasks; Section 4.1 "Benchmarks", double precision and 512 x 512 tiles in Section 4.1
 * "Methodology"), and solves with the factor. The tile task graph runs on one GPU inside a
 * persistent data-flow kernel: every thread block is a worker with its own ready queue,
 * and the pop / push / steal / activate operations of Section 2.2 place newly ready tasks
 * with HEFT (Algorithm 1), DADA(alpha) (Algorithm 2), work stealing (Section 4.3
 * "Comparison with work stealing") or a static owner-computes map.
 *
 * Conventions shared by every entry point
 *  - Matrices are column-major with a leading dimension (LAPACK), double precision.
 *  - Pointers named d... are DEVICE pointers on the current CUDA device; h... are host
 *    pointers. The caller owns all memory, including the workspaces; the library keeps no
 *    pointer after a call returns and allocates no device memory (chol_posv_host, too,
 *    works in a caller-provided device buffer).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls
 *    that take a stream are asynchronous with respect to the host: the return value only
 *    reports argument checks and launch errors; numerical status is written to device
 *    memory (dInfo) and is valid once the stream has reached that point.
 *  - Return values are chol_status codes. A negative code means nothing was launched,
 *    except CHOL_ERR_CUDA raised by a failed launch.
 */
#ifndef CHOL_GB300_H
#define CHOL_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CHOL_OK = 0,
  CHOL_ERR_INVALID_ARG = -1,  /* a size, leading dimension, option or pointer is invalid */
  CHOL_ERR_CUDA = -2,         /* a CUDA runtime call failed (cudaGetLastError has the cause) */
  CHOL_ERR_WORKSPACE = -3,    /* the workspace is smaller than the matching _workspace_size */
  CHOL_ERR_TIMEOUT = -4,      /* a device wait saw no progress for opts.timeout_ns (sync calls) */
  CHOL_ERR_UNSUPPORTED = -5,  /* the device is not sm_103 or the shape exceeds a limit */
  CHOL_ERR_NOT_SPD = 1        /* the matrix is not positive definite (sync calls) */
} chol_status;

/* Values written to *dInfo by the factorization (LAPACK convention for j > 0). */
#define CHOL_INFO_OK 0
/* j > 0: the leading minor of order j is not positive definite (pivot <= 0 or NaN). */
#define CHOL_INFO_TIMEOUT (-1)      /* a bounded device wait expired; results are undefined */
#define CHOL_INFO_QUEUE_FULL (-2)   /* internal: a ready queue overflowed (never expected) */
#define CHOL_INFO_BAD_ARG (-3)      /* batched calls: this matrix's size or leading dimension is invalid */

/* Ready-queue policies of the activate operation (Section 3). */
typedef enum {
  CHOL_POLICY_HEFT = 0,   /* Algorithm 1: priority order, earliest-finish-time worker */
  CHOL_POLICY_DADA = 1,   /* Algorithm 2: affinity phase up to alpha*lambda, then dual approx. */
  CHOL_POLICY_STEAL = 2,  /* successors stay on the finishing worker, FIFO, idle workers steal */
  CHOL_POLICY_STATIC = 3  /* owner computes: the worker is fixed by the tile a task writes */
} chol_policy;

/* Options of chol_factor. Initialise with chol_opts_default and change what is needed. */
typedef struct {
  int nb;                 /* tile order; 0 (default) = automatic: 128 for n <= 32768, else 256.
                             16 <= nb <= 1024 and ceil(n/nb) <= 1024 */
  int policy;             /* chol_policy */
  double alpha;           /* DADA affinity parameter, 0 <= alpha <= 1 (Section 3.2) */
  int steal;              /* 1: an idle worker steals from random victims (Section 2.1) */
  int workers_per_sm;     /* persistent thread blocks per SM: 1 or 2; 0 = 2 */
  int num_workers;        /* 0 = all SMs x workers_per_sm; else a smaller worker count */
  int queue_order;        /* 0 = by priority (bottom level), 1 = FIFO (arrival order) */
  int dada_max_iter;      /* bisection steps of Algorithm 2; 0 = 16 */
  double dada_eps;        /* stop when upper - lower <= dada_eps * first upper; 0 = 0.01 */
  long long cost_ns[4];   /* predicted time of one POTRF, TRSM, SYRK, GEMM tile task (ns);
                             0 = derived from the task's flops and a per-kind rate per SM (FP64:
                             7.5 GFLOP/s; FP32 forms: see chol_factor_lowp), divided among
                             the workers of an SM */
  long long timeout_ns;   /* a device wait that sees no progress for this long gives up and
                             writes CHOL_INFO_TIMEOUT; 0 = 10 s */
  int trace;              /* 1: record per task (worker, queue, start ns, end ns) */
  long long hold_task;    /* fault injection for tests of the bounded waits: the task with
                             this id gets one extra dependency, so it never becomes ready
                             and the run ends with CHOL_INFO_TIMEOUT; -1 (default) = none */
  int use_cp;             /* 1: communication prediction (DADA(alpha)+CP; transfer-aware HEFT):
                             a task placed on a worker that did not write one of its input
                             tiles last pays that tile's bytes / cp_gbs (Section 4.1) */
  double cp_gbs;          /* bandwidth per worker for that prediction, GB/s; 0 = 40 */
  int split;              /* 0 = every task runs on one worker; 1 (default) = the TRSMs of tile
                             rows k + 1 and k + 2 and the SYRK of tile row k + 1 (the critical
                             path), and any TRSM, SYRK or GEMM that starts while SMs idle with no
                             queued task for them, are cut into units -- 64-row TRSM bands,
                             64 x 64 (FP64) or 128 x 128 (FP32 FFMA) SYRK / GEMM blocks; the
                             tensor-core updates stay whole -- that idle workers take before
                             their own queues; 2 = every TRSM, SYRK and GEMM. The factor is
                             bitwise the same in every mode */
  int keep_next;          /* HEFT and DADA with priority queues: 1 (default) = a worker that
                             completes a task runs the most urgent task it made ready next when
                             that task outranks everything queued on it (it would be popped
                             first there anyway); 0 = every ready task is placed and queued */
} chol_opts;

void chol_opts_default(chol_opts *opts);
/* sizeof(chol_opts) as compiled into the library (for bindings that mirror the struct). */
size_t chol_opts_size(void);

/* ---------------------------------------------------------------------------------------
 * Factorization A = L L^T (Section 4.1: tile Cholesky DPOTRF; Section 2: data-flow
 * execution; Section 2.2: pop/push/steal/activate; Section 2.3: per-processor predicted
 * completion time-stamps; Algorithms 1 and 2: the activate policies).
 *
 * dA    n x n, leading dimension lda >= max(1, n). On entry the lower triangle holds A; on
 *       exit it holds L. The strict upper triangle is neither read nor written.
 * opts  host pointer, may be NULL (defaults).
 * dWork device workspace of at least chol_factor_workspace_size(n, opts) bytes, 256-byte
 *       aligned. Its contents on entry do not matter; on exit it holds the schedule state
 *       (and the trace when opts->trace is set, see chol_factor_trace_offset).
 * dInfo device int: CHOL_INFO_OK, j > 0 (the leading minor of order j is not positive
 *       definite; A is then left in an unspecified state) or a negative CHOL_INFO_*.
 * Runs one initialisation kernel and one persistent kernel on `stream`.
 */
size_t chol_factor_workspace_size(int n, const chol_opts *opts);
chol_status chol_factor(int n, double *dA, int lda, const chol_opts *opts, void *dWork,
                        size_t work_bytes, int *dInfo, void *stream);

/* Byte offset inside dWork of the trace written when opts->trace = 1: one record of four
 * int64 per task, in task-id order: {worker that ran it, worker whose queue it was taken
 * from, start time (ns, %globaltimer), end time (ns)}. -1 if tracing is off. */
long long chol_factor_trace_offset(int n, const chol_opts *opts);

/* ---------------------------------------------------------------------------------------
 * Solve A X = B with the factor from chol_factor: forward substitution L Y = B, then back
 * substitution L^T X = Y (the solves that consume the factor; the paper's experiments
 * stop at the factorization).
 *
 * dL    the array written by chol_factor (lower triangle used), leading dimension lda.
 * dB    n x nrhs, leading dimension ldb >= max(1, n); overwritten by X.
 * dWork at least chol_solve_workspace_size(n, nrhs) bytes.
 * dInfo device int or NULL: 0, or CHOL_INFO_TIMEOUT if a bounded wait expired.
 */
size_t chol_solve_workspace_size(int n, int nrhs);
chol_status chol_solve(int n, int nrhs, const double *dL, int lda, double *dB, int ldb,
                       void *dWork, size_t work_bytes, int *dInfo, void *stream);

/* Allocation-free chol_solve. The paper has no counterpart: this entry point is for callers
 * that cannot allocate device memory -- code that runs under a fixed device-memory budget in
 * which every allocation belongs to the host application, or inside a framework that hands
 * the library device pointers but no allocator -- and so cannot provide the workspace
 * chol_solve needs. Arguments, argument checks and results are those of chol_solve.
 *  - The workspace is a fixed 256 KiB array of this library in device global memory
 *    (each GPU that loads the library holds it until the process exits). Problems whose
 *    chol_solve_workspace_size(n, nrhs) exceeds 256 KiB -- ceil(n/32) * ceil(nrhs/32) >
 *    32704 -- are rejected with CHOL_ERR_UNSUPPORTED before anything is launched.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    with that device current and keeps it for the process; make that first call before
 *    any stream capture. After cudaDeviceReset the kept address is stale: do not call this
 *    entry point on a device that was reset.
 *  - Every call shares the one array and clears what it needs before use; two calls whose
 *    work overlaps on the GPU (different streams, no ordering between them) race on it.
 *  - Calls no cudaMalloc, cudaFree or other allocating routine.
 */
chol_status chol_solve_noalloc(int n, int nrhs, const double *dL, int lda, double *dB, int ldb,
                               int *dInfo, void *stream);

/* chol_solve with an FP32 factor (from chol_factor_f32 / chol_factor_lowp) and FP32
 * right-hand sides: the substitutions the mixed-precision refinement runs for each
 * correction (64-row blocks, inverted diagonal blocks). Workspace chol_solve_workspace_size. */
chol_status chol_solve_f32(int n, int nrhs, const float *dL, int lda, float *dB, int ldb, void *dWork,
                           size_t work_bytes, int *dInfo, void *stream);

/* One sweep only: uplo_t = 0 solves L Y = B, uplo_t = 1 solves L^T X = B, in place on dB. */
chol_status chol_trsm_sweep(int uplo_t, int n, int nrhs, const double *dL, int lda, double *dB,
                            int ldb, void *dWork, size_t work_bytes, int *dInfo, void *stream);

/* ---------------------------------------------------------------------------------------
 * Mixed precision (not in the paper): the same tile factorization in FP32, and a solver
 * that factors A in FP32 and wins the accuracy back by iterative refinement whose residual
 * r = b - A x and update x += d run in FP64 (classical iterative refinement).
 */
typedef enum {
  CHOL_F64 = 0,    /* FP64 (DFMA) tile bodies */
  CHOL_F32 = 1,    /* FP32 (FFMA) tile bodies */
  CHOL_BF16 = 2,   /* FP32 storage; SYRK/GEMM tile updates on the tensor cores (tcgen05) with
                      BF16 operands (8-bit significands) and FP32 accumulation; POTRF/TRSM FP32 */
  CHOL_BF16X3 = 3  /* as CHOL_BF16, but each FP32 operand is split into three BF16 terms
                      t0 + t1 + t2 and the six products t_i t_j (i + j <= 2) are accumulated
                      in FP32: an FP32-accurate GEMM tile update on the tensor cores. The SYRK
                      updates of the diagonal tiles run in FFMA: their products mostly share
                      a sign, and the tensor cores' accumulation errors then add up to a bias
                      that costs the refinement a step */
} chol_precision;

/* chol_factor on an FP32 matrix (same task graph, scheduler, options and workspace size). */
chol_status chol_factor_f32(int n, float *dA, int lda, const chol_opts *opts, void *dWork,
                            size_t work_bytes, int *dInfo, void *stream);

/* chol_factor_f32 with the tile bodies of `precision` (CHOL_F32, CHOL_BF16 or CHOL_BF16X3;
 * others return CHOL_ERR_INVALID_ARG), workspace chol_factor_lowp_workspace_size. A wait of the
 * tensor-core update that exceeds its 2 s limit ends the call with *dInfo = CHOL_INFO_TIMEOUT.
 * Default task costs (chol_opts.cost_ns = 0) come from per-SM rates measured on these bodies:
 * 40 (POTRF), 60 (TRSM), 140 (FFMA SYRK; 1000 on the tensor cores with one term) and
 * 250 / 1000 / 730 (GEMM: FFMA / one term / three terms) GFLOP/s. */
chol_status chol_factor_lowp(int precision, int n, float *dA, int lda, const chol_opts *opts, void *dWork,
                             size_t work_bytes, int *dInfo, void *stream);
/* Workspace of chol_factor_lowp in `precision`. For the BF16 forms with a tile size that is a
 * multiple of 32 and at most 256 it includes a side buffer of the panel tiles' BF16 terms
 * (T (T - 1) / 2 tiles of nb / 32 x NTERM x 16 KiB: 384 KiB per tile of 256 for CHOL_BF16X3),
 * written by each panel's TRSM and bulk-copied by the tile updates. */
size_t chol_factor_lowp_workspace_size(int precision, int n, const chol_opts *opts);

/* Solve A X = B to a normwise backward error <= tol (Rigal-Gaches, infinity norm, maximised
 * over the right-hand sides) with a factor in `low_precision` (CHOL_F32, CHOL_BF16 or
 * CHOL_BF16X3; others return CHOL_ERR_UNSUPPORTED) and at most max_iter refinement steps (the
 * first low-precision solve counts as one). The BF16 forms factor the diagonally scaled
 * matrix S A S, s_i the power of two with s_i^2 a_ii in [1/2, 2) (a_ii > 0; 1 otherwise), so
 * the scaling adds no rounding error, every diagonal entry lies in [1/2, 2) and every entry
 * in (-2, 2); they unscale each correction. Classical refinement converges when kappa(A) times
 * the factor's relative backward error is below 1: with plain BF16 operands (u = 2^-8) that
 * holds only for well-conditioned A; the steps are then taken to max_iter and *dBerr reports
 * the backward error reached.
 * dA    n x n FP64, lower triangle read (A is symmetric); not modified.
 * dB    n x nrhs FP64 (ldb), not modified; dX n x nrhs FP64 (ldx), overwritten by X.
 * opts  options of the low-precision factorization (tile size, policy, ...), may be NULL.
 * dWork at least chol_solve_refine_workspace_size(n, nrhs, opts) bytes, 256-B aligned.
 * dInfo device int: the low-precision factor's info (j > 0: A is not positive definite in
 *       that precision; X is then left at zero and *dBerr is +inf).
 * dIters, dBerr device int / double (nullable): steps taken and the final backward error.
 *       ||A||_inf in eta is the largest FP32 sum of |a_ij| over a row (relative error below
 *       n 2^-24, which scales eta by at most that factor). If those sums overflow FP32
 *       (entries near FLT_MAX), no step is taken, X is left at zero and *dBerr is NaN.
 * All steps run on `stream` with no host synchronisation: every step's kernels return at
 * once after convergence, so the call is one fixed sequence of launches.
 */
size_t chol_solve_refine_workspace_size(int n, int nrhs, const chol_opts *opts);  /* any form */
size_t chol_solve_refine_prec_workspace_size(int low_precision, int n, int nrhs, const chol_opts *opts);
chol_status chol_solve_refine(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb,
                              double *dX, int ldx, int low_precision, double tol, int max_iter,
                              const chol_opts *opts, void *dWork, size_t work_bytes, int *dInfo,
                              int *dIters, double *dBerr, void *stream);

/* ---------------------------------------------------------------------------------------
 * Reverse-mode derivatives (not in the paper: the differentiable form of the factorization).
 * Gradients with respect to the symmetric A are returned symmetric; gradients with respect
 * to L are lower triangular. FP64, asynchronous on `stream`, caller-owned workspaces.
 */

/* Abar = d<Lbar, chol(A)>/dA = (S + S^T)/2, S = L^-T Phi(L^T Lbar) L^-1, Phi = lower triangle
 * with the diagonal halved (I. Murray, "Differentiation of the Cholesky decomposition",
 * 2016). dL: the factor (lower triangle read). dLbar (n x n, ldlb): on entry Lbar (lower
 * triangle read), on exit the full symmetric Abar. Work: chol_backward_workspace_size(n). */
size_t chol_backward_workspace_size(int n);
chol_status chol_backward(int n, const double *dL, int lda, double *dLbar, int ldlb, void *dWork,
                          size_t work_bytes, void *stream);

/* For X = A^-1 B with A = L L^T (X from chol_solve): given Xbar, writes Bbar = A^-1 Xbar
 * (n x nrhs, ldbb) and Lbar = -tril((Bbar X^T + X Bbar^T) L) (n x n, ldlb, strict upper
 * triangle set to zero). Work: chol_solve_backward_workspace_size(n, nrhs). */
size_t chol_solve_backward_workspace_size(int n, int nrhs);
chol_status chol_solve_backward(int n, int nrhs, const double *dL, int lda, const double *dX, int ldx,
                                const double *dXbar, int ldxb, double *dBbar, int ldbb,
                                double *dLbar, int ldlb, void *dWork, size_t work_bytes,
                                void *stream);

/* dDst = lower triangle of dSrc with the strict upper triangle zeroed (n x n, FP64). */
chol_status chol_lower_copy(int n, const double *dSrc, int lds, double *dDst, int ldd, void *stream);

/* ---------------------------------------------------------------------------------------
 * Batched factor + solve of many independent SPD matrices of uneven sizes in one persistent
 * launch (not in the paper: its factorization applied to a batch). The batch is ordered on
 * the device by decreasing order (largest first) and each worker block takes the next matrix
 * from a counter, factors it with the blocked POTRF tile body and solves its right-hand
 * side. No host synchronisation: the call can be captured into a CUDA graph.
 *
 * precision  CHOL_F64 (double matrices) or CHOL_F32 (float matrices).
 * dN[batch]  orders, 0 <= n <= 4096 (device). dA[batch], dB[batch]: device arrays of device
 *            pointers to column-major matrices (leading dimension dLda[m]) and right-hand-side
 *            vectors; dB may be NULL (factor only) and entries of dB may be NULL.
 * dInfo[batch] per-matrix info (0, j > 0 not positive definite, CHOL_INFO_BAD_ARG).
 * bopts      launch shape (NULL = defaults); see chol_batched_autotune.
 * dWork      chol_batched_workspace_size(batch) bytes.
 */
typedef struct {
  int workers_per_sm;    /* worker blocks per SM: 1 or 2 */
  int lpt_order;         /* 1: largest matrices first; 0: in the given order */
  int wide_panel_min_n;  /* FP64: members of order >= this update their trailing matrix once per
                            64-column panel instead of once per 32-column block (the same
                            products, the two halves of a panel subtracted together); 0 = every
                            member, > 4096 = none. FP32 members always use 32-column blocks. */
} chol_batch_opts;
void chol_batch_opts_default(chol_batch_opts *o);
size_t chol_batched_workspace_size(int batch);
chol_status chol_posv_batched(int precision, int batch, const int *dN, void *const *dA, const int *dLda,
                              void *const *dB, int *dInfo, const chol_batch_opts *bopts, void *dWork,
                              size_t work_bytes, void *stream);
/* chol_posv_batched without right-hand sides: factor every matrix in place. */
chol_status chol_factor_batched(int precision, int batch, const int *dN, void *const *dA, const int *dLda,
                                int *dInfo, const chol_batch_opts *bopts, void *dWork, size_t work_bytes,
                                void *stream);
/* Forward and back substitution only: dL[m] holds the factor of matrix m (lower triangle, as
 * left by chol_factor_batched), dB[m] its right-hand-side vector, overwritten by the solution
 * (NULL entries are skipped). dInfo[m] = 0, or CHOL_INFO_BAD_ARG for an invalid size. */
chol_status chol_solve_batched(int precision, int batch, const int *dN, void *const *dL, const int *dLda,
                               void *const *dB, int *dInfo, const chol_batch_opts *bopts, void *dWork,
                               size_t work_bytes, void *stream);
/* Autotuner: times every launch shape (workers per SM x order, and for FP64 the size from which
 * members use 64-column panels: none, 384, 256, 128, all) on the given batch, copying
 * the matrices dAsrc into dAscratch before each run (both arrays of device pointers with the
 * same orders and leading dimensions), and writes the fastest shape to *best (and its time in
 * ms to *best_ms). Synchronises the stream. */
chol_status chol_batched_autotune(int precision, int batch, const int *dN, void *const *dAsrc,
                                  void *const *dAscratch, const int *dLda, int *dInfo, void *dWork,
                                  size_t work_bytes, chol_batch_opts *best, float *best_ms, void *stream);

/* ---------------------------------------------------------------------------------------
 * Host-buffer convenience: factor and solve from host memory (LAPACK dposv semantics).
 * hA (n x n, lda) is copied to the device, factored, and L is copied back into hA's lower
 * triangle; hB (n x nrhs, ldb) is overwritten by X. dStage is a device buffer of at least
 * chol_posv_host_stage_size(n, nrhs, opts) bytes that the call uses for A, B and the
 * workspaces. Synchronous: returns CHOL_ERR_NOT_SPD or CHOL_ERR_TIMEOUT from the info.
 * Host buffers may be pageable or pinned (pinned copies are faster).
 */
size_t chol_posv_host_stage_size(int n, int nrhs, const chol_opts *opts);
chol_status chol_posv_host(int n, int nrhs, double *hA, int lda, double *hB, int ldb,
                           const chol_opts *opts, void *dStage, size_t stage_bytes,
                           int *hInfo, void *stream);

/* ---------------------------------------------------------------------------------------
 * Tile LU factorization with incremental pivoting, the paper's second workload (Section 4.1
 * "Benchmarks": the PLASMA tile algorithm for DGETRF; Section 4.1 "Methodology": double
 * precision, an inner block IB), run by the same persistent data-flow kernel and policies
 * as chol_factor. Tasks per step k: GETRF(k) (LU with partial pivoting of the diagonal
 * tile), GESSM(k, j) (its transformation applied to A_kj), TSTRF(i, k) (LU with partial
 * pivoting of [U_kk; A_ik]), SSSSM(i, j, k) (that transformation applied to [A_kj; A_ij]).
 * Every kernel works on inner blocks of 32 columns (the inner block of these kernels); the
 * transformation of one block is its row interchanges in order, then the unit lower
 * triangle L11 of the block's pivot rows, then the elimination of the rows below with the
 * multipliers L21. Multipliers of a block are not interchanged by later blocks.
 *
 * dA    n x n general matrix, leading dimension lda >= max(1, n). On exit: its upper
 *       triangle is U; the strict lower triangle of a diagonal tile holds the multipliers
 *       of GETRF; tile (i, k), i > k, holds the multipliers of TSTRF(i, k).
 * dPiv  device ints, chol_lu_aux_size's piv_count of them: for tile column k the pivots of
 *       GETRF(k) at ((k T + k) nb) and of TSTRF(i, k) at ((k T + i) nb), one per column of
 *       the tile: the position (relative to the inner block's first row) interchanged with
 *       that column's diagonal position; for TSTRF positions 0..w-1 are rows of U_kk and
 *       w + r is row r of A_ik (w = the inner block's width).
 * dLw   device doubles, lw_count of them: the L11 blocks of TSTRF(i, k) at
 *       ((k T + i) 32 nb), a 32 x nb column-major array (block b's strict lower triangle in
 *       columns 32 b ..; zeros elsewhere).
 * opts  as chol_factor (policies, workers, ...); the tile order nb must be <= 256 (0 =
 *       automatic, as chol_factor). cost_ns[] are the GETRF, GESSM, TSTRF, SSSSM costs.
 * dWork at least chol_lu_workspace_size(n, opts) bytes, 256-byte aligned.
 * dInfo device int: 0, j > 0 (the first zero pivot met was in global column j: U is
 *       singular; the run stops and the outputs are unspecified) or a negative CHOL_INFO_*.
 * The caller owns every buffer; nothing is allocated. One initialisation kernel, one
 * bottom-level kernel and one persistent kernel run on `stream`.
 */
size_t chol_lu_workspace_size(int n, const chol_opts *opts);
chol_status chol_lu_aux_size(int n, const chol_opts *opts, long long *piv_count, long long *lw_count);
chol_status chol_lu_factor(int n, double *dA, int lda, int *dPiv, double *dLw, const chol_opts *opts,
                           void *dWork, size_t work_bytes, int *dInfo, void *stream);

/* Solve A X = B with the outputs of chol_lu_factor (same n and opts, so the same tiles):
 * the recorded transformations applied to B in factorization order, then back substitution
 * with U. dB n x nrhs (ldb >= max(1, n)) is overwritten by X. dWork: at least
 * chol_lu_solve_workspace_size(n, nrhs, opts) bytes, 256-byte aligned (ready flags of the
 * transformations and of the substitution). dInfo (device int, nullable): 0, or
 * CHOL_INFO_TIMEOUT if a bounded wait expired (X is then undefined). Two kernels on `stream`:
 * the transformations run as a wavefront over (tile row, tile column) nodes, the
 * substitution as the backward sweep of chol_solve with U. */
size_t chol_lu_solve_workspace_size(int n, int nrhs, const chol_opts *opts);
chol_status chol_lu_solve(int n, int nrhs, const double *dF, int lda, const int *dPiv, const double *dLw,
                          const chol_opts *opts, double *dB, int ldb, void *dWork, size_t work_bytes,
                          int *dInfo, void *stream);

/* ---------------------------------------------------------------------------------------
 * Introspection of the task graph and of the activate policies. These run on the HOST,
 * with host pointers, using the same code the persistent kernel runs; they exist so the
 * graph and the placement rules can be checked without a GPU.
 */

/* Number of tasks for T x T tiles: T + T(T-1) + T(T-1)(T-2)/6. */
long long chol_dag_task_count(int T);
/* Number of successor edges. */
long long chol_dag_edge_count(int T);
/* Fill, for every task id in [0, count): kind (0 POTRF, 1 TRSM, 2 SYRK, 3 GEMM), tile
 * indices (i, j, k) -- POTRF(k) = (k,k,k), TRSM(i,k) = (i,k,k), SYRK(i,k) = (i,i,k),
 * GEMM(i,j,k) = (i,j,k) --, the initial dependency count, and the successors in CSR form
 * (succ_ptr has count + 1 entries, succ has chol_dag_edge_count entries). Any output
 * pointer may be NULL. Returns CHOL_OK or CHOL_ERR_INVALID_ARG (T < 1 or T > 1024). */
chol_status chol_dag_describe(int T, int *kind, int *ti, int *tj, int *tk, int *indeg,
                              long long *succ_ptr, long long *succ);
/* Bottom level of every task: its cost plus the longest cost-weighted path to the exit
 * (the upward rank that orders the original HEFT, Section 3.1). cost_ns[4] per kind. */
chol_status chol_dag_bottom_levels(int T, const long long *cost_ns, long long *bl);

/* The same for the tile LU graph: count 1 + 2m + m^2 per step (m = T-1-k); kinds 0 GETRF
 * (k,k,k), 1 GESSM (k,j,k), 2 TSTRF (i,k,k), 3 SSSSM (i,j,k). */
long long chol_lu_dag_task_count(int T);
chol_status chol_lu_dag_describe(int T, int *kind, int *ti, int *tj, int *tk, int *indeg,
                                 long long *succ_ptr, long long *succ);
chol_status chol_lu_dag_bottom_levels(int T, const long long *cost_ns, long long *bl);

/* The bottom levels as the device computes them before every factor launch with
 * bottom-level queues (one block, step by step from k = T-1 down, per-step maxima in shared
 * memory): the Cholesky graph for lu = 0, the tile LU graph for lu = 1. cost_ns[4] is a HOST
 * array; dBl is DEVICE memory of chol_dag_task_count(T) (lu = 0) or chol_lu_dag_task_count(T)
 * (lu = 1) entries, all written. Asynchronous on `stream`; the values equal the host
 * functions' above. Returns CHOL_ERR_INVALID_ARG for T < 1, T > 1024 or a NULL pointer. */
chol_status chol_dag_bottom_levels_device(int lu, int T, const long long *cost_ns, long long *dBl,
                                          void *stream);

/* One activate operation on identical workers (Algorithm 1 for CHOL_POLICY_HEFT,
 * Algorithm 2 for CHOL_POLICY_DADA). Ready list of m tasks: task ids tid[m], processing
 * times p[m] (ns), priorities prio[m] (bottom levels), affinity worker aff[m] (-1: none)
 * and affinity score score[m] (bytes of the tile the task writes held by that worker).
 * With use_cp, comm[m] is the predicted cost of one input tile the chosen worker did not
 * write last, own3[3m] the workers that last wrote the task's input tiles (-1: none) and
 * nin[m] the number of input tiles; these may be NULL when use_cp = 0.
 * load[W]: each worker's predicted remaining busy time (ns). Writes the push order
 * out_tid[m] and the chosen worker out_worker[m]; *out_iters gets the number of
 * bisection steps (0 for HEFT). Host pointers. Ties go to the lowest worker index. */
chol_status chol_sched_activate(int policy, double alpha, int max_iter, double eps, int m,
                                const int *tid, const long long *p, const long long *prio,
                                const int *aff, const long long *score, int use_cp,
                                const long long *comm, const int *own3, const int *nin, int W,
                                const long long *load, int *out_tid, int *out_worker,
                                int *out_iters);
/* The same decision computed by one warp on the device (device pointers, all sizes as
 * above; m <= 1024, W <= 1024). Used to check that device and host agree. */
chol_status chol_sched_activate_device(int policy, double alpha, int max_iter, double eps, int m,
                                       const int *dtid, const long long *dp,
                                       const long long *dprio, const int *daff,
                                       const long long *dscore, int use_cp,
                                       const long long *dcomm, const int *down3, const int *dnin,
                                       int W, const long long *dload, int *dout_tid,
                                       int *dout_worker, int *dout_iters, void *stream);

/* ---------------------------------------------------------------------------------------
 * Measurement support (not part of the method): throughput probes of the FP64 units, the
 * denominator of the FP64 factor's roofline. Kind 0 keeps every thread on 16 independent
 * DFMA chains, a 4 x 4 register tile over fixed operands; kind 5 on 16 chains with operands
 * of their own; kind 6 on the 4 x 4 tile fed from shared memory as in the FP64 tile update
 * (iterations rounded up to 32, 256 threads); kinds 1-4 keep every warp
 * on 8 independent chains of FP64 warp MMAs, mma.sync shapes m8n8k4, m16n8k4, m16n8k8 and
 * m16n8k16. `iters` iterations per chain, grid `blocks` x `threads` (32..256, a multiple of
 * 32). chol_probe_fp64_flops returns the flops of such a launch (-1 for invalid arguments);
 * chol_probe_fp64 launches it on `stream` (dOut: one device double, written only by a
 * condition that never holds, so the compiler keeps the work). Time the launch with events
 * on the same stream. */
long long chol_probe_fp64_flops(int kind, int blocks, int threads, long long iters);
chol_status chol_probe_fp64(int kind, int blocks, int threads, long long iters, double *dOut, void *stream);

/* Library version string and the number of workers chol_factor would launch on the
 * current device for these options (0 if no usable device). */
const char *chol_version(void);
int chol_num_workers(const chol_opts *opts);

#ifdef __cplusplus
}
#endif

#endif /* CHOL_GB300_H */
