// Entry points shared between the library's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "../../include/chol.h"

namespace chol {

// tile bodies of the persistent factor kernel: Cholesky with FP64 DFMA, FP32 FFMA, FP32 with
// tensor-core BF16 updates (one or three operand terms); LU with incremental pivoting in FP64
enum { PREC_F64 = 0, PREC_F32 = 1, PREC_BF16 = 2, PREC_BF16X3 = 3, PREC_LU_F64 = 4 };

// Tile Cholesky of the n x n matrix at dA (double for PREC_F64, float for PREC_F32), or with
// PREC_LU_F64 the tile LU with incremental pivoting (pivots to lu_piv, L11 blocks to lu_lw).
chol_status factor_impl(int prec, int n, void *dA, int lda, const chol_opts *opts, void *dWork,
                        size_t work_bytes, int *dInfo, void *stream, int *lu_piv = nullptr,
                        double *lu_lw = nullptr);

// Tile size the LU entry points use for (n, opts) (0 if the options are invalid).
int lu_tile_size(int n, const chol_opts *opts);

// FP32 forward + back substitution in place; does nothing while *skip != 0 (skip nullable).
chol_status solve_f32(int n, int nrhs, const float *dL, int lda, float *dB, int ldb, void *dWork,
                      const int *skip, cudaStream_t s);

size_t solve_workspace_bytes(int n, int nrhs);

// U X = B in place with the upper triangle of the tiles (the tile LU's U): one backward sweep
// of the substitution kernel (workspace solve_workspace_bytes(n, nrhs)); its items are skipped
// once *prev_abort (nullable) is set. solve_upper_info merges the sweep's status into *dInfo.
chol_status solve_upper_f64(int n, int nrhs, const double *dU, int lda, double *dB, int ldb, void *dWork,
                            const int *prev_abort, cudaStream_t s);
chol_status solve_upper_info(void *dWork, int *dInfo, cudaStream_t s);

// Bottom levels of every task of the Cholesky (lu = false) or tile LU graph with T x T tiles
// and per-kind costs cost[4], written to dBl (device, one entry per task id) on stream s.
chol_status bottom_levels_device(bool lu, int T, const int64_t *cost, int64_t *dBl, cudaStream_t s);

}  // namespace chol
