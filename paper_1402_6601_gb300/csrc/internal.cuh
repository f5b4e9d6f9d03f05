// Entry points shared between the library's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "../../include/chol.h"

namespace chol {

// tile bodies of the factor: FP64 DFMA, FP32 FFMA, FP32 with tensor-core BF16 updates (one or
// three operand terms)
enum { PREC_F64 = 0, PREC_F32 = 1, PREC_BF16 = 2, PREC_BF16X3 = 3 };

// Tile Cholesky of the n x n matrix at dA (double for PREC_F64, float for PREC_F32).
chol_status factor_impl(int prec, int n, void *dA, int lda, const chol_opts *opts, void *dWork,
                        size_t work_bytes, int *dInfo, void *stream);

// FP32 forward + back substitution in place; does nothing while *skip != 0 (skip nullable).
chol_status solve_f32(int n, int nrhs, const float *dL, int lda, float *dB, int ldb, void *dWork,
                      const int *skip, cudaStream_t s);

size_t solve_workspace_bytes(int n, int nrhs);

}  // namespace chol
