/*
 * Oracle for the Cholesky factor and the triangular solves: TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may load this
 * library. The product path (the CUDA library under paper_1402_6601_gb300/) never calls it,
 * and the two share no code, header, table or constant.
 *
 * What it computes. The tile algorithm the paper schedules (PLASMA DPOTRF, Section 4.1
 * "Benchmarks", in double precision as stated in Section 4.1 "Methodology") reaches, for
 * any schedule that respects the data-flow dependencies (Section 2 "Execution flow"), the
 * Cholesky factor: the unique lower-triangular L with a positive diagonal such that
 * A = L L^T. The oracle writes that definition out as the column recurrence
 *
 *     l_jj = sqrt(a_jj - sum_{m<j} l_jm^2),
 *     l_ij = (a_ij - sum_{m<j} l_im l_jm) / l_jj        (i > j),
 *
 * with no blocking, no reordering of the sums (m increasing) and no fused multiply-add
 * (the build passes -ffp-contract=off so that x86 and Arm hosts give the same bits).
 * Solves are forward substitution L y = b and back substitution L^T x = y, again the plain
 * definitions. Everything is IEEE binary64.
 *
 * Pins (checked by the CPU tests, independent of this code): the symmetric Pascal matrix
 * whose factor is the lower Pascal matrix of binomial coefficients (exact to n = 20),
 * exact integer factors at any n, LAPACK on small random matrices, the uniqueness of the
 * factor of M M^T for random lower-triangular M, the non-SPD leading-minor index, and the
 * invariants ||A - L L^T||_F / ||A||_F and diag(L) > 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Lower Cholesky factor in place: A (n x n, column-major, leading dimension lda) is
 * overwritten on and below the diagonal by L; the strict upper triangle is not touched.
 * *info = 0 on success, or j (1-based) when the leading minor of order j is not positive
 * definite (a_jj - sum l_jm^2 is <= 0 or NaN); the columns before j then hold L, the rest
 * is left as it was. Returns *info. */
int oracle_cholesky(int n, double *A, long lda, int *info) {
  *info = 0;
  if (n <= 0) return 0;
  /* Row-major copy of L so that the dot products over m run through contiguous memory.
   * This only changes where the numbers are kept, not the arithmetic. */
  double *R = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
  if (!R) { *info = -1; return -1; }
  for (int j = 0; j < n; ++j) {
    const double *rj = R + (size_t)j * n;
    double s = A[(size_t)j * lda + j];
    for (int m = 0; m < j; ++m) s -= rj[m] * rj[m];
    if (!(s > 0.0)) { *info = j + 1; break; }
    const double ljj = sqrt(s);
    A[(size_t)j * lda + j] = ljj;
    R[(size_t)j * n + j] = ljj;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; ++i) {
      const double *ri = R + (size_t)i * n;
      double t = A[(size_t)j * lda + i];
      for (int m = 0; m < j; ++m) t -= ri[m] * rj[m];
      const double lij = t / ljj;
      A[(size_t)j * lda + i] = lij;
      R[(size_t)i * n + j] = lij;
    }
  }
  free(R);
  return *info;
}

/* Forward substitution L Y = B in place on B (n x nrhs, column-major, ldb); L is the lower
 * triangle of the n x n array at L (lda). y_i = (b_i - sum_{m<i} l_im y_m) / l_ii. */
void oracle_forward_solve(int n, int nrhs, const double *L, long lda, double *B, long ldb) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < nrhs; ++c) {
    double *b = B + (size_t)c * ldb;
    for (int i = 0; i < n; ++i) {
      double t = b[i];
      for (int m = 0; m < i; ++m) t -= L[(size_t)m * lda + i] * b[m];
      b[i] = t / L[(size_t)i * lda + i];
    }
  }
}

/* Back substitution L^T X = Y in place on B. x_i = (y_i - sum_{m>i} l_mi x_m) / l_ii. */
void oracle_backward_solve(int n, int nrhs, const double *L, long lda, double *B, long ldb) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < nrhs; ++c) {
    double *b = B + (size_t)c * ldb;
    for (int i = n - 1; i >= 0; --i) {
      const double *li = L + (size_t)i * lda;
      double t = b[i];
      for (int m = i + 1; m < n; ++m) t -= li[m] * b[m];
      b[i] = t / li[i];
    }
  }
}

/* Solve A X = B with the factor already in L: forward then back substitution. */
void oracle_cholesky_solve(int n, int nrhs, const double *L, long lda, double *B, long ldb) {
  oracle_forward_solve(n, nrhs, L, lda, B, ldb);
  oracle_backward_solve(n, nrhs, L, lda, B, ldb);
}
