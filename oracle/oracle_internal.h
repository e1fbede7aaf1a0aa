/* oracle_internal.h -- helpers shared by the oracle's own C files only.
 * Test infrastructure; never included by the CUDA library. */
#ifndef SAI_ORACLE_INTERNAL_H
#define SAI_ORACLE_INTERNAL_H
#include "oracle.h"
#include <stddef.h>

void* orc_xmalloc(size_t bytes);
void* orc_xcalloc(size_t count, size_t bytes);
int orc_csc_valid(const orc_csc* A);
int64_t orc_nnz(const orc_csc* A);

/* y = A x (A nrows x ncols) */
void orc_csc_matvec(const orc_csc* A, const double* x, double* y);
/* CSR copy (row_ptr[nrows+1], col_idx, val) with column indices ascending. */
void orc_csc_to_csr(const orc_csc* A, int64_t** row_ptr, int32_t** col_idx, double** val);
double orc_norm2(int32_t n, const double* x);
double orc_dot(int32_t n, const double* x, const double* y);
/* max_j sum_i |a_ij| */
double orc_norm1(const orc_csc* A);

/* Householder QR least squares, m >= c, column-major A (lda = m).
 * Returns ORC_OK or ORC_SINGULAR. */
int orc_dense_lsq(int32_t m, int32_t c, const double* A, const double* b, double* x);
/* Gaussian elimination with partial pivoting, column-major C (s x s). */
int orc_dense_lu_solve(int32_t s, const double* C, const double* g, double* z);

#endif
