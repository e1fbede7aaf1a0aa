/* oracle_core.c -- sparse and dense building blocks of the oracle.
 * Test infrastructure only: plain loops, FP64, no blocking. */
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

void* orc_xmalloc(size_t bytes) { return malloc(bytes ? bytes : 1); }
void* orc_xcalloc(size_t count, size_t bytes) { return calloc(count ? count : 1, bytes ? bytes : 1); }

void orc_csc_free(orc_csc* A)
{
    if (!A) return;
    free(A->col_ptr);
    free(A->row_idx);
    free(A->val);
    A->col_ptr = NULL;
    A->row_idx = NULL;
    A->val = NULL;
}

int64_t orc_nnz(const orc_csc* A) { return A->col_ptr[A->ncols]; }

/* Column pointers nondecreasing, rows in range and strictly ascending per column. */
int orc_csc_valid(const orc_csc* A)
{
    if (!A || A->nrows < 0 || A->ncols < 0 || !A->col_ptr) return 0;
    if (A->col_ptr[0] != 0) return 0;
    for (int32_t j = 0; j < A->ncols; ++j) {
        if (A->col_ptr[j + 1] < A->col_ptr[j]) return 0;
        for (int64_t t = A->col_ptr[j]; t < A->col_ptr[j + 1]; ++t) {
            int32_t i = A->row_idx[t];
            if (i < 0 || i >= A->nrows) return 0;
            if (t > A->col_ptr[j] && A->row_idx[t - 1] >= i) return 0;
        }
    }
    return 1;
}

void orc_csc_matvec(const orc_csc* A, const double* x, double* y)
{
    for (int32_t i = 0; i < A->nrows; ++i) y[i] = 0.0;
    for (int32_t j = 0; j < A->ncols; ++j) {
        double xj = x[j];
        for (int64_t t = A->col_ptr[j]; t < A->col_ptr[j + 1]; ++t) y[A->row_idx[t]] += A->val[t] * xj;
    }
}

void orc_csc_to_csr(const orc_csc* A, int64_t** row_ptr, int32_t** col_idx, double** val)
{
    int64_t nnz = orc_nnz(A);
    int64_t* rp = (int64_t*)orc_xcalloc((size_t)A->nrows + 1, sizeof(int64_t));
    int32_t* ci = (int32_t*)orc_xmalloc((size_t)nnz * sizeof(int32_t));
    double* v = (double*)orc_xmalloc((size_t)nnz * sizeof(double));
    for (int64_t t = 0; t < nnz; ++t) rp[A->row_idx[t] + 1]++;
    for (int32_t i = 0; i < A->nrows; ++i) rp[i + 1] += rp[i];
    int64_t* fill = (int64_t*)orc_xmalloc((size_t)(A->nrows + 1) * sizeof(int64_t));
    memcpy(fill, rp, (size_t)(A->nrows + 1) * sizeof(int64_t));
    /* columns visited in ascending order, so each row's columns come out sorted */
    for (int32_t j = 0; j < A->ncols; ++j)
        for (int64_t t = A->col_ptr[j]; t < A->col_ptr[j + 1]; ++t) {
            int64_t q = fill[A->row_idx[t]]++;
            ci[q] = j;
            v[q] = A->val[t];
        }
    free(fill);
    *row_ptr = rp;
    *col_idx = ci;
    *val = v;
}

double orc_dot(int32_t n, const double* x, const double* y)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

double orc_norm2(int32_t n, const double* x) { return sqrt(orc_dot(n, x, x)); }

double orc_norm1(const orc_csc* A)
{
    double best = 0.0;
    for (int32_t j = 0; j < A->ncols; ++j) {
        double s = 0.0;
        for (int64_t t = A->col_ptr[j]; t < A->col_ptr[j + 1]; ++t) s += fabs(A->val[t]);
        if (s > best) best = s;
    }
    return best;
}

/* Householder QR of the m x c matrix A, applied to b on the fly, then back
 * substitution with R (Golub & Van Loan, Householder LS). This is the "QR
 * decomposition" the paper names for the reduced problems, eq. (lsprob). */
int orc_dense_lsq(int32_t m, int32_t c, const double* A, const double* b, double* x)
{
    if (m < c || c < 0) return ORC_BAD_INPUT;
    double* Q = (double*)orc_xmalloc((size_t)m * (size_t)c * sizeof(double));
    double* y = (double*)orc_xmalloc((size_t)m * sizeof(double));
    double* diag = (double*)orc_xmalloc((size_t)c * sizeof(double));
    memcpy(Q, A, (size_t)m * (size_t)c * sizeof(double));
    memcpy(y, b, (size_t)m * sizeof(double));
    int status = ORC_OK;
    for (int32_t j = 0; j < c && status == ORC_OK; ++j) {
        double* qj = Q + (size_t)j * m;
        double nrm2 = 0.0;
        for (int32_t i = j; i < m; ++i) nrm2 += qj[i] * qj[i];
        double nrm = sqrt(nrm2);
        if (nrm == 0.0) {
            status = ORC_SINGULAR;
            break;
        }
        double alpha = (qj[j] >= 0.0) ? -nrm : nrm; /* R(j,j) */
        qj[j] -= alpha;                               /* v = x - alpha e_1 */
        double vtv = 0.0;
        for (int32_t i = j; i < m; ++i) vtv += qj[i] * qj[i];
        for (int32_t jj = j + 1; jj < c; ++jj) {
            double* qk = Q + (size_t)jj * m;
            double d = 0.0;
            for (int32_t i = j; i < m; ++i) d += qj[i] * qk[i];
            double f = 2.0 * d / vtv;
            for (int32_t i = j; i < m; ++i) qk[i] -= f * qj[i];
        }
        double d = 0.0;
        for (int32_t i = j; i < m; ++i) d += qj[i] * y[i];
        double f = 2.0 * d / vtv;
        for (int32_t i = j; i < m; ++i) y[i] -= f * qj[i];
        diag[j] = alpha;
    }
    if (status == ORC_OK) {
        for (int32_t j = c - 1; j >= 0; --j) {
            double s = y[j];
            for (int32_t jj = j + 1; jj < c; ++jj) s -= Q[(size_t)jj * m + j] * x[jj];
            x[j] = s / diag[j];
        }
    }
    free(Q);
    free(y);
    free(diag);
    return status;
}

/* Textbook Gaussian elimination with partial pivoting; the first row with
 * the largest |pivot| wins. Solves C z = g. */
int orc_dense_lu_solve(int32_t s, const double* C, const double* g, double* z)
{
    double* a = (double*)orc_xmalloc((size_t)s * (size_t)s * sizeof(double));
    double* rhs = (double*)orc_xmalloc((size_t)s * sizeof(double));
    memcpy(a, C, (size_t)s * (size_t)s * sizeof(double));
    memcpy(rhs, g, (size_t)s * sizeof(double));
#define A_(i, j) a[(size_t)(j) * s + (i)]
    int status = ORC_OK;
    for (int32_t k = 0; k < s; ++k) {
        int32_t piv = k;
        double best = fabs(A_(k, k));
        for (int32_t i = k + 1; i < s; ++i)
            if (fabs(A_(i, k)) > best) {
                best = fabs(A_(i, k));
                piv = i;
            }
        if (best == 0.0) {
            status = ORC_SINGULAR;
            break;
        }
        if (piv != k) {
            for (int32_t j = 0; j < s; ++j) {
                double t = A_(k, j);
                A_(k, j) = A_(piv, j);
                A_(piv, j) = t;
            }
            double t = rhs[k];
            rhs[k] = rhs[piv];
            rhs[piv] = t;
        }
        for (int32_t i = k + 1; i < s; ++i) {
            double l = A_(i, k) / A_(k, k);
            A_(i, k) = l;
            for (int32_t j = k + 1; j < s; ++j) A_(i, j) -= l * A_(k, j);
            rhs[i] -= l * rhs[k];
        }
    }
    if (status == ORC_OK) {
        for (int32_t i = s - 1; i >= 0; --i) {
            double t = rhs[i];
            for (int32_t j = i + 1; j < s; ++j) t -= A_(i, j) * z[j];
            z[i] = t / A_(i, i);
        }
    }
#undef A_
    free(a);
    free(rhs);
    return status;
}
