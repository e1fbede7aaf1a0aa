/* oracle_split.c -- dense-column detection and sparsification, section 4 of
 * the paper (threshold 10p with p = floor(nnz(A)/n); keep the diagonal and the
 * p-1 nonzeros nearest to it), which defines A = A~ + U V^T, eq. (split).
 * Test infrastructure only. */
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Section 4: p is the average number of nonzeros per column, rounded down. */
int32_t orc_avg_nnz(int32_t n, int64_t nnz)
{
    if (n <= 0) return 0;
    return (int32_t)(nnz / (int64_t)n);
}

/* Section 4: a column is irregular if its nonzero count exceeds 10p. The
 * comparison is strict by default; ge != 0 selects the "10p or more" wording
 * of section 1. */
int orc_detect(const orc_csc* A, double mult, double abs_tau, int ge,
               int32_t* J_out, int32_t* s_out, int32_t* p_out, double* tau_out)
{
    if (!orc_csc_valid(A) || A->nrows != A->ncols) return ORC_BAD_INPUT;
    int32_t n = A->ncols;
    int32_t p = orc_avg_nnz(n, orc_nnz(A));
    double tau = (abs_tau >= 0.0) ? abs_tau : mult * (double)p;
    int32_t s = 0;
    for (int32_t j = 0; j < n; ++j) {
        double cnt = (double)(A->col_ptr[j + 1] - A->col_ptr[j]);
        int dense = ge ? (cnt >= tau) : (cnt > tau);
        if (dense) J_out[s++] = j;
    }
    *s_out = s;
    *p_out = p;
    *tau_out = tau;
    return ORC_OK;
}

/* Section 4, first dropping approach: for an irregular column j keep a_jj
 * and the p-1 stored entries with the smallest distance |i - j|; on equal
 * distance the smaller row index is taken first. Everything dropped goes to
 * U, so A = A~ + U V^T holds entry by entry. */
/* off-diagonal entry of an irregular column, for the largest-magnitude rule */
typedef struct {
    double mag;
    int32_t row;
    int64_t pos;
} mag_entry;

/* |a_ij| descending, then the smaller row first */
static int cmp_mag(const void* x, const void* y)
{
    const mag_entry* a = (const mag_entry*)x;
    const mag_entry* b = (const mag_entry*)y;
    if (a->mag > b->mag) return -1;
    if (a->mag < b->mag) return 1;
    return (a->row > b->row) - (a->row < b->row);
}

int orc_split(const orc_csc* A, const int32_t* J, int32_t s, int32_t p_keep,
              orc_csc* At_out, orc_csc* U_out)
{
    return orc_split_rule(A, J, s, p_keep, 0, At_out, U_out);
}

/* rule 0 keeps the diagonal and the p_keep-1 entries nearest to it (the
 * choice of section 4); rule 1 keeps the diagonal and the p_keep-1 entries
 * of largest magnitude (the other rule named there), equal magnitudes to the
 * smaller row, or the p_keep largest when no diagonal is stored. */
int orc_split_rule(const orc_csc* A, const int32_t* J, int32_t s, int32_t p_keep, int32_t rule,
                   orc_csc* At_out, orc_csc* U_out)
{
    if (!orc_csc_valid(A) || A->nrows != A->ncols || s < 0 || p_keep < 1 || (rule != 0 && rule != 1))
        return ORC_BAD_INPUT;
    int32_t n = A->ncols;
    int64_t nnz = orc_nnz(A);
    /* map column -> position in J (or -1) */
    int32_t* slot = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    for (int32_t j = 0; j < n; ++j) slot[j] = -1;
    for (int32_t t = 0; t < s; ++t) {
        if (J[t] < 0 || J[t] >= n || (t > 0 && J[t] <= J[t - 1])) {
            free(slot);
            return ORC_BAD_INPUT;
        }
        slot[J[t]] = t;
    }
    /* keep[t] = 1 if entry t of A stays in A~ */
    char* keep = (char*)orc_xmalloc((size_t)nnz);
    for (int64_t t = 0; t < nnz; ++t) keep[t] = 1;
    for (int32_t j = 0; j < n; ++j) {
        if (slot[j] < 0) continue;
        int64_t b = A->col_ptr[j], e = A->col_ptr[j + 1];
        for (int64_t t = b; t < e; ++t) keep[t] = 0;
        if (rule == 1) {
            mag_entry* ent = (mag_entry*)orc_xmalloc((size_t)(e - b + 1) * sizeof(mag_entry));
            int64_t m = 0;
            int has_diag = 0;
            for (int64_t t = b; t < e; ++t) {
                if (A->row_idx[t] == j) {
                    keep[t] = 1;
                    has_diag = 1;
                    continue;
                }
                ent[m].mag = fabs(A->val[t]);
                ent[m].row = A->row_idx[t];
                ent[m].pos = t;
                ++m;
            }
            qsort(ent, (size_t)m, sizeof(mag_entry), cmp_mag);
            int64_t want = has_diag ? (int64_t)p_keep - 1 : (int64_t)p_keep;
            for (int64_t q = 0; q < m && q < want; ++q) keep[ent[q].pos] = 1;
            free(ent);
            continue;
        }
        /* first stored row >= j */
        int64_t mid = b;
        while (mid < e && A->row_idx[mid] < j) ++mid;
        int32_t kept = 0;
        int64_t lo = mid - 1, hi = mid;
        if (mid < e && A->row_idx[mid] == j) {
            keep[mid] = 1;
            kept = 1;
            hi = mid + 1;
        }
        while (kept < p_keep && (lo >= b || hi < e)) {
            int take_lo;
            if (lo < b) take_lo = 0;
            else if (hi >= e) take_lo = 1;
            else take_lo = ((int64_t)j - A->row_idx[lo]) <= ((int64_t)A->row_idx[hi] - j);
            if (take_lo) keep[lo--] = 1;
            else keep[hi++] = 1;
            ++kept;
        }
    }
    int64_t nk = 0;
    for (int64_t t = 0; t < nnz; ++t) nk += keep[t];
    At_out->nrows = n;
    At_out->ncols = n;
    At_out->col_ptr = (int64_t*)orc_xcalloc((size_t)n + 1, sizeof(int64_t));
    At_out->row_idx = (int32_t*)orc_xmalloc((size_t)nk * sizeof(int32_t));
    At_out->val = (double*)orc_xmalloc((size_t)nk * sizeof(double));
    U_out->nrows = n;
    U_out->ncols = s;
    U_out->col_ptr = (int64_t*)orc_xcalloc((size_t)s + 1, sizeof(int64_t));
    U_out->row_idx = (int32_t*)orc_xmalloc((size_t)(nnz - nk) * sizeof(int32_t));
    U_out->val = (double*)orc_xmalloc((size_t)(nnz - nk) * sizeof(double));
    int64_t qa = 0, qu = 0;
    for (int32_t j = 0; j < n; ++j) {
        for (int64_t t = A->col_ptr[j]; t < A->col_ptr[j + 1]; ++t) {
            if (keep[t]) {
                At_out->row_idx[qa] = A->row_idx[t];
                At_out->val[qa] = A->val[t];
                ++qa;
            } else {
                U_out->row_idx[qu] = A->row_idx[t];
                U_out->val[qu] = A->val[t];
                ++qu;
            }
        }
        At_out->col_ptr[j + 1] = qa;
        if (slot[j] >= 0) U_out->col_ptr[slot[j] + 1] = qu;
    }
    free(keep);
    free(slot);
    return ORC_OK;
}
