/* oracle_perm.c -- zero-diagonal repair before the method (section 5).
 *
 * TEST INFRASTRUCTURE (see oracle.h): plain sequential code, no tuning.
 *
 * Section 5 applies a row Dulmage-Mendelsohn permutation to the matrices
 * that have zero diagonals (MATLAB j = dmperm(A), A = A(j,:)) so that the
 * diagonal, which SPAI's initial pattern P(I) and the split keep, becomes
 * nonzero. With one output dmperm is a maximum transversal: a largest set
 * of stored nonzeros, no two in one row or column (Duff 1981; Pothen and
 * Fan 1990). Here:
 *   - an entry counts when it is stored with a nonzero value;
 *   - a zero-free diagonal is left alone (p = identity), since only the
 *     matrices with zero diagonals are permuted;
 *   - otherwise the columns whose diagonal is nonzero start matched to it,
 *     and each unmatched column, in ascending order, looks for an augmenting
 *     path by breadth-first search over the alternating paths (rows in
 *     ascending order, columns first in first out) and flips the first,
 *     hence shortest, one found; a column without one stays unmatched (a
 *     matching is maximum iff no augmenting path exists, and a column that
 *     finds none cannot find one later).
 * Shortest paths move as few rows as the search allows: the rows whose
 * diagonal was already nonzero stay in place unless a path needs them.
 * Several maximum transversals usually exist; only their size (the
 * structural rank) is unique.
 */
#include "oracle_internal.h"

#include <stdlib.h>
#include <string.h>

static int entry_counts(const orc_csc* A, int64_t t) { return A->val[t] != 0.0; }

/* the stored nonzero diagonal of column j, or 0 */
static int diag_nonzero(const orc_csc* A, int32_t j)
{
    for (int64_t t = A->col_ptr[j]; t < A->col_ptr[j + 1]; ++t)
        if (A->row_idx[t] == j) return entry_counts(A, t);
    return 0;
}

int orc_dmperm(const orc_csc* A, int32_t* p_out, int32_t* rank_out)
{
    if (!orc_csc_valid(A) || A->nrows != A->ncols || !p_out || !rank_out) return ORC_BAD_INPUT;
    const int32_t n = A->ncols;
    int32_t* match_col = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t)); /* row of column j */
    int32_t* match_row = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t)); /* column of row i */
    int32_t* seen = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));      /* search stamp per row */
    int32_t* via = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));       /* column that reached row i */
    int32_t* queue = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));     /* columns, first in first out */
    for (int32_t i = 0; i < n; ++i) {
        match_col[i] = -1;
        match_row[i] = -1;
        seen[i] = -1;
    }
    int32_t rank = 0;
    for (int32_t j = 0; j < n; ++j)
        if (diag_nonzero(A, j)) {
            match_col[j] = j;
            match_row[j] = j;
            ++rank;
        }
    for (int32_t j = 0; j < n && rank < n; ++j) {
        if (match_col[j] >= 0) continue;
        /* breadth-first search from the unmatched column j over alternating
         * paths: a row is reached from a column through any nonzero, a
         * column from its matched row; the first free row reached ends a
         * shortest augmenting path */
        int32_t head = 0, tail = 0, end = -1;
        queue[tail++] = j;
        while (head < tail && end < 0) {
            const int32_t c = queue[head++];
            for (int64_t t = A->col_ptr[c]; t < A->col_ptr[c + 1]; ++t) {
                const int32_t i = A->row_idx[t];
                if (!entry_counts(A, t) || seen[i] == j) continue;
                seen[i] = j;
                via[i] = c;
                if (match_row[i] < 0) {
                    end = i;
                    break;
                }
                queue[tail++] = match_row[i];
            }
        }
        if (end < 0) continue;  /* no augmenting path from j: column j stays unmatched */
        for (int32_t i = end;;) {  /* flip the path back to j */
            const int32_t c = via[i];
            const int32_t i_prev = match_col[c];
            match_col[c] = i;
            match_row[i] = c;
            if (c == j) break;
            i = i_prev;
        }
        ++rank;
    }
    for (int32_t j = 0; j < n; ++j) p_out[j] = match_col[j];
    *rank_out = rank;
    free(match_col);
    free(match_row);
    free(seen);
    free(via);
    free(queue);
    return ORC_OK;
}

typedef struct {
    int32_t row;
    double val;
} row_entry;

static int by_row(const void* a, const void* b)
{
    const int32_t x = ((const row_entry*)a)->row, y = ((const row_entry*)b)->row;
    return (x > y) - (x < y);
}

/* B = A(p,:): row j of B is row p[j] of A, i.e. entry (i, c) of A moves to
 * row pinv[i] of B, with pinv[p[j]] = j. */
int orc_permute_rows(const orc_csc* A, const int32_t* p, orc_csc* B_out)
{
    if (!orc_csc_valid(A) || A->nrows != A->ncols || !p || !B_out) return ORC_BAD_INPUT;
    const int32_t n = A->ncols;
    int32_t* pinv = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) pinv[i] = -1;
    for (int32_t j = 0; j < n; ++j) {
        if (p[j] < 0 || p[j] >= n || pinv[p[j]] >= 0) {  /* not a permutation */
            free(pinv);
            return ORC_BAD_INPUT;
        }
        pinv[p[j]] = j;
    }
    const int64_t nnz = orc_nnz(A);
    B_out->nrows = n;
    B_out->ncols = n;
    B_out->col_ptr = (int64_t*)orc_xmalloc((size_t)(n + 1) * sizeof(int64_t));
    B_out->row_idx = (int32_t*)orc_xmalloc((size_t)nnz * sizeof(int32_t));
    B_out->val = (double*)orc_xmalloc((size_t)nnz * sizeof(double));
    memcpy(B_out->col_ptr, A->col_ptr, (size_t)(n + 1) * sizeof(int64_t));
    int64_t longest = 0;
    for (int32_t c = 0; c < n; ++c)
        if (A->col_ptr[c + 1] - A->col_ptr[c] > longest) longest = A->col_ptr[c + 1] - A->col_ptr[c];
    row_entry* e = (row_entry*)orc_xmalloc((size_t)longest * sizeof(row_entry));
    for (int32_t c = 0; c < n; ++c) {
        const int64_t b = A->col_ptr[c], len = A->col_ptr[c + 1] - b;
        for (int64_t t = 0; t < len; ++t) {
            e[t].row = pinv[A->row_idx[b + t]];
            e[t].val = A->val[b + t];
        }
        qsort(e, (size_t)len, sizeof(row_entry), by_row);
        for (int64_t t = 0; t < len; ++t) {
            B_out->row_idx[b + t] = e[t].row;
            B_out->val[b + t] = e[t].val;
        }
    }
    free(e);
    free(pinv);
    return ORC_OK;
}
