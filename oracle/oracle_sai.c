/* oracle_sai.c -- the two F-norm-minimisation SAI builders of section 2:
 *   SPAI      (section 2.1, eqs. (candi), (ls1d), (muj), (rhoj)),
 *   PSAI(tol) (section 2.2, power pattern growth and eq. (tolk)), and
 *   PSAI(lfill), which keeps the lfill largest entries instead (section 2.2
 *   names it).
 * Both solve min ||A~ m_k - e_k|| column by column, eq. (subprob), through the
 * reduced problem min ||A^_k m^_k - e^_k||, eq. (lsprob), by Householder QR.
 * The reduced problem is rebuilt and refactored from scratch at every loop;
 * the CUDA path updates its QR incrementally, which gives the same solution.
 *
 * Readings where the paper is silent (the CUDA path takes the same ones):
 *  - L_k always contains row k, so e^_k is represented.
 *  - SPAI candidate rows are all rows of L_k (structural), not only those with
 *    r_k(i) != 0; a numerically exact zero test is not reproducible.
 *  - SPAI ranks candidates by the key (floor(rho_j^2/||r_k||^2 * 2^key_bits), j)
 *    ascending, so exactly tied candidates (symmetric stencils) are ordered by
 *    index and not by rounding noise.
 *  - PSAI(tol) grows the pattern from the undropped power sequence,
 *    S^(l+1) = P(a^(l+1)) u S_kept^(l), and emits the last LS solution
 *    restricted to its kept entries, without a re-solve.
 * Test infrastructure only. */
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const orc_csc* A;
    int32_t n;
    int64_t* rp;       /* CSR of A~ for the row access A~(L,:) */
    int32_t* ci;
    double* rv;
    double* colnorm2;  /* ||A~ e_j||^2 */
    int32_t* rowpos;   /* row -> position in L, or -1 */
    int32_t* colmark;  /* column marks for S membership / candidate dedupe */
    int32_t* L;        /* current row set, ascending */
    int32_t nL;
    double* r;         /* residual on L */
    int32_t* S;        /* current pattern */
    int32_t nS;
    double* m;         /* LS solution on S */
    int32_t* tmp;      /* scratch index list (capacity n) */
    double norm1;      /* ||A~||_1 */
} sai_ws;

static int ws_init(sai_ws* w, const orc_csc* A)
{
    memset(w, 0, sizeof(*w));
    w->A = A;
    w->n = A->ncols;
    orc_csc_to_csr(A, &w->rp, &w->ci, &w->rv);
    int32_t n = w->n;
    w->colnorm2 = (double*)orc_xcalloc((size_t)n, sizeof(double));
    for (int32_t j = 0; j < n; ++j)
        for (int64_t t = A->col_ptr[j]; t < A->col_ptr[j + 1]; ++t) w->colnorm2[j] += A->val[t] * A->val[t];
    w->rowpos = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    w->colmark = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) w->rowpos[i] = w->colmark[i] = -1;
    w->L = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    w->r = (double*)orc_xmalloc((size_t)n * sizeof(double));
    w->S = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    w->m = (double*)orc_xmalloc((size_t)n * sizeof(double));
    w->tmp = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    w->norm1 = orc_norm1(A);
    return ORC_OK;
}

static void ws_free(sai_ws* w)
{
    free(w->rp);
    free(w->ci);
    free(w->rv);
    free(w->colnorm2);
    free(w->rowpos);
    free(w->colmark);
    free(w->L);
    free(w->r);
    free(w->S);
    free(w->m);
    free(w->tmp);
}

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void reset_rows(sai_ws* w)
{
    for (int32_t t = 0; t < w->nL; ++t) w->rowpos[w->L[t]] = -1;
    w->nL = 0;
}

/* Reduced LS problem (lsprob) on the current pattern S of column k:
 * L = rows of A~(:,S) plus k, A^ = A~(L,S), e^ = e_k(L); solve by QR and
 * form r = A^ m^ - e^ explicitly. Leaves L/rowpos set for the caller. */
static int ls_on_pattern(sai_ws* w, int32_t k, double* rn_out)
{
    const orc_csc* A = w->A;
    w->nL = 0;
    w->rowpos[k] = 0;
    w->L[w->nL++] = k;
    for (int32_t t = 0; t < w->nS; ++t) {
        int32_t j = w->S[t];
        for (int64_t q = A->col_ptr[j]; q < A->col_ptr[j + 1]; ++q) {
            int32_t i = A->row_idx[q];
            if (w->rowpos[i] < 0) {
                w->rowpos[i] = 0;
                w->L[w->nL++] = i;
            }
        }
    }
    qsort(w->L, (size_t)w->nL, sizeof(int32_t), cmp_i32);
    for (int32_t t = 0; t < w->nL; ++t) w->rowpos[w->L[t]] = t;
    int32_t nL = w->nL, nS = w->nS;
    if (nL < nS) return ORC_SINGULAR;
    double* Ahat = (double*)orc_xcalloc((size_t)nL * (size_t)nS, sizeof(double));
    double* ehat = (double*)orc_xcalloc((size_t)nL, sizeof(double));
    for (int32_t t = 0; t < nS; ++t) {
        int32_t j = w->S[t];
        for (int64_t q = A->col_ptr[j]; q < A->col_ptr[j + 1]; ++q)
            Ahat[(size_t)t * nL + w->rowpos[A->row_idx[q]]] = A->val[q];
    }
    ehat[w->rowpos[k]] = 1.0;
    int st = orc_dense_lsq(nL, nS, Ahat, ehat, w->m);
    if (st == ORC_OK) {
        for (int32_t i = 0; i < nL; ++i) {
            double s = -ehat[i];
            for (int32_t t = 0; t < nS; ++t) s += Ahat[(size_t)t * nL + i] * w->m[t];
            w->r[i] = s;
        }
        *rn_out = orc_norm2(nL, w->r);
    }
    free(Ahat);
    free(ehat);
    return st;
}

typedef struct {
    uint64_t key;
    int32_t j;
} cand_t;

static int cmp_cand(const void* a, const void* b)
{
    const cand_t* x = (const cand_t*)a;
    const cand_t* y = (const cand_t*)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->j > y->j) - (x->j < y->j);
}

/* SPAI selection step (section 2.1): candidates J~ = N \ S, eq. (candi);
 * rho_j^2 = ||r||^2 - (r^T A e_j)^2 / ||A e_j||^2, eq. (rhoj); the mn
 * smallest are appended to S. Returns the number of indices added. */
static int32_t spai_augment(sai_ws* w, int32_t mn, int32_t key_bits, double rn)
{
    const orc_csc* A = w->A;
    int32_t nc = 0;
    for (int32_t t = 0; t < w->nS; ++t) w->colmark[w->S[t]] = 1;
    for (int32_t t = 0; t < w->nL; ++t) {
        int32_t i = w->L[t];
        for (int64_t q = w->rp[i]; q < w->rp[i + 1]; ++q) {
            int32_t j = w->ci[q];
            if (w->colmark[j] < 0) {
                w->colmark[j] = 2;
                w->tmp[nc++] = j;
            }
        }
    }
    cand_t* cand = (cand_t*)orc_xmalloc((size_t)nc * sizeof(cand_t));
    int32_t nvalid = 0;
    double rn2 = rn * rn;
    double scale = ldexp(1.0, key_bits);
    for (int32_t c = 0; c < nc; ++c) {
        int32_t j = w->tmp[c];
        if (w->colnorm2[j] == 0.0) continue;
        double d = 0.0; /* r^T A e_j over the stored entries of column j */
        for (int64_t q = A->col_ptr[j]; q < A->col_ptr[j + 1]; ++q) {
            int32_t pos = w->rowpos[A->row_idx[q]];
            if (pos >= 0) d += w->r[pos] * A->val[q];
        }
        double rho2 = rn2 - d * d / w->colnorm2[j];
        double t = rho2 / rn2;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        cand[nvalid].key = (uint64_t)floor(t * scale);
        cand[nvalid].j = j;
        ++nvalid;
    }
    qsort(cand, (size_t)nvalid, sizeof(cand_t), cmp_cand);
    int32_t take = nvalid < mn ? nvalid : mn;
    for (int32_t t = 0; t < w->nS; ++t) w->colmark[w->S[t]] = -1;
    for (int32_t c = 0; c < nc; ++c) w->colmark[w->tmp[c]] = -1;
    for (int32_t c = 0; c < take; ++c) w->S[w->nS++] = cand[c].j;
    free(cand);
    return take;
}

/* One SPAI column. On return w->S / w->m hold the pattern and values,
 * *loops the augmentation steps used, *res the final LS residual. */
static int spai_column(sai_ws* w, const orc_spai_params* prm, int32_t k, int32_t* loops, double* res,
                       int32_t* S_hist, int32_t cap_s, int32_t* S_off, double* res_hist)
{
    w->nS = 1;
    w->S[0] = k;
    int32_t l = 0;
    int32_t used = 0;
    if (S_off) S_off[0] = 0;
    for (;; ++l) {
        double rn = 0.0;
        int st = ls_on_pattern(w, k, &rn);
        if (st != ORC_OK) {
            reset_rows(w);
            return st;
        }
        if (S_hist) {
            if (used + w->nS > cap_s) {
                reset_rows(w);
                return ORC_NOMEM;
            }
            memcpy(S_hist + used, w->S, (size_t)w->nS * sizeof(int32_t));
            used += w->nS;
            S_off[l + 1] = used;
            res_hist[l] = rn;
        }
        *res = rn;
        if (rn <= prm->delta || l >= prm->max_aug) {
            reset_rows(w);
            break;
        }
        int32_t added = spai_augment(w, prm->mn, prm->key_bits, rn);
        reset_rows(w);
        if (added == 0) break;
    }
    *loops = l;
    return ORC_OK;
}

/* Append column k (pattern S, values m, or the entries flagged in keep) to
 * growing CSC storage, rows ascending. */
typedef struct {
    int32_t row;
    double v;
} entry_t;

static int cmp_entry(const void* a, const void* b)
{
    int32_t x = ((const entry_t*)a)->row, y = ((const entry_t*)b)->row;
    return (x > y) - (x < y);
}

typedef struct {
    int64_t cap, nnz;
    int32_t* row;
    double* val;
} grow_t;

static void grow_push(grow_t* g, int32_t row, double v)
{
    if (g->nnz == g->cap) {
        g->cap = g->cap ? 2 * g->cap : 1024;
        g->row = (int32_t*)realloc(g->row, (size_t)g->cap * sizeof(int32_t));
        g->val = (double*)realloc(g->val, (size_t)g->cap * sizeof(double));
    }
    g->row[g->nnz] = row;
    g->val[g->nnz] = v;
    g->nnz++;
}

static void emit_column(grow_t* g, const int32_t* S, const double* m, const char* keep, int32_t nS)
{
    entry_t* e = (entry_t*)orc_xmalloc((size_t)nS * sizeof(entry_t));
    int32_t ne = 0;
    for (int32_t t = 0; t < nS; ++t)
        if (!keep || keep[t]) {
            e[ne].row = S[t];
            e[ne].v = m[t];
            ++ne;
        }
    qsort(e, (size_t)ne, sizeof(entry_t), cmp_entry);
    for (int32_t t = 0; t < ne; ++t) grow_push(g, e[t].row, e[t].v);
    free(e);
}

int orc_spai(const orc_csc* At, const orc_spai_params* prm, int32_t c0, int32_t c1,
             orc_csc* M_out, int32_t* loops_out, double* res_out)
{
    if (!orc_csc_valid(At) || At->nrows != At->ncols || !prm || prm->mn < 1 || prm->max_aug < 0 ||
        prm->key_bits < 1 || prm->key_bits > 52)
        return ORC_BAD_INPUT;
    int32_t n = At->ncols;
    if (c0 < 0) c0 = 0;
    if (c1 > n) c1 = n;
    sai_ws w;
    ws_init(&w, At);
    grow_t g = {0, 0, NULL, NULL};
    M_out->nrows = n;
    M_out->ncols = n;
    M_out->col_ptr = (int64_t*)orc_xcalloc((size_t)n + 1, sizeof(int64_t));
    int st = ORC_OK;
    for (int32_t k = 0; k < n; ++k) {
        if (k >= c0 && k < c1 && st == ORC_OK) {
            int32_t loops = 0;
            double res = 0.0;
            st = spai_column(&w, prm, k, &loops, &res, NULL, 0, NULL, NULL);
            if (st == ORC_OK) {
                emit_column(&g, w.S, w.m, NULL, w.nS);
                loops_out[k] = loops;
                res_out[k] = res;
            }
        }
        M_out->col_ptr[k + 1] = g.nnz;
    }
    M_out->row_idx = g.row ? g.row : (int32_t*)orc_xmalloc(sizeof(int32_t));
    M_out->val = g.val ? g.val : (double*)orc_xmalloc(sizeof(double));
    ws_free(&w);
    return st;
}

int orc_spai_trace(const orc_csc* At, const orc_spai_params* prm, int32_t k,
                   int32_t* S_hist, int32_t cap_s, int32_t* S_off, double* res_hist)
{
    if (!orc_csc_valid(At) || At->nrows != At->ncols || k < 0 || k >= At->ncols) return -ORC_BAD_INPUT;
    sai_ws w;
    ws_init(&w, At);
    int32_t loops = 0;
    double res = 0.0;
    int st = spai_column(&w, prm, k, &loops, &res, S_hist, cap_s, S_off, res_hist);
    ws_free(&w);
    return st == ORC_OK ? loops + 1 : -st;
}

/* ---------------------------- PSAI(tol) ----------------------------------- */

/* One PSAI(tol) column (section 2.2). Loop l solves the LS problem on
 * S^(l), computes tol_k from the newly computed m_k, eq. (tolk), and either
 * stops (||r|| <= delta or l = lmax) emitting the entries |m_jk| > tol_k, or
 * grows S^(l+1) = P(a^(l+1)) u S_kept with a^(l+1) = |A~| a^(l). */
static int psai_column(sai_ws* w, const orc_psai_params* prm, int32_t k, char* keep, int32_t* loops,
                       double* res_pre, double* res_post, int32_t* S_hist, int32_t cap_s, int32_t* S_off,
                       double* res_hist)
{
    const orc_csc* A = w->A;
    int32_t n = w->n;
    int32_t* apat = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    int32_t na = 1;
    apat[0] = k;
    w->nS = 1;
    w->S[0] = k;
    int32_t used = 0;
    if (S_off) S_off[0] = 0;
    int st = ORC_OK;
    for (int32_t l = 0;; ++l) {
        double rn = 0.0;
        st = ls_on_pattern(w, k, &rn);
        if (st != ORC_OK) break;
        if (S_hist) {
            if (used + w->nS > cap_s) {
                st = ORC_NOMEM;
                break;
            }
            memcpy(S_hist + used, w->S, (size_t)w->nS * sizeof(int32_t));
            used += w->nS;
            S_off[l + 1] = used;
            res_hist[l] = rn;
        }
        if (prm->tol_mode == 2) {
            /* PSAI(lfill): keep the lfill entries of largest magnitude, equal
             * magnitudes to the smaller column index (counted one by one) */
            for (int32_t t = 0; t < w->nS; ++t) {
                int32_t rank = 0;
                for (int32_t u = 0; u < w->nS; ++u) {
                    const double mu = fabs(w->m[u]), mt = fabs(w->m[t]);
                    if (mu > mt || (mu == mt && w->S[u] < w->S[t])) ++rank;
                }
                keep[t] = (char)(rank < prm->lfill);
            }
        } else {
            double tolk = prm->tol;
            if (prm->tol_mode == 0) {
                int32_t nz = 0;
                for (int32_t t = 0; t < w->nS; ++t) nz += (w->m[t] != 0.0);
                tolk = (nz > 0 && w->norm1 > 0.0) ? prm->delta / ((double)nz * w->norm1) : 0.0;
            }
            for (int32_t t = 0; t < w->nS; ++t) keep[t] = (char)(fabs(w->m[t]) > tolk);
        }
        if (rn <= prm->delta || l >= prm->lmax) {
            /* residual of the emitted (dropped) column, on L */
            double* r2 = (double*)orc_xcalloc((size_t)w->nL, sizeof(double));
            r2[w->rowpos[k]] = -1.0;
            for (int32_t t = 0; t < w->nS; ++t) {
                if (!keep[t]) continue;
                int32_t j = w->S[t];
                for (int64_t q = A->col_ptr[j]; q < A->col_ptr[j + 1]; ++q)
                    r2[w->rowpos[A->row_idx[q]]] += A->val[q] * w->m[t];
            }
            *res_post = orc_norm2(w->nL, r2);
            free(r2);
            *res_pre = rn;
            *loops = l;
            break;
        }
        reset_rows(w);
        /* a^(l+1) = A~ a^(l), structurally: union of the column patterns */
        int32_t nb = 0;
        for (int32_t t = 0; t < na; ++t) {
            int32_t j = apat[t];
            for (int64_t q = A->col_ptr[j]; q < A->col_ptr[j + 1]; ++q) {
                int32_t i = A->row_idx[q];
                if (w->colmark[i] < 0) {
                    w->colmark[i] = 1;
                    w->tmp[nb++] = i;
                }
            }
        }
        for (int32_t t = 0; t < nb; ++t) w->colmark[w->tmp[t]] = -1;
        if (prm->growth == 1) {
            /* reading (C): S^(l+1) = S_kept^(l) u (P(a^(l+1)) \ P(a^(l))),
             * ascending; a dropped position never comes back */
            char* old_pat = (char*)orc_xcalloc((size_t)n, 1);
            char* in_next = (char*)orc_xcalloc((size_t)n, 1);
            int32_t* next = (int32_t*)orc_xmalloc(((size_t)w->nS + (size_t)nb + 1) * sizeof(int32_t));
            int32_t ns = 0;
            for (int32_t t = 0; t < na; ++t) old_pat[apat[t]] = 1;
            for (int32_t t = 0; t < w->nS; ++t)
                if (keep[t] && !in_next[w->S[t]]) {
                    in_next[w->S[t]] = 1;
                    next[ns++] = w->S[t];
                }
            for (int32_t t = 0; t < nb; ++t) {
                const int32_t i = w->tmp[t];
                if (!old_pat[i] && !in_next[i]) {
                    in_next[i] = 1;
                    next[ns++] = i;
                }
            }
            free(old_pat);
            free(in_next);
            if (ns == 0) {
                /* nothing kept and no new position: stop at loop l, emitting
                 * the (empty) kept set of this solution */
                free(next);
                *res_post = 1.0; /* the emitted column is empty: ||0 - e_k|| */
                *res_pre = rn;
                *loops = l;
                break;
            }
            memcpy(apat, w->tmp, (size_t)nb * sizeof(int32_t));
            na = nb;
            qsort(next, (size_t)ns, sizeof(int32_t), cmp_i32);
            memcpy(w->S, next, (size_t)ns * sizeof(int32_t));
            w->nS = ns;
            free(next);
            continue;
        }
        memcpy(apat, w->tmp, (size_t)nb * sizeof(int32_t));
        na = nb;
        /* S^(l+1) = P(a^(l+1)) u S_kept^(l), ascending */
        int32_t ns = 0;
        for (int32_t t = 0; t < na; ++t) {
            w->colmark[apat[t]] = 1;
            w->tmp[ns++] = apat[t];
        }
        for (int32_t t = 0; t < w->nS; ++t)
            if (keep[t] && w->colmark[w->S[t]] < 0) {
                w->colmark[w->S[t]] = 1;
                w->tmp[ns++] = w->S[t];
            }
        for (int32_t t = 0; t < ns; ++t) w->colmark[w->tmp[t]] = -1;
        qsort(w->tmp, (size_t)ns, sizeof(int32_t), cmp_i32);
        memcpy(w->S, w->tmp, (size_t)ns * sizeof(int32_t));
        w->nS = ns;
    }
    reset_rows(w);
    free(apat);
    return st;
}

int orc_psai(const orc_csc* At, const orc_psai_params* prm, int32_t c0, int32_t c1,
             orc_csc* M_out, int32_t* loops_out, double* res_pre, double* res_post)
{
    if (!orc_csc_valid(At) || At->nrows != At->ncols || !prm || prm->lmax < 0 || prm->tol_mode < 0 ||
        prm->tol_mode > 2 || (prm->tol_mode == 2 && prm->lfill < 1) || (prm->growth != 0 && prm->growth != 1))
        return ORC_BAD_INPUT;
    int32_t n = At->ncols;
    if (c0 < 0) c0 = 0;
    if (c1 > n) c1 = n;
    sai_ws w;
    ws_init(&w, At);
    char* keep = (char*)orc_xmalloc((size_t)n);
    grow_t g = {0, 0, NULL, NULL};
    M_out->nrows = n;
    M_out->ncols = n;
    M_out->col_ptr = (int64_t*)orc_xcalloc((size_t)n + 1, sizeof(int64_t));
    int st = ORC_OK;
    for (int32_t k = 0; k < n; ++k) {
        if (k >= c0 && k < c1 && st == ORC_OK) {
            int32_t loops = 0;
            double pre = 0.0, post = 0.0;
            st = psai_column(&w, prm, k, keep, &loops, &pre, &post, NULL, 0, NULL, NULL);
            if (st == ORC_OK) {
                emit_column(&g, w.S, w.m, keep, w.nS);
                loops_out[k] = loops;
                res_pre[k] = pre;
                res_post[k] = post;
            }
        }
        M_out->col_ptr[k + 1] = g.nnz;
    }
    M_out->row_idx = g.row ? g.row : (int32_t*)orc_xmalloc(sizeof(int32_t));
    M_out->val = g.val ? g.val : (double*)orc_xmalloc(sizeof(double));
    free(keep);
    ws_free(&w);
    return st;
}

int orc_psai_trace(const orc_csc* At, const orc_psai_params* prm, int32_t k,
                   int32_t* S_hist, int32_t cap_s, int32_t* S_off, double* res_hist)
{
    if (!orc_csc_valid(At) || At->nrows != At->ncols || k < 0 || k >= At->ncols) return -ORC_BAD_INPUT;
    sai_ws w;
    ws_init(&w, At);
    char* keep = (char*)orc_xmalloc((size_t)At->ncols);
    int32_t loops = 0;
    double pre = 0.0, post = 0.0;
    int st = psai_column(&w, prm, k, keep, &loops, &pre, &post, S_hist, cap_s, S_off, res_hist);
    free(keep);
    ws_free(&w);
    return st == ORC_OK ? loops + 1 : -st;
}
