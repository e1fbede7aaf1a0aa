/* oracle_smw.c -- Sherman-Morrison-Woodbury recovery (Theorem 1, eqs.
 * (update1), (composi)), the true relative residual (eq. (rrnorm)) and the
 * whole of Procedure * with the stopping rules of Theorem 2, eqs. (stopb)
 * and (stopU2) with c = 1 (section 4), optionally continued with the c the
 * recovery measures.  Test infrastructure only. */
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* eq. (composi): xhat = yhat - W (I + V^T W)^{-1} (V^T yhat). */
int orc_smw(int32_t n, int32_t s, const double* yhat, const double* W, const int32_t* J,
            double* x_out, double* z_out, double* c_out)
{
    if (s < 0 || n < 0) return ORC_BAD_INPUT;
    double* C = (double*)orc_xmalloc((size_t)s * (size_t)s * sizeof(double));
    double* g = (double*)orc_xmalloc((size_t)s * sizeof(double));
    for (int32_t t = 0; t < s; ++t) {
        g[t] = yhat[J[t]];                                    /* V^T yhat */
        for (int32_t i = 0; i < s; ++i)                       /* I + V^T W */
            C[(size_t)t * s + i] = (i == t ? 1.0 : 0.0) + W[(size_t)t * n + J[i]];
    }
    int st = orc_dense_lu_solve(s, C, g, z_out);
    if (st == ORC_OK) {
        for (int32_t i = 0; i < n; ++i) {
            double v = yhat[i];
            for (int32_t t = 0; t < s; ++t) v -= W[(size_t)t * n + i] * z_out[t];
            x_out[i] = v;
        }
        *c_out = orc_norm2(s, z_out);
    }
    free(C);
    free(g);
    return st;
}

/* eq. (rrnorm): rr = ||b - A x|| / ||b||. */
double orc_rel_resid(const orc_csc* A, const double* b, const double* x)
{
    int32_t n = A->nrows;
    double* ax = (double*)orc_xmalloc((size_t)n * sizeof(double));
    orc_csc_matvec(A, x, ax);
    double num = 0.0;
    for (int32_t i = 0; i < n; ++i) num += (b[i] - ax[i]) * (b[i] - ax[i]);
    free(ax);
    return sqrt(num) / orc_norm2(n, b);
}

/* Procedure *: step 1 split, then one M for A~, step 2 the s+1 solves with
 * the Theorem 2 thresholds (c = 1), step 3 the SMW recovery. */
int orc_solve(const orc_csc* A, const double* b, const orc_solve_params* prm,
              double* x_out, int32_t* iters_out, orc_solve_report* rep)
{
    if (!orc_csc_valid(A) || A->nrows != A->ncols || !prm || !rep) return ORC_BAD_INPUT;
    int32_t n = A->ncols;
    memset(rep, 0, sizeof(*rep));
    int32_t* J = (int32_t*)orc_xmalloc((size_t)n * sizeof(int32_t));
    int32_t s = 0, p = 0;
    double tau = 0.0;
    int st = orc_detect(A, prm->thresh_mult, prm->abs_tau, 0, J, &s, &p, &tau);
    if (st != ORC_OK) {
        free(J);
        return st;
    }
    orc_csc At = {0}, U = {0}, M = {0};
    st = orc_split(A, J, s, p > 0 ? p : 1, &At, &U);
    if (st != ORC_OK) {
        free(J);
        return st;
    }
    rep->s = s;
    rep->p = p;
    rep->tau = tau;
    rep->nnz_At = At.col_ptr[n];
    int32_t* loops = (int32_t*)orc_xcalloc((size_t)n, sizeof(int32_t));
    double* res = (double*)orc_xcalloc((size_t)n, sizeof(double));
    double* res2 = (double*)orc_xcalloc((size_t)n, sizeof(double));
    double delta;
    if (prm->sai == 0) {
        st = orc_spai(&At, &prm->spai, 0, n, &M, loops, res);
        delta = prm->spai.delta;
    } else {
        st = orc_psai(&At, &prm->psai, 0, n, &M, loops, res, res2);
        delta = prm->psai.delta;
    }
    if (st == ORC_OK) {
        rep->nnz_M = M.col_ptr[n];
        for (int32_t k = 0; k < n; ++k) {
            if (res[k] > delta) rep->n_c++;
            if (loops[k] > rep->l_m) rep->l_m = loops[k];
        }
        double bnorm = orc_norm2(n, b);
        double* Y = (double*)orc_xcalloc((size_t)(s + 1) * (size_t)n, sizeof(double)); /* [y, w_1..w_s] */
        double* rhs = (double*)orc_xmalloc((size_t)n * sizeof(double));
        double* tmp = (double*)orc_xmalloc((size_t)n * sizeof(double));
        double rW2 = 0.0, ry = 0.0;
        double* Bblk = prm->krylov == 4 ? (double*)orc_xmalloc((size_t)(s + 1) * (size_t)n * sizeof(double)) : NULL;
        double* blk_thr = prm->krylov == 4 ? (double*)orc_xmalloc((size_t)(s + 1) * sizeof(double)) : NULL;
        int blk_st = ORC_OK;
        int32_t* blk_it = prm->krylov == 4 ? (int32_t*)orc_xcalloc((size_t)(s + 1), sizeof(int32_t)) : NULL;
        rep->status = ORC_OK;
        for (int32_t q = 0; q <= s && st == ORC_OK; ++q) {
            double thr;
            if (q == 0) {
                memcpy(rhs, b, (size_t)n * sizeof(double));
                thr = 0.5 * prm->eps * bnorm;                          /* eq. (stopb) */
            } else {
                for (int32_t i = 0; i < n; ++i) rhs[i] = 0.0;
                for (int64_t t = U.col_ptr[q - 1]; t < U.col_ptr[q]; ++t) rhs[U.row_idx[t]] = U.val[t];
                thr = prm->eps * bnorm / (2.0 * sqrt((double)s));      /* eq. (stopU2), c = 1 */
            }
            int32_t it = 0;
            int ks;
            if (prm->krylov == 4) {
                /* block GMRES: all s+1 systems at once, at q = 0 */
                if (q == 0) {
                    blk_thr[0] = thr;
                    memcpy(Bblk, rhs, (size_t)n * sizeof(double));
                    for (int32_t t = 1; t <= s; ++t) {
                        double* bt = Bblk + (size_t)t * n;
                        for (int32_t i = 0; i < n; ++i) bt[i] = 0.0;
                        for (int64_t e = U.col_ptr[t - 1]; e < U.col_ptr[t]; ++e) bt[U.row_idx[e]] = U.val[e];
                        blk_thr[t] = prm->eps * bnorm / (2.0 * sqrt((double)s));
                    }
                    blk_st = orc_block_gmres(&At, &M, s + 1, Bblk, blk_thr, prm->restart, prm->maxit, Y, blk_it);
                }
                ks = blk_st;
                it = blk_it[q];
            } else if (prm->krylov == 0) ks = orc_bicgstab(&At, &M, rhs, thr, prm->maxit, Y + (size_t)q * n, &it);
            else if (prm->krylov == 2) ks = orc_cgs(&At, &M, rhs, thr, prm->maxit, Y + (size_t)q * n, &it);
            else if (prm->krylov == 3) ks = orc_bicg(&At, &M, rhs, thr, prm->maxit, Y + (size_t)q * n, &it);
            else ks = orc_gmres(&At, &M, rhs, thr, prm->restart, prm->maxit, Y + (size_t)q * n, &it);
            if (ks != ORC_OK && rep->status == ORC_OK) rep->status = ks;
            if (ks == ORC_BAD_INPUT) st = ks;
            if (iters_out) iters_out[q] = it;
            if (it > rep->iter_max) rep->iter_max = it;
            /* true residual of this system, for the Theorem 2 bound */
            orc_csc_matvec(&At, Y + (size_t)q * n, tmp);
            double rr2 = 0.0;
            for (int32_t i = 0; i < n; ++i) rr2 += (rhs[i] - tmp[i]) * (rhs[i] - tmp[i]);
            if (q == 0) ry = sqrt(rr2);
            else rW2 += rr2;
        }
        if (st == ORC_OK) {
            double* z = (double*)orc_xmalloc((size_t)(s > 0 ? s : 1) * sizeof(double));
            double c = 0.0;
            st = orc_smw(n, s, Y, Y + n, J, x_out, z, &c);
            rep->c_first = c;
            if (st == ORC_OK && prm->c_adapt && s > 0 && c > 1.0) {
                /* Theorem 2 bounds ||b - A xhat|| by ||r_y|| + c ||R_W||_F; with
                 * the c = 1 thresholds that exceeds eps ||b|| once c > 1. Reading
                 * of eq. (stopU2): its c is the c the recovery measures, so the
                 * u_j systems are continued from their iterates (a correction
                 * solve A~ d = u_j - A~ w_j, w_j += d) to eps ||b|| / (2 sqrt(s)
                 * 1.05 c) and x is recovered again. */
                const double thr2 = prm->eps * bnorm / (2.0 * sqrt((double)s) * 1.05 * c);
                double* D = (double*)orc_xcalloc((size_t)(s + 1) * (size_t)n, sizeof(double));
                double* R = (double*)orc_xcalloc((size_t)(s + 1) * (size_t)n, sizeof(double));
                double* th2 = (double*)orc_xmalloc((size_t)(s + 1) * sizeof(double));
                int32_t* it2 = (int32_t*)orc_xcalloc((size_t)(s + 1), sizeof(int32_t));
                th2[0] = 0.5 * prm->eps * bnorm;  /* system 0 has no correction: rhs 0 */
                for (int32_t q = 1; q <= s; ++q) {
                    double* rq = R + (size_t)q * n;
                    for (int64_t t = U.col_ptr[q - 1]; t < U.col_ptr[q]; ++t) rq[U.row_idx[t]] = U.val[t];
                    orc_csc_matvec(&At, Y + (size_t)q * n, tmp);
                    for (int32_t i = 0; i < n; ++i) rq[i] -= tmp[i];
                    th2[q] = thr2;
                }
                int ks2 = ORC_OK;
                if (prm->krylov == 4) {
                    ks2 = orc_block_gmres(&At, &M, s + 1, R, th2, prm->restart, prm->maxit, D, it2);
                } else {
                    for (int32_t q = 1; q <= s; ++q) {
                        int kq;
                        double* rq = R + (size_t)q * n;
                        double* dq = D + (size_t)q * n;
                        if (prm->krylov == 0) kq = orc_bicgstab(&At, &M, rq, thr2, prm->maxit, dq, &it2[q]);
                        else if (prm->krylov == 2) kq = orc_cgs(&At, &M, rq, thr2, prm->maxit, dq, &it2[q]);
                        else if (prm->krylov == 3) kq = orc_bicg(&At, &M, rq, thr2, prm->maxit, dq, &it2[q]);
                        else kq = orc_gmres(&At, &M, rq, thr2, prm->restart, prm->maxit, dq, &it2[q]);
                        if (kq != ORC_OK && ks2 == ORC_OK) ks2 = kq;
                    }
                }
                if (ks2 != ORC_OK && rep->status == ORC_OK) rep->status = ks2;
                rW2 = 0.0;
                for (int32_t q = 1; q <= s; ++q) {
                    double* wq = Y + (size_t)q * n;
                    double* dq = D + (size_t)q * n;
                    for (int32_t i = 0; i < n; ++i) wq[i] += dq[i];
                    const int32_t itq = (iters_out ? iters_out[q] : 0) + it2[q];
                    if (iters_out) iters_out[q] = itq;
                    if (itq > rep->iter_max) rep->iter_max = itq;
                    /* true residual of the continued w_q */
                    double* rq = R + (size_t)q * n;
                    for (int32_t i = 0; i < n; ++i) rq[i] = 0.0;
                    for (int64_t t = U.col_ptr[q - 1]; t < U.col_ptr[q]; ++t) rq[U.row_idx[t]] = U.val[t];
                    orc_csc_matvec(&At, wq, tmp);
                    for (int32_t i = 0; i < n; ++i) rW2 += (rq[i] - tmp[i]) * (rq[i] - tmp[i]);
                }
                st = orc_smw(n, s, Y, Y + n, J, x_out, z, &c);
                rep->c_rounds = 1;
                free(D);
                free(R);
                free(th2);
                free(it2);
            }
            if (st == ORC_OK) {
                rep->c = c;
                rep->rr = orc_rel_resid(A, b, x_out);
                rep->bound = ry + c * sqrt(rW2);
            }
            free(z);
        }
        free(Y);
        free(rhs);
        free(tmp);
        free(Bblk);
        free(blk_thr);
        free(blk_it);
    }
    free(loops);
    free(res);
    free(res2);
    free(J);
    orc_csc_free(&At);
    orc_csc_free(&U);
    orc_csc_free(&M);
    return st;
}
