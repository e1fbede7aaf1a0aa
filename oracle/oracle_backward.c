/* oracle_backward.c -- backward pass of x = A^{-1} b, written from the
 * method's own pieces. The paper has no backward pass: this is the adjoint
 * of Procedure * (section 3). With A = A~ + U V^T, A^T = A~^T + V U^T, so
 * Theorem 1 applied to A^T gives
 *     lambda = A^{-T} g = yhat - W (I + U^T W)^{-1} (U^T yhat),
 *     [yhat, W] = A~^{-T} [g, e_J1 .. e_Js],
 * and for a loss L with g = dL/dx: dL/db = lambda, dL/dA_ij = -lambda_i x_j.
 * The s+1 transposed systems are solved with the right preconditioner M^T
 * (M ~ A~^{-1} gives M^T ~ A~^{-T}) and the Theorem 2 thresholds taken from
 * ||g||. Test infrastructure only. */
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* B = A^T in CSC (the CSR arrays of A). */
int orc_csc_transpose(const orc_csc* A, orc_csc* B)
{
    int64_t* rp = NULL;
    int32_t* ci = NULL;
    double* v = NULL;
    orc_csc_to_csr(A, &rp, &ci, &v);
    B->nrows = A->ncols;
    B->ncols = A->nrows;
    B->col_ptr = rp;
    B->row_idx = ci;
    B->val = v;
    return ORC_OK;
}

/* Theorem 1 on A^T = A~^T + V U^T: lambda = yhat - W (I + U^T W)^{-1} U^T yhat.
 * W: n x s column-major; U: n x s CSC. */
int orc_smw_adjoint(int32_t n, int32_t s, const double* yhat, const double* W, const orc_csc* U,
                    double* lambda_out, double* z_out, double* c_out)
{
    if (s < 0 || n < 0) return ORC_BAD_INPUT;
    double* C = (double*)orc_xmalloc((size_t)s * (size_t)s * sizeof(double));
    double* g = (double*)orc_xmalloc((size_t)s * sizeof(double));
    for (int32_t a = 0; a < s; ++a) {
        double ga = 0.0;                                      /* (U^T yhat)_a */
        for (int64_t t = U->col_ptr[a]; t < U->col_ptr[a + 1]; ++t) ga += U->val[t] * yhat[U->row_idx[t]];
        g[a] = ga;
        for (int32_t b = 0; b < s; ++b) {                     /* (I + U^T W)_{ab} */
            double cab = (a == b) ? 1.0 : 0.0;
            for (int64_t t = U->col_ptr[a]; t < U->col_ptr[a + 1]; ++t)
                cab += U->val[t] * W[(size_t)b * n + U->row_idx[t]];
            C[(size_t)b * s + a] = cab;
        }
    }
    int st = orc_dense_lu_solve(s, C, g, z_out);
    if (st == ORC_OK) {
        for (int32_t i = 0; i < n; ++i) {
            double v = yhat[i];
            for (int32_t t = 0; t < s; ++t) v -= W[(size_t)t * n + i] * z_out[t];
            lambda_out[i] = v;
        }
        *c_out = orc_norm2(s, z_out);
    }
    free(C);
    free(g);
    return st;
}

/* The backward pass: detect, split, M as in orc_solve, then the s+1
 * transposed solves, orc_smw_adjoint and the gradients on A's pattern
 * (grad_vals aligned with A->val). rep->rr = ||g - A^T lambda|| / ||g||. */
int orc_backward(const orc_csc* A, const double* x, const double* g, const orc_solve_params* prm,
                 double* lambda_out, double* grad_vals, int32_t* iters_out, orc_solve_report* rep)
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
    orc_csc At = {0}, U = {0}, M = {0}, AtT = {0}, MT = {0};
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
    if (prm->sai == 0) st = orc_spai(&At, &prm->spai, 0, n, &M, loops, res);
    else st = orc_psai(&At, &prm->psai, 0, n, &M, loops, res, res2);
    if (st == ORC_OK) {
        rep->nnz_M = M.col_ptr[n];
        orc_csc_transpose(&At, &AtT);
        orc_csc_transpose(&M, &MT);
        double gnorm = orc_norm2(n, g);
        double* Y = (double*)orc_xcalloc((size_t)(s + 1) * (size_t)n, sizeof(double)); /* [yhat, w_1..w_s] */
        double* rhs = (double*)orc_xmalloc((size_t)n * sizeof(double));
        double* Bblk = prm->krylov == 4 ? (double*)orc_xmalloc((size_t)(s + 1) * (size_t)n * sizeof(double)) : NULL;
        double* blk_thr = prm->krylov == 4 ? (double*)orc_xmalloc((size_t)(s + 1) * sizeof(double)) : NULL;
        int blk_st = ORC_OK;
        int32_t* blk_it = prm->krylov == 4 ? (int32_t*)orc_xcalloc((size_t)(s + 1), sizeof(int32_t)) : NULL;
        rep->status = ORC_OK;
        for (int32_t q = 0; q <= s && st == ORC_OK; ++q) {
            double thr;
            if (q == 0) {
                memcpy(rhs, g, (size_t)n * sizeof(double));
                thr = 0.5 * prm->eps * gnorm;
            } else {
                for (int32_t i = 0; i < n; ++i) rhs[i] = 0.0;
                rhs[J[q - 1]] = 1.0;                              /* V e_q = e_{J_q} */
                thr = prm->eps * gnorm / (2.0 * sqrt((double)s));
            }
            int32_t it = 0;
            int ks;
            if (prm->krylov == 4) {
                /* block GMRES: all s+1 transposed systems at once, at q = 0 */
                if (q == 0) {
                    blk_thr[0] = thr;
                    memcpy(Bblk, rhs, (size_t)n * sizeof(double));
                    for (int32_t t = 1; t <= s; ++t) {
                        double* bt = Bblk + (size_t)t * n;
                        for (int32_t i = 0; i < n; ++i) bt[i] = 0.0;
                        bt[J[t - 1]] = 1.0;
                        blk_thr[t] = prm->eps * gnorm / (2.0 * sqrt((double)s));
                    }
                    blk_st = orc_block_gmres(&AtT, &MT, s + 1, Bblk, blk_thr, prm->restart, prm->maxit, Y, blk_it);
                }
                ks = blk_st;
                it = blk_it[q];
            } else if (prm->krylov == 0) ks = orc_bicgstab(&AtT, &MT, rhs, thr, prm->maxit, Y + (size_t)q * n, &it);
            else if (prm->krylov == 2) ks = orc_cgs(&AtT, &MT, rhs, thr, prm->maxit, Y + (size_t)q * n, &it);
            else if (prm->krylov == 3) ks = orc_bicg(&AtT, &MT, rhs, thr, prm->maxit, Y + (size_t)q * n, &it);
            else ks = orc_gmres(&AtT, &MT, rhs, thr, prm->restart, prm->maxit, Y + (size_t)q * n, &it);
            if (ks != ORC_OK && rep->status == ORC_OK) rep->status = ks;
            if (ks == ORC_BAD_INPUT) st = ks;
            if (iters_out) iters_out[q] = it;
            if (it > rep->iter_max) rep->iter_max = it;
        }
        if (st == ORC_OK) {
            double* z = (double*)orc_xmalloc((size_t)(s > 0 ? s : 1) * sizeof(double));
            double c = 0.0;
            st = orc_smw_adjoint(n, s, Y, Y + n, &U, lambda_out, z, &c);
            if (st == ORC_OK) {
                rep->c = c;
                /* ||g - A^T lambda|| / ||g||: (A^T lambda)_j = a_j^T lambda */
                double num = 0.0;
                for (int32_t j = 0; j < n; ++j) {
                    double t = 0.0;
                    for (int64_t q = A->col_ptr[j]; q < A->col_ptr[j + 1]; ++q) t += A->val[q] * lambda_out[A->row_idx[q]];
                    num += (g[j] - t) * (g[j] - t);
                    if (grad_vals)
                        for (int64_t q = A->col_ptr[j]; q < A->col_ptr[j + 1]; ++q)
                            grad_vals[q] = -lambda_out[A->row_idx[q]] * x[j];
                }
                rep->rr = sqrt(num) / gnorm;
            }
            free(z);
        }
        free(Y);
        free(rhs);
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
    orc_csc_free(&AtT);
    orc_csc_free(&MT);
    return st;
}
