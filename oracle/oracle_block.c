/* oracle_block.c -- block GMRES(m) for the s+1 systems (the block Krylov
 * alternative that section 3 names after Theorem 2 for eqs. (regprob) and
 * (auxi)).
 *
 * TEST INFRASTRUCTURE (see oracle.h): plain sequential FP64, no tuning.
 *
 * Textbook block GMRES (Vital 1990; Saad, Iterative Methods for Sparse
 * Linear Systems, 2nd ed., section 6.12) with right preconditioning, as
 * orc_gmres: the k right-hand sides B = [b1 .. bk] share one block Krylov
 * space of A~M, Y = M Z.
 *   cycle: R = B - A~ Y (B at the start); a column with ||R e_c|| < thr_c
 *          is frozen (done), the kb others form the cycle's block; stop when
 *          none is left; R_act = V_0 S (QR, diag(S) >= 0); G = [S; 0].
 *   step j = 0, 1, ..: W = A~ M V_j; for i = 0..j: H_ij = V_i^T W,
 *          W -= V_i H_ij (block modified Gram-Schmidt); W = V_{j+1} H_{j+1,j}
 *          (QR, diag >= 0). The block Hessenberg matrix Hbar ((j+2)k x (j+1)k)
 *          is reduced to triangular form by Householder reflections on rows
 *          q..q+k of each column q, applied to G as they are made; the least-
 *          squares residual of column c is ||G[(j+1)k : (j+2)k, c]||.
 *          The cycle ends when every column's residual is below its
 *          threshold, after m steps, or at maxit steps in all.
 *   end:   Z = V Rtri^{-1} G_top, Y += M Z, and the next cycle start tests
 *          the true residuals.
 * iters[c] counts the block steps column c took part in; one block step
 * applies A~ and M to each of the kb columns.
 * The dense QR of an n x k block is Householder QR with the Q factor formed
 * explicitly and the signs chosen so that diag(R) >= 0.
 */
#include "oracle_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Householder QR of the n x k column-major block W (overwritten by Q, n x k,
 * orthonormal columns); R (k x k, column-major, upper) gets diag >= 0. */
static void block_qr(int32_t n, int32_t k, double* W, double* R)
{
    double* A = (double*)orc_xmalloc((size_t)n * k * sizeof(double));
    double* beta = (double*)orc_xmalloc((size_t)k * sizeof(double));
    memcpy(A, W, (size_t)n * k * sizeof(double));
    for (int32_t c = 0; c < k; ++c) {
        double* a = A + (size_t)c * n;
        for (int32_t r = 0; r < k; ++r) R[(size_t)c * k + r] = 0.0;
        double nrm = 0.0;
        for (int32_t i = c; i < n; ++i) nrm += a[i] * a[i];
        nrm = sqrt(nrm);
        if (nrm == 0.0) {  /* nothing to reflect: the identity, R(c,c) = 0 */
            beta[c] = 0.0;
            continue;
        }
        const double alpha = a[c] >= 0.0 ? -nrm : nrm;
        /* v = a - alpha e_c stored in a[c..n), H = I - beta v v^T */
        a[c] -= alpha;
        double vv = 0.0;
        for (int32_t i = c; i < n; ++i) vv += a[i] * a[i];
        beta[c] = 2.0 / vv;
        for (int32_t d = c + 1; d < k; ++d) {
            double* b = A + (size_t)d * n;
            double t = 0.0;
            for (int32_t i = c; i < n; ++i) t += a[i] * b[i];
            t *= beta[c];
            for (int32_t i = c; i < n; ++i) b[i] -= t * a[i];
        }
        R[(size_t)c * k + c] = alpha;
    }
    /* R's strictly upper part of column d was left in A's rows 0..d-1 */
    for (int32_t d = 0; d < k; ++d)
        for (int32_t r = 0; r < d; ++r) R[(size_t)d * k + r] = A[(size_t)d * n + r];
    /* Q = H_0 H_1 .. H_{k-1} [e_0 .. e_{k-1}] */
    for (int32_t c = 0; c < k; ++c) {
        double* q = W + (size_t)c * n;
        for (int32_t i = 0; i < n; ++i) q[i] = 0.0;
        q[c] = 1.0;
        for (int32_t h = (c < k - 1 ? c : k - 1); h >= 0; --h) {
            if (beta[h] == 0.0) continue;
            const double* v = A + (size_t)h * n;
            double t = 0.0;
            for (int32_t i = h; i < n; ++i) t += v[i] * q[i];
            t *= beta[h];
            for (int32_t i = h; i < n; ++i) q[i] -= t * v[i];
        }
    }
    /* signs: diag(R) >= 0 */
    for (int32_t c = 0; c < k; ++c)
        if (R[(size_t)c * k + c] < 0.0) {
            for (int32_t d = c; d < k; ++d) R[(size_t)d * k + c] = -R[(size_t)d * k + c];
            double* q = W + (size_t)c * n;
            for (int32_t i = 0; i < n; ++i) q[i] = -q[i];
        }
    free(A);
    free(beta);
}

int orc_block_gmres(const orc_csc* At, const orc_csc* M, int32_t k, const double* B, const double* thr, int32_t m,
                    int32_t maxit, double* Y, int32_t* iters)
{
    const int32_t n = At->ncols;
    if (m < 1 || k < 1 || maxit < 0) return ORC_BAD_INPUT;
    const int32_t rows = (m + 1) * k, cols = m * k, L = k + 1;
    double* V = (double*)orc_xmalloc((size_t)(m + 1) * k * (size_t)n * sizeof(double));
    double* Hb = (double*)orc_xmalloc((size_t)rows * cols * sizeof(double));
    double* hv = (double*)orc_xmalloc((size_t)cols * L * sizeof(double));   /* reflector of column q */
    double* hbeta = (double*)orc_xmalloc((size_t)cols * sizeof(double));
    double* G = (double*)orc_xmalloc((size_t)rows * k * sizeof(double));
    double* Ys = (double*)orc_xmalloc((size_t)cols * k * sizeof(double));
    double* W = (double*)orc_xmalloc((size_t)n * k * sizeof(double));
    double* R = (double*)orc_xmalloc((size_t)n * k * sizeof(double));
    double* S = (double*)orc_xmalloc((size_t)k * k * sizeof(double));
    double* z = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* w = (double*)orc_xmalloc((size_t)n * sizeof(double));
    int32_t* act = (int32_t*)orc_xmalloc((size_t)k * sizeof(int32_t));  /* active columns of this cycle */
    int* done = (int*)orc_xcalloc((size_t)k, sizeof(int));
#define HB(i, q) Hb[(size_t)(q) * rows + (i)]
#define GG(i, c) G[(size_t)(c) * rows + (i)]
    for (size_t t = 0; t < (size_t)n * k; ++t) {
        Y[t] = 0.0;
        R[t] = B[t];
    }
    for (int32_t c = 0; c < k; ++c) iters[c] = 0;
    int32_t it = 0;
    int status = ORC_MAXITER;
    for (;;) {
        /* cycle start: a column whose true residual meets its threshold is
         * frozen; the others form this cycle's block */
        int32_t kb = 0;
        for (int32_t c = 0; c < k; ++c) {
            if (done[c]) continue;
            if (orc_norm2(n, R + (size_t)c * n) < thr[c]) done[c] = 1;
            else act[kb++] = c;
        }
        if (kb == 0) {
            status = ORC_OK;
            break;
        }
        if (it >= maxit) break;
        for (int32_t a = 0; a < kb; ++a) memcpy(V + (size_t)a * n, R + (size_t)act[a] * n, (size_t)n * sizeof(double));
        block_qr(n, kb, V, S);
        for (size_t t = 0; t < (size_t)rows * k; ++t) G[t] = 0.0;
        for (int32_t c = 0; c < kb; ++c)
            for (int32_t r = 0; r <= c; ++r) GG(r, c) = S[(size_t)c * kb + r];
        for (size_t t = 0; t < (size_t)rows * cols; ++t) Hb[t] = 0.0;
        int32_t jdone = 0;
        for (int32_t j = 0; j < m && it < maxit; ++j) {
            const double* Vj = V + (size_t)j * kb * n;
            for (int32_t c = 0; c < kb; ++c) {
                orc_csc_matvec(M, Vj + (size_t)c * n, z);
                orc_csc_matvec(At, z, W + (size_t)c * n);
            }
            for (int32_t i = 0; i <= j; ++i) {  /* block modified Gram-Schmidt */
                const double* Vi = V + (size_t)i * kb * n;
                for (int32_t c = 0; c < kb; ++c)
                    for (int32_t r = 0; r < kb; ++r) HB(i * kb + r, j * kb + c) = orc_dot(n, Vi + (size_t)r * n,
                                                                                        W + (size_t)c * n);
                for (int32_t c = 0; c < kb; ++c) {
                    double* wc = W + (size_t)c * n;
                    for (int32_t r = 0; r < kb; ++r) {
                        const double h = HB(i * kb + r, j * kb + c);
                        const double* vr = Vi + (size_t)r * n;
                        for (int32_t q = 0; q < n; ++q) wc[q] -= h * vr[q];
                    }
                }
            }
            block_qr(n, kb, W, S);
            memcpy(V + (size_t)(j + 1) * kb * n, W, (size_t)n * kb * sizeof(double));
            for (int32_t c = 0; c < kb; ++c)
                for (int32_t r = 0; r <= c; ++r) HB((j + 1) * kb + r, j * kb + c) = S[(size_t)c * kb + r];
            /* the earlier reflections, in order, on the new block column */
            for (int32_t q = 0; q < j * kb; ++q) {
                const double* v = hv + (size_t)q * L;
                for (int32_t c = j * kb; c < (j + 1) * kb; ++c) {
                    double t = 0.0;
                    for (int32_t l = 0; l <= kb; ++l) t += v[l] * HB(q + l, c);
                    t *= hbeta[q];
                    for (int32_t l = 0; l <= kb; ++l) HB(q + l, c) -= t * v[l];
                }
            }
            /* new reflections: column q's rows q+1..q+kb to zero */
            for (int32_t q = j * kb; q < (j + 1) * kb; ++q) {
                double* v = hv + (size_t)q * L;
                double nrm = 0.0;
                for (int32_t l = 0; l <= kb; ++l) {
                    v[l] = HB(q + l, q);
                    nrm += v[l] * v[l];
                }
                nrm = sqrt(nrm);
                if (nrm == 0.0) {
                    hbeta[q] = 0.0;
                    continue;
                }
                const double alpha = v[0] >= 0.0 ? -nrm : nrm;
                v[0] -= alpha;
                double vv = 0.0;
                for (int32_t l = 0; l <= kb; ++l) vv += v[l] * v[l];
                hbeta[q] = 2.0 / vv;
                HB(q, q) = alpha;
                for (int32_t l = 1; l <= kb; ++l) HB(q + l, q) = 0.0;
                for (int32_t c = q + 1; c < (j + 1) * kb; ++c) {
                    double t = 0.0;
                    for (int32_t l = 0; l <= kb; ++l) t += v[l] * HB(q + l, c);
                    t *= hbeta[q];
                    for (int32_t l = 0; l <= kb; ++l) HB(q + l, c) -= t * v[l];
                }
                for (int32_t c = 0; c < kb; ++c) {
                    double t = 0.0;
                    for (int32_t l = 0; l <= kb; ++l) t += v[l] * GG(q + l, c);
                    t *= hbeta[q];
                    for (int32_t l = 0; l <= kb; ++l) GG(q + l, c) -= t * v[l];
                }
            }
            ++it;
            for (int32_t a = 0; a < kb; ++a) iters[act[a]]++;
            jdone = j + 1;
            int all = 1;
            for (int32_t c = 0; c < kb; ++c) {
                double e = 0.0;
                for (int32_t r = (j + 1) * kb; r < (j + 2) * kb; ++r) e += GG(r, c) * GG(r, c);
                if (!(sqrt(e) < thr[act[c]])) all = 0;
            }
            if (all) break;
        }
        /* Ys = Rtri^{-1} G_top, Z = V Ys, Y += M Z, R = B - A~ Y */
        const int32_t nt = jdone * kb;
        for (int32_t c = 0; c < kb && status != ORC_BREAKDOWN; ++c)
            for (int32_t i = nt - 1; i >= 0; --i) {
                double t = GG(i, c);
                for (int32_t q = i + 1; q < nt; ++q) t -= HB(i, q) * Ys[(size_t)c * cols + q];
                if (HB(i, i) == 0.0) {
                    status = ORC_BREAKDOWN;
                    break;
                }
                Ys[(size_t)c * cols + i] = t / HB(i, i);
            }
        if (status == ORC_BREAKDOWN) break;
        for (int32_t a = 0; a < kb; ++a) {
            const int32_t c = act[a];
            for (int32_t q = 0; q < n; ++q) w[q] = 0.0;
            for (int32_t i = 0; i < nt; ++i) {
                const double* vi = V + (size_t)i * n;  /* basis vector i = block i/kb, column i%kb */
                const double y = Ys[(size_t)a * cols + i];
                for (int32_t q = 0; q < n; ++q) w[q] += y * vi[q];
            }
            orc_csc_matvec(M, w, z);
            double* yc = Y + (size_t)c * n;
            for (int32_t q = 0; q < n; ++q) yc[q] += z[q];
            orc_csc_matvec(At, yc, w);
            for (int32_t q = 0; q < n; ++q) R[(size_t)c * n + q] = B[(size_t)c * n + q] - w[q];
        }
    }
#undef HB
#undef GG
    free(V);
    free(Hb);
    free(hv);
    free(hbeta);
    free(G);
    free(Ys);
    free(W);
    free(R);
    free(S);
    free(z);
    free(w);
    free(act);
    free(done);
    return status;
}
