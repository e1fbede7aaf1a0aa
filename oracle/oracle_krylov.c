/* oracle_krylov.c -- right-preconditioned Krylov solvers used for the s+1
 * systems A~ y = b, A~ w_j = u_j, eqs. (regprob) and (auxi); section 5 runs
 * BiCGStab with x0 = 0 and at most 500 iterations, and mentions GMRES.
 * Textbook recurrences (van der Vorst's BiCGStab; restarted GMRES with
 * modified Gram-Schmidt and Givens rotations), one system at a time, FP64.
 * Test infrastructure only. */
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* BiCGStab on A~ M z = rhs, returning y = M z directly. The residual is
 * tested after the half step (s) and after the full step (r); an exit at
 * the half step still counts a full iteration. */
int orc_bicgstab(const orc_csc* At, const orc_csc* M, const double* rhs, double thr,
                 int32_t maxit, double* y, int32_t* iters)
{
    int32_t n = At->ncols;
    double* r = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* rh = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* p = (double*)orc_xcalloc((size_t)n, sizeof(double));
    double* v = (double*)orc_xcalloc((size_t)n, sizeof(double));
    double* ph = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* s = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* sh = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* t = (double*)orc_xmalloc((size_t)n * sizeof(double));
    for (int32_t i = 0; i < n; ++i) {
        y[i] = 0.0;
        r[i] = rhs[i];
        rh[i] = rhs[i];
    }
    int status = ORC_MAXITER;
    int32_t it = 0;
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    if (orc_norm2(n, r) < thr) {
        status = ORC_OK;
    } else {
        for (it = 1; it <= maxit; ++it) {
            double rho = orc_dot(n, rh, r);
            if (rho == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            if (it == 1) {
                memcpy(p, r, (size_t)n * sizeof(double));
            } else {
                double beta = (rho / rho_prev) * (alpha / omega);
                for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            }
            orc_csc_matvec(M, p, ph);
            orc_csc_matvec(At, ph, v);
            double rv = orc_dot(n, rh, v);
            if (rv == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            alpha = rho / rv;
            for (int32_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
            if (orc_norm2(n, s) < thr) {
                for (int32_t i = 0; i < n; ++i) y[i] += alpha * ph[i];
                memcpy(r, s, (size_t)n * sizeof(double));
                status = ORC_OK;
                break;
            }
            orc_csc_matvec(M, s, sh);
            orc_csc_matvec(At, sh, t);
            double tt = orc_dot(n, t, t);
            if (tt == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            omega = orc_dot(n, t, s) / tt;
            for (int32_t i = 0; i < n; ++i) {
                y[i] += alpha * ph[i] + omega * sh[i];
                r[i] = s[i] - omega * t[i];
            }
            if (orc_norm2(n, r) < thr) {
                status = ORC_OK;
                break;
            }
            if (omega == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            rho_prev = rho;
        }
        if (it > maxit) it = maxit;
    }
    *iters = it;
    free(r);
    free(rh);
    free(p);
    free(v);
    free(ph);
    free(s);
    free(sh);
    free(t);
    return status;
}



/* BiCG on A~ M z = rhs, returning y = M z: the shadow sequence runs with
 * (A~ M)^T = M^T A~^T, shadow residual = rhs; the residual is tested after
 * each iteration (section 5 names BiCG among the other solvers tried). */
int orc_bicg(const orc_csc* At, const orc_csc* M, const double* rhs, double thr, int32_t maxit, double* y,
             int32_t* iters)
{
    int32_t n = At->ncols;
    orc_csc AtT, MT;
    if (orc_csc_transpose(At, &AtT) != ORC_OK) return ORC_NOMEM;
    if (orc_csc_transpose(M, &MT) != ORC_OK) {
        orc_csc_free(&AtT);
        return ORC_NOMEM;
    }
    double* r = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* rs = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* p = (double*)orc_xcalloc((size_t)n, sizeof(double));
    double* ps = (double*)orc_xcalloc((size_t)n, sizeof(double));
    double* z = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* q = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* zs = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* qs = (double*)orc_xmalloc((size_t)n * sizeof(double));
    for (int32_t i = 0; i < n; ++i) {
        y[i] = 0.0;
        r[i] = rhs[i];
        rs[i] = rhs[i];
    }
    int status = ORC_MAXITER;
    int32_t it = 0;
    double rho_prev = 1.0;
    if (orc_norm2(n, r) < thr) {
        status = ORC_OK;
    } else {
        for (it = 1; it <= maxit; ++it) {
            double rho = orc_dot(n, rs, r);
            if (rho == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            if (it == 1) {
                memcpy(p, r, (size_t)n * sizeof(double));
                memcpy(ps, rs, (size_t)n * sizeof(double));
            } else {
                double beta = rho / rho_prev;
                for (int32_t i = 0; i < n; ++i) {
                    p[i] = r[i] + beta * p[i];
                    ps[i] = rs[i] + beta * ps[i];
                }
            }
            orc_csc_matvec(M, p, z);      /* z = M p        */
            orc_csc_matvec(At, z, q);     /* q = A~ M p     */
            orc_csc_matvec(&AtT, ps, zs); /* A~^T ps        */
            orc_csc_matvec(&MT, zs, qs);  /* M^T A~^T ps    */
            double sigma = orc_dot(n, ps, q);
            if (sigma == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            double alpha = rho / sigma;
            for (int32_t i = 0; i < n; ++i) {
                y[i] += alpha * z[i];
                r[i] -= alpha * q[i];
                rs[i] -= alpha * qs[i];
            }
            if (orc_norm2(n, r) < thr) {
                status = ORC_OK;
                break;
            }
            rho_prev = rho;
        }
        if (it > maxit) it = maxit;
    }
    *iters = it;
    free(r);
    free(rs);
    free(p);
    free(ps);
    free(z);
    free(q);
    free(zs);
    free(qs);
    orc_csc_free(&AtT);
    orc_csc_free(&MT);
    return status;
}

/* CGS (Sonneveld's conjugate gradient squared) on A~ M z = rhs, returning
 * y = M z directly: two applications of A~ M per iteration, the recursive
 * residual tested after each iteration (section 5 names CGS among the other
 * solvers tried). */
int orc_cgs(const orc_csc* At, const orc_csc* M, const double* rhs, double thr, int32_t maxit, double* y,
            int32_t* iters)
{
    int32_t n = At->ncols;
    double* r = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* rh = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* u = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* p = (double*)orc_xcalloc((size_t)n, sizeof(double));
    double* q = (double*)orc_xcalloc((size_t)n, sizeof(double));
    double* ph = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* v = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* w = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* wh = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* qh = (double*)orc_xmalloc((size_t)n * sizeof(double));
    for (int32_t i = 0; i < n; ++i) {
        y[i] = 0.0;
        r[i] = rhs[i];
        rh[i] = rhs[i];
    }
    int status = ORC_MAXITER;
    int32_t it = 0;
    double rho_prev = 1.0;
    if (orc_norm2(n, r) < thr) {
        status = ORC_OK;
    } else {
        for (it = 1; it <= maxit; ++it) {
            double rho = orc_dot(n, rh, r);
            if (rho == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            if (it == 1) {
                memcpy(u, r, (size_t)n * sizeof(double));
                memcpy(p, u, (size_t)n * sizeof(double));
            } else {
                double beta = rho / rho_prev;
                for (int32_t i = 0; i < n; ++i) {
                    u[i] = r[i] + beta * q[i];
                    p[i] = u[i] + beta * (q[i] + beta * p[i]);
                }
            }
            orc_csc_matvec(M, p, ph);
            orc_csc_matvec(At, ph, v);
            double sigma = orc_dot(n, rh, v);
            if (sigma == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            double alpha = rho / sigma;
            for (int32_t i = 0; i < n; ++i) {
                q[i] = u[i] - alpha * v[i];
                w[i] = u[i] + q[i];
            }
            orc_csc_matvec(M, w, wh);
            orc_csc_matvec(At, wh, qh);
            for (int32_t i = 0; i < n; ++i) {
                y[i] += alpha * wh[i];
                r[i] -= alpha * qh[i];
            }
            if (orc_norm2(n, r) < thr) {
                status = ORC_OK;
                break;
            }
            rho_prev = rho;
        }
        if (it > maxit) it = maxit;
    }
    *iters = it;
    free(r);
    free(rh);
    free(u);
    free(p);
    free(q);
    free(ph);
    free(v);
    free(w);
    free(wh);
    free(qh);
    return status;
}

/* Restarted GMRES(m) on A~ M z = rhs, y = M z. Arnoldi by modified
 * Gram-Schmidt, least squares by Givens rotations; the cycle stops when the
 * rotated residual estimate |g_{j+1}| < thr; each restart recomputes the
 * true residual rhs - A~ y. */
int orc_gmres(const orc_csc* At, const orc_csc* M, const double* rhs, double thr,
              int32_t m, int32_t maxit, double* y, int32_t* iters)
{
    int32_t n = At->ncols;
    if (m < 1) return ORC_BAD_INPUT;
    double* V = (double*)orc_xmalloc((size_t)(m + 1) * (size_t)n * sizeof(double));
    double* H = (double*)orc_xcalloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double* cs = (double*)orc_xmalloc((size_t)m * sizeof(double));
    double* sn = (double*)orc_xmalloc((size_t)m * sizeof(double));
    double* g = (double*)orc_xmalloc((size_t)(m + 1) * sizeof(double));
    double* u = (double*)orc_xmalloc((size_t)m * sizeof(double));
    double* z = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* w = (double*)orc_xmalloc((size_t)n * sizeof(double));
    double* r = (double*)orc_xmalloc((size_t)n * sizeof(double));
#define H_(i, j) H[(size_t)(j) * (m + 1) + (i)]
    for (int32_t i = 0; i < n; ++i) {
        y[i] = 0.0;
        r[i] = rhs[i];
    }
    int32_t it = 0;
    int status = ORC_MAXITER;
    for (;;) {
        double beta = orc_norm2(n, r);
        if (beta < thr) {
            status = ORC_OK;
            break;
        }
        if (it >= maxit) break;
        for (int32_t i = 0; i < n; ++i) V[i] = r[i] / beta;
        for (int32_t i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int32_t jdone = 0;
        int conv = 0;
        for (int32_t j = 0; j < m && it < maxit; ++j) {
            double* vj = V + (size_t)j * n;
            orc_csc_matvec(M, vj, z);
            orc_csc_matvec(At, z, w);
            for (int32_t i = 0; i <= j; ++i) {
                double* vi = V + (size_t)i * n;
                double h = orc_dot(n, vi, w);
                H_(i, j) = h;
                for (int32_t q = 0; q < n; ++q) w[q] -= h * vi[q];
            }
            double hn = orc_norm2(n, w);
            H_(j + 1, j) = hn;
            if (hn != 0.0) {
                double* vn = V + (size_t)(j + 1) * n;
                for (int32_t q = 0; q < n; ++q) vn[q] = w[q] / hn;
            }
            for (int32_t i = 0; i < j; ++i) {
                double a = H_(i, j), b = H_(i + 1, j);
                H_(i, j) = cs[i] * a + sn[i] * b;
                H_(i + 1, j) = -sn[i] * a + cs[i] * b;
            }
            double a = H_(j, j), b = H_(j + 1, j);
            double den = sqrt(a * a + b * b);
            if (den == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                cs[j] = a / den;
                sn[j] = b / den;
            }
            H_(j, j) = cs[j] * a + sn[j] * b;
            H_(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            jdone = j + 1;
            if (fabs(g[j + 1]) < thr) {
                conv = 1;
                break;
            }
        }
        /* u = H(0:jdone,0:jdone)^{-1} g(0:jdone); y += M (V u) */
        for (int32_t i = jdone - 1; i >= 0; --i) {
            double t = g[i];
            for (int32_t q = i + 1; q < jdone; ++q) t -= H_(i, q) * u[q];
            if (H_(i, i) == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            u[i] = t / H_(i, i);
        }
        if (status == ORC_BREAKDOWN) break;
        for (int32_t q = 0; q < n; ++q) w[q] = 0.0;
        for (int32_t i = 0; i < jdone; ++i) {
            double* vi = V + (size_t)i * n;
            for (int32_t q = 0; q < n; ++q) w[q] += u[i] * vi[q];
        }
        orc_csc_matvec(M, w, z);
        for (int32_t q = 0; q < n; ++q) y[q] += z[q];
        if (conv) {
            status = ORC_OK;
            break;
        }
        if (it >= maxit) break;
        orc_csc_matvec(At, y, w);
        for (int32_t q = 0; q < n; ++q) r[q] = rhs[q] - w[q];
    }
#undef H_
    *iters = it;
    free(V);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(u);
    free(z);
    free(w);
    free(r);
    return status;
}
