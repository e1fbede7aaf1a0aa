/*
 * oracle.h -- plain, sequential FP64 CPU oracle for the split + SAI +
 * Krylov + Sherman-Morrison-Woodbury method of Jia & Zhang,
 * "An approach to making SPAI and PSAI preconditioning effective for large
 * irregular sparse linear systems" (arXiv 1211.6866).
 *
 * THIS IS TEST INFRASTRUCTURE. It exists only so that tests, the smoke check
 * and the CPU-baseline leg of the benchmark can check and time the CUDA path.
 * The product path never calls it. It shares no code, header, table or
 * constant with the CUDA library, and neither side includes the other.
 *
 * Every routine is written for clarity, not speed: dense O(n) marker arrays,
 * qsort, textbook Householder QR and textbook Krylov recurrences, all FP64.
 *
 * Sparse matrices are CSC: col_ptr[n+1] (int64), row_idx[nnz] (int32, sorted
 * ascending inside each column, no duplicates), val[nnz] (double).
 * Arrays returned through orc_csc outputs are malloc'd by the oracle and
 * released with orc_csc_free(). All other outputs are caller-allocated.
 */
#ifndef SAI_ORACLE_H
#define SAI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nrows;
    int32_t ncols;
    int64_t* col_ptr;
    int32_t* row_idx;
    double* val;
} orc_csc;

enum {
    ORC_OK = 0,
    ORC_BAD_INPUT = 1,
    ORC_SINGULAR = 2,      /* an LS matrix or the s x s SMW matrix is singular */
    ORC_MAXITER = 3,       /* Krylov iteration limit reached */
    ORC_BREAKDOWN = 4,     /* BiCGStab rho = 0 or omega = 0 */
    ORC_NOMEM = 5
};

void orc_csc_free(orc_csc* A);

/* ---- section 4: dense-column detection and split (eq. (split)) ---------- */

/* p = floor(nnz(A)/n), the average number of nonzeros per column (section 4). */
int32_t orc_avg_nnz(int32_t n, int64_t nnz);

/* Irregular columns: nnz(a_j) > tau (or >= tau when ge != 0), tau = mult*p,
 * or tau = abs_tau when abs_tau >= 0. J_out (capacity n) gets the ascending
 * list, *s_out its length, *p_out and *tau_out the values used. */
int orc_detect(const orc_csc* A, double mult, double abs_tau, int ge,
               int32_t* J_out, int32_t* s_out, int32_t* p_out, double* tau_out);

/* Sparsify the s columns J of A: keep the diagonal and the p_keep-1 stored
 * entries nearest to it (|i-j| ascending, ties to the smaller row), or the
 * p_keep nearest entries when the diagonal is not stored. Outputs A~ (n x n)
 * and U (n x s, column t holds the dropped entries of column J[t]). */
int orc_split(const orc_csc* A, const int32_t* J, int32_t s, int32_t p_keep,
              orc_csc* At_out, orc_csc* U_out);
/* the same with a keep rule: 0 = the diagonal and the p_keep-1 nearest entries
 * (as orc_split), 1 = the diagonal and the p_keep-1 entries of largest
 * magnitude (ties to the smaller row; p_keep largest without a diagonal) */
int orc_split_rule(const orc_csc* A, const int32_t* J, int32_t s, int32_t p_keep, int32_t rule,
                   orc_csc* At_out, orc_csc* U_out);

/* ---- section 2.1: SPAI (Grote-Huckle adaptive augmentation) -------------- */

typedef struct {
    double delta;      /* stop when ||A~ m_k - e_k|| <= delta            */
    int32_t mn;        /* most profitable indices added per loop        */
    int32_t max_aug;   /* maximum number of augmentation steps          */
    int32_t key_bits;  /* rho^2/||r||^2 quantised to 2^-key_bits        */
} orc_spai_params;

/* Builds columns [c0, c1) of M ~ A~^{-1} (other columns left empty).
 * loops_out[k] = augmentation steps used, res_out[k] = final ||r_k||.
 * Both arrays have length n (entries outside [c0,c1) untouched). */
int orc_spai(const orc_csc* At, const orc_spai_params* prm, int32_t c0, int32_t c1,
             orc_csc* M_out, int32_t* loops_out, double* res_out);

/* One column with its full trace: after loop l the pattern is
 * S_hist[S_off[l] .. S_off[l+1]) and the LS residual res_hist[l].
 * Capacities: S_hist >= cap_s, S_off >= max_aug+2, res_hist >= max_aug+1.
 * Returns the number of loops recorded (>= 1) or a negative error. */
int orc_spai_trace(const orc_csc* At, const orc_spai_params* prm, int32_t k,
                   int32_t* S_hist, int32_t cap_s, int32_t* S_off, double* res_hist);

/* ---- section 2.2: PSAI(tol) (power pattern growth + dropping) ------------ */

typedef struct {
    double delta;      /* stop tolerance on the pre-drop residual            */
    double tol;        /* fixed dropping tolerance (tol_mode = 1)            */
    int32_t tol_mode;  /* 0: tol_k = delta/(nnz(m_k) ||A~||_1), eq. (tolk);  */
                       /* 1: tol_k = tol                                    */
    int32_t lmax;      /* loops l = 0..lmax                                 */
    int32_t lfill;     /* tol_mode 2, PSAI(lfill): keep the lfill entries of */
                       /* largest magnitude (ties to the smaller index)      */
    int32_t growth;    /* 0: S' = P(a^(l+1)) u S_kept (reading A);          */
                       /* 1: S' = S_kept u (P(a^(l+1)) \ P(a^(l))) (reading C) */
} orc_psai_params;

/* Builds columns [c0,c1) of M. loops_out[k] = last loop index l used,
 * res_pre[k] = LS residual before dropping, res_post[k] = ||A~ m_k - e_k||
 * of the emitted (dropped) column. */
int orc_psai(const orc_csc* At, const orc_psai_params* prm, int32_t c0, int32_t c1,
             orc_csc* M_out, int32_t* loops_out, double* res_pre, double* res_post);

/* One column with its trace: patterns before each LS solve (as for SPAI)
 * and the pre-drop residual of every loop. */
int orc_psai_trace(const orc_csc* At, const orc_psai_params* prm, int32_t k,
                   int32_t* S_hist, int32_t cap_s, int32_t* S_off, double* res_hist);

/* ---- right-preconditioned Krylov solvers (section 5) ---------------------- */

/* Solves A~ y = rhs with right preconditioner M: A~ M z = rhs, y = M z.
 * x0 = 0; stops when the recursively updated residual norm < thr.
 * *iters = loop passes started. Returns ORC_OK, ORC_MAXITER or ORC_BREAKDOWN. */
int orc_bicgstab(const orc_csc* At, const orc_csc* M, const double* rhs, double thr,
                 int32_t maxit, double* y, int32_t* iters);

/* Restarted GMRES(m), modified Gram-Schmidt Arnoldi, Givens rotations,
 * stop on the Givens residual estimate < thr; *iters counts inner steps. */
/* BiCG on A~ M z = rhs returning y = M z, shadow sequence with M^T A~^T;
 * the residual is tested after each iteration. */
int orc_bicg(const orc_csc* At, const orc_csc* M, const double* rhs, double thr, int32_t maxit, double* y,
             int32_t* iters);

/* CGS on A~ M z = rhs returning y = M z; the recursive residual is tested
 * after each iteration (two applications of A~ M). */
int orc_cgs(const orc_csc* At, const orc_csc* M, const double* rhs, double thr, int32_t maxit, double* y,
            int32_t* iters);

int orc_gmres(const orc_csc* At, const orc_csc* M, const double* rhs, double thr,
              int32_t restart, int32_t maxit, double* y, int32_t* iters);

/* ---- section 3 / Theorem 2: SMW recovery and true residual --------------- */

/* xhat = yhat - W (I + V^T W)^{-1} V^T yhat (eq. (composi)), W n x s column
 * major, V = [e_J0 ... e_J(s-1)]. z_out (s) = (I+V^T W)^{-1} V^T yhat,
 * *c_out = ||z||_2. */
int orc_smw(int32_t n, int32_t s, const double* yhat, const double* W, const int32_t* J,
            double* x_out, double* z_out, double* c_out);

/* rr = ||b - A x|| / ||b|| (eq. (rrnorm)). */
double orc_rel_resid(const orc_csc* A, const double* b, const double* x);

/* ---- Procedure * ----------------------------------------------------------- */

typedef struct {
    double thresh_mult;   /* 10 */
    double abs_tau;       /* < 0: use thresh_mult * p */
    int32_t sai;          /* 0: SPAI, 1: PSAI(tol) */
    orc_spai_params spai;
    orc_psai_params psai;
    int32_t krylov;       /* 0: BiCGStab, 1: GMRES(restart), 2: CGS, 3: BiCG,
                             4: block GMRES(restart) over all s+1 systems */
    int32_t restart;
    int32_t maxit;
    double eps;
    int32_t c_adapt;      /* 1: when SMW's c = ||z|| exceeds 1, continue the u_j systems to
                             eq. (stopU2) with that c (times 1.05) and recover x again */
    int32_t reserved;
} orc_solve_params;

typedef struct {
    int32_t s, p;
    double tau;
    int64_t nnz_At, nnz_M;
    int32_t n_c;          /* columns whose final (pre-drop) residual > delta */
    int32_t l_m;          /* largest loop count used by the SAI builder */
    int32_t iter_max;     /* max Krylov iterations over the s+1 systems */
    int32_t status;       /* first non-OK Krylov status, else OK */
    double c;             /* ||(I+V^T W)^{-1} V^T y|| */
    double rr;            /* ||b - A xhat|| / ||b|| */
    double bound;         /* ||r_y|| + c ||R_W||_F  (Theorem 2, eq. (rry)) */
    double c_first;       /* c of the first recovery (c when no second round ran) */
    int32_t c_rounds;     /* 1 when the u_j systems were continued with the measured c */
    int32_t reserved;
} orc_solve_report;

/* Full Procedure *: split, build M, s+1 Krylov solves, SMW, rr.
 * iters_out (s+1, may be NULL) gets the per-system iteration counts
 * in the order [b, u_1, ..., u_s]. */
int orc_solve(const orc_csc* A, const double* b, const orc_solve_params* prm,
              double* x_out, int32_t* iters_out, orc_solve_report* rep);

/* ---- backward pass (not in the paper: the adjoint of Procedure *) ------- */

/* B = A^T in CSC (arrays malloc'd, free with orc_csc_free). */
int orc_csc_transpose(const orc_csc* A, orc_csc* B);

/* Theorem 1 on A^T = A~^T + V U^T:
 * lambda = yhat - W (I + U^T W)^{-1} (U^T yhat); W n x s column-major, U n x s CSC. */
int orc_smw_adjoint(int32_t n, int32_t s, const double* yhat, const double* W, const orc_csc* U,
                    double* lambda_out, double* z_out, double* c_out);

/* Backward pass of x = A^{-1} b for g = dL/dx: split and M as in orc_solve,
 * [yhat, W] = A~^{-T}[g, e_J] by the s+1 solves with right preconditioner
 * M^T and the Theorem 2 thresholds from ||g||, lambda by orc_smw_adjoint,
 * grad_vals[q] = -lambda_i x_j for A's stored entry q = (i, j) (may be NULL).
 * rep->rr = ||g - A^T lambda|| / ||g||, rep->c = ||z||. */
int orc_backward(const orc_csc* A, const double* x, const double* g, const orc_solve_params* prm,
                 double* lambda_out, double* grad_vals, int32_t* iters_out, orc_solve_report* rep);

/* ---- block Krylov alternative for the s+1 systems (section 3) ---------- */

/* Block GMRES(m) with right preconditioning on A~ M Z = B, Y = M Z, for the
 * k right-hand sides of B (n x k column-major); Y (n x k column-major) out.
 * At each cycle start a column whose true residual ||B e_c - A~ Y e_c|| is
 * below thr[c] is frozen and the others form the cycle's block; the
 * cycle's block steps stop when every column's least-squares residual is
 * below its threshold (or after m steps). iters[c] (k entries) = the block
 * steps column c took part in. Returns ORC_OK, ORC_MAXITER (maxit block
 * steps) or ORC_BREAKDOWN (a zero pivot of the reduced block Hessenberg
 * matrix). */
int orc_block_gmres(const orc_csc* At, const orc_csc* M, int32_t k, const double* B, const double* thr, int32_t m,
                    int32_t maxit, double* Y, int32_t* iters);

/* ---- section 5 preprocessing: zero-diagonal repair (row DM permutation) -- */

/* A maximum transversal of A (MATLAB dmperm with one output): p_out[j] = the
 * row matched to column j, or -1; *rank_out = the number of matched columns
 * (the structural rank). Entries count when stored with a nonzero value. A
 * zero-free diagonal gives p = identity; otherwise the nonzero diagonal
 * entries start the matching and shortest augmenting paths (breadth-first
 * search) from the unmatched columns (ascending) complete it. */
int orc_dmperm(const orc_csc* A, int32_t* p_out, int32_t* rank_out);

/* B = A(p,:) (row j of B is row p[j] of A); p must be a permutation of
 * 0..n-1 (ORC_BAD_INPUT otherwise). Arrays malloc'd, free with orc_csc_free. */
int orc_permute_rows(const orc_csc* A, const int32_t* p, orc_csc* B_out);

#ifdef __cplusplus
}
#endif
#endif
