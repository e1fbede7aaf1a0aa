/*
 * saismw.h -- C ABI of the GB300 (sm_103a) implementation of Jia & Zhang's
 * approach for irregular sparse systems A x = b (arXiv 1211.6866):
 *
 *   1. split A = A~ + U V^T              (section 3, eq. (split); section 4)
 *   2. build M ~ A~^{-1} by SPAI or PSAI  (section 2.1, section 2.2)
 *   3. solve the s+1 systems A~ y = b, A~ w_j = u_j with right
 *      preconditioner M                   (eqs. (regprob), (auxi); section 5)
 *   4. recover x = y - W (I + V^T W)^{-1} V^T y        (eq. (composi))
 *      with the stopping rules of Theorem 2, eqs. (stopb), (stopU2), c = 1.
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers unless the comment says "host".
 *    The caller owns them; the library never frees or keeps them beyond the
 *    call (except where a handle documents a copy).
 *  - Sparse inputs are CSC: col_ptr[n+1] int64 (col_ptr[0] = 0), row_idx[nnz]
 *    int32 strictly ascending inside each column, val[nnz] double.
 *  - Dense multi-right-hand-side blocks are n x k ROW-MAJOR (the k values of a
 *    row are contiguous, element (i,c) at [i*k + c]).
 *  - Handles own their device buffers and release them in *_destroy.
 *  - All work is enqueued on `stream`. Calls that return sizes or reports to
 *    the host synchronise the stream before returning.
 *  - Errors: the first error is returned; no C++ exception crosses the ABI;
 *    outputs are unspecified unless SAI_OK is returned, except that
 *    SAI_MAXITER still returns the last iterates and a filled report.
 *  - One CUDA device: the device current at the call.
 */
#ifndef SAISMW_H
#define SAISMW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sai_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    SAI_OK = 0,
    SAI_INVALID_ARG = 1,       /* bad size, NULL pointer, unsorted rows, ... */
    SAI_CUDA_ERROR = 2,        /* a CUDA runtime call failed, or a bounded wait inside a
                                  kernel (the GMRES update's copy ring) gave up */
    SAI_OOM = 3,               /* device allocation failed */
    SAI_PATTERN_OVERFLOW = 4,  /* an SAI column outgrew the largest workspace tier */
    SAI_MAXITER = 5,           /* a Krylov system hit maxit (iterates still returned) */
    SAI_BREAKDOWN = 6,         /* BiCGStab rho = 0 / omega = 0, GMRES zero pivot */
    SAI_SINGULAR = 7,          /* singular LS matrix A^_k or singular I + V^T W */
    SAI_NOT_IMPLEMENTED = 8
} sai_status;

/* Returns a static, NUL-terminated name for a status code. */
const char* sai_status_string(sai_status st);

/* View of a caller-owned square CSC matrix on the device. */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int64_t* col_ptr;
    const int32_t* row_idx;
    const double* val;
} sai_csc_view;

/* ----------------------------------------------------------------------
 * Step 1: split (section 4, first dropping approach; eq. (split)).
 * p = floor(nnz(A)/n). Column j is irregular when nnz(a_j) > tau with
 * tau = thresh_mult * p (paper: 10, "8p to 15p work as well"), or
 * tau = abs_tau when abs_tau >= 0; ge != 0 uses >= instead of > (the
 * "10p or more" wording of section 1). Each irregular column keeps its
 * diagonal and the p_keep-1 stored entries nearest to it (|i-j| ascending,
 * ties to the smaller row; p_keep nearest when no diagonal is stored);
 * p_keep <= 0 means p_keep = p (the paper's choice p^ = p). Dropped entries
 * form U (n x s), V = [e_J0 ... e_J(s-1)] with J ascending.
 * abs_tau = +infinity keeps every column: A~ = A and s = 0, so the builders
 * and sai_solve work on A itself (the S-SPAI / S-PSAI baselines of
 * section 5).
 * ---------------------------------------------------------------------- */
typedef struct {
    double thresh_mult;
    double abs_tau;
    int32_t ge;
    int32_t p_keep;
    int32_t keep_rule; /* 0: the diagonal and the p_keep-1 entries nearest to it
                          (the paper's choice); 1: the diagonal and the p_keep-1
                          entries of largest magnitude (the other rule of section 4;
                          ties to the smaller row; p_keep largest without a
                          diagonal). Other values: SAI_INVALID_ARG. */
    int32_t zero_diag; /* sai_solve only: 1 applies the zero-diagonal repair of
                          section 5 first (see sai_dmperm): when A has a zero on
                          its diagonal, the method runs on A(p,:) x = b(p) with p
                          a maximum transversal (SAI_SINGULAR when A is
                          structurally singular). 0: off. sai_split_create and
                          sai_solve_batched take 0 only (SAI_INVALID_ARG). */
} sai_split_params;

typedef struct sai_split_s* sai_split;

typedef struct {
    int32_t n, s, p, p_keep;
    double tau;
    int64_t nnz_At, nnz_U;
    double norm1_At;  /* ||A~||_1 = max_j sum_i |a~_ij| (used by eq. (tolk)) */
} sai_split_info;

/* Builds A~ (CSC and CSR), U (CSC) and J on the device from A.
 * The handle keeps its own copies; A may be freed after the call returns.
 * Rows must be strictly ascending per column (SAI_INVALID_ARG otherwise). */
sai_status sai_split_create(const sai_csc_view* A, const sai_split_params* prm,
                            sai_stream_t stream, sai_split* out);
sai_status sai_split_get_info(sai_split h, sai_split_info* info);
/* Copies the split to caller buffers sized from sai_split_get_info
 * (At: n+1, nnz_At, nnz_At; U: s+1, nnz_U, nnz_U; J: s). NULL pointers are
 * skipped. */
sai_status sai_split_copy_out(sai_split h, int64_t* At_col_ptr, int32_t* At_row_idx, double* At_val,
                              int64_t* U_col_ptr, int32_t* U_row_idx, double* U_val, int32_t* J,
                              sai_stream_t stream);
void sai_split_destroy(sai_split h);

/* ----------------------------------------------------------------------
 * Zero-diagonal repair (section 5, before the method): the paper permutes
 * the rows of the matrices that have zeros on the diagonal with MATLAB's
 * dmperm so that the diagonal, which the split keeps and SPAI's initial
 * pattern P(I) starts from, becomes nonzero.
 * ---------------------------------------------------------------------- */

/* A maximum transversal of the square A: p[j] (device, n entries, caller
 * owned) = the row matched to column j, or -1 when column j stays unmatched;
 * A(p,:) has a zero-free diagonal when *rank_out == n. An entry counts when
 * it is stored with a nonzero value. A zero-free diagonal gives the
 * identity; otherwise the nonzero diagonal entries start the matching and
 * phases of shortest augmenting paths complete it (ties to the smaller
 * column and row, so p is reproducible). rank_out (host): the number of
 * matched columns, the structural rank of A. moved_out (host, may be NULL):
 * the number of columns j with p[j] != j. Rows must be strictly ascending
 * per column (SAI_INVALID_ARG otherwise). Synchronises the stream. */
sai_status sai_dmperm(const sai_csc_view* A, int32_t* p, int32_t* rank_out, int32_t* moved_out,
                      sai_stream_t stream);

/* B = A(p,:): row j of B is row p[j] of A (entry (i, c) of A becomes entry
 * (pinv[i], c) of B, pinv[p[j]] = j). p: device, a permutation of 0..n-1
 * (SAI_INVALID_ARG otherwise). B: caller-owned device CSC arrays of
 * n+1, nnz and nnz entries, rows ascending per column; the values are A's,
 * bit for bit. Synchronises the stream. */
sai_status sai_permute_rows(const sai_csc_view* A, const int32_t* p, int64_t* B_col_ptr, int32_t* B_row_idx,
                            double* B_val, sai_stream_t stream);

/* ----------------------------------------------------------------------
 * Step 2: sparse approximate inverse M ~ A~^{-1}, min ||A~ M - I||_F,
 * decoupled into n independent problems min ||A~ m_k - e_k|| (eq. (subprob))
 * solved through the reduced problems (lsprob) by Householder QR, updated
 * incrementally as the pattern grows. Initial pattern S_k^(0) = {k}.
 * The reduced row set L_k always contains k.
 * ---------------------------------------------------------------------- */
typedef enum { SAI_FP64 = 0, SAI_FP32_REFINE64 = 1 } sai_precision;

/* SPAI (section 2.1, eqs. (candi), (ls1d), (muj), (rhoj)). Loop: solve,
 * stop when ||r_k|| <= delta or max_aug augmentation steps were made,
 * otherwise add the mn candidates j in N \ S (N = columns touching the rows
 * of L_k) with the smallest keys (floor(rho_j^2/||r_k||^2 * 2^key_bits), j).
 * key_bits in [1, 31]; 20 is the default reading. */
typedef struct {
    double delta;      /* paper: 0.4 (section 5.1) */
    int32_t mn;        /* paper: 5, at most 8 here */
    int32_t max_aug;   /* paper: l_max = 20 loops, i.e. 19 augmentations */
    int32_t key_bits;
    int32_t precision; /* SAI_FP64, or SAI_FP32_REFINE64: Householder QR of the
                          reduced problems in FP32, then per loop one FP64
                          refinement step by the corrected semi-normal
                          equations; residuals, stop tests and SPAI keys use
                          the refined solution in FP64 */
} sai_spai_params;

/* PSAI(tol) (section 2.2). Loop l = 0..lmax: solve on S^(l), drop
 * |m_jk| <= tol_k with tol_k = delta/(nnz(m_k) ||A~||_1) (tol_mode 0,
 * eq. (tolk)) or tol_k = tol (tol_mode 1), or keep only the lfill largest
 * (tol_mode 2, PSAI(lfill)); stop when the pre-drop residual <= delta or
 * l = lmax and emit the kept entries of that solution; else
 * S^(l+1) = P(|A~| a^(l)) u S_kept^(l) with a^(0) = e_k. */
typedef struct {
    double delta;      /* paper: 0.4 */
    double tol;
    int32_t tol_mode;
    int32_t lmax;      /* paper: 10 */
    int32_t precision; /* as for SPAI; the drop test uses the refined solution */
    int32_t lfill;     /* tol_mode 2 only: PSAI(lfill) keeps the lfill entries of
                          largest magnitude of each newly computed m_k (equal
                          magnitudes to the smaller column index), >= 1 */
    int32_t growth;    /* 0: S^(l+1) = P(a^(l+1)) u S_kept^(l) (reading A, the
                          default); 1: S^(l+1) = S_kept^(l) u (P(a^(l+1)) \ P(a^(l))),
                          dropped positions never return (reading C); a column
                          whose next pattern would be empty stops and emits its
                          (empty) kept set. Other values: SAI_INVALID_ARG. */
    int32_t reserved;  /* 0 */
} sai_psai_params;

typedef struct sai_precond_s* sai_precond;

/* Schedule of the SAI build (not part of the method). warps_t0: warps per
 * block of the shared-memory tiers (4 or 8); blocks_per_sm_t12: blocks per
 * SM of the global-memory tiers (1, 2 or 4); heavy_first: 1 puts the columns
 * of A~ with more than twice the average entry count at the head of the work
 * queue; first_tier: the workspace every column starts in -- 0: tier 0 (|L|
 * <= 64 rows, |S| <= 16 columns, one column per warp), 1: the small tier
 * (|L| <= 32, |S| <= 8) with four columns per warp (8-lane groups), 2: the
 * small tier with two columns per warp (16-lane groups), 3: the small tier
 * with one column per lane (32 per warp, each lane running its column's
 * steps alone); a column that outgrows its tier restarts in the next one. ms: the sampled build time
 * measured by sai_build_autotune (0 otherwise). Default {8, 2, 0, 0}.
 * warps_t0, blocks_per_sm_t12 and heavy_first never change M. first_tier
 * sets how many lanes sum each reduction of the columns the small tier
 * finishes, so M's values can differ in the last bits between first_tier 0
 * and 1, 2 or 3 (the same first_tier always gives the same bits). */
typedef struct {
    int32_t warps_t0;
    int32_t blocks_per_sm_t12;
    int32_t heavy_first;
    int32_t first_tier;
    float ms;
} sai_build_config;

typedef struct {
    sai_build_config chosen;
    int32_t sample_columns;      /* columns of the strided sample timed */
    int32_t ncand;
    sai_build_config cand[12];   /* every candidate with its time */
} sai_build_tuning;

typedef struct {
    int32_t n;
    int64_t nnz_M;
    int32_t n_c;        /* columns whose final (pre-drop) residual > delta */
    int32_t l_m;        /* largest loop index used over all columns */
    int32_t n_tier[6];  /* columns finished per workspace tier: 0 shared memory (|L| <= 64,
                           |S| <= 16), 1-3 global memory (|L| <= 256 / 1024 / 2048, |S| <= 64 /
                           128 / 128), 4 the small shared-memory tier (first_tier 1 or 2),
                           5 the large-pattern tier (|L| <= 4096, |S| <= 2048, one warp per
                           column and per SM) */
    double build_ms;    /* device time of the build, CUDA events */
} sai_precond_info;

sai_status sai_build_spai(sai_split h, const sai_spai_params* prm, sai_stream_t stream, sai_precond* out);
sai_status sai_build_psai(sai_split h, const sai_psai_params* prm, sai_stream_t stream, sai_precond* out);
sai_status sai_precond_get_info(sai_precond P, sai_precond_info* info);

/* Autotuner of the build schedule: times the build of a strided sample of
 * h's columns (every max(1, n/65536)-th, at least 4096 when n allows) under
 * candidate configurations, with sai = 0 (SPAI, spai params) or 1 (PSAI,
 * psai params), and makes the fastest the process-wide configuration of
 * that builder's later builds (SPAI and PSAI keep one each). The search
 * takes one coordinate at a time: first_tier (the workspace shape and
 * columns per warp of the first tier) x warps_t0 with {blocks_per_sm_t12 2,
 * heavy_first 0} (first_tier 3 with warps_t0 8 only), then heavy_first 1 on
 * the best of those, then blocks_per_sm_t12 1 and 4 on the best so far (ten
 * candidates). out (host) receives the candidates and the choice.
 * Synchronises the stream. */
sai_status sai_build_autotune(sai_split h, int32_t sai, const sai_spai_params* spai, const sai_psai_params* psai,
                              sai_stream_t stream, sai_build_tuning* out);
/* Sets the process-wide build configuration of both builders; NULL restores
 * the default. Returns SAI_INVALID_ARG for values outside the candidate
 * ranges. */
sai_status sai_build_set_config(const sai_build_config* cfg);
/* M as CSC (rows ascending per column): col_ptr n+1, row_idx/val nnz_M.
 * loops[n]: augmentation steps (SPAI) or last loop index (PSAI).
 * res[n]: final LS residual (pre-drop for PSAI). res_post[n] (PSAI only,
 * else zeros): ||A~ m_k - e_k|| of the emitted column. NULLs skipped. */
sai_status sai_precond_copy_out(sai_precond P, int64_t* col_ptr, int32_t* row_idx, double* val,
                                int32_t* loops, double* res, double* res_post, sai_stream_t stream);
void sai_precond_destroy(sai_precond P);
/* A preconditioner handle for a given M (n x n CSC on the device, rows
 * ascending per column, caller-owned and only read): for an M saved from
 * an earlier build (sai_precond_copy_out) and loaded again, so that later
 * right-hand sides skip the build (the paper keeps M for sequences of
 * right-hand sides). The arrays are copied and checked
 * (SAI_INVALID_ARG on a malformed CSC); the CSR copy is built; the
 * per-column statistics are zeros. Synchronises the stream. */
sai_status sai_precond_create(const sai_csc_view* M, sai_stream_t stream, sai_precond* out);

/* ----------------------------------------------------------------------
 * Step 3: k systems A~ X(:,c) = B(:,c) solved together, right
 * preconditioned (A~ M z = b, x = M z), x0 = 0, one SpMM with A~ and one
 * with M per operator application for all right-hand sides at once.
 * System c stops when its residual norm < thr[c] (host array); converged
 * systems are frozen. BiCGStab tests after the half and the full step (a
 * half-step exit counts a full iteration); GMRES(restart) tests the Givens
 * residual estimate and restarts from the true residual; CGS (conjugate
 * gradient squared, two applications of A~ M per iteration) and BiCG (one
 * application of A~ M and one of its transpose M^T A~^T per iteration) test
 * the recursive residual after each iteration. Block GMRES(restart)
 * (SAI_BGMRES, the block Krylov alternative named after Theorem 2) runs the
 * systems still active at a cycle start as one block of a shared block
 * Krylov space (block Arnoldi with two passes of block classical
 * Gram-Schmidt and a shifted Cholesky QR of each new block, Householder
 * reduction of the block Hessenberg matrix); it tests every system's
 * least-squares residual after each block step, ends the cycle when all
 * meet their thresholds and restarts from the true residuals; iters counts
 * block steps (each applies A~ and M to every active system).
 * ---------------------------------------------------------------------- */
typedef enum { SAI_BICGSTAB = 0, SAI_GMRES = 1, SAI_CGS = 2, SAI_BICG = 3, SAI_BGMRES = 4 } sai_krylov_method;

typedef struct {
    int32_t method;
    int32_t restart;   /* GMRES(m) and block GMRES(m), 1..255; ignored by the others */
    int32_t maxit;     /* paper: 500 */
    int32_t precision; /* SAI_FP64, or SAI_FP32_REFINE64 (GMRES and block GMRES):
                          FP32 inner solves of A~ d = r/||r|| refined in FP64 --
                          r = b - A~ x, x += ||r|| d and every stop test in FP64;
                          maxit then bounds the total inner iterations */
    double inner_tol;  /* relative inner tolerance of the refined form; <= 0 -> 1e-4 */
    int32_t transpose; /* 0: solve A~ y = b with right preconditioner M (Procedure *);
                          1: solve A~^T y = b with right preconditioner M^T (the
                          adjoint solves of sai_backward) */
} sai_krylov_params;

/* B, X: n x k row-major device blocks. thr, iters, status: host arrays of k.
 * k: 1..256 for GMRES and its refined form; 1..32 for block GMRES (FP64,
 * or refined: FP32 inner block solves, FP64 outside, as for GMRES);
 * 1..262144 for FP64 BiCGStab, CGS and BiCG (SAI_INVALID_ARG beyond). The solver keeps about 10 n x k FP64 blocks of
 * its own (BiCGStab) and returns SAI_OOM when they do not fit.
 * Returns SAI_OK, SAI_MAXITER or SAI_BREAKDOWN (the first non-OK system
 * status), or an error. Synchronises the stream. */
sai_status sai_krylov_solve(sai_split h, sai_precond P, int32_t k, const double* B, const double* thr,
                            const sai_krylov_params* prm, double* X, int32_t* iters, int32_t* status,
                            sai_stream_t stream);

/* ----------------------------------------------------------------------
 * Step 4: SMW recovery, eq. (composi):
 *   xhat = yhat - What (I + V^T What)^{-1} (V^T yhat)
 * Y: n x (s+1) row-major, column 0 = yhat, columns 1..s = What.
 * x: n. c_out (host, may be NULL): c = ||(I + V^T What)^{-1} V^T yhat||.
 * Gaussian elimination with partial pivoting on the s x s matrix (the
 * largest |pivot|, the first row on ties): one thread block for s <= 256, a
 * blocked right-looking LU (panels of 16 columns, FP64 tiles for the
 * trailing update) for larger s. SAI_SINGULAR on a zero pivot, after which
 * x is not valid.
 * ---------------------------------------------------------------------- */
sai_status sai_smw_recover(sai_split h, const double* Y, double* x, double* c_out, sai_stream_t stream);

/* The same recovery without any device allocation, for callers that cannot
 * allocate: code whose device memory is entirely owned by a host framework's
 * pool or a fixed budget, or that runs where an allocation would synchronise
 * or is not permitted. The paper has no counterpart; it is an interface
 * convenience. Inputs are explicit instead of a split handle: n, s, J (s
 * ascending row indices of V, device), Y (n x (s+1) row-major, device), x
 * (n, device output), c_out (host, may be NULL).
 * Scratch: a static device array of about 516 KB (s <= 256) that every
 * device loading the library holds until the process exits; s > 256 returns
 * SAI_INVALID_ARG. Every call looks up the array's device address in the
 * current context (cudaGetSymbolAddress, which allocates nothing); the first
 * call on a device may also load the library's module there, so make that
 * first call before any stream capture. All calls share the array, so calls
 * that overlap on the GPU (other streams or threads) race: serialise them.
 * On SAI_SINGULAR (a zero pivot) x holds yhat, column 0 of Y, uncorrected.
 * Synchronises the stream. */
sai_status sai_smw_recover_noalloc(int32_t n, int32_t s, const int32_t* J, const double* Y, double* x,
                                   double* c_out, sai_stream_t stream);

/* rr = ||b - A x|| / ||b|| (eq. (rrnorm)) for a caller CSC matrix;
 * rr_out is a host pointer. Synchronises the stream. */
sai_status sai_rel_resid(const sai_csc_view* A, const double* b, const double* x, double* rr_out,
                         sai_stream_t stream);

/* ----------------------------------------------------------------------
 * Procedure *: split, build M, the s+1 solves with the Theorem 2
 * thresholds ||r_y|| < (eps/2)||b|| and ||r_wj|| < eps ||b|| / (2 sqrt(s)),
 * SMW recovery and rr. b, x: device n-vectors.
 * ---------------------------------------------------------------------- */
typedef struct {
    sai_split_params split;
    int32_t sai;                  /* 0: SPAI, 1: PSAI(tol) */
    sai_spai_params spai;
    sai_psai_params psai;
    sai_krylov_params krylov;
    double eps;                   /* paper: 1e-8 */
    int32_t c_adapt;              /* 0: c = 1 in eq. (stopU2) (the paper's setting). 1: when the
                                     recovery's c = ||z|| exceeds 1, the u_j systems are continued
                                     from their iterates to eps ||b|| / (2 sqrt(s) 1.05 c) and x is
                                     recovered again, so that Theorem 2 bounds the residual by
                                     eps ||b|| (one extra round at most) */
    int32_t reserved;             /* 0 */
} sai_solve_params;

typedef struct {
    sai_split_info split;
    sai_precond_info precond;
    int32_t status;               /* worst Krylov status (sai_status) */
    int32_t iter_max;             /* max iterations over the s+1 systems */
    double c;
    double rr;                    /* ||b - A xhat|| / ||b|| */
    double ms_split, ms_build, ms_krylov, ms_smw;  /* device time per step
                                     (ms_split includes the zero-diagonal repair) */
    int32_t moved;                /* zero_diag: columns j with p[j] != j (0: A kept) */
    int32_t c_rounds;             /* c_adapt: 1 when the u_j systems were continued (the
                                     iteration counts include both rounds; c is the last one) */
} sai_solve_report;

/* iters (host, may be NULL): s+1 iteration counts in the order [b, u_1..u_s];
 * pass capacity in iters_cap (counts beyond it are not written). */
sai_status sai_solve(const sai_csc_view* A, const double* b, const sai_solve_params* prm, double* x,
                     int32_t* iters, int32_t iters_cap, sai_solve_report* rep, sai_stream_t stream);

/* ----------------------------------------------------------------------
 * Steps 3-5 of Procedure * on an existing split and preconditioner (one
 * split and one M serve any number of right-hand sides), and the backward
 * pass of x = A^{-1} b.
 * ---------------------------------------------------------------------- */
typedef struct {
    sai_krylov_params krylov;
    double eps;                   /* Theorem 2 thresholds as in sai_solve_params */
} sai_stage_params;

/* x = A^{-1} b from the s+1 solves with h's A~ and P's M, the Theorem 2
 * thresholds (from ||b||), SMW recovery and rr. A: the matrix h was split
 * from (device CSC, used for rr only). b, x: device n-vectors. rep: split and
 * precond fields from the handles, ms_split = ms_build = 0. iters: as in
 * sai_solve. */
sai_status sai_solve_with(const sai_csc_view* A, sai_split h, sai_precond P, const double* b,
                          const sai_stage_params* prm, double* x, int32_t* iters, int32_t iters_cap,
                          sai_solve_report* rep, sai_stream_t stream);

/* Backward pass of x = A^{-1} b for a loss L with g = dL/dx. Not in the
 * paper: the adjoint of Procedure * built from the same pieces. With
 * A^T = A~^T + V U^T, lambda = A^{-T} g is recovered by Theorem 1 applied to
 * A^T:
 *   [yhat, What] = A~^{-T} [g, e_J1 .. e_Js]      (s+1 solves, preconditioner M^T)
 *   lambda = yhat - What (I + U^T What)^{-1} (U^T yhat)
 * with the Theorem 2 thresholds taken from ||g||. Outputs (device):
 *   lambda     n      = dL/db
 *   grad_vals  nnz(A) = dL/dA on A's stored pattern, aligned with A->val:
 *                       -lambda_i x_j for the entry (i, j)
 * A: the matrix h was split from (device CSC); x: the forward solution
 * (device n-vector). rep->rr = ||g - A^T lambda|| / ||g||, rep->c = ||z||,
 * rep->status / iter_max / ms_krylov / ms_smw as in sai_solve; iters: the
 * s+1 adjoint iteration counts. grad_vals may be NULL (skipped). */
sai_status sai_backward(const sai_csc_view* A, sai_split h, sai_precond P, const double* x, const double* g,
                        const sai_stage_params* prm, double* lambda, double* grad_vals, int32_t* iters,
                        int32_t iters_cap, sai_solve_report* rep, sai_stream_t stream);

/* ----------------------------------------------------------------------
 * Batches of independent systems: Procedure * for nmat irregular matrices of
 * different orders in one call. Each matrix is split on its own (its own p
 * and threshold); the columns of all the A~_i are built in one persistent
 * SAI launch (the block-diagonal A~ of the batch: every column's least-squares
 * problem only sees its own matrix); the sum(s_i + 1) Krylov systems of the
 * batch run together in one batched FP64 BiCGStab (each system on its own
 * matrix, with the Theorem 2 thresholds of its matrix), the whole iteration
 * loop as one CUDA graph launch (a conditional while node); then SMW and rr
 * per matrix. prm->c_adapt = 1 continues, for each matrix whose c exceeds 1,
 * its u_j systems with that c (as sai_solve does) in a second batched pass. Supported: SPAI, and PSAI with a fixed tolerance (tol_mode 1; the
 * tol_k of eq. (tolk) is per matrix and is not taken in a batch), both
 * precisions of the build; BiCGStab in FP64 (GMRES and the refined Krylov form
 * return SAI_NOT_IMPLEMENTED).
 *   A: host array of nmat CSC views (device arrays), b, x: host arrays of nmat
 *   device n_i-vectors. items (host, nmat): per-matrix results; rep (host):
 *   batch totals. Returns the worst system status or an error.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t status;    /* worst Krylov status of the matrix's s+1 systems */
    int32_t iter_max;  /* max iterations over its s+1 systems */
    int32_t s, p;      /* irregular columns found, p = floor(nnz/n) */
    double c;          /* ||(I + V^T What)^{-1} V^T yhat|| (of the last recovery) */
    double rr;         /* ||b - A x|| / ||b|| */
    int32_t c_rounds;  /* prm->c_adapt: 1 when this matrix's u_j systems were continued */
    int32_t reserved;
} sai_batch_item;

typedef struct {
    int64_t columns;   /* columns of M built (sum of n_i) */
    int64_t nnz_M;
    int32_t systems;   /* Krylov systems, sum of (s_i + 1) */
    int32_t iter_max;
    double ms_split, ms_build, ms_krylov, ms_smw;  /* device time per step */
} sai_batch_report;

sai_status sai_solve_batched(int32_t nmat, const sai_csc_view* A, const double* const* b,
                             const sai_solve_params* prm, double* const* x, sai_batch_item* items,
                             sai_batch_report* rep, sai_stream_t stream);

/* The SAI build of a batch alone (section 2 on each matrix's A~_i): each
 * matrix split on its own (prm->split), the regular parts stacked as the
 * block-diagonal A~ of the batch (matrix m's rows and columns start at the sum
 * of the earlier orders), one build over all its columns (prm->sai with
 * prm->spai or prm->psai; the same limits as sai_solve_batched). *out: the
 * preconditioner of the stacked A~, owned by the caller (sai_precond_destroy);
 * its diagonal blocks are the M_i that sai_solve_batched uses. */
sai_status sai_build_batched(int32_t nmat, const sai_csc_view* A, const sai_solve_params* prm,
                             sai_stream_t stream, sai_precond* out);
/* The build-schedule autotuner (as sai_build_autotune) on the stacked A~ of a
 * batch, split and stacked as sai_build_batched does; the fastest
 * configuration becomes the process-wide one, so a later sai_solve_batched
 * builds with it. Synchronises the stream. */
sai_status sai_build_autotune_batched(int32_t nmat, const sai_csc_view* A, const sai_solve_params* prm,
                                      sai_stream_t stream, sai_build_tuning* out);

/* ----------------------------------------------------------------------
 * Diagnostics (not part of the paper's method): launch counting and the
 * per-kernel measurements behind the roofline figures.
 * ---------------------------------------------------------------------- */
#define SAI_PROF_MAX_SITES 12

typedef struct {
    char name[24];
    int64_t launches;   /* launches of this site while the profile was open */
    int64_t timed;      /* launches bracketed by CUDA events (every 7th) */
    double ms;          /* device time of all launches: mean timed duration x launches */
    double bytes;       /* algorithmic bytes moved by all launches */
    double flops;       /* algorithmic floating-point operations of all launches */
    double flops32;     /* the FP32 ones among them (the refined build's QR, the FP32
                           Krylov sites); the rest are FP64 */
} sai_profile_site;

typedef struct {
    uint64_t launches;  /* all kernel launches of the library while open */
    int32_t nsites;
    sai_profile_site site[SAI_PROF_MAX_SITES];
} sai_profile_report;

/* Total number of kernel launches made by the library in this process. */
uint64_t sai_launch_count(void);
/* Opens a profile: resets the counters, counts every launch of the profiled
 * sites (SAI build, Krylov SpMV, GMRES projections and updates, BiCGStab
 * vector kernels) and brackets one launch in seven of each site with CUDA
 * events on its stream. */
sai_status sai_profile_begin(void);
/* Closes the profile: synchronises the device, fills *out. */
sai_status sai_profile_end(sai_profile_report* out);

#ifdef __cplusplus
}
#endif
#endif /* SAISMW_H */
