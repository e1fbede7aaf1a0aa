// internal.h -- host-side declarations shared by the saismw CUDA sources.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "saismw.h"

// Ownership mode of a device buffer: handles returned to the user allocate
// synchronously (cudaMalloc); buffers that live inside one call use the
// stream-ordered pool of the call's stream.
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    bool async = false;
    Buf() = default;
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    ~Buf() { release(); }
    sai_status alloc(size_t nbytes, cudaStream_t s, bool use_async);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Exclusive scan of n counts into out[0..n] (out[n] = total), int64 output.
sai_status sai_scan_counts_i32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st);
sai_status sai_scan_counts_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);

// CSC (ncols columns, rows < nrows) -> CSR with ascending column indices.
// Output buffers are allocated in `mode_async` mode on st.
sai_status sai_csc_to_csr(int32_t nrows, int32_t ncols, int64_t nnz, const int64_t* cp, const int32_t* ri,
                          const double* cv, Buf& rp, Buf& ci, Buf& rv, cudaStream_t st, bool mode_async);

// Checks CSC structure on the device: col_ptr[0]=0, nondecreasing, last = nnz,
// rows in [0,nrows) strictly ascending per column.
sai_status sai_validate_csc(int32_t nrows, int32_t ncols, int64_t nnz, const int64_t* cp, const int32_t* ri,
                            cudaStream_t st);

// Y = A X (mode 0) or Y = B - A X (mode 1), A in CSR (n rows), X/Y/B n x k row-major.
sai_status sai_spmm(int32_t n, const int64_t* rp, const int32_t* ci, const double* v, int32_t k, const double* X,
                    double* Y, const double* B, int mode, cudaStream_t st);

// y = A x for a CSC matrix via gather over a CSR copy is done by callers; this
// helper computes ||b - A x||^2 and ||b||^2 with A in CSC (one pass, atomics-free).
sai_status sai_csc_residual_norms(int32_t n, const int64_t* cp, const int32_t* ri, const double* cv,
                                  const double* b, const double* x, double* out2_host, cudaStream_t st);

// Handle internals --------------------------------------------------------
struct sai_split_s {
    int32_t n = 0, s = 0, p = 0, p_keep = 0;
    double tau = 0.0, norm1 = 0.0;
    int64_t nnz_At = 0, nnz_U = 0;
    Buf At_cp, At_ri, At_v;      // CSC of A~
    Buf Atr_rp, Atr_ci, Atr_v;   // CSR of A~
    Buf U_cp, U_ri, U_v;         // CSC of U (n x s)
    Buf J;                       // int32[s]
    Buf colnorm2;                // ||A~ e_j||^2
    float ms = 0.f;
};

struct sai_precond_s {
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t n_c = 0, l_m = 0;
    int32_t n_tier[6] = {0, 0, 0, 0, 0, 0};
    float ms = 0.f;
    Buf M_cp, M_ri, M_v;     // CSC
    Buf Mr_rp, Mr_ci, Mr_v;  // CSR
    Buf loops, res, res_post;
};

sai_status sai_split_build(const sai_csc_view* A, const sai_split_params* prm, cudaStream_t st, bool async,
                           sai_split_s* h);
sai_status sai_spai_build(const sai_split_s* h, const sai_spai_params* prm, cudaStream_t st, bool async,
                          sai_precond_s* P);
sai_status sai_psai_build(const sai_split_s* h, const sai_psai_params* prm, cudaStream_t st, bool async,
                          sai_precond_s* P);
sai_status sai_krylov_run(const sai_split_s* h, const sai_precond_s* P, int32_t k, const double* B,
                          const double* thr, const sai_krylov_params* prm, double* X, int32_t* iters,
                          int32_t* status, cudaStream_t st);
sai_status sai_smw_run(const sai_split_s* h, const double* Y, double* x, double* c_out, cudaStream_t st);
sai_status sai_build_autotune_run(const sai_split_s* h, int32_t sai, const sai_spai_params* sp,
                                  const sai_psai_params* pp, cudaStream_t st, sai_build_tuning* out);
sai_status sai_build_set_config_run(const sai_build_config* cfg);
// Theorem 1 for A^T = A~^T + V U^T: x = yhat - What (I + U^T What)^{-1} (U^T yhat)
sai_status sai_smw_adj_run(const sai_split_s* h, const double* Y, double* x, double* c_out, cudaStream_t st);

// Zero-diagonal repair (section 5): maximum transversal p (p[j] = row of
// column j, -1 if unmatched), B = A(p,:), and y = x(p).
sai_status sai_dmperm_run(const sai_csc_view* A, int32_t* p, int32_t* rank_out, int32_t* moved_out, cudaStream_t st);
sai_status sai_permute_rows_run(const sai_csc_view* A, const int32_t* p, int64_t* Bcp, int32_t* Bri, double* Bv,
                                cudaStream_t st);
sai_status sai_gather_vec(int32_t n, const int32_t* p, const double* x, double* y, cudaStream_t st);

void sai_pool_init_once();
// Library-owned non-blocking stream of the current device (for graph capture), or nullptr.
cudaStream_t sai_aux_stream();

// Device-side algorithmic work per profiled site ([site][0] bytes, [1] flops),
// one accumulator per translation unit.
sai_status sai_krylov_work_reset();
sai_status sai_krylov_work_read(double* out /* PROF_NSITES x 2 */);
sai_status sai_build_work_reset();
sai_status sai_build_work_read(double* out /* PROF_NSITES x 2 */, double* flops32 /* FP32 flops of the build */);
sai_status sai_batch_work_reset();
sai_status sai_batch_work_read(double* out /* PROF_NSITES x 2 */);
