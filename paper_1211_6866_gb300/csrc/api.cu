// api.cu -- extern "C" entry points declared in include/saismw.h.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <new>
#include <string.h>
#include <vector>

#include "internal.h"

// ---------------------------------------------------------------- accounting
static std::atomic<unsigned long long> g_launches{0};
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
// Events are created up front when a profile opens, so that bracketing a
// launch costs two cudaEventRecord calls and no allocation.
static std::vector<cudaEvent_t> g_ev_pool;
static std::atomic<size_t> g_ev_next{0};
struct ProfPair {
    size_t a, b;  // event pair in the pool
    bool all;     // from the fully timed head of the site's launches
};
static std::vector<ProfPair> g_prof_ev[PROF_NSITES];
static const char* k_site_names[PROF_NSITES] = {"sai_build",          "krylov_spmm",     "gmres_project",
                                                "gmres_update",       "bicgstab_vector", "krylov_spmm_fp32",
                                                "gmres_project_fp32", "gmres_update_fp32", "gmres_step"};
static const size_t k_ev_pool = 1 << 16;

unsigned sai_count_grid(unsigned g)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return g;
}

void sai_count_grid_add(long long d) { g_launches.fetch_add((unsigned long long)d, std::memory_order_relaxed); }

bool sai_prof_on() { return g_prof.load(std::memory_order_relaxed); }

void sai_internal_note_cuda_error(cudaError_t e, const char* what, const char* file, int line)
{
    if (getenv("SAISMW_VERBOSE"))
        fprintf(stderr, "saismw: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
}

// The stream-ordered pool keeps freed blocks for reuse instead of returning
// them to the driver after every synchronisation.
void sai_pool_init_once()
{
    static int done_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (done_dev == dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done_dev = dev;
}

static inline cudaStream_t S(sai_stream_t s) { return (cudaStream_t)s; }

cudaStream_t sai_aux_stream()
{
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}

// Every launch of a profiled site is counted; the first k_prof_all launches
// of a site and then one in k_prof_stride are timed with a pair of events (a
// uniform subsample of the frequent sites' launches, every launch of the rare
// ones), which keeps the event overhead out of the timed region.
static const long long k_prof_stride = 7;
static const long long k_prof_all = 16;
static std::atomic<long long> g_site_calls[PROF_NSITES];

ProfScope::ProfScope(int site_, cudaStream_t st_) : site(site_), st(st_)
{
    if (!sai_prof_on()) return;
    const long long c = g_site_calls[site].fetch_add(1);
    if (c >= k_prof_all && c % k_prof_stride != 0) return;
    all = c < k_prof_all;
    const size_t i = g_ev_next.fetch_add(2);
    if (i + 1 >= g_ev_pool.size()) return;
    idx = (long long)i;
    cudaEventRecord(g_ev_pool[i], st);
}

ProfScope::~ProfScope()
{
    if (idx < 0) return;
    const size_t i = (size_t)idx;
    cudaEventRecord(g_ev_pool[i + 1], st);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_ev[site].push_back(ProfPair{i, i + 1, all});
}

extern "C" {

uint64_t sai_launch_count(void) { return g_launches.load(); }

sai_status sai_profile_begin(void)
{
    SAI_CUDA(cudaDeviceSynchronize());
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (auto& v : g_prof_ev) v.clear();
        for (auto& c : g_site_calls) c.store(0);
        if (g_ev_pool.empty()) {
            g_ev_pool.resize(k_ev_pool);
            for (auto& e : g_ev_pool) SAI_CUDA(cudaEventCreate(&e));
        }
        g_ev_next.store(0);
    }
    SAI_TRY(sai_krylov_work_reset());
    SAI_TRY(sai_build_work_reset());
    SAI_TRY(sai_batch_work_reset());
    SAI_CUDA(cudaDeviceSynchronize());
    g_launches.store(0);
    g_prof.store(true);
    return SAI_OK;
}

sai_status sai_profile_end(sai_profile_report* out)
{
    if (!out) return SAI_INVALID_ARG;
    g_prof.store(false);
    SAI_CUDA(cudaDeviceSynchronize());
    memset(out, 0, sizeof(*out));
    out->launches = g_launches.load();
    double wk[PROF_NSITES * 2], wb[PROF_NSITES * 2], wt[PROF_NSITES * 2], wb32 = 0.0;
    SAI_TRY(sai_krylov_work_read(wk));
    SAI_TRY(sai_build_work_read(wb, &wb32));
    SAI_TRY(sai_batch_work_read(wt));
    std::lock_guard<std::mutex> lk(g_prof_mu);
    out->nsites = PROF_NSITES;
    for (int q = 0; q < PROF_NSITES; ++q) {
        sai_profile_site& ps = out->site[q];
        strncpy(ps.name, k_site_names[q], sizeof(ps.name) - 1);
        ps.launches = (int64_t)g_site_calls[q].load();
        // the head launches are all timed; the rest are a 1-in-k_prof_stride
        // sample scaled to the launches after the head
        double ms_head = 0.0, ms_tail = 0.0;
        size_t n_head = 0, n_tail = 0;
        for (auto& pr : g_prof_ev[q]) {
            float t = 0.f;
            cudaEventElapsedTime(&t, g_ev_pool[pr.a], g_ev_pool[pr.b]);
            if (pr.all) {
                ms_head += t;
                ++n_head;
            } else {
                ms_tail += t;
                ++n_tail;
            }
        }
        const double rest = (double)ps.launches - (double)n_head;
        ps.ms = ms_head + (n_tail ? ms_tail * rest / (double)n_tail : 0.0);
        const size_t timed = n_head + n_tail;
        ps.timed = (int64_t)timed;
        g_prof_ev[q].clear();
        ps.bytes = wk[2 * q] + wb[2 * q] + wt[2 * q];
        // all flops, and their FP32 share: the whole of an FP32 Krylov site,
        // the QR of the refined build
        const double b32 = q == PROF_SAI_BUILD ? wb32 : 0.0;
        ps.flops = wk[2 * q + 1] + wb[2 * q + 1] + wt[2 * q + 1] + b32;
        const size_t ln = strlen(k_site_names[q]);
        const bool fp32_site = ln > 5 && strcmp(k_site_names[q] + ln - 5, "_fp32") == 0;
        ps.flops32 = fp32_site ? ps.flops : b32;
    }
    return SAI_OK;
}

const char* sai_status_string(sai_status st)
{
    switch (st) {
    case SAI_OK: return "SAI_OK";
    case SAI_INVALID_ARG: return "SAI_INVALID_ARG";
    case SAI_CUDA_ERROR: return "SAI_CUDA_ERROR";
    case SAI_OOM: return "SAI_OOM";
    case SAI_PATTERN_OVERFLOW: return "SAI_PATTERN_OVERFLOW";
    case SAI_MAXITER: return "SAI_MAXITER";
    case SAI_BREAKDOWN: return "SAI_BREAKDOWN";
    case SAI_SINGULAR: return "SAI_SINGULAR";
    case SAI_NOT_IMPLEMENTED: return "SAI_NOT_IMPLEMENTED";
    }
    return "SAI_UNKNOWN";
}

sai_status sai_split_create(const sai_csc_view* A, const sai_split_params* prm, sai_stream_t stream, sai_split* out)
{
    if (!out) return SAI_INVALID_ARG;
    *out = nullptr;
    if (prm && prm->zero_diag != 0) return SAI_INVALID_ARG;  // the repair belongs to sai_solve
    sai_pool_init_once();
    sai_split_s* h = new (std::nothrow) sai_split_s();
    if (!h) return SAI_OOM;
    sai_status st = sai_split_build(A, prm, S(stream), false, h);
    if (st != SAI_OK) {
        delete h;
        return st;
    }
    *out = h;
    return SAI_OK;
}

sai_status sai_split_get_info(sai_split h, sai_split_info* info)
{
    if (!h || !info) return SAI_INVALID_ARG;
    info->n = h->n;
    info->s = h->s;
    info->p = h->p;
    info->p_keep = h->p_keep;
    info->tau = h->tau;
    info->nnz_At = h->nnz_At;
    info->nnz_U = h->nnz_U;
    info->norm1_At = h->norm1;
    return SAI_OK;
}

sai_status sai_split_copy_out(sai_split h, int64_t* At_col_ptr, int32_t* At_row_idx, double* At_val,
                              int64_t* U_col_ptr, int32_t* U_row_idx, double* U_val, int32_t* J,
                              sai_stream_t stream)
{
    if (!h) return SAI_INVALID_ARG;
    cudaStream_t st = S(stream);
    const cudaMemcpyKind D = cudaMemcpyDeviceToDevice;
    if (At_col_ptr) SAI_CUDA(cudaMemcpyAsync(At_col_ptr, h->At_cp.p, sizeof(int64_t) * (h->n + 1), D, st));
    if (At_row_idx && h->nnz_At) SAI_CUDA(cudaMemcpyAsync(At_row_idx, h->At_ri.p, sizeof(int32_t) * h->nnz_At, D, st));
    if (At_val && h->nnz_At) SAI_CUDA(cudaMemcpyAsync(At_val, h->At_v.p, sizeof(double) * h->nnz_At, D, st));
    if (U_col_ptr) SAI_CUDA(cudaMemcpyAsync(U_col_ptr, h->U_cp.p, sizeof(int64_t) * (h->s + 1), D, st));
    if (U_row_idx && h->nnz_U) SAI_CUDA(cudaMemcpyAsync(U_row_idx, h->U_ri.p, sizeof(int32_t) * h->nnz_U, D, st));
    if (U_val && h->nnz_U) SAI_CUDA(cudaMemcpyAsync(U_val, h->U_v.p, sizeof(double) * h->nnz_U, D, st));
    if (J && h->s) SAI_CUDA(cudaMemcpyAsync(J, h->J.p, sizeof(int32_t) * h->s, D, st));
    return SAI_OK;
}

void sai_split_destroy(sai_split h) { delete h; }

sai_status sai_build_autotune(sai_split h, int32_t sai, const sai_spai_params* spai, const sai_psai_params* psai,
                              sai_stream_t stream, sai_build_tuning* out)
{
    sai_pool_init_once();
    return sai_build_autotune_run(h, sai, spai, psai, S(stream), out);
}

sai_status sai_build_set_config(const sai_build_config* cfg) { return sai_build_set_config_run(cfg); }

sai_status sai_build_spai(sai_split h, const sai_spai_params* prm, sai_stream_t stream, sai_precond* out)
{
    if (!out) return SAI_INVALID_ARG;
    *out = nullptr;
    sai_pool_init_once();
    sai_precond_s* P = new (std::nothrow) sai_precond_s();
    if (!P) return SAI_OOM;
    sai_status st = sai_spai_build(h, prm, S(stream), false, P);
    if (st != SAI_OK) {
        delete P;
        return st;
    }
    *out = P;
    return SAI_OK;
}

sai_status sai_build_psai(sai_split h, const sai_psai_params* prm, sai_stream_t stream, sai_precond* out)
{
    if (!out) return SAI_INVALID_ARG;
    *out = nullptr;
    sai_pool_init_once();
    sai_precond_s* P = new (std::nothrow) sai_precond_s();
    if (!P) return SAI_OOM;
    sai_status st = sai_psai_build(h, prm, S(stream), false, P);
    if (st != SAI_OK) {
        delete P;
        return st;
    }
    *out = P;
    return SAI_OK;
}

sai_status sai_precond_create(const sai_csc_view* M, sai_stream_t stream, sai_precond* out)
{
    if (!out) return SAI_INVALID_ARG;
    *out = nullptr;
    if (!M || M->n < 0 || M->nnz < 0 || (M->n > 0 && !M->col_ptr) || (M->nnz > 0 && (!M->row_idx || !M->val)))
        return SAI_INVALID_ARG;
    sai_pool_init_once();
    cudaStream_t st = S(stream);
    const int32_t n = M->n;
    const int64_t nnz = M->nnz;
    SAI_TRY(sai_validate_csc(n, n, nnz, M->col_ptr, M->row_idx, st));
    std::unique_ptr<sai_precond_s> P(new (std::nothrow) sai_precond_s());
    if (!P) return SAI_OOM;
    P->n = n;
    P->nnz = nnz;
    const size_t nn = (size_t)(n > 0 ? n : 1), nz = (size_t)(nnz > 0 ? nnz : 1);
    SAI_TRY(P->M_cp.alloc(sizeof(int64_t) * (nn + 1), st, false));
    SAI_TRY(P->M_ri.alloc(sizeof(int32_t) * nz, st, false));
    SAI_TRY(P->M_v.alloc(sizeof(double) * nz, st, false));
    SAI_TRY(P->loops.alloc(sizeof(int32_t) * nn, st, false));
    SAI_TRY(P->res.alloc(sizeof(double) * nn, st, false));
    SAI_TRY(P->res_post.alloc(sizeof(double) * nn, st, false));
    const cudaMemcpyKind D = cudaMemcpyDeviceToDevice;
    SAI_CUDA(cudaMemcpyAsync(P->M_cp.p, M->col_ptr, sizeof(int64_t) * ((size_t)n + 1), D, st));
    if (nnz > 0) {
        SAI_CUDA(cudaMemcpyAsync(P->M_ri.p, M->row_idx, sizeof(int32_t) * (size_t)nnz, D, st));
        SAI_CUDA(cudaMemcpyAsync(P->M_v.p, M->val, sizeof(double) * (size_t)nnz, D, st));
    }
    SAI_CUDA(cudaMemsetAsync(P->loops.p, 0, sizeof(int32_t) * nn, st));
    SAI_CUDA(cudaMemsetAsync(P->res.p, 0, sizeof(double) * nn, st));
    SAI_CUDA(cudaMemsetAsync(P->res_post.p, 0, sizeof(double) * nn, st));
    SAI_TRY(sai_csc_to_csr(n, n, nnz, P->M_cp.as<int64_t>(), P->M_ri.as<int32_t>(), P->M_v.as<double>(), P->Mr_rp,
                           P->Mr_ci, P->Mr_v, st, false));
    SAI_CUDA(cudaStreamSynchronize(st));
    *out = P.release();
    return SAI_OK;
}

sai_status sai_precond_get_info(sai_precond P, sai_precond_info* info)
{
    if (!P || !info) return SAI_INVALID_ARG;
    info->n = P->n;
    info->nnz_M = P->nnz;
    info->n_c = P->n_c;
    info->l_m = P->l_m;
    for (int q = 0; q < 6; ++q) info->n_tier[q] = P->n_tier[q];
    info->build_ms = P->ms;
    return SAI_OK;
}

sai_status sai_precond_copy_out(sai_precond P, int64_t* col_ptr, int32_t* row_idx, double* val, int32_t* loops,
                                double* res, double* res_post, sai_stream_t stream)
{
    if (!P) return SAI_INVALID_ARG;
    cudaStream_t st = S(stream);
    const cudaMemcpyKind D = cudaMemcpyDeviceToDevice;
    if (col_ptr) SAI_CUDA(cudaMemcpyAsync(col_ptr, P->M_cp.p, sizeof(int64_t) * (P->n + 1), D, st));
    if (row_idx && P->nnz) SAI_CUDA(cudaMemcpyAsync(row_idx, P->M_ri.p, sizeof(int32_t) * P->nnz, D, st));
    if (val && P->nnz) SAI_CUDA(cudaMemcpyAsync(val, P->M_v.p, sizeof(double) * P->nnz, D, st));
    if (loops && P->n) SAI_CUDA(cudaMemcpyAsync(loops, P->loops.p, sizeof(int32_t) * P->n, D, st));
    if (res && P->n) SAI_CUDA(cudaMemcpyAsync(res, P->res.p, sizeof(double) * P->n, D, st));
    if (res_post && P->n) SAI_CUDA(cudaMemcpyAsync(res_post, P->res_post.p, sizeof(double) * P->n, D, st));
    return SAI_OK;
}

void sai_precond_destroy(sai_precond P) { delete P; }

sai_status sai_krylov_solve(sai_split h, sai_precond P, int32_t k, const double* B, const double* thr,
                            const sai_krylov_params* prm, double* X, int32_t* iters, int32_t* status,
                            sai_stream_t stream)
{
    sai_pool_init_once();
    return sai_krylov_run(h, P, k, B, thr, prm, X, iters, status, S(stream));
}

sai_status sai_smw_recover(sai_split h, const double* Y, double* x, double* c_out, sai_stream_t stream)
{
    sai_pool_init_once();
    return sai_smw_run(h, Y, x, c_out, S(stream));
}

sai_status sai_rel_resid(const sai_csc_view* A, const double* b, const double* x, double* rr_out,
                         sai_stream_t stream)
{
    if (!A || !rr_out || A->n < 0 || (A->n > 0 && (!b || !x || !A->col_ptr))) return SAI_INVALID_ARG;
    sai_pool_init_once();
    double nn[2] = {0.0, 0.0};
    SAI_TRY(sai_csc_residual_norms(A->n, A->col_ptr, A->row_idx, A->val, b, x, nn, S(stream)));
    *rr_out = nn[1] > 0.0 ? sqrt(nn[0] / nn[1]) : sqrt(nn[0]);
    return SAI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- Procedure *
namespace {

// column 0 of the n x (s+1) row-major block B (the rest is cleared first)
__global__ void k_put_col0(int32_t n, int32_t s, const double* b, double* B)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) B[i * ((int64_t)s + 1)] = b[i];
}

// B = [b, 0 .. 0] as an n x (s+1) row-major block
sai_status fill_rhs(int32_t n, int32_t s, const double* b, double* B, cudaStream_t st)
{
    if (n <= 0) return SAI_OK;
    SAI_CUDA(cudaMemsetAsync(B, 0, sizeof(double) * (size_t)n * ((size_t)s + 1), st));
    k_put_col0<<<SAI_GRID(sai_div_up(n, 256)), 256, 0, st>>>(n, s, b, B);
    return SAI_OK;
}

__global__ void k_scatter_U(int32_t s, const int64_t* Ucp, const int32_t* Uri, const double* Uv, double* B)
{
    const int t = blockIdx.x;
    const int64_t ld = (int64_t)s + 1;
    for (int64_t q = Ucp[t] + threadIdx.x; q < Ucp[t + 1]; q += blockDim.x) B[(int64_t)Uri[q] * ld + 1 + t] = Uv[q];
}

__global__ void k_sumsq(int32_t n, const double* b, double* out)
{
    __shared__ double sh[1024];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += b[i] * b[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) t += sh[q];
        *out = t;
    }
}

struct Ev {
    cudaEvent_t e = nullptr;
    Ev() { cudaEventCreate(&e); }
    ~Ev() { cudaEventDestroy(e); }
};

// B = [g, e_J1 .. e_Js]: right-hand sides of the adjoint solves (V's columns)
__global__ void k_set_units(int32_t s, const int32_t* J, double* B)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < s) B[(int64_t)J[t] * (s + 1) + 1 + t] = 1.0;
}

// Per block: sum over its columns j of (g_j - (A^T lambda)_j)^2, one warp per
// column, warps summed in order.
__global__ void k_adj_resid(int32_t n, const int64_t* cp, const int32_t* ri, const double* v, const double* lam,
                            const double* g, double* partial)
{
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double mine = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * nw + wid; j < n; j += (int64_t)gridDim.x * nw) {
        double acc = 0.0;
        for (int64_t q = cp[j] + lane; q < cp[j + 1]; q += 32) acc = fma(v[q], lam[ri[q]], acc);
        acc = warp_sum(acc);
        const double r = g[j] - acc;
        mine = fma(r, r, mine);
    }
    if (lane == 0) sh[wid] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_sum_in_order(int32_t m, const double* a, double* out)
{
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < m; ++i) t += a[i];
        *out = t;
    }
}

// dL/dA(i,j) = -lambda_i x_j on A's stored pattern, one warp per column
__global__ void k_grad_vals(int32_t n, const int64_t* cp, const int32_t* ri, const double* lam, const double* x,
                            double* gv)
{
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const double xj = x[j];
    for (int64_t q = cp[j] + lane; q < cp[j + 1]; q += 32) gv[q] = -lam[ri[q]] * xj;
}

void report_handles(const sai_split_s& h, const sai_precond_s& P, sai_solve_report* rep)
{
    rep->split.n = h.n;
    rep->split.s = h.s;
    rep->split.p = h.p;
    rep->split.p_keep = h.p_keep;
    rep->split.tau = h.tau;
    rep->split.nnz_At = h.nnz_At;
    rep->split.nnz_U = h.nnz_U;
    rep->split.norm1_At = h.norm1;
    rep->precond.n = P.n;
    rep->precond.nnz_M = P.nnz;
    rep->precond.n_c = P.n_c;
    rep->precond.l_m = P.l_m;
    for (int q = 0; q < 6; ++q) rep->precond.n_tier[q] = P.n_tier[q];
    rep->precond.build_ms = P.ms;
}

// ||v||_2 of a device n-vector, read back to the host
sai_status host_norm(int32_t n, const double* v, double* out, cudaStream_t st)
{
    Buf nb;
    SAI_TRY(nb.alloc(sizeof(double), st, true));
    k_sumsq<<<SAI_GRID(1), 1024, 0, st>>>(n, v, nb.as<double>());
    SAI_CUDA(cudaGetLastError());
    double vv = 0.0;
    SAI_CUDA(cudaMemcpyAsync(&vv, nb.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    *out = sqrt(vv);
    return SAI_OK;
}

// The s+1 solves with the Theorem 2 thresholds of eqs. (stopb) and (stopU2),
// taken from rnorm = ||b|| (or ||g|| for the adjoint solves), with c = cu in
// eq. (stopU2) (1 unless a continuation round tightens it). Returns an
// error, or SAI_OK with *kst the worst system status.
sai_status stage_solves(const sai_split_s& h, const sai_precond_s& P, const double* B, double rnorm,
                        const sai_krylov_params& kp, double eps, double* Y, int32_t* iters, int32_t iters_cap,
                        int32_t* imax, sai_status* kst, cudaStream_t st, double cu = 1.0)
{
    const int32_t s = h.s, k = s + 1;
    double* thr = (double*)malloc(sizeof(double) * k);
    int32_t* it = (int32_t*)malloc(sizeof(int32_t) * k);
    int32_t* stt = (int32_t*)malloc(sizeof(int32_t) * k);
    if (!thr || !it || !stt) {
        free(thr);
        free(it);
        free(stt);
        return SAI_OOM;
    }
    thr[0] = 0.5 * eps * rnorm;
    for (int t = 1; t < k; ++t) thr[t] = eps * rnorm / (2.0 * sqrt((double)s) * cu);
    const sai_status r = sai_krylov_run(&h, &P, k, B, thr, &kp, Y, it, stt, st);
    if (r == SAI_OK || r == SAI_MAXITER || r == SAI_BREAKDOWN) {
        int m = 0;
        for (int t = 0; t < k; ++t) {
            if (it[t] > m) m = it[t];
            if (iters && t < iters_cap) iters[t] = it[t];
        }
        *imax = m;
        *kst = r;
    }
    free(thr);
    free(it);
    free(stt);
    return (r == SAI_OK || r == SAI_MAXITER || r == SAI_BREAKDOWN) ? SAI_OK : r;
}

// Y += D over n x k values
__global__ void k_add_block(int64_t m, const double* __restrict__ D, double* __restrict__ Y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        Y[i] += D[i];
}

// Steps 3-5 of Procedure * on the handles: B = [b, u_1..u_s], the solves,
// SMW recovery, rr. c_adapt: when the recovery's c exceeds 1, one more round
// continues the u_j systems (correction solves A~ d = u_j - A~ w_j to the
// eq. (stopU2) threshold with c = 1.05 c, w_j += d) and recovers x again.
sai_status solve_steps(const sai_csc_view* A, const sai_split_s& h, const sai_precond_s& P, const double* b,
                       const sai_krylov_params& kp, double eps, double* x, int32_t* iters, int32_t iters_cap,
                       sai_solve_report* rep, cudaEvent_t e_solve, cudaEvent_t e_smw, cudaEvent_t e_end,
                       cudaStream_t st, int c_adapt = 0)
{
    const int32_t n = h.n, s = h.s, k = s + 1;
    Buf Bb, Yb;
    SAI_TRY(Bb.alloc(sizeof(double) * (size_t)n * k + 8, st, true));
    SAI_TRY(Yb.alloc(sizeof(double) * (size_t)n * k + 8, st, true));
    SAI_TRY(fill_rhs(n, s, b, Bb.as<double>(), st));
    if (s > 0)
        k_scatter_U<<<SAI_GRID(s), 256, 0, st>>>(s, h.U_cp.as<int64_t>(), h.U_ri.as<int32_t>(), h.U_v.as<double>(),
                                       Bb.as<double>());
    SAI_CUDA(cudaGetLastError());
    double bnorm = 0.0;
    SAI_TRY(host_norm(n, b, &bnorm, st));
    SAI_CUDA(cudaEventRecord(e_solve, st));
    int32_t imax = 0;
    sai_status kst = SAI_OK;
    SAI_TRY(stage_solves(h, P, Bb.as<double>(), bnorm, kp, eps, Yb.as<double>(), iters, iters_cap, &imax, &kst, st));
    double c = 0.0;
    if (c_adapt && s > 0) {
        SAI_TRY(sai_smw_run(&h, Yb.as<double>(), x, &c, st));
        if (c > 1.0) {
            // R = B - A~ Y; its column 0 is cleared (the y system is not continued)
            Buf Rb, Db;
            SAI_TRY(Rb.alloc(sizeof(double) * (size_t)n * k + 8, st, true));
            SAI_TRY(Db.alloc(sizeof(double) * (size_t)n * k + 8, st, true));
            SAI_TRY(sai_spmm(n, h.Atr_rp.as<int64_t>(), h.Atr_ci.as<int32_t>(), h.Atr_v.as<double>(), k,
                             Yb.as<double>(), Rb.as<double>(), Bb.as<double>(), 1, st));
            SAI_CUDA(cudaMemset2DAsync(Rb.p, sizeof(double) * (size_t)k, 0, sizeof(double), (size_t)n, st));
            std::vector<int32_t> it2((size_t)k, 0);
            int32_t imax2 = 0;
            sai_status kst2 = SAI_OK;
            SAI_TRY(stage_solves(h, P, Rb.as<double>(), bnorm, kp, eps, Db.as<double>(), it2.data(), k, &imax2, &kst2,
                                 st, 1.05 * c));
            const int64_t m = (int64_t)n * k;
            k_add_block<<<SAI_GRID(sai_div_up(m, 256) < 4096u ? sai_div_up(m, 256) : 4096u), 256, 0, st>>>(
                m, Db.as<double>(), Yb.as<double>());
            SAI_CUDA(cudaGetLastError());
            imax = 0;
            for (int32_t t = 0; t < k; ++t) {
                const int32_t tot = (iters && t < iters_cap ? iters[t] : 0) + it2[t];
                if (iters && t < iters_cap) iters[t] = tot;
                imax = tot > imax ? tot : imax;
            }
            if (kst == SAI_OK) kst = kst2;
            rep->c_rounds = 1;
        }
    }
    SAI_CUDA(cudaEventRecord(e_smw, st));
    SAI_TRY(sai_smw_run(&h, Yb.as<double>(), x, &c, st));
    SAI_CUDA(cudaEventRecord(e_end, st));
    double nn[2] = {0.0, 0.0};
    SAI_TRY(sai_csc_residual_norms(A->n, A->col_ptr, A->row_idx, A->val, b, x, nn, st));
    report_handles(h, P, rep);
    rep->status = kst;
    rep->iter_max = imax;
    rep->c = c;
    rep->rr = nn[1] > 0.0 ? sqrt(nn[0] / nn[1]) : sqrt(nn[0]);
    return kst;
}

float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

sai_status solve_impl(const sai_csc_view* A, const double* b, const sai_solve_params* prm, double* x,
                      int32_t* iters, int32_t iters_cap, sai_solve_report* rep, cudaStream_t st)
{
    if (!A || !prm || !rep || (A->n > 0 && (!b || !x)) || (prm->split.zero_diag != 0 && prm->split.zero_diag != 1) ||
        (prm->c_adapt != 0 && prm->c_adapt != 1))
        return SAI_INVALID_ARG;
    *rep = sai_solve_report{};
    Ev e0, e1, e2, e3, e4, e5;
    SAI_CUDA(cudaEventRecord(e0.e, st));
    // zero-diagonal repair (section 5): the method then runs on A(p,:) x = b(p)
    Buf pb, bcp, bri, bv, bb;
    sai_csc_view Ap = *A;
    if (prm->split.zero_diag && A->n > 0) {
        SAI_TRY(pb.alloc(sizeof(int32_t) * (size_t)A->n, st, true));
        int32_t rank = 0, moved = 0;
        SAI_TRY(sai_dmperm_run(A, pb.as<int32_t>(), &rank, &moved, st));
        if (rank < A->n) return SAI_SINGULAR;
        rep->moved = moved;
        if (moved > 0) {
            SAI_TRY(bcp.alloc(sizeof(int64_t) * ((size_t)A->n + 1), st, true));
            SAI_TRY(bri.alloc(sizeof(int32_t) * (size_t)A->nnz + 4, st, true));
            SAI_TRY(bv.alloc(sizeof(double) * (size_t)A->nnz + 8, st, true));
            SAI_TRY(bb.alloc(sizeof(double) * (size_t)A->n, st, true));
            SAI_TRY(sai_permute_rows_run(A, pb.as<int32_t>(), bcp.as<int64_t>(), bri.as<int32_t>(), bv.as<double>(),
                                         st));
            SAI_TRY(sai_gather_vec(A->n, pb.as<int32_t>(), b, bb.as<double>(), st));
            Ap.col_ptr = bcp.as<int64_t>();
            Ap.row_idx = bri.as<int32_t>();
            Ap.val = bv.as<double>();
            A = &Ap;
            b = bb.as<double>();
        }
    }
    sai_split_s h;
    SAI_TRY(sai_split_build(A, &prm->split, st, true, &h));
    SAI_CUDA(cudaEventRecord(e1.e, st));
    sai_precond_s P;
    if (prm->sai == 0) SAI_TRY(sai_spai_build(&h, &prm->spai, st, true, &P));
    else SAI_TRY(sai_psai_build(&h, &prm->psai, st, true, &P));
    SAI_CUDA(cudaEventRecord(e2.e, st));
    const sai_status r = solve_steps(A, h, P, b, prm->krylov, prm->eps, x, iters, iters_cap, rep, e3.e, e4.e, e5.e,
                                     st, prm->c_adapt);
    if (r != SAI_OK && r != SAI_MAXITER && r != SAI_BREAKDOWN) return r;
    rep->ms_split = elapsed(e0.e, e1.e);
    rep->ms_build = elapsed(e1.e, e2.e);
    rep->ms_krylov = elapsed(e2.e, e4.e);  // includes forming B and ||b||
    rep->ms_smw = elapsed(e4.e, e5.e);
    return r;
}

sai_status solve_with_impl(const sai_csc_view* A, const sai_split_s* h, const sai_precond_s* P, const double* b,
                           const sai_stage_params* prm, double* x, int32_t* iters, int32_t iters_cap,
                           sai_solve_report* rep, cudaStream_t st)
{
    if (!A || !h || !P || !prm || !rep || A->n != h->n || P->n != h->n || (h->n > 0 && (!b || !x)))
        return SAI_INVALID_ARG;
    *rep = sai_solve_report{};
    Ev e0, e1, e2, e3;
    SAI_CUDA(cudaEventRecord(e0.e, st));
    const sai_status r = solve_steps(A, *h, *P, b, prm->krylov, prm->eps, x, iters, iters_cap, rep, e1.e, e2.e,
                                     e3.e, st);
    if (r != SAI_OK && r != SAI_MAXITER && r != SAI_BREAKDOWN) return r;
    rep->ms_krylov = elapsed(e0.e, e2.e);
    rep->ms_smw = elapsed(e2.e, e3.e);
    return r;
}

// Backward pass: Theorem 1 on A^T = A~^T + V U^T (see saismw.h).
sai_status backward_impl(const sai_csc_view* A, const sai_split_s* h, const sai_precond_s* P, const double* x,
                         const double* g, const sai_stage_params* prm, double* lambda, double* grad_vals,
                         int32_t* iters, int32_t iters_cap, sai_solve_report* rep, cudaStream_t st)
{
    if (!A || !h || !P || !prm || !rep || A->n != h->n || P->n != h->n ||
        (h->n > 0 && (!x || !g || !lambda || !A->col_ptr)))
        return SAI_INVALID_ARG;
    *rep = sai_solve_report{};
    const int32_t n = h->n, s = h->s, k = s + 1;
    Ev e0, e1, e2;
    SAI_CUDA(cudaEventRecord(e0.e, st));
    Buf Bb, Yb;
    SAI_TRY(Bb.alloc(sizeof(double) * (size_t)n * k + 8, st, true));
    SAI_TRY(Yb.alloc(sizeof(double) * (size_t)n * k + 8, st, true));
    SAI_TRY(fill_rhs(n, s, g, Bb.as<double>(), st));
    if (s > 0) k_set_units<<<SAI_GRID(sai_div_up(s, 256)), 256, 0, st>>>(s, h->J.as<int32_t>(), Bb.as<double>());
    SAI_CUDA(cudaGetLastError());
    double gnorm = 0.0;
    SAI_TRY(host_norm(n, g, &gnorm, st));
    sai_krylov_params kp = prm->krylov;
    kp.transpose = 1;
    int32_t imax = 0;
    sai_status kst = SAI_OK;
    SAI_TRY(stage_solves(*h, *P, Bb.as<double>(), gnorm, kp, prm->eps, Yb.as<double>(), iters, iters_cap, &imax,
                         &kst, st));
    SAI_CUDA(cudaEventRecord(e1.e, st));
    double c = 0.0;
    SAI_TRY(sai_smw_adj_run(h, Yb.as<double>(), lambda, &c, st));
    if (grad_vals && n > 0)
        k_grad_vals<<<SAI_GRID(sai_div_up((int64_t)n * 32, 256)), 256, 0, st>>>(n, A->col_ptr, A->row_idx, lambda, x,
                                                                            grad_vals);
    SAI_CUDA(cudaEventRecord(e2.e, st));
    // adjoint residual ||g - A^T lambda|| / ||g||
    int64_t rb = sai_div_up((int64_t)(n > 0 ? n : 1) * 32, 256);
    if (rb > 1024) rb = 1024;
    Buf part, out;
    SAI_TRY(part.alloc(sizeof(double) * (size_t)rb, st, true));
    SAI_TRY(out.alloc(sizeof(double), st, true));
    k_adj_resid<<<SAI_GRID(rb), 256, 0, st>>>(n, A->col_ptr, A->row_idx, A->val, lambda, g, part.as<double>());
    k_sum_in_order<<<SAI_GRID(1), 32, 0, st>>>((int32_t)rb, part.as<double>(), out.as<double>());
    SAI_CUDA(cudaGetLastError());
    double rr2 = 0.0;
    SAI_CUDA(cudaMemcpyAsync(&rr2, out.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    report_handles(*h, *P, rep);
    rep->status = kst;
    rep->iter_max = imax;
    rep->c = c;
    rep->rr = gnorm > 0.0 ? sqrt(rr2) / gnorm : sqrt(rr2);
    rep->ms_krylov = elapsed(e0.e, e1.e);
    rep->ms_smw = elapsed(e1.e, e2.e);
    return kst;
}

}  // namespace

extern "C" sai_status sai_solve(const sai_csc_view* A, const double* b, const sai_solve_params* prm, double* x,
                                int32_t* iters, int32_t iters_cap, sai_solve_report* rep, sai_stream_t stream)
{
    sai_pool_init_once();
    return solve_impl(A, b, prm, x, iters, iters_cap, rep, S(stream));
}

extern "C" sai_status sai_solve_with(const sai_csc_view* A, sai_split h, sai_precond P, const double* b,
                                     const sai_stage_params* prm, double* x, int32_t* iters, int32_t iters_cap,
                                     sai_solve_report* rep, sai_stream_t stream)
{
    sai_pool_init_once();
    return solve_with_impl(A, h, P, b, prm, x, iters, iters_cap, rep, S(stream));
}

extern "C" sai_status sai_backward(const sai_csc_view* A, sai_split h, sai_precond P, const double* x,
                                   const double* g, const sai_stage_params* prm, double* lambda, double* grad_vals,
                                   int32_t* iters, int32_t iters_cap, sai_solve_report* rep, sai_stream_t stream)
{
    sai_pool_init_once();
    return backward_impl(A, h, P, x, g, prm, lambda, grad_vals, iters, iters_cap, rep, S(stream));
}

extern "C" sai_status sai_dmperm(const sai_csc_view* A, int32_t* p, int32_t* rank_out, int32_t* moved_out,
                                 sai_stream_t stream)
{
    sai_pool_init_once();
    return sai_dmperm_run(A, p, rank_out, moved_out, S(stream));
}

extern "C" sai_status sai_permute_rows(const sai_csc_view* A, const int32_t* p, int64_t* B_col_ptr,
                                       int32_t* B_row_idx, double* B_val, sai_stream_t stream)
{
    sai_pool_init_once();
    const sai_status r = sai_permute_rows_run(A, p, B_col_ptr, B_row_idx, B_val, S(stream));
    if (r != SAI_OK) return r;
    SAI_CUDA(cudaStreamSynchronize(S(stream)));
    return SAI_OK;
}
