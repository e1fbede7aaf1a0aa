// krylov.cu -- the s+1 right-preconditioned Krylov solves of Procedure *
// (A~ y = b, A~ w_j = u_j, eqs. (regprob), (auxi)) for k systems at once.
//
// Layout: inside the solver every block of k vectors is stored system-major
// (system c's vector is contiguous, leading dimension ld = n rounded up to 32),
// so each warp streams 256 contiguous bytes of one system and no lane idles.
// The caller's n x k row-major B and X are transposed on entry and exit.
//
// Work distribution: device-side lists of the systems that take part in a
// step (list[0] = count, list[1..] = system indices, ascending) are rebuilt
// by the single-block control kernels; data-parallel kernels loop over the
// items (system in the list) x (row tile or row chunk), so converged systems
// cost nothing and the host never needs to know which systems are active.
// Inner products are formed per (system, row chunk) by one warp and summed
// in a fixed order, so results do not depend on scheduling.
//
// BiCGStab: van der Vorst's recurrence on A~ M z = b with y = M z updated
// directly; stop tests after the half step (s) and the full step (r).
// GMRES(m): Arnoldi with classical Gram-Schmidt, re-applied for a system
// only when its norm falls below 1/sqrt(2) of the pre-projection norm (the
// Daniel-Gragg-Kaufman-Stewart criterion); Givens rotations; stop on the
// rotated residual |g_{j+1}|; restart from the true residual b - A~ y.
#include <math.h>

#include "internal.h"

namespace {

constexpr int CTRL = 256;      // threads of the single-block control kernels (>= k)
constexpr int CHUNK = 1024;    // rows per (system, chunk) reduction item (one warp)
constexpr int TILE = 256;      // rows per SpMV item (one block)
constexpr int PJ = 32;         // basis vectors per register-tiled projection pass
constexpr int IT_WARPS = 8;    // warps per block of the item kernels

enum { ST_OK = 0, ST_MAXITER = 5, ST_BREAKDOWN = 6 };  // same values as sai_status

int g_sms = 0;

// ---------------------------------------------------------------- accounting
__device__ double d_kwork[PROF_NSITES * 2];

struct Dims {
    double n, nnzA, nnzM;
};

__device__ __forceinline__ void kwork_add(int site, double bytes, double flops)
{
    atomicAdd(&d_kwork[2 * site], bytes);
    atomicAdd(&d_kwork[2 * site + 1], flops);
}

// one SpMV launch over k_act systems: matrix once, x read once, y written
__device__ __forceinline__ void spmm_work(double n, double nnz, int kact)
{
    if (kact > 0) kwork_add(PROF_SPMM, 8.0 * (n + 1) + 12.0 * nnz + 16.0 * n * kact, 2.0 * nnz * kact);
}

// ---------------------------------------------------------------- lists
// Rebuild list (count + ascending indices) from mask; called by thread 0 of a
// single-block kernel after the mask is final.
__device__ __forceinline__ void build_list(int k, const int* mask, int* list)
{
    int q = 0;
    for (int c = 0; c < k; ++c)
        if (mask[c]) list[1 + q++] = c;
    list[0] = q;
}

// ---------------------------------------------------------------- layout
__global__ void k_to_soa(int64_t n, int k, int64_t ld, const double* __restrict__ B, double* __restrict__ Bs)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e - i * k);
        Bs[(int64_t)c * ld + i] = B[e];
    }
}

__global__ void k_from_soa(int64_t n, int k, int64_t ld, const double* __restrict__ Xs, double* __restrict__ X)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e - i * k);
        X[e] = Xs[(int64_t)c * ld + i];
    }
}

// ---------------------------------------------------------------- SpMV over a list
// Y[c] = A X[c] (mode 0) or B[c] - A X[c] (mode 1) for the systems in list.
// Items are (row tile, system), tile-major, so the systems of a tile reuse
// the tile's matrix rows from cache. One thread per row (CSR).
template <int MODE>
__global__ void __launch_bounds__(TILE) k_spmv(int32_t n, int64_t ld, const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ ci, const double* __restrict__ v,
                                               const double* __restrict__ X, double* __restrict__ Y,
                                               const double* __restrict__ B, const int* __restrict__ list)
{
    const int cnt = list[0];
    const int64_t tiles = ((int64_t)n + TILE - 1) / TILE;
    for (int64_t it = blockIdx.x; it < tiles * cnt; it += gridDim.x) {
        const int64_t tile = it / cnt;
        const int c = list[1 + (int)(it - tile * cnt)];
        const int64_t row = tile * TILE + threadIdx.x;
        if (row >= n) continue;
        const double* xc = X + (int64_t)c * ld;
        double acc = 0.0;
        const int64_t b = rp[row], e = rp[row + 1];
        for (int64_t t = b; t < e; ++t) acc = fma(v[t], xc[ci[t]], acc);
        if (MODE == 0) Y[(int64_t)c * ld + row] = acc;
        else Y[(int64_t)c * ld + row] = B[(int64_t)c * ld + row] - acc;
    }
}

template <int MODE>
void spmv(int32_t n, int64_t ld, const int64_t* rp, const int32_t* ci, const double* v, int k, const double* X,
          double* Y, const double* B, const int* list, cudaStream_t st)
{
    const int64_t tiles = ((int64_t)n + TILE - 1) / TILE;
    int64_t g = tiles * k;
    const int64_t cap = (int64_t)g_sms * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    k_spmv<MODE><<<SAI_GRID(g), TILE, 0, st>>>(n, ld, rp, ci, v, X, Y, B, list);
}

// ---------------------------------------------------------------- item kernels
// An item is (system in list, row chunk of CHUNK rows) handled by one warp.
struct Items {
    int32_t n;
    int64_t ld;
    int nch;  // chunks per system
};

__host__ __device__ __forceinline__ int nchunks(int64_t n) { return (int)((n + CHUNK - 1) / CHUNK); }

int item_blocks(int64_t n, int k)
{
    int64_t items = (int64_t)nchunks(n) * k;
    int64_t b = (items + IT_WARPS - 1) / IT_WARPS;
    const int64_t cap = (int64_t)g_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// Loops the calling warp over its items: c = system, q_ = chunk, [r0, r1) = rows.
#define FOR_ITEMS(I, list, cvar, r0, r1)                                                              \
    const int cnt_ = (list)[0];                                                                       \
    const int lane_ = threadIdx.x & 31;                                                               \
    const int64_t w0_ = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;                        \
    const int64_t nw_ = ((int64_t)gridDim.x * blockDim.x) >> 5;                                       \
    for (int64_t it_ = w0_; it_ < (int64_t)cnt_ * (I).nch; it_ += nw_)                                \
        for (int cvar = (list)[1 + (int)(it_ % cnt_)], q_ = (int)(it_ / cnt_), once_ = 1; once_;      \
             once_ = 0)                                                                               \
            for (int64_t r0 = (int64_t)q_ * CHUNK, r1 = min((int64_t)(I).n, r0 + CHUNK); once_; once_ = 0)

// partial index of item (c, q), dot d: [d][c][q]
__device__ __forceinline__ size_t pidx(int d, int c, int q, int k, int nch)
{
    return ((size_t)d * k + c) * nch + q;
}

// ---------------------------------------------------------------- per-system state
struct Sys {
    double *thr, *rho, *rho_old, *alpha, *omega, *beta, *hn;
    int *active, *iters, *status, *mode, *go;
    int *lact, *lgo, *lall;  // lists
};

__device__ __forceinline__ double sum_chunks(const double* part, int d, int c, int k, int nch)
{
    double s = 0.0;
    for (int q = 0; q < nch; ++q) s += part[pidx(d, c, q, k, nch)];
    return s;
}

// ================================================================== BiCGStab
__global__ void k_bicg_init(Items I, int k, const double* __restrict__ Bs, double* x, double* r, double* rh,
                            double* p, double* v, const int* list, double* part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        double acc = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            const double b = Bs[o + i];
            x[o + i] = 0.0;
            r[o + i] = b;
            rh[o + i] = b;
            p[o + i] = 0.0;
            v[o + i] = 0.0;
            acc = fma(b, b, acc);
        }
        acc = warp_sum(acc);
        if (lane_ == 0) part[pidx(0, c, q_, k, I.nch)] = acc;
    }
}

__global__ void k_bicg_f0(int k, int nch, const double* part, Sys S)
{
    const int c = threadIdx.x;
    if (c < k) {
        const double bb = sum_chunks(part, 0, c, k, nch);
        S.iters[c] = 0;
        S.rho[c] = bb;  // r^T rhat with r = rhat = b
        S.alpha[c] = 1.0;
        S.omega[c] = 1.0;
        S.mode[c] = 1;
        S.go[c] = 0;
        if (sqrt(bb) < S.thr[c]) {
            S.active[c] = 0;
            S.status[c] = ST_OK;
        } else {
            S.active[c] = 1;
            S.status[c] = ST_MAXITER;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) build_list(k, S.active, S.lact);
}

// iteration start: count it, test rho, form beta
__global__ void k_bicg_start(int k, int maxit, Sys S)
{
    const int c = threadIdx.x;
    if (c < k && S.active[c]) {
        if (S.iters[c] >= maxit) {
            S.active[c] = 0;
            S.status[c] = ST_MAXITER;
        } else {
            S.iters[c] += 1;
            if (S.rho[c] == 0.0) {
                S.active[c] = 0;
                S.status[c] = ST_BREAKDOWN;
            } else {
                S.beta[c] = S.iters[c] == 1 ? 0.0 : (S.rho[c] / S.rho_old[c]) * (S.alpha[c] / S.omega[c]);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) build_list(k, S.active, S.lact);
}

__global__ void k_bicg_p(Items I, const double* __restrict__ r, double* p, const double* __restrict__ v, Sys S)
{
    FOR_ITEMS(I, S.lact, c, r0, r1)
    {
        const double be = S.beta[c], om = S.omega[c];
        const bool first = S.iters[c] == 1;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32)
            p[o + i] = first ? r[o + i] : r[o + i] + be * (p[o + i] - om * v[o + i]);
    }
}

// ND inner products (a0,b0), (a1,b1) over the systems of list
template <int ND>
__global__ void k_dots(Items I, int k, const double* a0, const double* b0, const double* a1, const double* b1,
                       const int* list, double* part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        double s0 = 0.0, s1 = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            s0 = fma(a0[o + i], b0[o + i], s0);
            if (ND > 1) s1 = fma(a1[o + i], b1[o + i], s1);
        }
        s0 = warp_sum(s0);
        if (ND > 1) s1 = warp_sum(s1);
        if (lane_ == 0) {
            part[pidx(0, c, q_, k, I.nch)] = s0;
            if (ND > 1) part[pidx(1, c, q_, k, I.nch)] = s1;
        }
    }
}

__global__ void k_bicg_f1(int k, int nch, const double* part, Sys S, Dims D)
{
    const int c = threadIdx.x;
    const int k1 = S.lact[0];
    if (c == 0 && k1 > 0) {
        spmm_work(D.n, D.nnzM, k1);
        spmm_work(D.n, D.nnzA, k1);
        kwork_add(PROF_BICG_VEC, 8.0 * D.n * k1 * (4 + 2), D.n * k1 * (3 + 2));  // p update, rhat^T v
    }
    if (c < k && S.active[c]) {
        const double rv = sum_chunks(part, 0, c, k, nch);
        if (rv == 0.0) {
            S.active[c] = 0;
            S.status[c] = ST_BREAKDOWN;
        } else {
            S.alpha[c] = S.rho[c] / rv;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) build_list(k, S.active, S.lact);
}

__global__ void k_bicg_s(Items I, int k, const double* __restrict__ r, const double* __restrict__ v, double* s,
                         Sys S, double* part)
{
    FOR_ITEMS(I, S.lact, c, r0, r1)
    {
        const double al = S.alpha[c];
        double acc = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            const double sv = r[o + i] - al * v[o + i];
            s[o + i] = sv;
            acc = fma(sv, sv, acc);
        }
        acc = warp_sum(acc);
        if (lane_ == 0) part[pidx(0, c, q_, k, I.nch)] = acc;
    }
}

__global__ void k_bicg_f2(int k, int nch, const double* part, Sys S, Dims D)
{
    const int c = threadIdx.x;
    const int k2 = S.lact[0];
    if (c == 0 && k2 > 0) kwork_add(PROF_BICG_VEC, 8.0 * D.n * k2 * 3, D.n * k2 * 4.0);  // s, ||s||
    if (c < k) {
        if (S.active[c]) {
            const double ss = sum_chunks(part, 0, c, k, nch);
            S.mode[c] = sqrt(ss) < S.thr[c] ? 2 : 1;
            S.go[c] = S.mode[c] == 1;
        } else {
            S.go[c] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) build_list(k, S.go, S.lgo);
}

__global__ void k_bicg_f3(int k, int nch, const double* part, Sys S, Dims D)
{
    const int c = threadIdx.x;
    const int k3 = S.lgo[0];
    if (c == 0 && k3 > 0) {
        spmm_work(D.n, D.nnzM, k3);
        spmm_work(D.n, D.nnzA, k3);
        kwork_add(PROF_BICG_VEC, 8.0 * D.n * k3 * 2, D.n * k3 * 4.0);  // t^T s, t^T t
    }
    if (c < k && S.go[c]) {
        const double ts = sum_chunks(part, 0, c, k, nch), tt = sum_chunks(part, 1, c, k, nch);
        if (tt == 0.0) {
            S.active[c] = 0;
            S.go[c] = 0;
            S.status[c] = ST_BREAKDOWN;
        } else {
            S.omega[c] = ts / tt;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) build_list(k, S.active, S.lact);
}

__global__ void k_bicg_xr(Items I, int k, double* x, double* r, const double* __restrict__ rh,
                          const double* __restrict__ ph, const double* __restrict__ sh, const double* __restrict__ s,
                          const double* __restrict__ t, Sys S, double* part)
{
    FOR_ITEMS(I, S.lact, c, r0, r1)
    {
        const double al = S.alpha[c], om = S.omega[c];
        const bool half = S.mode[c] == 2;
        double a0 = 0.0, a1 = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            double rv;
            if (half) {
                x[o + i] += al * ph[o + i];
                rv = s[o + i];
            } else {
                x[o + i] += al * ph[o + i] + om * sh[o + i];
                rv = s[o + i] - om * t[o + i];
            }
            r[o + i] = rv;
            a0 = fma(rv, rv, a0);
            a1 = fma(rh[o + i], rv, a1);
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        if (lane_ == 0) {
            part[pidx(0, c, q_, k, I.nch)] = a0;
            part[pidx(1, c, q_, k, I.nch)] = a1;
        }
    }
}

__global__ void k_bicg_f4(int k, int nch, const double* part, Sys S, Dims D, int* any_active)
{
    const int c = threadIdx.x;
    const int k4 = S.lact[0];
    if (c == 0 && k4 > 0) kwork_add(PROF_BICG_VEC, 8.0 * D.n * k4 * 8, D.n * k4 * 10.0);  // x, r, two dots
    if (c < k && S.active[c]) {
        const double rr = sum_chunks(part, 0, c, k, nch), rhr = sum_chunks(part, 1, c, k, nch);
        if (S.mode[c] == 2 || sqrt(rr) < S.thr[c]) {
            S.active[c] = 0;
            S.status[c] = ST_OK;
        } else if (S.omega[c] == 0.0) {
            S.active[c] = 0;
            S.status[c] = ST_BREAKDOWN;
        } else {
            S.rho_old[c] = S.rho[c];
            S.rho[c] = rhr;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        build_list(k, S.active, S.lact);
        *any_active = S.lact[0] > 0;
    }
}

// ================================================================== GMRES(m)
struct Gm {
    int m;
    int64_t vstride;  // k * ld: distance between basis vectors V_i
    double* V;        // (m+1) blocks of k systems
    double* H;        // k x m x (m+1): column j of system c at H[(c*m + j)*(m+1)]
    double* cs;       // k x m
    double* sn;       // k x m
    double* g;        // k x (m+1)
    double* h;        // 2 x (m+1) x k  (projection passes)
    double* u;        // k x m
    double* ww;       // k: ||w||^2 before the projection
    double* hn2;      // k: ||w||^2 after it
    int *cyc, *adv, *jd, *done, *conv, *reo;
    int *lcyc, *ladv, *lreo;  // lists
};

__global__ void k_gm_init(Items I, int k, const double* __restrict__ Bs, double* x, double* r, const int* list,
                          double* part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        double acc = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            const double b = Bs[o + i];
            x[o + i] = 0.0;
            r[o + i] = b;
            acc = fma(b, b, acc);
        }
        acc = warp_sum(acc);
        if (lane_ == 0) part[pidx(0, c, q_, k, I.nch)] = acc;
    }
}

__global__ void k_norm2(Items I, int k, const double* __restrict__ r, const int* list, double* part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        double acc = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) acc = fma(r[o + i], r[o + i], acc);
        acc = warp_sum(acc);
        if (lane_ == 0) part[pidx(0, c, q_, k, I.nch)] = acc;
    }
}

// cycle start: true residual norm, stop tests, g = beta e_1
__global__ void k_gm_cycle_start(int k, int nch, const double* part, int maxit, Sys S, Gm G, int first,
                                 int* any_cyc)
{
    const int c = threadIdx.x;
    if (c < k) {
        if (first) {
            S.iters[c] = 0;
            G.done[c] = 0;
            S.status[c] = ST_MAXITER;
        }
        G.cyc[c] = 0;
        G.adv[c] = 0;
        G.conv[c] = 0;
        G.jd[c] = 0;
        G.reo[c] = 0;
        if (!G.done[c]) {
            const double beta = sqrt(sum_chunks(part, 0, c, k, nch));
            if (beta < S.thr[c]) {
                G.done[c] = 1;
                S.status[c] = ST_OK;
            } else if (S.iters[c] >= maxit) {
                G.done[c] = 1;
                S.status[c] = ST_MAXITER;
            } else {
                G.cyc[c] = 1;
                G.adv[c] = 1;
                S.beta[c] = beta;
                for (int i = 0; i <= G.m; ++i) G.g[(size_t)c * (G.m + 1) + i] = 0.0;
                G.g[(size_t)c * (G.m + 1)] = beta;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        build_list(k, G.cyc, G.lcyc);
        build_list(k, G.adv, G.ladv);
        G.lreo[0] = 0;
        *any_cyc = G.lcyc[0] > 0;
    }
}

__global__ void k_gm_v0(Items I, const double* __restrict__ r, Sys S, Gm G)
{
    FOR_ITEMS(I, G.lcyc, c, r0, r1)
    {
        const double inv = 1.0 / S.beta[c];
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) G.V[o + i] = r[o + i] * inv;
    }
}

// Projection h_i = V_i^T w (i in [i0, i0+ni)) and ||w||^2 for the systems of
// list: each warp item keeps NI+1 accumulators in registers and streams its
// chunk of w and of the ni basis vectors once.
template <int NI>
__global__ void __launch_bounds__(IT_WARPS * 32) k_gm_proj(Items I, int k, int i0, int ni,
                                                          const double* __restrict__ w, Gm G, const int* list,
                                                          double* __restrict__ part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        double acc[NI + 1];
#pragma unroll
        for (int i = 0; i <= NI; ++i) acc[i] = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        const double* Vp = G.V + (int64_t)i0 * G.vstride + o;
        for (int64_t row = r0 + lane_; row < r1; row += 32) {
            const double wv = w[o + row];
#pragma unroll
            for (int i = 0; i < NI; ++i)
                if (i < ni) acc[i] = fma(Vp[(int64_t)i * G.vstride + row], wv, acc[i]);
            acc[NI] = fma(wv, wv, acc[NI]);
        }
#pragma unroll
        for (int i = 0; i <= NI; ++i) acc[i] = warp_sum(acc[i]);
        if (lane_ == 0) {
            double* pp = part + ((size_t)c * I.nch + q_) * (PJ + 1);
#pragma unroll
            for (int i = 0; i < NI; ++i)
                if (i < ni) pp[i] = acc[i];
            pp[PJ] = acc[NI];
        }
    }
}

// h[pass][i0+i][c] for i < ni and ww[c] from the chunk partials; one warp per
// (listed system, i); slot PJ is ||w||^2
__global__ void k_gm_fin(int k, int nch, int i0, int ni, const double* __restrict__ part, const int* list,
                         double* __restrict__ h, double* __restrict__ ww)
{
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int cnt = list[0];
    if (q >= (int64_t)cnt * (ni + 1)) return;
    const int s = (int)(q / (ni + 1)), i = (int)(q - (int64_t)s * (ni + 1));
    const int c = list[1 + s];
    const int slot = i < ni ? i : PJ;
    double sum = 0.0;
    for (int b = lane; b < nch; b += 32) sum += part[((size_t)c * nch + b) * (PJ + 1) + slot];
    sum = warp_sum(sum);
    if (lane == 0) {
        if (i < ni) h[(size_t)(i0 + i) * k + c] = sum;
        else if (ww) ww[c] = sum;
    }
}

// w -= sum_{i in chunk} V_i h_i for the systems of list; the last chunk also
// writes ||w||^2 partials (one per item)
template <int NI>
__global__ void __launch_bounds__(IT_WARPS * 32) k_gm_upd(Items I, int k, int i0, int ni, double* __restrict__ w,
                                                         Gm G, const double* __restrict__ h, const int* list,
                                                         int last, double* __restrict__ part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        double hc[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) hc[i] = i < ni ? h[(size_t)(i0 + i) * k + c] : 0.0;
        const int64_t o = (int64_t)c * I.ld;
        const double* Vp = G.V + (int64_t)i0 * G.vstride + o;
        double acc = 0.0;
        for (int64_t row = r0 + lane_; row < r1; row += 32) {
            double wv = w[o + row];
#pragma unroll
            for (int i = 0; i < NI; ++i)
                if (i < ni) wv = fma(-Vp[(int64_t)i * G.vstride + row], hc[i], wv);
            w[o + row] = wv;
            acc = fma(wv, wv, acc);
        }
        if (last) {
            acc = warp_sum(acc);
            if (lane_ == 0) part[(size_t)c * I.nch + q_] = acc;
        }
    }
}

// ||w||^2 after a projection pass (one warp per listed system). Pass 0 marks
// the systems that need a second pass: ||w_after||^2 < ||w_before||^2 / 2.
__global__ void k_gm_finnorm(int k, int nch, const double* __restrict__ part, Gm G, int pass)
{
    const int* list = pass == 0 ? G.ladv : G.lreo;
    const int cnt = list[0];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = wid; s < cnt; s += blockDim.x >> 5) {
        const int c = list[1 + s];
        double sum = 0.0;
        for (int b = lane; b < nch; b += 32) sum += part[(size_t)c * nch + b];
        sum = warp_sum(sum);
        if (lane == 0) {
            G.hn2[c] = sum;
            if (pass == 0) G.reo[c] = sum < 0.5 * G.ww[c];
        }
    }
    __syncthreads();
    if (pass == 0 && threadIdx.x == 0) {
        int q = 0;
        for (int s = 0; s < cnt; ++s) {
            const int c = list[1 + s];
            if (G.reo[c]) G.lreo[1 + q++] = c;
        }
        G.lreo[0] = q;
    }
}

// H(:,j) = h0 (+ h1), ||w||, Givens rotations, residual estimate, stop tests
__global__ void k_gm_givens(int k, int j, int maxit, Sys S, Gm G, Dims D, int* any_adv)
{
    const int c = threadIdx.x;
    if (c == 0) {
        const int ka = G.ladv[0], kr = G.lreo[0];
        if (ka > 0) {
            spmm_work(D.n, D.nnzM, ka);
            spmm_work(D.n, D.nnzA, ka);
            const double p = (double)(ka + kr);  // projection passes
            kwork_add(PROF_GM_DOTS, 8.0 * D.n * p * (j + 2), D.n * p * (2.0 * (j + 1) + 2.0));
            kwork_add(PROF_GM_UPDATE, 8.0 * D.n * p * (j + 3), D.n * p * (2.0 * (j + 1) + 2.0));
        }
    }
    if (c < k && G.adv[c]) {
        const int m = G.m;
        double* Hc = G.H + ((size_t)c * m + j) * (m + 1);
        const bool two = G.reo[c] != 0;
        for (int i = 0; i <= j; ++i)
            Hc[i] = G.h[(size_t)i * k + c] + (two ? G.h[((size_t)(m + 1) + i) * k + c] : 0.0);
        const double hn = sqrt(G.hn2[c]);
        Hc[j + 1] = hn;
        S.hn[c] = hn;
        double* csc = G.cs + (size_t)c * m;
        double* snc = G.sn + (size_t)c * m;
        for (int i = 0; i < j; ++i) {
            const double a = Hc[i], b = Hc[i + 1];
            Hc[i] = csc[i] * a + snc[i] * b;
            Hc[i + 1] = -snc[i] * a + csc[i] * b;
        }
        const double a = Hc[j], b = Hc[j + 1];
        const double den = sqrt(a * a + b * b);
        if (den == 0.0) {
            csc[j] = 1.0;
            snc[j] = 0.0;
        } else {
            csc[j] = a / den;
            snc[j] = b / den;
        }
        Hc[j] = csc[j] * a + snc[j] * b;
        Hc[j + 1] = 0.0;
        double* gc = G.g + (size_t)c * (m + 1);
        gc[j + 1] = -snc[j] * gc[j];
        gc[j] = csc[j] * gc[j];
        S.iters[c] += 1;
        G.jd[c] = j + 1;
        if (fabs(gc[j + 1]) < S.thr[c]) {
            G.adv[c] = 0;
            G.conv[c] = 1;
        } else if (S.iters[c] >= maxit) {
            G.adv[c] = 0;
        }
    }
    __syncthreads();
    if (c < k) G.reo[c] = 0;
    if (threadIdx.x == 0) {
        build_list(k, G.adv, G.ladv);
        G.lreo[0] = 0;
        *any_adv = G.ladv[0] > 0;
    }
}

__global__ void k_gm_normalize(Items I, int j, const double* __restrict__ w, Sys S, Gm G)
{
    FOR_ITEMS(I, G.ladv, c, r0, r1)
    {
        const double hn = S.hn[c];
        const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
        const int64_t o = (int64_t)c * I.ld;
        double* Vn = G.V + (int64_t)(j + 1) * G.vstride + o;
        for (int64_t i = r0 + lane_; i < r1; i += 32) Vn[i] = w[o + i] * inv;
    }
}

// u = H(0:jd,0:jd)^{-1} g(0:jd) per system (upper triangular)
__global__ void k_gm_trisolve(int k, Sys S, Gm G)
{
    const int c = threadIdx.x;
    if (c < k && G.cyc[c]) {
        const int m = G.m, jd = G.jd[c];
        const double* gc = G.g + (size_t)c * (m + 1);
        double* uc = G.u + (size_t)c * m;
        for (int i = 0; i < m; ++i) uc[i] = 0.0;
        for (int i = jd - 1; i >= 0; --i) {
            double t = gc[i];
            for (int q = i + 1; q < jd; ++q) t -= G.H[((size_t)c * m + q) * (m + 1) + i] * uc[q];
            const double d = G.H[((size_t)c * m + i) * (m + 1) + i];
            if (d == 0.0) {
                S.status[c] = ST_BREAKDOWN;
                G.done[c] = 1;
                G.cyc[c] = 0;
                for (int q = 0; q < m; ++q) uc[q] = 0.0;
                break;
            }
            uc[i] = t / d;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) build_list(k, G.cyc, G.lcyc);
}

// w = V u per system (the caller forms z = M w and x += z)
__global__ void k_gm_combine(Items I, double* w, Gm G)
{
    FOR_ITEMS(I, G.lcyc, c, r0, r1)
    {
        const int jd = G.jd[c];
        const double* uc = G.u + (size_t)c * G.m;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            double s = 0.0;
            for (int q = 0; q < jd; ++q) s = fma(G.V[(int64_t)q * G.vstride + o + i], uc[q], s);
            w[o + i] = s;
        }
    }
}

__global__ void k_gm_xadd(Items I, double* x, const double* __restrict__ z, Gm G)
{
    FOR_ITEMS(I, G.lcyc, c, r0, r1)
    {
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) x[o + i] += z[o + i];
    }
}

// end of a cycle: converged systems are done; a system that used its last
// iteration inside the cycle ends with MAXITER; the rest need a residual
__global__ void k_gm_cycle_end(int k, int maxit, Sys S, Gm G, int* any_left)
{
    const int c = threadIdx.x;
    if (c < k) {
        if (G.cyc[c] && G.conv[c]) {
            G.done[c] = 1;
            S.status[c] = ST_OK;
        } else if (G.cyc[c] && S.iters[c] >= maxit) {
            G.done[c] = 1;
            S.status[c] = ST_MAXITER;
        }
        G.cyc[c] = !G.done[c];  // reused as "needs a residual"
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        build_list(k, G.cyc, G.lcyc);
        *any_left = G.lcyc[0] > 0;
    }
}

__global__ void k_list_all(int k, int* list)
{
    if (threadIdx.x == 0) {
        for (int c = 0; c < k; ++c) list[1 + c] = c;
        list[0] = k;
    }
}

// ---------------------------------------------------------------- host helpers
template <int NI>
void proj_t(const Items& I, int k, int i0, int ni, const double* w, const Gm& G, const int* list, double* part,
            cudaStream_t st)
{
    k_gm_proj<NI><<<SAI_GRID(item_blocks(I.n, k)), IT_WARPS * 32, 0, st>>>(I, k, i0, ni, w, G, list, part);
}

template <int NI>
void upd_t(const Items& I, int k, int i0, int ni, double* w, const Gm& G, const double* h, const int* list, int last,
           double* part, cudaStream_t st)
{
    k_gm_upd<NI><<<SAI_GRID(item_blocks(I.n, k)), IT_WARPS * 32, 0, st>>>(I, k, i0, ni, w, G, h, list, last, part);
}

// One classical Gram-Schmidt pass of w against V_0..V_j for the systems of list.
void cgs_pass(const Items& I, int k, int j, int pass, double* w, const Gm& G, const int* list, double* part,
              double* part2, cudaStream_t st)
{
    double* h = G.h + (size_t)pass * (G.m + 1) * k;
    for (int i0 = 0; i0 <= j; i0 += PJ) {
        const int ni = (j + 1 - i0) < PJ ? (j + 1 - i0) : PJ;
        {
            ProfScope ps(PROF_GM_DOTS, st);
            if (ni <= 8) proj_t<8>(I, k, i0, ni, w, G, list, part, st);
            else if (ni <= 16) proj_t<16>(I, k, i0, ni, w, G, list, part, st);
            else proj_t<32>(I, k, i0, ni, w, G, list, part, st);
        }
        const int64_t warps = (int64_t)k * (ni + 1);
        k_gm_fin<<<SAI_GRID(sai_div_up(warps * 32, 256)), 256, 0, st>>>(k, I.nch, i0, ni, part, list, h,
                                                                       (i0 == 0 && pass == 0) ? G.ww : nullptr);
    }
    for (int i0 = 0; i0 <= j; i0 += PJ) {
        const int ni = (j + 1 - i0) < PJ ? (j + 1 - i0) : PJ;
        const int last = (i0 + PJ > j) ? 1 : 0;
        ProfScope ps(PROF_GM_UPDATE, st);
        if (ni <= 8) upd_t<8>(I, k, i0, ni, w, G, h, list, last, part2, st);
        else if (ni <= 16) upd_t<16>(I, k, i0, ni, w, G, h, list, last, part2, st);
        else upd_t<32>(I, k, i0, ni, w, G, h, list, last, part2, st);
    }
    k_gm_finnorm<<<SAI_GRID(1), 1024, 0, st>>>(k, I.nch, part2, G, pass);
}

}  // namespace

sai_status sai_krylov_run(const sai_split_s* h, const sai_precond_s* P, int32_t k, const double* B,
                          const double* thr, const sai_krylov_params* prm, double* X, int32_t* iters,
                          int32_t* status, cudaStream_t st)
{
    if (!h || !P || !prm || !thr || !iters || !status || k < 1 || k > CTRL) return SAI_INVALID_ARG;
    if (prm->maxit < 0 || (prm->method == SAI_GMRES && prm->restart < 1)) return SAI_INVALID_ARG;
    if (prm->method != SAI_BICGSTAB && prm->method != SAI_GMRES) return SAI_INVALID_ARG;
    const int32_t n = h->n;
    if (n > 0 && (!B || !X)) return SAI_INVALID_ARG;
    if (g_sms == 0) {
        int dev = 0;
        SAI_CUDA(cudaGetDevice(&dev));
        SAI_CUDA(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int64_t ld = ((int64_t)n + 31) / 32 * 32;
    const size_t blk = (size_t)ld * k;  // one system-major block of k vectors
    Items I;
    I.n = n;
    I.ld = ld;
    I.nch = nchunks(n > 0 ? n : 1);
    const int ib = item_blocks(n > 0 ? n : 1, k);
    const int64_t* Ar = h->Atr_rp.as<int64_t>();
    const int32_t* Ac = h->Atr_ci.as<int32_t>();
    const double* Av = h->Atr_v.as<double>();
    const int64_t* Mr = P->Mr_rp.as<int64_t>();
    const int32_t* Mc = P->Mr_ci.as<int32_t>();
    const double* Mv = P->Mr_v.as<double>();
    int64_t tg = sai_div_up((int64_t)n * k > 0 ? (int64_t)n * k : 1, 256);
    if (tg > (int64_t)g_sms * 8) tg = (int64_t)g_sms * 8;
    const int tgrid = (int)tg;

    Buf sysd, sysi, part, part2, flag, Bs, Xs;
    SAI_TRY(sysd.alloc(sizeof(double) * 7 * k, st, true));
    SAI_TRY(sysi.alloc(sizeof(int) * (5 * k + 3 * (k + 1)), st, true));
    SAI_TRY(part.alloc(sizeof(double) * (size_t)k * I.nch * (PJ + 1), st, true));
    SAI_TRY(part2.alloc(sizeof(double) * (size_t)k * I.nch * 2, st, true));
    SAI_TRY(flag.alloc(sizeof(int) * 4, st, true));
    SAI_TRY(Bs.alloc(sizeof(double) * blk + 8, st, true));
    SAI_TRY(Xs.alloc(sizeof(double) * blk + 8, st, true));
    Sys S;
    double* d = sysd.as<double>();
    S.thr = d;
    S.rho = d + k;
    S.rho_old = d + 2 * k;
    S.alpha = d + 3 * k;
    S.omega = d + 4 * k;
    S.beta = d + 5 * k;
    S.hn = d + 6 * k;
    int* ii = sysi.as<int>();
    S.active = ii;
    S.iters = ii + k;
    S.status = ii + 2 * k;
    S.mode = ii + 3 * k;
    S.go = ii + 4 * k;
    S.lact = ii + 5 * k;
    S.lgo = S.lact + (k + 1);
    S.lall = S.lgo + (k + 1);
    SAI_CUDA(cudaMemcpyAsync(S.thr, thr, sizeof(double) * k, cudaMemcpyHostToDevice, st));
    SAI_CUDA(cudaMemsetAsync(ii, 0, sizeof(int) * (5 * k + 3 * (k + 1)), st));
    SAI_CUDA(cudaMemsetAsync(Bs.p, 0, sizeof(double) * blk, st));
    SAI_CUDA(cudaMemsetAsync(Xs.p, 0, sizeof(double) * blk, st));
    int* fl = flag.as<int>();
    int hflag = 0;
    Dims D;
    D.n = (double)n;
    D.nnzA = (double)h->nnz_At;
    D.nnzM = (double)P->nnz;
    const int check_every = 4;
    double* Bsd = Bs.as<double>();
    double* Xsd = Xs.as<double>();
    if (n > 0) k_to_soa<<<SAI_GRID(tgrid), 256, 0, st>>>(n, k, ld, B, Bsd);
    k_list_all<<<SAI_GRID(1), 32, 0, st>>>(k, S.lall);
    SAI_CUDA(cudaGetLastError());

    if (prm->method == SAI_BICGSTAB) {
        Buf vecs;
        SAI_TRY(vecs.alloc(sizeof(double) * blk * 8 + 8, st, true));
        SAI_CUDA(cudaMemsetAsync(vecs.p, 0, sizeof(double) * blk * 8, st));
        double* r = vecs.as<double>();
        double* rh = r + blk;
        double* p = rh + blk;
        double* v = p + blk;
        double* ph = v + blk;
        double* s = ph + blk;
        double* sh = s + blk;
        double* t = sh + blk;
        double* pt = part.as<double>();
        const int nch = I.nch;
        k_bicg_init<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Bsd, Xsd, r, rh, p, v, S.lall, pt);
        k_bicg_f0<<<SAI_GRID(1), CTRL, 0, st>>>(k, nch, pt, S);
        SAI_CUDA(cudaGetLastError());
        for (int it = 0; it < prm->maxit; ++it) {
            k_bicg_start<<<SAI_GRID(1), CTRL, 0, st>>>(k, prm->maxit, S);
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_bicg_p<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, r, p, v, S);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<0>(n, ld, Mr, Mc, Mv, k, p, ph, nullptr, S.lact, st);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<0>(n, ld, Ar, Ac, Av, k, ph, v, nullptr, S.lact, st);
            }
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_dots<1><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, rh, v, nullptr, nullptr, S.lact, pt);
            }
            k_bicg_f1<<<SAI_GRID(1), CTRL, 0, st>>>(k, nch, pt, S, D);
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_bicg_s<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, r, v, s, S, pt);
            }
            k_bicg_f2<<<SAI_GRID(1), CTRL, 0, st>>>(k, nch, pt, S, D);
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<0>(n, ld, Mr, Mc, Mv, k, s, sh, nullptr, S.lgo, st);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<0>(n, ld, Ar, Ac, Av, k, sh, t, nullptr, S.lgo, st);
            }
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_dots<2><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, t, s, t, t, S.lgo, pt);
            }
            k_bicg_f3<<<SAI_GRID(1), CTRL, 0, st>>>(k, nch, pt, S, D);
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_bicg_xr<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Xsd, r, rh, ph, sh, s, t, S, pt);
            }
            k_bicg_f4<<<SAI_GRID(1), CTRL, 0, st>>>(k, nch, pt, S, D, fl);
            SAI_CUDA(cudaGetLastError());
            if ((it + 1) % check_every == 0 || it + 1 == prm->maxit) {
                SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
                SAI_CUDA(cudaStreamSynchronize(st));
                if (!hflag) break;
            }
        }
        // systems still active after maxit passes
        k_bicg_start<<<SAI_GRID(1), CTRL, 0, st>>>(k, prm->maxit, S);
    } else {
        const int m = prm->restart;
        Gm G;
        G.m = m;
        G.vstride = (int64_t)blk;
        Buf vb, hb, ibuf, wb;
        SAI_TRY(vb.alloc(sizeof(double) * blk * (m + 1) + 8, st, true));
        SAI_TRY(wb.alloc(sizeof(double) * blk * 3 + 8, st, true));
        SAI_CUDA(cudaMemsetAsync(wb.p, 0, sizeof(double) * blk * 3, st));
        const size_t hsz = (size_t)k * (m + 1) * m + 2 * (size_t)k * m + (size_t)k * (m + 1) +
                           2 * (size_t)(m + 1) * k + (size_t)k * m + 2 * (size_t)k;
        SAI_TRY(hb.alloc(sizeof(double) * hsz, st, true));
        SAI_TRY(ibuf.alloc(sizeof(int) * (6 * k + 3 * (k + 1)), st, true));
        SAI_CUDA(cudaMemsetAsync(hb.p, 0, sizeof(double) * hsz, st));
        G.V = vb.as<double>();
        double* hp = hb.as<double>();
        G.H = hp;
        hp += (size_t)k * (m + 1) * m;
        G.cs = hp;
        hp += (size_t)k * m;
        G.sn = hp;
        hp += (size_t)k * m;
        G.g = hp;
        hp += (size_t)k * (m + 1);
        G.h = hp;
        hp += 2 * (size_t)(m + 1) * k;
        G.u = hp;
        hp += (size_t)k * m;
        G.ww = hp;
        G.hn2 = hp + k;
        int* ip = ibuf.as<int>();
        G.cyc = ip;
        G.adv = ip + k;
        G.jd = ip + 2 * k;
        G.done = ip + 3 * k;
        G.conv = ip + 4 * k;
        G.reo = ip + 5 * k;
        G.lcyc = ip + 6 * k;
        G.ladv = G.lcyc + (k + 1);
        G.lreo = G.ladv + (k + 1);
        SAI_CUDA(cudaMemsetAsync(ip, 0, sizeof(int) * (6 * k + 3 * (k + 1)), st));
        double* r = wb.as<double>();
        double* w = r + blk;
        double* z = w + blk;
        double* pt = part.as<double>();
        double* pt2 = part2.as<double>();
        k_gm_init<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Bsd, Xsd, r, S.lall, pt2);
        int first = 1;
        for (;;) {
            k_gm_cycle_start<<<SAI_GRID(1), CTRL, 0, st>>>(k, I.nch, pt2, prm->maxit, S, G, first, fl);
            first = 0;
            SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            if (!hflag) break;
            k_gm_v0<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, r, S, G);
            for (int j = 0; j < m; ++j) {
                const double* vj = G.V + (size_t)j * blk;
                {
                    ProfScope ps(PROF_SPMM, st);
                    spmv<0>(n, ld, Mr, Mc, Mv, k, vj, z, nullptr, G.ladv, st);
                }
                {
                    ProfScope ps(PROF_SPMM, st);
                    spmv<0>(n, ld, Ar, Ac, Av, k, z, w, nullptr, G.ladv, st);
                }
                cgs_pass(I, k, j, 0, w, G, G.ladv, pt, pt2, st);
                cgs_pass(I, k, j, 1, w, G, G.lreo, pt, pt2, st);
                k_gm_givens<<<SAI_GRID(1), CTRL, 0, st>>>(k, j, prm->maxit, S, G, D, fl);
                k_gm_normalize<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, j, w, S, G);
                SAI_CUDA(cudaGetLastError());
                if ((j + 1) % check_every == 0 || j + 1 == m) {
                    SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
                    SAI_CUDA(cudaStreamSynchronize(st));
                    if (!hflag) break;
                }
            }
            k_gm_trisolve<<<SAI_GRID(1), CTRL, 0, st>>>(k, S, G);
            k_gm_combine<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, w, G);
            spmv<0>(n, ld, Mr, Mc, Mv, k, w, z, nullptr, G.lcyc, st);
            k_gm_xadd<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, Xsd, z, G);
            k_gm_cycle_end<<<SAI_GRID(1), CTRL, 0, st>>>(k, prm->maxit, S, G, fl);
            spmv<1>(n, ld, Ar, Ac, Av, k, Xsd, r, Bsd, G.lcyc, st);
            k_norm2<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, r, G.lcyc, pt2);
            SAI_CUDA(cudaGetLastError());
        }
    }
    if (n > 0) k_from_soa<<<SAI_GRID(tgrid), 256, 0, st>>>(n, k, ld, Xsd, X);
    SAI_CUDA(cudaGetLastError());
    SAI_CUDA(cudaMemcpyAsync(iters, S.iters, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaMemcpyAsync(status, S.status, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    sai_status worst = SAI_OK;
    for (int c = 0; c < k; ++c)
        if (status[c] != SAI_OK && worst == SAI_OK) worst = (sai_status)status[c];
    return worst;
}

sai_status sai_krylov_work_reset()
{
    double z[PROF_NSITES * 2] = {};
    SAI_CUDA(cudaMemcpyToSymbol(d_kwork, z, sizeof(z)));
    return SAI_OK;
}

sai_status sai_krylov_work_read(double* out)
{
    SAI_CUDA(cudaMemcpyFromSymbol(out, d_kwork, sizeof(double) * PROF_NSITES * 2));
    return SAI_OK;
}
