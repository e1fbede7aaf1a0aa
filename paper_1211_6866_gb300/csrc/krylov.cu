// krylov.cu -- the s+1 right-preconditioned Krylov solves of Procedure *
// (A~ y = b, A~ w_j = u_j, eqs. (regprob), (auxi)) for k right-hand sides at
// once. Every operator application is one SpMM over the n x k row-major block
// (all systems share A~ and M); every inner product is a per-system
// reduction with fixed-order partial sums (deterministic). Each system keeps
// its own scalars, iteration count, stop threshold and status on the device;
// a converged system is frozen (masked out of the SpMMs and updates).
//
// BiCGStab: van der Vorst's recurrence on A~ M z = b with y = M z updated
// directly; stop tests after the half step (s) and the full step (r).
// GMRES(m): Arnoldi with classical Gram-Schmidt applied twice (CGS2), Givens
// rotations, stop on the rotated residual |g_{j+1}|, restart from the true
// residual b - A~ y.
#include <math.h>

#include "internal.h"

namespace {

constexpr int KT = 256;  // threads per block of the row x system kernels

// thread -> (row offset tr, system c), RB rows per block step
struct RC {
    int RB, tr, c;
    bool ok;
};
__device__ __forceinline__ RC rowc(int k)
{
    RC r;
    r.RB = KT / k;
    r.tr = threadIdx.x / k;
    r.c = threadIdx.x - r.tr * k;
    r.ok = r.tr < r.RB;
    return r;
}

int kblocks(int64_t n, int k)
{
    int RB = KT / k;
    int64_t b = (n + RB - 1) / RB;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

// Writes the block's per-system sums of v[0..ND) to part[d][blockIdx][c].
template <int ND>
__device__ __forceinline__ void block_partials(const double (&v)[ND], const RC& rc, int k, double* part)
{
    __shared__ double sh[ND][KT];
#pragma unroll
    for (int d = 0; d < ND; ++d) sh[d][threadIdx.x] = rc.ok ? v[d] : 0.0;
    __syncthreads();
    if (threadIdx.x < k) {
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            double s = 0.0;
            for (int q = 0; q < rc.RB; ++q) s += sh[d][q * k + threadIdx.x];
            part[((size_t)d * gridDim.x + blockIdx.x) * k + threadIdx.x] = s;
        }
    }
}

__device__ __forceinline__ double fin(const double* part, int d, int nblk, int k, int c)
{
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[((size_t)d * nblk + b) * k + c];
    return s;
}

// ------------------------------------------------------------------ masked SpMM
template <int G, int MODE>
__global__ void __launch_bounds__(256) k_spmm_m(int32_t n, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ ci, const double* __restrict__ v, int32_t k,
                                                const double* __restrict__ X, double* __restrict__ Y,
                                                const double* __restrict__ B, const int* __restrict__ mask)
{
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, c0 = lane % G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row0 = warp * RPW; row0 < n; row0 += nwarps * RPW) {
        const int64_t row = row0 + sub;
        if (row >= n) continue;
        const int64_t b = rp[row], e = rp[row + 1];
        for (int c = c0; c < k; c += G) {
            if (mask && !mask[c]) continue;
            double acc = 0.0;
            for (int64_t t = b; t < e; ++t) acc = fma(v[t], X[(int64_t)ci[t] * k + c], acc);
            if (MODE == 0) Y[row * k + c] = acc;
            else Y[row * k + c] = B[row * k + c] - acc;
        }
    }
}

template <int MODE>
void spmm_m(int32_t n, const int64_t* rp, const int32_t* ci, const double* v, int32_t k, const double* X, double* Y,
            const double* B, const int* mask, cudaStream_t st)
{
    int G = 1;
    while (G < k && G < 32) G <<= 1;
    const int rpw = 32 / G;
    int64_t warps = (n + rpw - 1) / rpw;
    int64_t blocks = (warps * 32 + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    const unsigned g = (unsigned)blocks;
    switch (G) {
    case 1: k_spmm_m<1, MODE><<<SAI_GRID(g), 256, 0, st>>>(n, rp, ci, v, k, X, Y, B, mask); break;
    case 2: k_spmm_m<2, MODE><<<SAI_GRID(g), 256, 0, st>>>(n, rp, ci, v, k, X, Y, B, mask); break;
    case 4: k_spmm_m<4, MODE><<<SAI_GRID(g), 256, 0, st>>>(n, rp, ci, v, k, X, Y, B, mask); break;
    case 8: k_spmm_m<8, MODE><<<SAI_GRID(g), 256, 0, st>>>(n, rp, ci, v, k, X, Y, B, mask); break;
    case 16: k_spmm_m<16, MODE><<<SAI_GRID(g), 256, 0, st>>>(n, rp, ci, v, k, X, Y, B, mask); break;
    default: k_spmm_m<32, MODE><<<SAI_GRID(g), 256, 0, st>>>(n, rp, ci, v, k, X, Y, B, mask); break;
    }
}

// ------------------------------------------------------------------ shared state
struct Sys {  // per-system state, arrays of k
    double *thr, *rho, *rho_old, *alpha, *omega, *beta, *hn;
    int *active, *iters, *status, *mode, *go;
};

enum { ST_OK = 0, ST_MAXITER = 5, ST_BREAKDOWN = 6 };  // same values as sai_status

// Algorithmic work of the profiled sites, accumulated by the single-block
// finalize kernels from the number of systems that took part in each launch.
__device__ double d_kwork[PROF_NSITES * 2];

struct Dims {  // sizes for the work accounting
    double n, nnzA, nnzM;
};

__device__ __forceinline__ void kwork_add(int site, double bytes, double flops)
{
    atomicAdd(&d_kwork[2 * site], bytes);
    atomicAdd(&d_kwork[2 * site + 1], flops);
}

// one SpMM launch over the k_act unmasked systems: matrix once, X read once, Y written
__device__ __forceinline__ void spmm_work(double n, double nnz, int kact)
{
    if (kact > 0) kwork_add(PROF_SPMM, 8.0 * (n + 1) + 12.0 * nnz + 16.0 * n * kact, 2.0 * nnz * kact);
}

// ================================================================== BiCGStab
__global__ void k_bicg_init(int64_t n, int k, const double* B, double* x, double* r, double* rh, double* p,
                            double* v, double* part)
{
    const RC rc = rowc(k);
    double acc[1] = {0.0};
    if (rc.ok)
        for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
            const int64_t e = row * k + rc.c;
            const double b = B[e];
            x[e] = 0.0;
            r[e] = b;
            rh[e] = b;
            p[e] = 0.0;
            v[e] = 0.0;
            acc[0] = fma(b, b, acc[0]);
        }
    block_partials<1>(acc, rc, k, part);
}

__global__ void k_bicg_f0(int k, int nblk, const double* part, Sys S)
{
    const int c = threadIdx.x;
    if (c >= k) return;
    const double bb = fin(part, 0, nblk, k, c);
    S.iters[c] = 0;
    S.rho[c] = bb;  // r^T rhat with r = rhat = b
    S.alpha[c] = 1.0;
    S.omega[c] = 1.0;
    if (sqrt(bb) < S.thr[c]) {
        S.active[c] = 0;
        S.status[c] = ST_OK;
    } else {
        S.active[c] = 1;
        S.status[c] = ST_MAXITER;
    }
}

// iteration start: count it, test rho, form beta
__global__ void k_bicg_start(int k, int maxit, Sys S)
{
    const int c = threadIdx.x;
    if (c >= k || !S.active[c]) return;
    if (S.iters[c] >= maxit) {
        S.active[c] = 0;
        S.status[c] = ST_MAXITER;
        return;
    }
    S.iters[c] += 1;
    if (S.rho[c] == 0.0) {
        S.active[c] = 0;
        S.status[c] = ST_BREAKDOWN;
        return;
    }
    S.beta[c] = S.iters[c] == 1 ? 0.0 : (S.rho[c] / S.rho_old[c]) * (S.alpha[c] / S.omega[c]);
}

__global__ void k_bicg_p(int64_t n, int k, const double* r, double* p, const double* v, Sys S)
{
    const RC rc = rowc(k);
    if (!rc.ok || !S.active[rc.c]) return;
    const double be = S.beta[rc.c], om = S.omega[rc.c];
    const bool first = S.iters[rc.c] == 1;
    for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
        const int64_t e = row * k + rc.c;
        p[e] = first ? r[e] : r[e] + be * (p[e] - om * v[e]);
    }
}

__global__ void k_dot1(int64_t n, int k, const double* a, const double* b, const int* mask, double* part)
{
    const RC rc = rowc(k);
    double acc[1] = {0.0};
    if (rc.ok && mask[rc.c])
        for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
            const int64_t e = row * k + rc.c;
            acc[0] = fma(a[e], b[e], acc[0]);
        }
    block_partials<1>(acc, rc, k, part);
}

__global__ void k_bicg_f1(int k, int nblk, const double* part, Sys S, Dims D)
{
    const int c = threadIdx.x;
    const int k1 = __syncthreads_count(c < k && S.active[c]);
    if (c == 0 && k1 > 0) {
        spmm_work(D.n, D.nnzM, k1);
        spmm_work(D.n, D.nnzA, k1);
        kwork_add(PROF_BICG_VEC, 8.0 * D.n * k1 * (4 + 2), D.n * k1 * (3 + 2));  // p update, r^T v
    }
    if (c >= k || !S.active[c]) return;
    const double rv = fin(part, 0, nblk, k, c);
    if (rv == 0.0) {
        S.active[c] = 0;
        S.status[c] = ST_BREAKDOWN;
        return;
    }
    S.alpha[c] = S.rho[c] / rv;
}

__global__ void k_bicg_s(int64_t n, int k, const double* r, const double* v, double* s, Sys S, double* part)
{
    const RC rc = rowc(k);
    double acc[1] = {0.0};
    if (rc.ok && S.active[rc.c]) {
        const double al = S.alpha[rc.c];
        for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
            const int64_t e = row * k + rc.c;
            const double sv = r[e] - al * v[e];
            s[e] = sv;
            acc[0] = fma(sv, sv, acc[0]);
        }
    }
    block_partials<1>(acc, rc, k, part);
}

__global__ void k_bicg_f2(int k, int nblk, const double* part, Sys S, Dims D)
{
    const int c = threadIdx.x;
    const int k2 = __syncthreads_count(c < k && S.active[c]);
    if (c == 0 && k2 > 0) kwork_add(PROF_BICG_VEC, 8.0 * D.n * k2 * 3, D.n * k2 * 4.0);  // s = r - alpha v, ||s||
    if (c >= k) return;
    if (!S.active[c]) {
        S.go[c] = 0;
        return;
    }
    const double ss = fin(part, 0, nblk, k, c);
    S.mode[c] = sqrt(ss) < S.thr[c] ? 2 : 1;
    S.go[c] = S.mode[c] == 1;
}

__global__ void k_dot2(int64_t n, int k, const double* t, const double* s, const int* mask, double* part)
{
    const RC rc = rowc(k);
    double acc[2] = {0.0, 0.0};
    if (rc.ok && mask[rc.c])
        for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
            const int64_t e = row * k + rc.c;
            acc[0] = fma(t[e], s[e], acc[0]);
            acc[1] = fma(t[e], t[e], acc[1]);
        }
    block_partials<2>(acc, rc, k, part);
}

__global__ void k_bicg_f3(int k, int nblk, const double* part, Sys S, Dims D)
{
    const int c = threadIdx.x;
    const int k3 = __syncthreads_count(c < k && S.go[c]);
    if (c == 0 && k3 > 0) {
        spmm_work(D.n, D.nnzM, k3);
        spmm_work(D.n, D.nnzA, k3);
        kwork_add(PROF_BICG_VEC, 8.0 * D.n * k3 * 2, D.n * k3 * 4.0);  // t^T s, t^T t
    }
    if (c >= k || !S.go[c]) return;
    const double ts = fin(part, 0, nblk, k, c), tt = fin(part, 1, nblk, k, c);
    if (tt == 0.0) {
        S.active[c] = 0;
        S.go[c] = 0;
        S.status[c] = ST_BREAKDOWN;
        return;
    }
    S.omega[c] = ts / tt;
}

__global__ void k_bicg_xr(int64_t n, int k, double* x, double* r, const double* rh, const double* ph,
                          const double* sh, const double* s, const double* t, Sys S, double* part)
{
    const RC rc = rowc(k);
    double acc[2] = {0.0, 0.0};
    if (rc.ok && S.active[rc.c]) {
        const double al = S.alpha[rc.c], om = S.omega[rc.c];
        const bool half = S.mode[rc.c] == 2;
        for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
            const int64_t e = row * k + rc.c;
            double rv;
            if (half) {
                x[e] += al * ph[e];
                rv = s[e];
            } else {
                x[e] += al * ph[e] + om * sh[e];
                rv = s[e] - om * t[e];
            }
            r[e] = rv;
            acc[0] = fma(rv, rv, acc[0]);
            acc[1] = fma(rh[e], rv, acc[1]);
        }
    }
    block_partials<2>(acc, rc, k, part);
}

__global__ void k_bicg_f4(int k, int nblk, const double* part, Sys S, Dims D, int* any_active)
{
    const int c = threadIdx.x;
    const int k4 = __syncthreads_count(c < k && S.active[c]);
    if (c == 0 && k4 > 0) kwork_add(PROF_BICG_VEC, 8.0 * D.n * k4 * 8, D.n * k4 * 10.0);  // x, r, two dots
    int act = 0;
    if (c < k && S.active[c]) {
        const double rr = fin(part, 0, nblk, k, c), rhr = fin(part, 1, nblk, k, c);
        if (S.mode[c] == 2 || sqrt(rr) < S.thr[c]) {
            S.active[c] = 0;
            S.status[c] = ST_OK;
        } else if (S.omega[c] == 0.0) {
            S.active[c] = 0;
            S.status[c] = ST_BREAKDOWN;
        } else {
            S.rho_old[c] = S.rho[c];
            S.rho[c] = rhr;
            act = 1;
        }
    }
    act = __syncthreads_or(act);
    if (threadIdx.x == 0) *any_active = act;
}

// ================================================================== GMRES(m)
struct Gm {
    int m;
    double* V;     // (m+1) blocks of n x k
    double* H;     // k x (m+1) x m, column j of system c at H[(c*m + j)*(m+1)]
    double* cs;    // k x m
    double* sn;    // k x m
    double* g;     // k x (m+1)
    double* h;     // 2 x (m+1) x k  (CGS passes)
    double* u;     // k x m
    int *cyc, *adv, *jd, *done, *conv;
};

__global__ void k_gm_init(int64_t n, int k, const double* B, double* x, double* r, double* part)
{
    const RC rc = rowc(k);
    double acc[1] = {0.0};
    if (rc.ok)
        for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
            const int64_t e = row * k + rc.c;
            x[e] = 0.0;
            r[e] = B[e];
            acc[0] = fma(B[e], B[e], acc[0]);
        }
    block_partials<1>(acc, rc, k, part);
}

__global__ void k_norm2(int64_t n, int k, const double* r, const int* mask, double* part)
{
    const RC rc = rowc(k);
    double acc[1] = {0.0};
    if (rc.ok && (!mask || mask[rc.c]))
        for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
            const int64_t e = row * k + rc.c;
            acc[0] = fma(r[e], r[e], acc[0]);
        }
    block_partials<1>(acc, rc, k, part);
}

// cycle start: true residual norm, stop tests, g = beta e_1
__global__ void k_gm_cycle_start(int k, int nblk, const double* part, int maxit, Sys S, Gm G, int first,
                                 int* any_cyc)
{
    const int c = threadIdx.x;
    int act = 0;
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
        if (!G.done[c]) {
            const double beta = sqrt(fin(part, 0, nblk, k, c));
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
                act = 1;
            }
        }
    }
    act = __syncthreads_or(act);
    if (threadIdx.x == 0) *any_cyc = act;
}

__global__ void k_gm_v0(int64_t n, int k, const double* r, Sys S, Gm G)
{
    const RC rc = rowc(k);
    if (!rc.ok || !G.cyc[rc.c]) return;
    const double inv = 1.0 / S.beta[rc.c];
    for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
        const int64_t e = row * k + rc.c;
        G.V[e] = r[e] * inv;
    }
}

// partial[i][blk][c] = sum_rows V_i(row,c) w(row,c), i = 0..j
__global__ void k_gm_dots(int64_t n, int k, int j, const double* w, Gm G, double* part)
{
    const RC rc = rowc(k);
    __shared__ double sh[KT];
    const bool on = rc.ok && G.adv[rc.c];
    const size_t blk = (size_t)n * k;
    for (int i = 0; i <= j; ++i) {
        double acc = 0.0;
        if (on) {
            const double* Vi = G.V + (size_t)i * blk;
            for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
                const int64_t e = row * k + rc.c;
                acc = fma(Vi[e], w[e], acc);
            }
        }
        sh[threadIdx.x] = rc.ok ? acc : 0.0;
        __syncthreads();
        if (threadIdx.x < k) {
            double s = 0.0;
            for (int q = 0; q < rc.RB; ++q) s += sh[q * k + threadIdx.x];
            part[((size_t)i * gridDim.x + blockIdx.x) * k + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// h[pass][i][c] = sum over blocks, for i <= j
__global__ void k_gm_fin_h(int k, int j, int nblk, const double* part, Gm G, int pass)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (j + 1) * k) return;
    const int i = t / k, c = t - i * k;
    if (!G.adv[c]) return;
    G.h[((size_t)pass * (G.m + 1) + i) * k + c] = fin(part, i, nblk, k, c);
}

// w -= sum_i V_i h[pass][i]; pass 1 also accumulates ||w||^2
__global__ void k_gm_update(int64_t n, int k, int j, double* w, Gm G, int pass, double* part)
{
    const RC rc = rowc(k);
    double acc[1] = {0.0};
    const size_t blk = (size_t)n * k;
    if (rc.ok && G.adv[rc.c]) {
        const double* hh = G.h + (size_t)pass * (G.m + 1) * k;
        for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
            const int64_t e = row * k + rc.c;
            double wv = w[e];
            for (int i = 0; i <= j; ++i) wv = fma(-G.V[(size_t)i * blk + e], hh[(size_t)i * k + rc.c], wv);
            w[e] = wv;
            acc[0] = fma(wv, wv, acc[0]);
        }
    }
    if (pass == 1) block_partials<1>(acc, rc, k, part);
}

// H(:,j) = h0 + h1, ||w||, Givens rotations, residual estimate, stop tests
__global__ void k_gm_givens(int k, int j, int nblk, const double* part, int maxit, Sys S, Gm G, Dims D,
                            int* any_adv)
{
    const int c = threadIdx.x;
    const int ka = __syncthreads_count(c < k && G.adv[c]);
    if (c == 0 && ka > 0) {
        spmm_work(D.n, D.nnzM, ka);
        spmm_work(D.n, D.nnzA, ka);
        // two CGS passes: V_0..j and w read (+ w written by the update)
        kwork_add(PROF_GM_DOTS, 2.0 * 8.0 * D.n * ka * (j + 2), 2.0 * 2.0 * D.n * ka * (j + 1));
        kwork_add(PROF_GM_UPDATE, 2.0 * 8.0 * D.n * ka * (j + 3), 2.0 * 2.0 * D.n * ka * (j + 1) + 2.0 * D.n * ka);
    }
    int act = 0;
    if (c < k && G.adv[c]) {
        const int m = G.m;
        double* Hc = G.H + ((size_t)c * m + j) * (m + 1);
        for (int i = 0; i <= j; ++i) Hc[i] = G.h[(size_t)i * k + c] + G.h[((size_t)(m + 1) + i) * k + c];
        const double hn = sqrt(fin(part, 0, nblk, k, c));
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
        } else {
            act = 1;
        }
    }
    act = __syncthreads_or(act);
    if (threadIdx.x == 0) *any_adv = act;
}

__global__ void k_gm_normalize(int64_t n, int k, int j, const double* w, Sys S, Gm G)
{
    const RC rc = rowc(k);
    if (!rc.ok || !G.adv[rc.c]) return;
    const double hn = S.hn[rc.c];
    const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
    double* Vn = G.V + (size_t)(j + 1) * n * k;
    for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
        const int64_t e = row * k + rc.c;
        Vn[e] = w[e] * inv;
    }
}

// u = H(0:jd,0:jd)^{-1} g(0:jd) per system (upper triangular)
__global__ void k_gm_trisolve(int k, Sys S, Gm G)
{
    const int c = threadIdx.x;
    if (c >= k || !G.cyc[c]) return;
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
            return;
        }
        uc[i] = t / d;
    }
}

// w = V u (per system), then the caller forms z = M w and x += z
__global__ void k_gm_combine(int64_t n, int k, int jmax, double* w, Gm G)
{
    const RC rc = rowc(k);
    if (!rc.ok || !G.cyc[rc.c]) return;
    const size_t blk = (size_t)n * k;
    const int jd = G.jd[rc.c];
    const double* uc = G.u + (size_t)rc.c * G.m;
    for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
        const int64_t e = row * k + rc.c;
        double s = 0.0;
        for (int i = 0; i < jd && i < jmax; ++i) s = fma(G.V[(size_t)i * blk + e], uc[i], s);
        w[e] = s;
    }
}

__global__ void k_gm_xadd(int64_t n, int k, double* x, const double* z, Gm G)
{
    const RC rc = rowc(k);
    if (!rc.ok || !G.cyc[rc.c]) return;
    for (int64_t row = (int64_t)blockIdx.x * rc.RB + rc.tr; row < n; row += (int64_t)gridDim.x * rc.RB) {
        const int64_t e = row * k + rc.c;
        x[e] += z[e];
    }
}

__global__ void k_gm_cycle_end(int k, int maxit, Sys S, Gm G, int* any_left)
{
    const int c = threadIdx.x;
    int left = 0;
    if (c < k) {
        if (G.cyc[c] && G.conv[c]) {
            G.done[c] = 1;
            S.status[c] = ST_OK;
        } else if (G.cyc[c] && S.iters[c] >= maxit) {
            G.done[c] = 1;  // limit reached: no further residual test
            S.status[c] = ST_MAXITER;
        }
        if (!G.done[c]) {
            G.cyc[c] = 1;  // reused as "needs residual" mask
            left = 1;
        } else {
            G.cyc[c] = 0;
        }
    }
    left = __syncthreads_or(left);
    if (threadIdx.x == 0) *any_left = left;
}

}  // namespace

sai_status sai_krylov_run(const sai_split_s* h, const sai_precond_s* P, int32_t k, const double* B,
                          const double* thr, const sai_krylov_params* prm, double* X, int32_t* iters,
                          int32_t* status, cudaStream_t st)
{
    if (!h || !P || !prm || !thr || !iters || !status || k < 1 || k > KT) return SAI_INVALID_ARG;
    if (prm->maxit < 0 || (prm->method == SAI_GMRES && prm->restart < 1)) return SAI_INVALID_ARG;
    if (prm->method != SAI_BICGSTAB && prm->method != SAI_GMRES) return SAI_INVALID_ARG;
    const int32_t n = h->n;
    if (n > 0 && (!B || !X)) return SAI_INVALID_ARG;
    const size_t blk = (size_t)n * k;
    const int nb = kblocks(n, k);
    const int64_t* Ar = h->Atr_rp.as<int64_t>();
    const int32_t* Ac = h->Atr_ci.as<int32_t>();
    const double* Av = h->Atr_v.as<double>();
    const int64_t* Mr = P->Mr_rp.as<int64_t>();
    const int32_t* Mc = P->Mr_ci.as<int32_t>();
    const double* Mv = P->Mr_v.as<double>();

    Buf sysd, sysi, part, flag;
    SAI_TRY(sysd.alloc(sizeof(double) * 7 * k, st, true));
    SAI_TRY(sysi.alloc(sizeof(int) * 10 * k, st, true));
    const int m = prm->method == SAI_GMRES ? prm->restart : 1;
    const int ndots = prm->method == SAI_GMRES ? (m + 1) : 2;
    SAI_TRY(part.alloc(sizeof(double) * (size_t)ndots * nb * k, st, true));
    SAI_TRY(flag.alloc(sizeof(int) * 4, st, true));
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
    SAI_CUDA(cudaMemcpyAsync(S.thr, thr, sizeof(double) * k, cudaMemcpyHostToDevice, st));
    SAI_CUDA(cudaMemsetAsync(ii, 0, sizeof(int) * 10 * k, st));
    int* fl = flag.as<int>();
    int hflag = 0;
    Dims D;
    D.n = (double)n;
    D.nnzA = (double)h->nnz_At;
    D.nnzM = (double)P->nnz;
    const int check_every = 4;

    if (prm->method == SAI_BICGSTAB) {
        Buf vecs;
        SAI_TRY(vecs.alloc(sizeof(double) * blk * 8 + 8, st, true));
        double* r = vecs.as<double>();
        double* rh = r + blk;
        double* p = rh + blk;
        double* v = p + blk;
        double* ph = v + blk;
        double* s = ph + blk;
        double* sh = s + blk;
        double* t = sh + blk;
        k_bicg_init<<<SAI_GRID(nb), KT, 0, st>>>(n, k, B, X, r, rh, p, v, part.as<double>());
        k_bicg_f0<<<SAI_GRID(1), KT, 0, st>>>(k, nb, part.as<double>(), S);
        SAI_CUDA(cudaGetLastError());
        for (int it = 0; it < prm->maxit; ++it) {
            k_bicg_start<<<SAI_GRID(1), KT, 0, st>>>(k, prm->maxit, S);
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_bicg_p<<<SAI_GRID(nb), KT, 0, st>>>(n, k, r, p, v, S);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmm_m<0>(n, Mr, Mc, Mv, k, p, ph, nullptr, S.active, st);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmm_m<0>(n, Ar, Ac, Av, k, ph, v, nullptr, S.active, st);
            }
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_dot1<<<SAI_GRID(nb), KT, 0, st>>>(n, k, rh, v, S.active, part.as<double>());
            }
            k_bicg_f1<<<SAI_GRID(1), KT, 0, st>>>(k, nb, part.as<double>(), S, D);
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_bicg_s<<<SAI_GRID(nb), KT, 0, st>>>(n, k, r, v, s, S, part.as<double>());
            }
            k_bicg_f2<<<SAI_GRID(1), KT, 0, st>>>(k, nb, part.as<double>(), S, D);
            {
                ProfScope ps(PROF_SPMM, st);
                spmm_m<0>(n, Mr, Mc, Mv, k, s, sh, nullptr, S.go, st);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmm_m<0>(n, Ar, Ac, Av, k, sh, t, nullptr, S.go, st);
            }
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_dot2<<<SAI_GRID(nb), KT, 0, st>>>(n, k, t, s, S.go, part.as<double>());
            }
            k_bicg_f3<<<SAI_GRID(1), KT, 0, st>>>(k, nb, part.as<double>(), S, D);
            {
                ProfScope ps(PROF_BICG_VEC, st);
                k_bicg_xr<<<SAI_GRID(nb), KT, 0, st>>>(n, k, X, r, rh, ph, sh, s, t, S, part.as<double>());
            }
            k_bicg_f4<<<SAI_GRID(1), KT, 0, st>>>(k, nb, part.as<double>(), S, D, fl);
            SAI_CUDA(cudaGetLastError());
            if ((it + 1) % check_every == 0 || it + 1 == prm->maxit) {
                SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
                SAI_CUDA(cudaStreamSynchronize(st));
                if (!hflag) break;
            }
        }
        // systems still active after maxit passes
        k_bicg_start<<<SAI_GRID(1), KT, 0, st>>>(k, prm->maxit, S);
    } else {
        Gm G;
        G.m = m;
        Buf vb, hb, ib, wb;
        SAI_TRY(vb.alloc(sizeof(double) * blk * (m + 1) + 8, st, true));
        SAI_TRY(wb.alloc(sizeof(double) * blk * 3 + 8, st, true));
        const size_t hsz = (size_t)k * (m + 1) * m + 2 * (size_t)k * m + (size_t)k * (m + 1) +
                           2 * (size_t)(m + 1) * k + (size_t)k * m;
        SAI_TRY(hb.alloc(sizeof(double) * hsz, st, true));
        SAI_TRY(ib.alloc(sizeof(int) * 5 * k, st, true));
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
        int* ip = ib.as<int>();
        G.cyc = ip;
        G.adv = ip + k;
        G.jd = ip + 2 * k;
        G.done = ip + 3 * k;
        G.conv = ip + 4 * k;
        SAI_CUDA(cudaMemsetAsync(ip, 0, sizeof(int) * 5 * k, st));
        double* r = wb.as<double>();
        double* w = r + blk;
        double* z = w + blk;
        k_gm_init<<<SAI_GRID(nb), KT, 0, st>>>(n, k, B, X, r, part.as<double>());
        int first = 1;
        for (;;) {
            k_gm_cycle_start<<<SAI_GRID(1), KT, 0, st>>>(k, nb, part.as<double>(), prm->maxit, S, G, first, fl);
            first = 0;
            SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            if (!hflag) break;
            k_gm_v0<<<SAI_GRID(nb), KT, 0, st>>>(n, k, r, S, G);
            int jmax = 0;
            for (int j = 0; j < m; ++j) {
                const double* vj = G.V + (size_t)j * blk;
                {
                    ProfScope ps(PROF_SPMM, st);
                    spmm_m<0>(n, Mr, Mc, Mv, k, vj, z, nullptr, G.adv, st);
                }
                {
                    ProfScope ps(PROF_SPMM, st);
                    spmm_m<0>(n, Ar, Ac, Av, k, z, w, nullptr, G.adv, st);
                }
                for (int pass = 0; pass < 2; ++pass) {
                    {
                        ProfScope ps(PROF_GM_DOTS, st);
                        k_gm_dots<<<SAI_GRID(nb), KT, 0, st>>>(n, k, j, w, G, part.as<double>());
                    }
                    k_gm_fin_h<<<SAI_GRID(sai_div_up((int64_t)(j + 1) * k, 256)), 256, 0, st>>>(k, j, nb, part.as<double>(),
                                                                                       G, pass);
                    {
                        ProfScope ps(PROF_GM_UPDATE, st);
                        k_gm_update<<<SAI_GRID(nb), KT, 0, st>>>(n, k, j, w, G, pass, part.as<double>());
                    }
                }
                k_gm_givens<<<SAI_GRID(1), KT, 0, st>>>(k, j, nb, part.as<double>(), prm->maxit, S, G, D, fl);
                k_gm_normalize<<<SAI_GRID(nb), KT, 0, st>>>(n, k, j, w, S, G);
                SAI_CUDA(cudaGetLastError());
                jmax = j + 1;
                if ((j + 1) % check_every == 0 || j + 1 == m) {
                    SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
                    SAI_CUDA(cudaStreamSynchronize(st));
                    if (!hflag) break;
                }
            }
            k_gm_trisolve<<<SAI_GRID(1), KT, 0, st>>>(k, S, G);
            k_gm_combine<<<SAI_GRID(nb), KT, 0, st>>>(n, k, jmax, w, G);
            spmm_m<0>(n, Mr, Mc, Mv, k, w, z, nullptr, G.cyc, st);
            k_gm_xadd<<<SAI_GRID(nb), KT, 0, st>>>(n, k, X, z, G);
            k_gm_cycle_end<<<SAI_GRID(1), KT, 0, st>>>(k, prm->maxit, S, G, fl);
            spmm_m<1>(n, Ar, Ac, Av, k, X, r, B, G.cyc, st);
            k_norm2<<<SAI_GRID(nb), KT, 0, st>>>(n, k, r, G.cyc, part.as<double>());
            SAI_CUDA(cudaGetLastError());
        }
    }
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
