// batch.cu -- Procedure * (§3) for a batch of independent irregular systems.
//
// Split: each matrix on its own (sai_split_build: its own p and threshold),
//   several at a time on worker streams.
// Build: the A~_i are laid side by side as the block-diagonal A~ of the batch
//   (CSC and CSR copied with row / column offsets) and M is built for all of
//   its columns in one persistent launch of the SAI kernel: the column problems
//   of a block only reach rows and columns of that block, so each M_i is the
//   one its matrix alone would give.
// Solve: the sum(s_i + 1) right-hand sides [b_i, u_i1 .. u_is_i] are Krylov
//   systems of different lengths, stored one after another. Work items are
//   (system, chunk of BR rows), listed once for the whole batch: one block
//   each in the SpMV (a thread per row), one warp each in the vector kernels;
//   a stopped system's items return at once. Inner products are summed per
//   item in a fixed order and per system over its items in order. The
//   control kernels run one warp (or thread) per system. Groups of 8
//   iterations are captured once as a CUDA graph and replayed, with one host
//   check of the "any system still running" flag per group.
// SMW: one block per matrix solves its s_i x s_i system (partial pivoting);
//   then x_i = yhat_i - What_i z_i, and rr per matrix.
#include <math.h>

#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

constexpr int BR = 256;  // rows per work item (one block, one thread per row)

enum { B_OK = 0, B_MAXITER = 5, B_BREAKDOWN = 6 };  // same values as sai_status

// System table of the batch (device arrays).
struct BSys {
    int32_t nsys;
    const int64_t* off;     // start of system c's vectors in the batch vectors
    const int32_t* len;     // n of its matrix
    const int32_t* row0;    // first row of its matrix in the block-diagonal A~
    const int32_t* first;   // first item of system c (first[nsys] = item count)
    const int32_t* it_sys;  // system of item q
    const int32_t* it_r0;   // first local row of item q
    const int32_t* nsm;     // systems of c's matrix (s + 1)
    int32_t nitems;
};

// Algorithmic work of the batched BiCGStab, added per system by the control
// kernels and read by the profile: an SpMV reads its matrix block once for
// all the systems of the matrix (a 1/(s+1) share per system) and the
// system's input and output vectors once.
__device__ double d_bwork[PROF_NSITES * 2];

struct BWork {
    const int64_t* Arp;  // CSR row pointers of the block-diagonal A~ and M
    const int64_t* Mrp;
};

__device__ __forceinline__ void bwork_add(int site, double bytes, double flops)
{
    atomicAdd(&d_bwork[2 * site], bytes);
    atomicAdd(&d_bwork[2 * site + 1], flops);
}

// the two SpMVs (M, then A~) of one half iteration of system c
__device__ void bwork_pair(const BSys& Y, const BWork& Wk, int c)
{
    const int64_t r0 = Y.row0[c], n = Y.len[c];
    const double nA = (double)(Wk.Arp[r0 + n] - Wk.Arp[r0]), nM = (double)(Wk.Mrp[r0 + n] - Wk.Mrp[r0]);
    const double bytes = (12.0 * (nA + nM) + 16.0 * (double)(n + 1)) / (double)Y.nsm[c] + 32.0 * (double)n;
    bwork_add(PROF_SPMM, bytes, 2.0 * (nA + nM));
}

// Per-system BiCGStab state.
struct BState {
    double *thr, *rho, *rho_old, *alpha, *omega, *beta;
    int *active, *iters, *status, *mode, *go;
};

// Sum of the item partials of system c, in item order (one warp).
__device__ __forceinline__ double sys_sum(const BSys& Y, const double* part, int c)
{
    const int lane = threadIdx.x & 31;
    double a = 0.0;
    for (int q = Y.first[c] + lane; q < Y.first[c + 1]; q += 32) a += part[q];
    return warp_sum(a);
}

// y_c = A~ x_c (mode 0) for the systems with flag set, over their own block;
// A~ in CSR with global row / column indices (block diagonal).
__global__ void __launch_bounds__(BR) k_b_spmv(BSys Y, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                               const double* __restrict__ v, const double* __restrict__ X,
                                               double* __restrict__ Yv, const int* flags)
{
    for (int32_t q = blockIdx.x; q < Y.nitems; q += gridDim.x) {
        const int c = Y.it_sys[q];
        if (!flags[c]) continue;
        const int64_t i = Y.it_r0[q] + threadIdx.x;
        if (i >= Y.len[c]) continue;
        const int64_t o = Y.off[c];
        const int32_t r0 = Y.row0[c];
        const int64_t b = rp[r0 + i], e = rp[r0 + i + 1];
        double acc = 0.0;
        for (int64_t q0 = b; q0 < e; q0 += 8) {
            int32_t col[8];
            double a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                col[u] = q0 + u < e ? ci[q0 + u] - r0 : 0;
                a[u] = q0 + u < e ? v[q0 + u] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc = fma(a[u], X[o + col[u]], acc);
        }
        Yv[o + i] = acc;
    }
}

// The vector kernels take one warp per item (system, BR rows): lane l holds
// rows r0 + l + 32 t (t < RPL), whose loads are independent, and the item's
// partial sums are reduced by shuffles, in a fixed order.
constexpr int RPL = BR / 32;
#define FOR_WARP_ITEMS(Y, q)                                                                                 \
    for (int32_t q = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); q < (Y).nitems;      \
         q += (int32_t)(((int64_t)gridDim.x * blockDim.x) >> 5))

__global__ void __launch_bounds__(BR) k_b_init(BSys Y, const double* __restrict__ B, double* x, double* r, double* rh,
                                               double* p, double* v, double* part)
{
    const int lane = threadIdx.x & 31;
    FOR_WARP_ITEMS(Y, q)
    {
        const int c = Y.it_sys[q];
        const int64_t o = Y.off[c], r0 = Y.it_r0[q], n = Y.len[c];
        double a = 0.0;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int64_t i = r0 + lane + 32 * t;
            if (i < n) {
                const double bv = B[o + i];
                x[o + i] = 0.0;
                r[o + i] = bv;
                rh[o + i] = bv;
                p[o + i] = 0.0;
                v[o + i] = 0.0;
                a = fma(bv, bv, a);
            }
        }
        a = warp_sum(a);
        if (lane == 0) part[q] = a;
    }
}

// one warp per system
__global__ void k_b_f0(BSys Y, const double* part, BState S)
{
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (c >= Y.nsys) return;
    const double bb = sys_sum(Y, part, c);
    if ((threadIdx.x & 31) == 0) {
        S.iters[c] = 0;
        S.rho[c] = bb;
        S.alpha[c] = 1.0;
        S.omega[c] = 1.0;
        S.mode[c] = 1;
        S.go[c] = 0;
        if (sqrt(bb) < S.thr[c]) {
            S.active[c] = 0;
            S.status[c] = B_OK;
        } else {
            S.active[c] = 1;
            S.status[c] = B_MAXITER;
        }
    }
}

__global__ void k_b_start(int32_t nsys, int maxit, BState S)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nsys || !S.active[c]) return;
    if (S.iters[c] >= maxit) {
        S.active[c] = 0;
        S.status[c] = B_MAXITER;
    } else {
        S.iters[c] += 1;
        if (S.rho[c] == 0.0) {
            S.active[c] = 0;
            S.status[c] = B_BREAKDOWN;
        } else {
            S.beta[c] = S.iters[c] == 1 ? 0.0 : (S.rho[c] / S.rho_old[c]) * (S.alpha[c] / S.omega[c]);
        }
    }
}

__global__ void __launch_bounds__(BR) k_b_p(BSys Y, const double* __restrict__ r, double* p, const double* __restrict__ v,
                                            BState S)
{
    const int lane = threadIdx.x & 31;
    FOR_WARP_ITEMS(Y, q)
    {
        const int c = Y.it_sys[q];
        if (!S.active[c]) continue;
        const int64_t o = Y.off[c], r0 = Y.it_r0[q], n = Y.len[c];
        const double be = S.beta[c], om = S.omega[c];
        const bool first = S.iters[c] == 1;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int64_t i = r0 + lane + 32 * t;
            if (i < n) p[o + i] = first ? r[o + i] : r[o + i] + be * (p[o + i] - om * v[o + i]);
        }
    }
}

template <int ND>
__global__ void __launch_bounds__(BR) k_b_dots(BSys Y, const double* a0, const double* b0, const double* a1,
                                               const double* b1, const int* flags, double* part)
{
    const int lane = threadIdx.x & 31;
    FOR_WARP_ITEMS(Y, q)
    {
        const int c = Y.it_sys[q];
        if (!flags[c]) continue;
        const int64_t o = Y.off[c], r0 = Y.it_r0[q], n = Y.len[c];
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int64_t i = r0 + lane + 32 * t;
            if (i < n) {
                s0 = fma(a0[o + i], b0[o + i], s0);
                if (ND > 1) s1 = fma(a1[o + i], b1[o + i], s1);
            }
        }
        s0 = warp_sum(s0);
        if (ND > 1) s1 = warp_sum(s1);
        if (lane == 0) {
            part[q] = s0;
            if (ND > 1) part[Y.nitems + q] = s1;
        }
    }
}

__global__ void k_b_f1(BSys Y, const double* part, BState S, BWork Wk)
{
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (c >= Y.nsys || !S.active[c]) return;
    const double rv = sys_sum(Y, part, c);
    if ((threadIdx.x & 31) == 0) {
        bwork_pair(Y, Wk, c);
        bwork_add(PROF_BICG_VEC, 8.0 * Y.len[c] * (4 + 2), (double)Y.len[c] * (3 + 2));  // p update, rhat^T v
        if (rv == 0.0) {
            S.active[c] = 0;
            S.status[c] = B_BREAKDOWN;
        } else {
            S.alpha[c] = S.rho[c] / rv;
        }
    }
}

__global__ void __launch_bounds__(BR) k_b_s(BSys Y, const double* __restrict__ r, const double* __restrict__ v, double* s,
                                            BState S, double* part)
{
    const int lane = threadIdx.x & 31;
    FOR_WARP_ITEMS(Y, q)
    {
        const int c = Y.it_sys[q];
        if (!S.active[c]) continue;
        const int64_t o = Y.off[c], r0 = Y.it_r0[q], n = Y.len[c];
        const double al = S.alpha[c];
        double a = 0.0;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int64_t i = r0 + lane + 32 * t;
            if (i < n) {
                const double sv = r[o + i] - al * v[o + i];
                s[o + i] = sv;
                a = fma(sv, sv, a);
            }
        }
        a = warp_sum(a);
        if (lane == 0) part[q] = a;
    }
}

__global__ void k_b_f2(BSys Y, const double* part, BState S)
{
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (c >= Y.nsys) return;
    if (!S.active[c]) {
        if ((threadIdx.x & 31) == 0) S.go[c] = 0;
        return;
    }
    const double ss = sys_sum(Y, part, c);
    if ((threadIdx.x & 31) == 0) {
        bwork_add(PROF_BICG_VEC, 8.0 * Y.len[c] * 3, 4.0 * Y.len[c]);  // s, ||s||
        S.mode[c] = sqrt(ss) < S.thr[c] ? 2 : 1;
        S.go[c] = S.mode[c] == 1;
    }
}

__global__ void k_b_f3(BSys Y, const double* part, BState S, BWork Wk)
{
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (c >= Y.nsys || !S.go[c]) return;
    const double ts = sys_sum(Y, part, c);
    const double tt = sys_sum(Y, part + Y.nitems, c);
    if ((threadIdx.x & 31) == 0) {
        bwork_pair(Y, Wk, c);
        bwork_add(PROF_BICG_VEC, 8.0 * Y.len[c] * 2, 4.0 * Y.len[c]);  // t^T s, t^T t
        if (tt == 0.0) {
            S.active[c] = 0;
            S.go[c] = 0;
            S.status[c] = B_BREAKDOWN;
        } else {
            S.omega[c] = ts / tt;
        }
    }
}

__global__ void __launch_bounds__(BR) k_b_xr(BSys Y, double* x, double* r, const double* __restrict__ rh,
                                             const double* __restrict__ ph, const double* __restrict__ sh_,
                                             const double* __restrict__ s, const double* __restrict__ t, BState S,
                                             double* part)
{
    const int lane = threadIdx.x & 31;
    FOR_WARP_ITEMS(Y, q)
    {
        const int c = Y.it_sys[q];
        if (!S.active[c]) continue;
        const int64_t o = Y.off[c], r0 = Y.it_r0[q], n = Y.len[c];
        const double al = S.alpha[c], om = S.omega[c];
        const bool half = S.mode[c] == 2;
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
            const int64_t i = r0 + lane + 32 * u;
            if (i < n) {
                double rv;
                if (half) {
                    x[o + i] += al * ph[o + i];
                    rv = s[o + i];
                } else {
                    x[o + i] += al * ph[o + i] + om * sh_[o + i];
                    rv = s[o + i] - om * t[o + i];
                }
                r[o + i] = rv;
                a0 = fma(rv, rv, a0);
                a1 = fma(rh[o + i], rv, a1);
            }
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        if (lane == 0) {
            part[q] = a0;
            part[Y.nitems + q] = a1;
        }
    }
}

__global__ void k_b_f4(BSys Y, const double* part, BState S)
{
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (c >= Y.nsys || !S.active[c]) return;
    const double rr = sys_sum(Y, part, c);
    const double rhr = sys_sum(Y, part + Y.nitems, c);
    if ((threadIdx.x & 31) == 0) {
        bwork_add(PROF_BICG_VEC, 8.0 * Y.len[c] * 8, 10.0 * Y.len[c]);  // x, r, two dots
        if (S.mode[c] == 2 || sqrt(rr) < S.thr[c]) {
            S.active[c] = 0;
            S.status[c] = B_OK;
        } else if (S.omega[c] == 0.0) {
            S.active[c] = 0;
            S.status[c] = B_BREAKDOWN;
        } else {
            S.rho_old[c] = S.rho[c];
            S.rho[c] = rhr;
        }
    }
}

__global__ void k_b_any(int32_t nsys, const int* active, int* any)
{
    __shared__ int f;
    if (threadIdx.x == 0) f = 0;
    __syncthreads();
    int a = 0;
    for (int c = threadIdx.x; c < nsys; c += blockDim.x) a |= active[c];
    if (a) f = 1;
    __syncthreads();
    if (threadIdx.x == 0) *any = f;
}

// The condition of the while node that runs the whole batched loop: true
// while a system is active and fewer than max_body bodies have run.
// nbody counts the bodies (for the launch count), any mirrors the flag.
__global__ void k_b_cond(int32_t nsys, const int* active, int* any, int* nbody, int max_body,
                         cudaGraphConditionalHandle h)
{
    __shared__ int f;
    if (threadIdx.x == 0) f = 0;
    __syncthreads();
    int a = 0;
    for (int c = threadIdx.x; c < nsys; c += blockDim.x) a |= active[c];
    if (a) f = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nb = *nbody + 1;
        *nbody = nb;
        *any = f;
        cudaGraphSetConditional(h, (f && nb < max_body) ? 1u : 0u);
    }
}

// R = B - R on the systems with sel set (R holds A~ X there)
__global__ void __launch_bounds__(BR) k_b_resid(BSys Y, const double* __restrict__ B, const int* sel, double* R)
{
    const int lane = threadIdx.x & 31;
    FOR_WARP_ITEMS(Y, q)
    {
        const int c = Y.it_sys[q];
        if (!sel[c]) continue;
        const int64_t o = Y.off[c], r0 = Y.it_r0[q], n = Y.len[c];
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int64_t i = r0 + lane + 32 * t;
            if (i < n) R[o + i] = B[o + i] - R[o + i];
        }
    }
}

// X += D on the systems with sel set
__global__ void __launch_bounds__(BR) k_b_acc(BSys Y, const double* __restrict__ D, const int* sel, double* X)
{
    const int lane = threadIdx.x & 31;
    FOR_WARP_ITEMS(Y, q)
    {
        const int c = Y.it_sys[q];
        if (!sel[c]) continue;
        const int64_t o = Y.off[c], r0 = Y.it_r0[q], n = Y.len[c];
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int64_t i = r0 + lane + 32 * t;
            if (i < n) X[o + i] += D[o + i];
        }
    }
}

// B = [b_i, u_i1 .. u_is] per matrix (U_i scattered into its systems)
__global__ void k_b_rhs_b(int32_t n, const double* __restrict__ b, double* __restrict__ B)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) B[i] = b[i];
}

__global__ void k_b_rhs_u(int32_t s, const int64_t* Ucp, const int32_t* Uri, const double* Uv, int32_t n, double* B)
{
    const int t = blockIdx.x;  // column t of U goes to the system at B + (t + 1) * n
    for (int64_t q = Ucp[t] + threadIdx.x; q < Ucp[t + 1]; q += blockDim.x) B[(int64_t)(t + 1) * n + Uri[q]] = Uv[q];
}

// Batched SMW: block m solves (I + What_m(J_m,:)) z = yhat_m(J_m) with partial
// pivoting (the first largest |pivot| wins), C in shared memory.
struct BSmw {
    const int64_t* xoff;   // start of matrix m's first system (yhat) in X
    const int32_t* n;      // order of matrix m
    const int32_t* s;      // irregular columns of matrix m
    const int64_t* joff;   // start of J_m in the concatenated J
    const int32_t* J;
    double* z;             // concatenated z_m (offset joff)
    double* c;             // ||z_m||
    int* err;              // singular flag per matrix
};

__global__ void k_b_smw(BSmw W, const double* __restrict__ X, int smax)
{
    extern __shared__ double smem[];
    const int m = blockIdx.x;
    const int s = W.s[m], n = W.n[m];
    double* C = smem;                // s x s column-major
    double* g = smem + (size_t)smax * smax;
    __shared__ int piv_s;
    const int64_t xo = W.xoff[m];
    const int32_t* J = W.J + W.joff[m];
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int col = e / s, row = e - col * s;
        C[(size_t)col * s + row] = (row == col ? 1.0 : 0.0) + X[xo + (int64_t)(col + 1) * n + J[row]];
    }
    for (int a = threadIdx.x; a < s; a += blockDim.x) g[a] = X[xo + J[a]];
    __syncthreads();
    for (int k = 0; k < s; ++k) {
        if (threadIdx.x == 0) {
            int p = k;
            double best = fabs(C[(size_t)k * s + k]);
            for (int i = k + 1; i < s; ++i)
                if (fabs(C[(size_t)k * s + i]) > best) {
                    best = fabs(C[(size_t)k * s + i]);
                    p = i;
                }
            piv_s = best > 0.0 ? p : -1;
        }
        __syncthreads();
        const int p = piv_s;
        if (p < 0) {
            if (threadIdx.x == 0) W.err[m] = 1;
            return;
        }
        if (p != k) {
            for (int j = threadIdx.x; j < s; j += blockDim.x) {
                const double t = C[(size_t)j * s + k];
                C[(size_t)j * s + k] = C[(size_t)j * s + p];
                C[(size_t)j * s + p] = t;
            }
            if (threadIdx.x == 0) {
                const double t = g[k];
                g[k] = g[p];
                g[p] = t;
            }
        }
        __syncthreads();
        const double akk = C[(size_t)k * s + k];
        const double gk = g[k];
        for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) {
            const double l = C[(size_t)k * s + i] / akk;
            C[(size_t)k * s + i] = l;
            for (int j = k + 1; j < s; ++j) C[(size_t)j * s + i] -= l * C[(size_t)j * s + k];
            g[i] -= l * gk;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* z = W.z + W.joff[m];
        double cc = 0.0;
        for (int j = s - 1; j >= 0; --j) {
            double t = g[j];
            for (int i = j + 1; i < s; ++i) t -= C[(size_t)i * s + j] * z[i];
            z[j] = t / C[(size_t)j * s + j];
        }
        for (int j = 0; j < s; ++j) cc += z[j] * z[j];
        W.c[m] = sqrt(cc);
        W.err[m] = 0;
    }
}

__global__ void k_b_xhat(int32_t n, int32_t s, const double* __restrict__ X, const double* __restrict__ z,
                         double* __restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = X[i];
    for (int t = 0; t < s; ++t) v = fma(-X[(int64_t)(t + 1) * n + i], z[t], v);
    x[i] = v;
}

__global__ void k_b_add_i64(int64_t cnt, const int64_t* __restrict__ a, int64_t add, int64_t* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + add;
}

__global__ void k_b_add_i32(int64_t cnt, const int32_t* __restrict__ a, int32_t add, int32_t* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + add;
}

struct Ev {
    cudaEvent_t e = nullptr;
    Ev() { cudaEventCreate(&e); }
    ~Ev() { cudaEventDestroy(e); }
};

float ms_between(cudaEvent_t a, cudaEvent_t b)
{
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    return t;
}

unsigned grid_for(int64_t work, int64_t cap)
{
    int64_t g = work < cap ? work : cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// The block-diagonal A~ of a batch (CSC and CSR with row / column offsets,
// ||a~_j||^2, the largest ||A~_i||_1) from the matrices' split handles;
// R0[m] = first row of matrix m.
sai_status stack_splits(int32_t nmat, const std::vector<std::unique_ptr<sai_split_s>>& hs, sai_split_s& bd,
                        std::vector<int64_t>& R0, int64_t cap, cudaStream_t st)
{
    R0.assign(nmat + 1, 0);
    std::vector<int64_t> Z0(nmat + 1, 0);
    double norm1 = 0.0;
    for (int32_t m = 0; m < nmat; ++m) {
        R0[m + 1] = R0[m] + hs[m]->n;
        Z0[m + 1] = Z0[m] + hs[m]->nnz_At;
        norm1 = hs[m]->norm1 > norm1 ? hs[m]->norm1 : norm1;
    }
    const int64_t N = R0[nmat], NZ = Z0[nmat];
    if (N > INT32_MAX - 1) return SAI_INVALID_ARG;
    bd.n = (int32_t)N;
    bd.nnz_At = NZ;
    bd.norm1 = norm1;
    SAI_TRY(bd.At_cp.alloc(sizeof(int64_t) * (size_t)(N + 1), st, true));
    SAI_TRY(bd.At_ri.alloc(sizeof(int32_t) * (size_t)(NZ > 0 ? NZ : 1), st, true));
    SAI_TRY(bd.At_v.alloc(sizeof(double) * (size_t)(NZ > 0 ? NZ : 1), st, true));
    SAI_TRY(bd.Atr_rp.alloc(sizeof(int64_t) * (size_t)(N + 1), st, true));
    SAI_TRY(bd.Atr_ci.alloc(sizeof(int32_t) * (size_t)(NZ > 0 ? NZ : 1), st, true));
    SAI_TRY(bd.Atr_v.alloc(sizeof(double) * (size_t)(NZ > 0 ? NZ : 1), st, true));
    SAI_TRY(bd.colnorm2.alloc(sizeof(double) * (size_t)N, st, true));
    for (int32_t m = 0; m < nmat; ++m) {
        const sai_split_s& h = *hs[m];
        const int64_t n = h.n, z = h.nnz_At;
        const unsigned gz = grid_for(sai_div_up(z > n ? z : n, 256), cap);
        k_b_add_i64<<<SAI_GRID(gz), 256, 0, st>>>(n, h.At_cp.as<int64_t>(), Z0[m], bd.At_cp.as<int64_t>() + R0[m]);
        k_b_add_i64<<<SAI_GRID(gz), 256, 0, st>>>(n, h.Atr_rp.as<int64_t>(), Z0[m], bd.Atr_rp.as<int64_t>() + R0[m]);
        if (z > 0) {
            k_b_add_i32<<<SAI_GRID(gz), 256, 0, st>>>(z, h.At_ri.as<int32_t>(), (int32_t)R0[m],
                                                      bd.At_ri.as<int32_t>() + Z0[m]);
            k_b_add_i32<<<SAI_GRID(gz), 256, 0, st>>>(z, h.Atr_ci.as<int32_t>(), (int32_t)R0[m],
                                                      bd.Atr_ci.as<int32_t>() + Z0[m]);
            SAI_CUDA(cudaMemcpyAsync(bd.At_v.as<double>() + Z0[m], h.At_v.p, sizeof(double) * z,
                                     cudaMemcpyDeviceToDevice, st));
            SAI_CUDA(cudaMemcpyAsync(bd.Atr_v.as<double>() + Z0[m], h.Atr_v.p, sizeof(double) * z,
                                     cudaMemcpyDeviceToDevice, st));
        }
        SAI_CUDA(cudaMemcpyAsync(bd.colnorm2.as<double>() + R0[m], h.colnorm2.p, sizeof(double) * n,
                                 cudaMemcpyDeviceToDevice, st));
    }
    SAI_CUDA(cudaMemcpyAsync(bd.At_cp.as<int64_t>() + N, &Z0[nmat], sizeof(int64_t), cudaMemcpyHostToDevice, st));
    SAI_CUDA(cudaMemcpyAsync(bd.Atr_rp.as<int64_t>() + N, &Z0[nmat], sizeof(int64_t), cudaMemcpyHostToDevice, st));
    SAI_CUDA(cudaGetLastError());

    return SAI_OK;
}

sai_status batched_impl(int32_t nmat, const sai_csc_view* A, const double* const* b, const sai_solve_params* prm,
                        double* const* x, sai_batch_item* items, sai_batch_report* rep, cudaStream_t st)
{
    if (nmat < 1 || !A || !b || !prm || !x || !items || !rep) return SAI_INVALID_ARG;
    if (prm->krylov.method != SAI_BICGSTAB || prm->krylov.precision != SAI_FP64 || prm->krylov.transpose)
        return SAI_NOT_IMPLEMENTED;
    if (prm->sai == 1 && prm->psai.tol_mode == 0) return SAI_NOT_IMPLEMENTED;
    if (prm->krylov.maxit < 0 || prm->split.zero_diag != 0) return SAI_INVALID_ARG;
    *rep = sai_batch_report{};
    int dev = 0, sms = 0;
    SAI_CUDA(cudaGetDevice(&dev));
    SAI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = (int64_t)sms * 8;
    Ev e0, e1, e2, e3, e4;
    SAI_CUDA(cudaEventRecord(e0.e, st));

    // ---- split: each matrix on its own. A split waits on the host for its
    // counts, so the matrices are spread over worker streams, each driven by
    // a host thread, and those waits overlap. The worker streams start after
    // st, st waits for all of them, and they wait for st again before the
    // split handles (whose buffers they own) are freed.
    for (int32_t m = 0; m < nmat; ++m)
        if (A[m].n < 1 || !b[m] || !x[m]) return SAI_INVALID_ARG;
    const int nthr = nmat < 8 ? nmat : 8;
    struct Workers {
        std::vector<cudaStream_t> s;
        ~Workers()
        {
            for (cudaStream_t q : s) cudaStreamDestroy(q);
        }
    } wk;
    {
        cudaEvent_t ev = nullptr;
        SAI_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        SAI_CUDA(cudaEventRecord(ev, st));
        for (int t = 0; t < nthr; ++t) {
            cudaStream_t q = nullptr;
            if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) {
                cudaEventDestroy(ev);
                return SAI_CUDA_ERROR;
            }
            wk.s.push_back(q);
            SAI_CUDA(cudaStreamWaitEvent(q, ev, 0));
        }
        cudaEventDestroy(ev);
    }
    std::vector<std::unique_ptr<sai_split_s>> hs((size_t)nmat);
    struct Join {  // destroyed before hs: the worker streams wait for st's use of the splits
        const std::vector<cudaStream_t>& s;
        cudaStream_t main;
        ~Join()
        {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                cudaStreamSynchronize(main);
                return;
            }
            cudaEventRecord(ev, main);
            for (cudaStream_t q : s) cudaStreamWaitEvent(q, ev, 0);
            cudaEventDestroy(ev);
        }
    } join{wk.s, st};
    {
        std::vector<sai_status> tst((size_t)nthr, SAI_OK);
        std::vector<std::thread> th;
        for (int t = 0; t < nthr; ++t)
            th.emplace_back([&, t] {
                if (cudaSetDevice(dev) != cudaSuccess) {
                    tst[t] = SAI_CUDA_ERROR;
                    return;
                }
                for (int32_t m = t; m < nmat && tst[t] == SAI_OK; m += nthr) {
                    hs[m].reset(new sai_split_s);
                    tst[t] = sai_split_build(&A[m], &prm->split, wk.s[t], true, hs[m].get());
                }
            });
        for (auto& h : th) h.join();
        for (int t = 0; t < nthr; ++t) {
            cudaEvent_t ev = nullptr;
            SAI_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            SAI_CUDA(cudaEventRecord(ev, wk.s[t]));
            SAI_CUDA(cudaStreamWaitEvent(st, ev, 0));
            cudaEventDestroy(ev);
        }
        for (int t = 0; t < nthr; ++t)
            if (tst[t] != SAI_OK) return tst[t];
    }
    SAI_CUDA(cudaEventRecord(e1.e, st));

    // ---- the block-diagonal A~ of the batch (CSC and CSR), ||a~_j||^2
    std::vector<int64_t> R0;
    sai_split_s bd;
    SAI_TRY(stack_splits(nmat, hs, bd, R0, cap, st));
    const int64_t N = R0[nmat];

    // ---- one SAI build for every column of the batch
    sai_precond_s P;
    if (prm->sai == 0) SAI_TRY(sai_spai_build(&bd, &prm->spai, st, true, &P));
    else SAI_TRY(sai_psai_build(&bd, &prm->psai, st, true, &P));
    SAI_CUDA(cudaEventRecord(e2.e, st));

    // ---- system table: matrix m owns systems sys0[m] .. sys0[m] + s_m
    std::vector<int32_t> sys0(nmat + 1, 0);
    for (int32_t m = 0; m < nmat; ++m) sys0[m + 1] = sys0[m] + hs[m]->s + 1;
    const int32_t nsys = sys0[nmat];
    std::vector<int64_t> off(nsys);
    std::vector<int32_t> len(nsys), row0(nsys), first(nsys + 1), nsm(nsys);
    std::vector<int64_t> xoff(nmat), joff(nmat + 1, 0);
    std::vector<int32_t> nvec(nmat), svec(nmat);
    int64_t o = 0;
    int32_t nit = 0;
    int smax = 1;
    for (int32_t m = 0; m < nmat; ++m) {
        xoff[m] = o;
        nvec[m] = hs[m]->n;
        svec[m] = hs[m]->s;
        joff[m + 1] = joff[m] + hs[m]->s;
        smax = hs[m]->s > smax ? hs[m]->s : smax;
        for (int32_t c = sys0[m]; c < sys0[m + 1]; ++c) {
            off[c] = o;
            len[c] = hs[m]->n;
            row0[c] = (int32_t)R0[m];
            nsm[c] = hs[m]->s + 1;
            first[c] = nit;
            o += hs[m]->n;
            nit += (hs[m]->n + BR - 1) / BR;
        }
    }
    first[nsys] = nit;
    const int64_t NV = o;
    std::vector<int32_t> it_sys(nit), it_r0(nit);
    for (int32_t c = 0; c < nsys; ++c)
        for (int32_t q = first[c]; q < first[c + 1]; ++q) {
            it_sys[q] = c;
            it_r0[q] = (q - first[c]) * BR;
        }
    Buf tab, vecs, bst, bsi, part, misc;
    const size_t tab_bytes = sizeof(int64_t) * (nsys + nmat + nmat + 1) +
                             sizeof(int32_t) * (4 * (size_t)nsys + 1 + 2 * (size_t)nit + 2 * (size_t)nmat + joff[nmat] + 1);
    SAI_TRY(tab.alloc(tab_bytes + 64, st, true));
    char* tp = tab.as<char>();
    auto put = [&](const void* src, size_t bytes) -> char* {
        char* at = tp;
        if (bytes) cudaMemcpyAsync(at, src, bytes, cudaMemcpyHostToDevice, st);
        tp += (bytes + 7) & ~size_t(7);
        return at;
    };
    BSys Y;
    Y.nsys = nsys;
    Y.nitems = nit;
    Y.off = (const int64_t*)put(off.data(), sizeof(int64_t) * nsys);
    Y.len = (const int32_t*)put(len.data(), sizeof(int32_t) * nsys);
    Y.row0 = (const int32_t*)put(row0.data(), sizeof(int32_t) * nsys);
    Y.first = (const int32_t*)put(first.data(), sizeof(int32_t) * (nsys + 1));
    Y.it_sys = (const int32_t*)put(it_sys.data(), sizeof(int32_t) * nit);
    Y.it_r0 = (const int32_t*)put(it_r0.data(), sizeof(int32_t) * nit);
    Y.nsm = (const int32_t*)put(nsm.data(), sizeof(int32_t) * nsys);
    BSmw W;
    W.xoff = (const int64_t*)put(xoff.data(), sizeof(int64_t) * nmat);
    W.n = (const int32_t*)put(nvec.data(), sizeof(int32_t) * nmat);
    W.s = (const int32_t*)put(svec.data(), sizeof(int32_t) * nmat);
    W.joff = (const int64_t*)put(joff.data(), sizeof(int64_t) * (nmat + 1));
    {
        int32_t* Jcat = (int32_t*)tp;
        for (int32_t m = 0; m < nmat; ++m)
            if (hs[m]->s > 0)
                SAI_CUDA(cudaMemcpyAsync(Jcat + joff[m], hs[m]->J.p, sizeof(int32_t) * hs[m]->s,
                                         cudaMemcpyDeviceToDevice, st));
        W.J = Jcat;
        tp += (sizeof(int32_t) * (size_t)joff[nmat] + 7) & ~size_t(7);
    }
    SAI_TRY(vecs.alloc(sizeof(double) * (size_t)NV * 11 + 64, st, true));
    SAI_CUDA(cudaMemsetAsync(vecs.p, 0, sizeof(double) * (size_t)NV * 11, st));
    double* Bv = vecs.as<double>();
    double* X = Bv + NV;
    double* r = X + NV;
    double* rh = r + NV;
    double* p = rh + NV;
    double* v = p + NV;
    double* ph = v + NV;
    double* s = ph + NV;
    double* sh = s + NV;
    double* t = sh + NV;
    SAI_TRY(bst.alloc(sizeof(double) * 6 * (size_t)nsys, st, true));
    SAI_TRY(bsi.alloc(sizeof(int) * (5 * (size_t)nsys + 2), st, true));
    SAI_TRY(part.alloc(sizeof(double) * 2 * (size_t)(nit > 0 ? nit : 1), st, true));
    SAI_TRY(misc.alloc(sizeof(double) * ((size_t)joff[nmat] + 2 * (size_t)nmat + 4), st, true));
    BState S;
    double* dp = bst.as<double>();
    S.thr = dp;
    S.rho = dp + nsys;
    S.rho_old = dp + 2 * nsys;
    S.alpha = dp + 3 * nsys;
    S.omega = dp + 4 * nsys;
    S.beta = dp + 5 * nsys;
    int* ip = bsi.as<int>();
    S.active = ip;
    S.iters = ip + nsys;
    S.status = ip + 2 * nsys;
    S.mode = ip + 3 * nsys;
    S.go = ip + 4 * nsys;
    int* any = ip + 5 * nsys;
    SAI_CUDA(cudaMemsetAsync(ip, 0, sizeof(int) * (5 * (size_t)nsys + 2), st));

    // right-hand sides and the Theorem 2 thresholds of each matrix
    std::vector<double> thr(nsys);
    for (int32_t m = 0; m < nmat; ++m) {
        const sai_split_s& h = *hs[m];
        double* Bm = Bv + xoff[m];
        k_b_rhs_b<<<SAI_GRID(sai_div_up(h.n, 256)), 256, 0, st>>>(h.n, b[m], Bm);
        if (h.s > 0)
            k_b_rhs_u<<<SAI_GRID(h.s), 256, 0, st>>>(h.s, h.U_cp.as<int64_t>(), h.U_ri.as<int32_t>(),
                                                     h.U_v.as<double>(), h.n, Bm);
    }
    SAI_CUDA(cudaGetLastError());
    {
        // ||b_m||: item partials of each matrix's first system, summed on the host in item order
        k_b_init<<<SAI_GRID(grid_for(sai_div_up(nit, BR / 32), cap)), BR, 0, st>>>(Y, Bv, X, r, rh, p, v, part.as<double>());
        std::vector<double> hp(nit);
        SAI_CUDA(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * nit, cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        for (int32_t m = 0; m < nmat; ++m) {
            const int32_t c0 = sys0[m];
            double bb = 0.0;
            for (int32_t q = first[c0]; q < first[c0 + 1]; ++q) bb += hp[q];
            const double bn = sqrt(bb);
            thr[c0] = 0.5 * prm->eps * bn;  // eq. (stopb)
            for (int32_t c = c0 + 1; c < sys0[m + 1]; ++c)
                thr[c] = prm->eps * bn / (2.0 * sqrt((double)hs[m]->s));  // eq. (stopU2), c = 1
        }
    }
    SAI_CUDA(cudaMemcpyAsync(S.thr, thr.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
    SAI_CUDA(cudaEventRecord(e3.e, st));

    // ---- batched BiCGStab (right preconditioning: A~ M z = rhs, y = M z)
    const int64_t *Ar = bd.Atr_rp.as<int64_t>(), *Mr = P.Mr_rp.as<int64_t>();
    const int32_t *Ac = bd.Atr_ci.as<int32_t>(), *Mc = P.Mr_ci.as<int32_t>();
    const double *Av = bd.Atr_v.as<double>(), *Mv = P.Mr_v.as<double>();
    const unsigned gi = grid_for(nit, cap);                   // SpMV: one block per item
    const unsigned gw = grid_for(sai_div_up(nit, BR / 32), cap);  // vector kernels: one warp per item
    const unsigned gs = sai_div_up((int64_t)nsys * 32, 256), gt = sai_div_up(nsys, 256);
    double* pt = part.as<double>();
    const int maxit = prm->krylov.maxit;
    BWork Wk;
    Wk.Arp = Ar;
    Wk.Mrp = Mr;
    double* Xd = X;  // the iterates of the current pass
    // profile scopes act only while a profile is open, when no graph is captured
    auto iteration = [&](cudaStream_t q) {
        k_b_start<<<SAI_GRID(gt), 256, 0, q>>>(nsys, maxit, S);
        {
            ProfScope ps(PROF_BICG_VEC, q);
            k_b_p<<<SAI_GRID(gw), BR, 0, q>>>(Y, r, p, v, S);
        }
        {
            ProfScope ps(PROF_SPMM, q);
            k_b_spmv<<<SAI_GRID(gi), BR, 0, q>>>(Y, Mr, Mc, Mv, p, ph, S.active);
        }
        {
            ProfScope ps(PROF_SPMM, q);
            k_b_spmv<<<SAI_GRID(gi), BR, 0, q>>>(Y, Ar, Ac, Av, ph, v, S.active);
        }
        {
            ProfScope ps(PROF_BICG_VEC, q);
            k_b_dots<1><<<SAI_GRID(gw), BR, 0, q>>>(Y, rh, v, nullptr, nullptr, S.active, pt);
        }
        k_b_f1<<<SAI_GRID(gs), 256, 0, q>>>(Y, pt, S, Wk);
        {
            ProfScope ps(PROF_BICG_VEC, q);
            k_b_s<<<SAI_GRID(gw), BR, 0, q>>>(Y, r, v, s, S, pt);
        }
        k_b_f2<<<SAI_GRID(gs), 256, 0, q>>>(Y, pt, S);
        {
            ProfScope ps(PROF_SPMM, q);
            k_b_spmv<<<SAI_GRID(gi), BR, 0, q>>>(Y, Mr, Mc, Mv, s, sh, S.go);
        }
        {
            ProfScope ps(PROF_SPMM, q);
            k_b_spmv<<<SAI_GRID(gi), BR, 0, q>>>(Y, Ar, Ac, Av, sh, t, S.go);
        }
        {
            ProfScope ps(PROF_BICG_VEC, q);
            k_b_dots<2><<<SAI_GRID(gw), BR, 0, q>>>(Y, t, s, t, t, S.go, pt);
        }
        k_b_f3<<<SAI_GRID(gs), 256, 0, q>>>(Y, pt, S, Wk);
        {
            ProfScope ps(PROF_BICG_VEC, q);
            k_b_xr<<<SAI_GRID(gw), BR, 0, q>>>(Y, Xd, r, rh, ph, sh, s, t, S, pt);
        }
        k_b_f4<<<SAI_GRID(gs), 256, 0, q>>>(Y, pt, S);
    };
    constexpr int ITERS_PER_CHECK = 8, LAUNCHES = ITERS_PER_CHECK * 14 + 1;
    int* nbody = any + 1;  // body runs of the while graph
    // One pass of the batched BiCGStab from x = 0 on the right-hand sides
    // Bsrc (thresholds in S.thr), iterates into Xdst. Without an open
    // profile the whole loop is one CUDA graph launch: a conditional while
    // node whose body runs ITERS_PER_CHECK iterations and then k_b_cond,
    // which keeps the loop going while any system is active and fewer than
    // maxit iterations have run. Where that graph cannot be built, groups of
    // ITERS_PER_CHECK iterations run as a captured graph with one host check
    // of the "any system active" flag per group. Both run on a library
    // stream ordered after the caller's; iterations past maxit change nothing
    // (k_b_start retires those systems).
    auto run_pass = [&](const double* Bsrc, double* Xdst) -> sai_status {
        Xd = Xdst;
        k_b_init<<<SAI_GRID(gw), BR, 0, st>>>(Y, Bsrc, Xdst, r, rh, p, v, pt);
        k_b_f0<<<SAI_GRID(gs), 256, 0, st>>>(Y, pt, S);
        SAI_CUDA(cudaMemsetAsync(any, 0, sizeof(int) * 2, st));
        SAI_CUDA(cudaGetLastError());
        cudaStream_t q = st;
        cudaEvent_t ev_in = nullptr, ev_out = nullptr;
        cudaGraphExec_t gexec = nullptr;
        bool whole = false;  // gexec is the whole loop
        const int max_body = (maxit + ITERS_PER_CHECK - 1) / ITERS_PER_CHECK;
        if (!sai_prof_on()) {
            cudaStream_t aux = sai_aux_stream();
            if (aux) {
                SAI_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
                SAI_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
                SAI_CUDA(cudaEventRecord(ev_in, st));
                SAI_CUDA(cudaStreamWaitEvent(aux, ev_in, 0));
                q = aux;
                // the whole loop: a while node around the body
                cudaGraph_t graph = nullptr;
                cudaError_t e = max_body > 0 ? cudaGraphCreate(&graph, 0) : cudaErrorNotSupported;
                cudaGraphConditionalHandle hnd = 0;
                if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hnd, graph, 1, cudaGraphCondAssignDefault);
                cudaGraph_t body = nullptr;
                if (e == cudaSuccess) {
                    cudaGraphNodeParams np = {};
                    np.type = cudaGraphNodeTypeConditional;
                    np.conditional.handle = hnd;
                    np.conditional.type = cudaGraphCondTypeWhile;
                    np.conditional.size = 1;
                    cudaGraphNode_t node = nullptr;
                    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
                    if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
                }
                if (e == cudaSuccess)
                    e = cudaStreamBeginCaptureToGraph(q, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    for (int k = 0; k < ITERS_PER_CHECK; ++k) iteration(q);
                    k_b_cond<<<SAI_GRID(1), 1024, 0, q>>>(nsys, S.active, any, nbody, max_body, hnd);
                    cudaGraph_t cap_g = nullptr;
                    e = cudaStreamEndCapture(q, &cap_g);
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (e == cudaSuccess) {
                    whole = true;
                } else {
                    gexec = nullptr;
                    (void)cudaGetLastError();
                    // groups of iterations with host checks
                    graph = nullptr;
                    SAI_CUDA(cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal));
                    for (int k = 0; k < ITERS_PER_CHECK; ++k) iteration(q);
                    k_b_any<<<SAI_GRID(1), 1024, 0, q>>>(nsys, S.active, any);
                    e = cudaStreamEndCapture(q, &graph);
                    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
                    if (graph) cudaGraphDestroy(graph);
                    if (e != cudaSuccess) {
                        gexec = nullptr;
                        (void)cudaGetLastError();
                    }
                }
                sai_count_grid_add(-(long long)LAUNCHES);  // captured, not run: counted at replay
            }
        }
        sai_status kst = SAI_OK;
        if (whole) {
            if (cudaGraphLaunch(gexec, q) != cudaSuccess) kst = SAI_CUDA_ERROR;
            int nb = 0;
            if (kst == SAI_OK) {
                SAI_CUDA(cudaMemcpyAsync(&nb, nbody, sizeof(int), cudaMemcpyDeviceToHost, q));
                SAI_CUDA(cudaStreamSynchronize(q));
            }
            sai_count_grid_add((long long)nb * LAUNCHES);
        } else {
            int hflag = 0;
            for (int it = 0; it < maxit; it += ITERS_PER_CHECK) {
                if (gexec) {
                    if (cudaGraphLaunch(gexec, q) != cudaSuccess) {
                        kst = SAI_CUDA_ERROR;
                        break;
                    }
                    sai_count_grid_add(LAUNCHES);
                } else {
                    for (int k = 0; k < ITERS_PER_CHECK; ++k) iteration(q);
                    k_b_any<<<SAI_GRID(1), 1024, 0, q>>>(nsys, S.active, any);
                }
                SAI_CUDA(cudaGetLastError());
                SAI_CUDA(cudaMemcpyAsync(&hflag, any, sizeof(int), cudaMemcpyDeviceToHost, q));
                SAI_CUDA(cudaStreamSynchronize(q));
                if (!hflag) break;
            }
        }
        if (gexec) cudaGraphExecDestroy(gexec);
        k_b_start<<<SAI_GRID(gt), 256, 0, q>>>(nsys, maxit, S);  // systems still running after maxit
        if (ev_in) {
            cudaEventRecord(ev_out, q);
            cudaStreamWaitEvent(st, ev_out, 0);
            cudaEventDestroy(ev_in);
            cudaEventDestroy(ev_out);
        }
        SAI_CUDA(cudaGetLastError());
        return kst;
    };
    SAI_TRY(run_pass(Bv, X));

    // ---- SMW per matrix, x_m = yhat_m - What_m z_m, rr per matrix
    double* zcat = misc.as<double>();
    double* cvec = zcat + joff[nmat];
    int* errv = (int*)(cvec + nmat);
    W.z = zcat;
    W.c = cvec;
    W.err = errv;
    const size_t smw_smem = sizeof(double) * ((size_t)smax * smax + smax);
    if (smw_smem > 48 * 1024)
        SAI_CUDA(cudaFuncSetAttribute(k_b_smw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw_smem));
    auto smw_all = [&]() -> sai_status {
        SAI_CUDA(cudaMemsetAsync(cvec, 0, sizeof(double) * nmat, st));
        SAI_CUDA(cudaMemsetAsync(errv, 0, sizeof(int) * nmat, st));
        k_b_smw<<<SAI_GRID(nmat), 256, smw_smem, st>>>(W, X, smax);
        SAI_CUDA(cudaGetLastError());
        return SAI_OK;
    };
    std::vector<int> it_h(nsys), st_h(nsys), err_h(nmat);
    std::vector<double> c_h(nmat);
    std::vector<int32_t> rounds(nmat, 0);
    if (prm->c_adapt) {
        // Theorem 2 with the measured c: a matrix whose c = ||z_m|| exceeds 1
        // has its u_j systems continued from their iterates (correction
        // solves A~ d = u_j - A~ w_j to eps ||b_m|| / (2 sqrt(s_m) 1.05 c_m),
        // w_j += d) before the recovery
        SAI_TRY(smw_all());
        SAI_CUDA(cudaMemcpyAsync(c_h.data(), cvec, sizeof(double) * nmat, cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaMemcpyAsync(it_h.data(), S.iters, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaMemcpyAsync(st_h.data(), S.status, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        std::vector<int> sel(nsys, 0);
        std::vector<double> thr2(thr);
        bool any_sel = false;
        for (int32_t m = 0; m < nmat; ++m)
            if (hs[m]->s > 0 && c_h[m] > 1.0) {
                rounds[m] = 1;
                any_sel = true;
                for (int32_t c = sys0[m] + 1; c < sys0[m + 1]; ++c) {
                    sel[c] = 1;
                    thr2[c] = thr[c] / (1.05 * c_h[m]);
                }
            }
        if (any_sel) {
            Buf extra;
            SAI_TRY(extra.alloc(sizeof(double) * 2 * (size_t)NV + sizeof(int) * (size_t)nsys + 64, st, true));
            double* R = extra.as<double>();
            double* D = R + NV;
            int* dsel = (int*)(D + NV);  // the continued systems
            SAI_CUDA(cudaMemcpyAsync(dsel, sel.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
            SAI_CUDA(cudaMemsetAsync(R, 0, sizeof(double) * (size_t)NV, st));
            k_b_spmv<<<SAI_GRID(gi), BR, 0, st>>>(Y, Ar, Ac, Av, X, R, dsel);
            k_b_resid<<<SAI_GRID(gw), BR, 0, st>>>(Y, Bv, dsel, R);
            SAI_CUDA(cudaGetLastError());
            SAI_CUDA(cudaMemcpyAsync(S.thr, thr2.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
            SAI_TRY(run_pass(R, D));
            k_b_acc<<<SAI_GRID(gw), BR, 0, st>>>(Y, D, dsel, X);
            SAI_CUDA(cudaGetLastError());
            std::vector<int> it2(nsys), st2(nsys);
            SAI_CUDA(cudaMemcpyAsync(it2.data(), S.iters, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaMemcpyAsync(st2.data(), S.status, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            for (int32_t c = 0; c < nsys; ++c)
                if (sel[c]) {
                    it_h[c] += it2[c];
                    if (st_h[c] == B_OK) st_h[c] = st2[c];
                }
            SAI_CUDA(cudaMemcpyAsync(S.iters, it_h.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
            SAI_CUDA(cudaMemcpyAsync(S.status, st_h.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
            SAI_CUDA(cudaStreamSynchronize(st));  // extra (and the host vectors) go out of scope
        }
    }
    SAI_CUDA(cudaEventRecord(e4.e, st));
    SAI_TRY(smw_all());
    for (int32_t m = 0; m < nmat; ++m)
        k_b_xhat<<<SAI_GRID(sai_div_up(hs[m]->n, 256)), 256, 0, st>>>(hs[m]->n, hs[m]->s, X + xoff[m], zcat + joff[m],
                                                                     x[m]);
    SAI_CUDA(cudaGetLastError());
    Ev e5;
    SAI_CUDA(cudaEventRecord(e5.e, st));
    SAI_CUDA(cudaMemcpyAsync(it_h.data(), S.iters, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaMemcpyAsync(st_h.data(), S.status, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaMemcpyAsync(err_h.data(), errv, sizeof(int) * nmat, cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaMemcpyAsync(c_h.data(), cvec, sizeof(double) * nmat, cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    sai_status worst = SAI_OK;
    for (int32_t m = 0; m < nmat; ++m) {
        sai_batch_item& it = items[m];
        it = sai_batch_item{};
        it.s = hs[m]->s;
        it.p = hs[m]->p;
        it.c = c_h[m];
        it.c_rounds = rounds[m];
        for (int32_t c = sys0[m]; c < sys0[m + 1]; ++c) {
            if (it_h[c] > it.iter_max) it.iter_max = it_h[c];
            if (st_h[c] != B_OK && it.status == SAI_OK) it.status = st_h[c];
        }
        if (err_h[m]) it.status = SAI_SINGULAR;
        double nn[2] = {0.0, 0.0};
        SAI_TRY(sai_csc_residual_norms(A[m].n, A[m].col_ptr, A[m].row_idx, A[m].val, b[m], x[m], nn, st));
        it.rr = nn[1] > 0.0 ? sqrt(nn[0] / nn[1]) : sqrt(nn[0]);
        if (it.iter_max > rep->iter_max) rep->iter_max = it.iter_max;
        if (it.status != SAI_OK && worst == SAI_OK) worst = (sai_status)it.status;
    }
    rep->columns = N;
    rep->nnz_M = P.nnz;
    rep->systems = nsys;
    rep->ms_split = ms_between(e0.e, e1.e);
    rep->ms_build = ms_between(e1.e, e2.e);
    rep->ms_krylov = ms_between(e2.e, e4.e);
    rep->ms_smw = ms_between(e4.e, e5.e);
    return worst;
}

}  // namespace

namespace {

// The matrices split one after another on st and stacked (for the build-only
// entry points; sai_solve_batched splits on worker streams).
sai_status split_and_stack(int32_t nmat, const sai_csc_view* A, const sai_solve_params* prm,
                           std::vector<std::unique_ptr<sai_split_s>>& hs, sai_split_s& bd, cudaStream_t st)
{
    if (nmat < 1 || !A || !prm || prm->split.zero_diag != 0) return SAI_INVALID_ARG;
    if (prm->sai == 1 && prm->psai.tol_mode == 0) return SAI_NOT_IMPLEMENTED;
    int dev = 0, sms = 0;
    SAI_CUDA(cudaGetDevice(&dev));
    SAI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    hs.resize((size_t)nmat);
    for (int32_t m = 0; m < nmat; ++m) {
        if (A[m].n < 1) return SAI_INVALID_ARG;
        hs[m].reset(new (std::nothrow) sai_split_s);
        if (!hs[m]) return SAI_OOM;
        SAI_TRY(sai_split_build(&A[m], &prm->split, st, true, hs[m].get()));
    }
    std::vector<int64_t> R0;
    return stack_splits(nmat, hs, bd, R0, (int64_t)sms * 8, st);
}

}  // namespace

extern "C" sai_status sai_build_batched(int32_t nmat, const sai_csc_view* A, const sai_solve_params* prm,
                                        sai_stream_t stream, sai_precond* out)
{
    if (!out) return SAI_INVALID_ARG;
    *out = nullptr;
    sai_pool_init_once();
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<std::unique_ptr<sai_split_s>> hs;
    sai_split_s bd;
    SAI_TRY(split_and_stack(nmat, A, prm, hs, bd, st));
    sai_precond_s* P = new (std::nothrow) sai_precond_s();
    if (!P) return SAI_OOM;
    const sai_status r = prm->sai == 0 ? sai_spai_build(&bd, &prm->spai, st, false, P)
                                       : sai_psai_build(&bd, &prm->psai, st, false, P);
    if (r != SAI_OK) {
        delete P;
        return r;
    }
    *out = P;
    return SAI_OK;
}

extern "C" sai_status sai_build_autotune_batched(int32_t nmat, const sai_csc_view* A, const sai_solve_params* prm,
                                                 sai_stream_t stream, sai_build_tuning* out)
{
    if (!out) return SAI_INVALID_ARG;
    sai_pool_init_once();
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<std::unique_ptr<sai_split_s>> hs;
    sai_split_s bd;
    SAI_TRY(split_and_stack(nmat, A, prm, hs, bd, st));
    return sai_build_autotune_run(&bd, prm->sai, &prm->spai, &prm->psai, st, out);
}

extern "C" sai_status sai_solve_batched(int32_t nmat, const sai_csc_view* A, const double* const* b,
                                        const sai_solve_params* prm, double* const* x, sai_batch_item* items,
                                        sai_batch_report* rep, sai_stream_t stream)
{
    sai_pool_init_once();
    return batched_impl(nmat, A, b, prm, x, items, rep, (cudaStream_t)stream);
}

sai_status sai_batch_work_reset()
{
    double z[PROF_NSITES * 2] = {};
    SAI_CUDA(cudaMemcpyToSymbol(d_bwork, z, sizeof(z)));
    return SAI_OK;
}

sai_status sai_batch_work_read(double* out)
{
    SAI_CUDA(cudaMemcpyFromSymbol(out, d_bwork, sizeof(double) * PROF_NSITES * 2));
    return SAI_OK;
}
