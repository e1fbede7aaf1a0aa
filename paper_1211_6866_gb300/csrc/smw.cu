// smw.cu -- Sherman-Morrison-Woodbury recovery of x (Theorem 1; eq.
// (composi)): xhat = yhat - What (I + V^T What)^{-1} (V^T yhat), with
// V = [e_J0 .. e_J(s-1)], so V^T What is What(J,:) and V^T yhat is yhat(J).
//   k_smw_gather   C = I + What(J,:) (column-major s x s), g = yhat(J)
//   k_lu_solve     Gaussian elimination with partial pivoting (first largest
//                  |pivot| wins), one block; z = C^{-1} g, c = ||z||
//   k_smw_update   xhat(i) = yhat(i) - sum_t What(i,t) z_t, one thread per row
// and its adjoint for A^T = A~^T + V U^T (the backward pass), where the small
// system is C = I + U^T What, g = U^T yhat (k_smw_gather_adj).
#include <math.h>

#include "internal.h"

namespace {

int g_smw_sms = 0;
int g_num_sms_smw()
{
    if (g_smw_sms == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            g_smw_sms = v;
        else
            return 1;
    }
    return g_smw_sms;
}

__global__ void k_smw_gather(int32_t n, int32_t s, const int32_t* J, const double* Y, double* C, double* g)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)s * s) return;
    const int col = (int)(t / s), row = (int)(t - (int64_t)col * s);  // C(row, col)
    const int64_t ld = (int64_t)s + 1;
    C[(int64_t)col * s + row] = (row == col ? 1.0 : 0.0) + Y[(int64_t)J[row] * ld + 1 + col];
    if (col == 0) g[row] = Y[(int64_t)J[row] * ld];
}

// Adjoint form (A^T = A~^T + V U^T): C = I + U^T What (column-major s x s),
// g = U^T yhat. One warp per (row a of U^T, column b of Y), b = 0 is yhat.
__global__ void k_smw_gather_adj(int32_t s, const int64_t* Ucp, const int32_t* Uri, const double* Uv,
                                 const double* Y, double* C, double* g)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)s * (s + 1)) return;
    const int a = (int)(w % s), b = (int)(w / s);
    const int64_t ld = (int64_t)s + 1;
    double acc = 0.0;
    for (int64_t q = Ucp[a] + lane; q < Ucp[a + 1]; q += 32) acc = fma(Uv[q], Y[(int64_t)Uri[q] * ld + b], acc);
    acc = warp_sum(acc);
    if (lane == 0) {
        if (b == 0) g[a] = acc;
        else C[(int64_t)(b - 1) * s + a] = (a == b - 1 ? 1.0 : 0.0) + acc;
    }
}

__global__ void k_lu_solve(int32_t s, double* C, double* g, double* z, double* c_out, int* err)
{
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    __shared__ int piv_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = 0; k < s; ++k) {
        double best = -1.0;
        int bidx = s;
        for (int i = k + tid; i < s; i += nt) {
            const double a = fabs(C[(int64_t)k * s + i]);
            if (a > best) {
                best = a;
                bidx = i;
            }
        }
        bv[tid] = best;
        bi[tid] = bidx;
        __syncthreads();
        for (int w = nt >> 1; w > 0; w >>= 1) {
            if (tid < w) {
                const double ov = bv[tid + w];
                const int oi = bi[tid + w];
                if (ov > bv[tid] || (ov == bv[tid] && oi < bi[tid])) {
                    bv[tid] = ov;
                    bi[tid] = oi;
                }
            }
            __syncthreads();
        }
        if (tid == 0) piv_s = (bv[0] > 0.0) ? bi[0] : -1;
        __syncthreads();
        const int piv = piv_s;
        if (piv < 0) {
            if (tid == 0) *err = 1;
            return;
        }
        if (piv != k) {
            for (int j = tid; j < s; j += nt) {
                const double tmp = C[(int64_t)j * s + k];
                C[(int64_t)j * s + k] = C[(int64_t)j * s + piv];
                C[(int64_t)j * s + piv] = tmp;
            }
            if (tid == 0) {
                const double tmp = g[k];
                g[k] = g[piv];
                g[piv] = tmp;
            }
        }
        __syncthreads();
        const double akk = C[(int64_t)k * s + k];
        const double gk = g[k];
        for (int i = k + 1 + tid; i < s; i += nt) {
            const double l = C[(int64_t)k * s + i] / akk;
            C[(int64_t)k * s + i] = l;
            for (int j = k + 1; j < s; ++j) C[(int64_t)j * s + i] -= l * C[(int64_t)j * s + k];
            g[i] -= l * gk;
        }
        __syncthreads();
    }
    for (int i = tid; i < s; i += nt) z[i] = g[i];
    __syncthreads();
    for (int j = s - 1; j >= 0; --j) {
        if (tid == 0) z[j] = z[j] / C[(int64_t)j * s + j];
        __syncthreads();
        const double zj = z[j];
        for (int i = tid; i < j; i += nt) z[i] -= C[(int64_t)j * s + i] * zj;
        __syncthreads();
    }
    double acc = 0.0;
    for (int i = tid; i < s; i += nt) acc += z[i] * z[i];
    bv[tid] = acc;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int q = 0; q < nt; ++q) t += bv[q];
        *c_out = sqrt(t);
    }
}

__global__ void k_smw_update(int32_t n, int32_t s, const double* Y, const double* z, double* x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t ld = (int64_t)s + 1;
    const double* row = Y + i * ld;
    double v = row[0];
    for (int t = 0; t < s; ++t) v = fma(-row[1 + t], z[t], v);
    x[i] = v;
}


// ---------------------------------------------------------------- large s
// For s > LU_SMALL the s x s system is solved by a blocked right-looking LU
// with the same partial pivoting (largest |pivot|, the first row on ties),
// panels of LU_NB columns:
//   k_lu_panel   one block factors columns [k0, k0 + kb) over rows [k0, s)
//   k_lu_swap    applies the panel's interchanges to the other columns and g
//   k_lu_trsm    U12 = L11^{-1} A12, one thread per trailing column
//   k_lu_gemm    A22 -= L21 U12 on 64 x 64 tiles in FP64
//   k_lu_trsv    L y = Pg, U z = y in blocks of 32 rows, one block; c = ||z||
// After a zero pivot the panel sets *err and every later kernel returns
// without touching C, so no unwritten pivot index is ever read.
constexpr int LU_SMALL = 256;
constexpr int LU_NB = 16;

__global__ void __launch_bounds__(1024) k_lu_panel(int32_t s, int32_t k0, int32_t kb, double* C, int32_t* piv,
                                                   int* err)
{
    __shared__ double wv[32];
    __shared__ int wi[32];
    __shared__ int pv_s;
    if (*err) return;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nwarps = nt >> 5;
    for (int j = k0; j < k0 + kb; ++j) {
        double* cj = C + (int64_t)j * s;
        double best = -1.0;
        int bidx = s;
        for (int i = j + tid; i < s; i += nt) {
            const double a = fabs(cj[i]);
            if (a > best) {
                best = a;
                bidx = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(SAI_FULL, best, o);
            const int oi = __shfl_xor_sync(SAI_FULL, bidx, o);
            if (ov > best || (ov == best && oi < bidx)) {
                best = ov;
                bidx = oi;
            }
        }
        if (lane == 0) {
            wv[wid] = best;
            wi[wid] = bidx;
        }
        __syncthreads();
        if (wid == 0) {
            best = lane < nwarps ? wv[lane] : -1.0;
            bidx = lane < nwarps ? wi[lane] : s;
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(SAI_FULL, best, o);
                const int oi = __shfl_xor_sync(SAI_FULL, bidx, o);
                if (ov > best || (ov == best && oi < bidx)) {
                    best = ov;
                    bidx = oi;
                }
            }
            if (lane == 0) pv_s = (best > 0.0 && bidx < s) ? bidx : -1;
        }
        __syncthreads();
        const int p = pv_s;
        if (p < 0) {
            if (tid == 0) *err = 1;
            return;
        }
        if (tid == 0) piv[j] = p;
        if (p != j)
            for (int c = k0 + tid; c < k0 + kb; c += nt) {
                const double t = C[(int64_t)c * s + j];
                C[(int64_t)c * s + j] = C[(int64_t)c * s + p];
                C[(int64_t)c * s + p] = t;
            }
        __syncthreads();
        const double ajj = cj[j];
        for (int i = j + 1 + tid; i < s; i += nt) {
            const double l = cj[i] / ajj;
            cj[i] = l;
            for (int c = j + 1; c < k0 + kb; ++c) C[(int64_t)c * s + i] -= l * C[(int64_t)c * s + j];
        }
        __syncthreads();
    }
}

// thread t < s: column t (outside the panel); thread s: g
__global__ void k_lu_swap(int32_t s, int32_t k0, int32_t kb, double* C, double* g, const int32_t* piv,
                          const int* err)
{
    if (*err) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > s || (t >= k0 && t < k0 + kb)) return;
    double* v = t < s ? C + t * s : g;
    for (int j = k0; j < k0 + kb; ++j) {
        const int p = piv[j];
        if (p <= j || p >= s) continue;
        const double a = v[j];
        v[j] = v[p];
        v[p] = a;
    }
}

__global__ void k_lu_trsm(int32_t s, int32_t k0, int32_t kb, double* C, const int* err)
{
    if (*err) return;
    const int64_t c = (int64_t)k0 + kb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s) return;
    double x[LU_NB];
    double* col = C + c * s + k0;
#pragma unroll
    for (int r = 0; r < LU_NB; ++r) {
        if (r < kb) {
            double v = col[r];
            for (int q = 0; q < r; ++q) v -= C[(int64_t)(k0 + q) * s + k0 + r] * x[q];
            x[r] = v;
            col[r] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_lu_gemm(int32_t s, int32_t k0, int32_t kb, double* C, const int* err)
{
    __shared__ double Ls[LU_NB][64];
    __shared__ double Us[LU_NB][65];
    if (*err) return;
    const int k1 = k0 + kb;
    const int m = s - k1;
    const int nt = (m + 63) / 64;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int64_t blk = blockIdx.x; blk < (int64_t)nt * nt; blk += gridDim.x) {
        const int i0 = k1 + (int)(blk % nt) * 64, c0 = k1 + (int)(blk / nt) * 64;
        for (int e = tid; e < kb * 64; e += 256) {
            const int q = e / 64, ii = e % 64;
            Ls[q][ii] = i0 + ii < s ? C[(int64_t)(k0 + q) * s + i0 + ii] : 0.0;
        }
        for (int e = tid; e < kb * 64; e += 256) {
            const int q = e % kb, cc = e / kb;
            Us[q][cc] = c0 + cc < s ? C[(int64_t)(c0 + cc) * s + k0 + q] : 0.0;
        }
        __syncthreads();
        double acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
        for (int q = 0; q < kb; ++q) {
            double l[4], u[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) l[a] = Ls[q][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) u[b] = Us[q][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(l[a], u[b], acc[a][b]);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = c0 + ty + 16 * b;
            if (c >= s) continue;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int i = i0 + tx + 16 * a;
                if (i < s) C[(int64_t)c * s + i] -= acc[a][b];
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_lu_trsv(int32_t s, const double* C, const double* g, double* z,
                                                  double* c_out, const int* err)
{
    __shared__ double yb[32];
    __shared__ double red[32];
    if (*err) return;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < s; i += nt) z[i] = g[i];
    __syncthreads();
    for (int j0 = 0; j0 < s; j0 += 32) {  // L y = Pg, unit diagonal
        const int jb = s - j0 < 32 ? s - j0 : 32;
        if (wid == 0) {
            double v = lane < jb ? z[j0 + lane] : 0.0;
            for (int jj = 0; jj < jb; ++jj) {
                const double yj = __shfl_sync(SAI_FULL, v, jj);
                if (lane > jj && lane < jb) v -= C[(int64_t)(j0 + jj) * s + j0 + lane] * yj;
            }
            if (lane < jb) {
                z[j0 + lane] = v;
                yb[lane] = v;
            }
        }
        __syncthreads();
        for (int i = j0 + jb + tid; i < s; i += nt) {
            double v = z[i];
            for (int jj = 0; jj < jb; ++jj) v -= C[(int64_t)(j0 + jj) * s + i] * yb[jj];
            z[i] = v;
        }
        __syncthreads();
    }
    for (int j1 = s; j1 > 0; j1 -= 32) {  // U z = y
        const int j0 = j1 - 32 > 0 ? j1 - 32 : 0, jb = j1 - j0;
        if (wid == 0) {
            double v = lane < jb ? z[j0 + lane] : 0.0;
            for (int jj = jb - 1; jj >= 0; --jj) {
                if (lane == jj) v = v / C[(int64_t)(j0 + jj) * s + j0 + jj];
                const double zj = __shfl_sync(SAI_FULL, v, jj);
                if (lane < jj) v -= C[(int64_t)(j0 + jj) * s + j0 + lane] * zj;
            }
            if (lane < jb) {
                z[j0 + lane] = v;
                yb[lane] = v;
            }
        }
        __syncthreads();
        for (int i = tid; i < j0; i += nt) {
            double v = z[i];
            for (int jj = 0; jj < jb; ++jj) v -= C[(int64_t)(j0 + jj) * s + i] * yb[jj];
            z[i] = v;
        }
        __syncthreads();
    }
    double acc = 0.0;
    for (int i = tid; i < s; i += nt) acc = fma(z[i], z[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) t += red[w];
        *c_out = sqrt(t);
    }
}

// C = I + U^T What, g = U^T yhat for large s: a warp forms 64 consecutive
// columns b of Y = [yhat, What] for one column a of U, summing over U's
// entries in stored order. Items are column-chunk-major, so the warps
// running together read the same 64 columns of Y (n x 64 values, in L2).
__global__ void k_smw_gather_adj_big(int32_t s, const int64_t* Ucp, const int32_t* Uri, const double* Uv,
                                     const double* Y, double* C, double* g)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ld = (int64_t)s + 1;
    const int64_t nbc = (ld + 63) / 64;
    for (int64_t it = w0; it < (int64_t)s * nbc; it += nw) {
        const int a = (int)(it % s);
        const int64_t b0 = (it / s) * 64;
        const int64_t ba = b0 + lane, bb = b0 + 32 + lane;
        double acc0 = 0.0, acc1 = 0.0;
        const int64_t q0 = Ucp[a], q1 = Ucp[a + 1];
        for (int64_t qb = q0; qb < q1; qb += 32) {
            const int64_t q = qb + lane;
            const int32_t ri = q < q1 ? Uri[q] : 0;
            const double uv = q < q1 ? Uv[q] : 0.0;
            const int m = q1 - qb < 32 ? (int)(q1 - qb) : 32;
            for (int e = 0; e < m; ++e) {
                const int64_t i = __shfl_sync(SAI_FULL, ri, e);
                const double u = __shfl_sync(SAI_FULL, uv, e);
                const double* row = Y + i * ld;
                if (ba < ld) acc0 = fma(u, row[ba], acc0);
                if (bb < ld) acc1 = fma(u, row[bb], acc1);
            }
        }
        if (ba < ld) {
            if (ba == 0) g[a] = acc0;
            else C[(ba - 1) * s + a] = (a == ba - 1 ? 1.0 : 0.0) + acc0;
        }
        if (bb < ld) C[(bb - 1) * s + a] = (a == bb - 1 ? 1.0 : 0.0) + acc1;
    }
}

// xhat(i) = yhat(i) - sum_t What(i,t) z_t for large s, one warp per row
__global__ void k_smw_update_big(int32_t n, int32_t s, const double* Y, const double* z, double* x)
{
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t ld = (int64_t)s + 1;
    const double* row = Y + i * ld;
    double v = 0.0;
    for (int t = lane; t < s; t += 32) v = fma(row[1 + t], z[t], v);
    v = warp_sum(v);
    if (lane == 0) x[i] = row[0] - v;
}

// LU solve of the s x s system C z = g (C, g overwritten) for large s.
sai_status lu_big(int32_t s, double* C, double* g, double* z, double* c_out, int* err, cudaStream_t st)
{
    Buf pivb;
    SAI_TRY(pivb.alloc(sizeof(int32_t) * (size_t)s, st, true));
    int32_t* piv = pivb.as<int32_t>();
    for (int k0 = 0; k0 < s; k0 += LU_NB) {
        const int kb = s - k0 < LU_NB ? s - k0 : LU_NB;
        k_lu_panel<<<SAI_GRID(1), 1024, 0, st>>>(s, k0, kb, C, piv, err);
        k_lu_swap<<<SAI_GRID(sai_div_up((int64_t)s + 1, 256)), 256, 0, st>>>(s, k0, kb, C, g, piv, err);
        const int m = s - k0 - kb;
        if (m > 0) {
            k_lu_trsm<<<SAI_GRID(sai_div_up(m, 128)), 128, 0, st>>>(s, k0, kb, C, err);
            const int64_t nt = (m + 63) / 64;
            const int64_t gb = nt * nt < (int64_t)g_num_sms_smw() * 8 ? nt * nt : (int64_t)g_num_sms_smw() * 8;
            k_lu_gemm<<<SAI_GRID(gb), 256, 0, st>>>(s, k0, kb, C, err);
        }
    }
    k_lu_trsv<<<SAI_GRID(1), 1024, 0, st>>>(s, C, g, z, c_out, err);
    SAI_CUDA(cudaGetLastError());
    return SAI_OK;
}

}  // namespace

namespace {

sai_status smw_common(const sai_split_s* h, const double* Y, double* x, double* c_out, bool adjoint, cudaStream_t st)
{
    if (!h || (h->n > 0 && (!Y || !x))) return SAI_INVALID_ARG;
    const int32_t n = h->n, s = h->s;
    const size_t ss = (size_t)(s > 0 ? s : 1);
    Buf C, g, z, cbuf, err;
    SAI_TRY(C.alloc(sizeof(double) * ss * ss, st, true));
    SAI_TRY(g.alloc(sizeof(double) * ss, st, true));
    SAI_TRY(z.alloc(sizeof(double) * ss, st, true));
    SAI_TRY(cbuf.alloc(sizeof(double), st, true));
    SAI_TRY(err.alloc(sizeof(int), st, true));
    SAI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    SAI_CUDA(cudaMemsetAsync(cbuf.p, 0, sizeof(double), st));
    if (s > 0) {
        if (!adjoint)
            k_smw_gather<<<SAI_GRID(sai_div_up((int64_t)s * s, 256)), 256, 0, st>>>(n, s, h->J.as<int32_t>(), Y,
                                                                                   C.as<double>(), g.as<double>());
        else if (s <= LU_SMALL)
            k_smw_gather_adj<<<SAI_GRID(sai_div_up((int64_t)s * (s + 1) * 32, 256)), 256, 0, st>>>(
                s, h->U_cp.as<int64_t>(), h->U_ri.as<int32_t>(), h->U_v.as<double>(), Y, C.as<double>(),
                g.as<double>());
        else {
            const int64_t items = (int64_t)s * (((int64_t)s + 1 + 63) / 64);
            const int64_t gb = sai_div_up(items, 8) < (int64_t)g_num_sms_smw() * 16 ? sai_div_up(items, 8)
                                                                                   : (int64_t)g_num_sms_smw() * 16;
            k_smw_gather_adj_big<<<SAI_GRID(gb), 256, 0, st>>>(s, h->U_cp.as<int64_t>(), h->U_ri.as<int32_t>(),
                                                               h->U_v.as<double>(), Y, C.as<double>(),
                                                               g.as<double>());
        }
        if (s <= LU_SMALL)
            k_lu_solve<<<SAI_GRID(1), 1024, 0, st>>>(s, C.as<double>(), g.as<double>(), z.as<double>(),
                                                     cbuf.as<double>(), err.as<int>());
        else
            SAI_TRY(lu_big(s, C.as<double>(), g.as<double>(), z.as<double>(), cbuf.as<double>(), err.as<int>(), st));
    }
    if (n > 0 && s <= LU_SMALL) k_smw_update<<<SAI_GRID(sai_div_up(n, 256)), 256, 0, st>>>(n, s, Y, z.as<double>(), x);
    else if (n > 0)
        k_smw_update_big<<<SAI_GRID(sai_div_up((int64_t)n * 32, 256)), 256, 0, st>>>(n, s, Y, z.as<double>(), x);
    SAI_CUDA(cudaGetLastError());
    int herr = 0;
    double hc = 0.0;
    SAI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaMemcpyAsync(&hc, cbuf.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    if (herr) return SAI_SINGULAR;
    if (c_out) *c_out = hc;
    return SAI_OK;
}

}  // namespace

sai_status sai_smw_run(const sai_split_s* h, const double* Y, double* x, double* c_out, cudaStream_t st)
{
    return smw_common(h, Y, x, c_out, false, st);
}

sai_status sai_smw_adj_run(const sai_split_s* h, const double* Y, double* x, double* c_out, cudaStream_t st)
{
    return smw_common(h, Y, x, c_out, true, st);
}

// ---------------------------------------------------------------- allocation-free variant
// sai_smw_recover_noalloc: the same SMW recovery for callers that cannot
// allocate device memory -- code that runs where every device byte is owned
// by a host framework's own pool or a fixed budget, or where an allocation
// would synchronise or is not permitted. Its scratch (the s x s matrix, two
// s-vectors, c and an error flag) is this file-scope array, reserved once on
// every device that loads the library and held until the process exits.
namespace {

constexpr int NOALLOC_MAX_S = 256;
constexpr size_t NOALLOC_C_OFF = 0;
constexpr size_t NOALLOC_G_OFF = NOALLOC_C_OFF + sizeof(double) * NOALLOC_MAX_S * NOALLOC_MAX_S;
constexpr size_t NOALLOC_Z_OFF = NOALLOC_G_OFF + sizeof(double) * NOALLOC_MAX_S;
constexpr size_t NOALLOC_CV_OFF = NOALLOC_Z_OFF + sizeof(double) * NOALLOC_MAX_S;
constexpr size_t NOALLOC_ERR_OFF = NOALLOC_CV_OFF + 256;
constexpr size_t NOALLOC_BYTES = NOALLOC_ERR_OFF + 256;

static __device__ __align__(256) unsigned char g_smw_noalloc_scratch[NOALLOC_BYTES];

// Device address of the scratch array in the current device's context (the
// host-side symbol is only a stand-in, not a device address). Looked up on
// every call: the lookup allocates nothing, and an address kept from an
// earlier context (before a cudaDeviceReset, say) would no longer be valid.
sai_status noalloc_scratch(unsigned char** out)
{
    void* p = nullptr;
    SAI_CUDA(cudaGetSymbolAddress(&p, g_smw_noalloc_scratch));
    *out = (unsigned char*)p;
    return SAI_OK;
}

}  // namespace

extern "C" sai_status sai_smw_recover_noalloc(int32_t n, int32_t s, const int32_t* J, const double* Y, double* x,
                                              double* c_out, sai_stream_t stream)
{
    if (n < 0 || s < 0 || s > n || (n > 0 && (!Y || !x)) || (s > 0 && !J)) return SAI_INVALID_ARG;
    if (s > NOALLOC_MAX_S) return SAI_INVALID_ARG;  // beyond the static scratch
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    SAI_TRY(noalloc_scratch(&base));
    double* C = (double*)(base + NOALLOC_C_OFF);
    double* g = (double*)(base + NOALLOC_G_OFF);
    double* z = (double*)(base + NOALLOC_Z_OFF);
    double* cval = (double*)(base + NOALLOC_CV_OFF);
    int* err = (int*)(base + NOALLOC_ERR_OFF);
    // the array keeps the previous call's contents: clear what must start at
    // zero; z too, so that a zero pivot (z left unwritten) gives x = yhat
    SAI_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    SAI_CUDA(cudaMemsetAsync(cval, 0, sizeof(double), st));
    if (s > 0) SAI_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * (size_t)s, st));
    if (s > 0) {
        k_smw_gather<<<SAI_GRID(sai_div_up((int64_t)s * s, 256)), 256, 0, st>>>(n, s, J, Y, C, g);
        k_lu_solve<<<SAI_GRID(1), 1024, 0, st>>>(s, C, g, z, cval, err);
    }
    if (n > 0) k_smw_update<<<SAI_GRID(sai_div_up(n, 256)), 256, 0, st>>>(n, s, Y, z, x);
    SAI_CUDA(cudaGetLastError());
    int herr = 0;
    double hc = 0.0;
    SAI_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaMemcpyAsync(&hc, cval, sizeof(double), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    if (herr) return SAI_SINGULAR;
    if (c_out) *c_out = hc;
    return SAI_OK;
}
