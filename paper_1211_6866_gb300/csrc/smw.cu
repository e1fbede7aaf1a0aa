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

#include <mutex>

#include "internal.h"

namespace {

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
        else
            k_smw_gather_adj<<<SAI_GRID(sai_div_up((int64_t)s * (s + 1) * 32, 256)), 256, 0, st>>>(
                s, h->U_cp.as<int64_t>(), h->U_ri.as<int32_t>(), h->U_v.as<double>(), Y, C.as<double>(),
                g.as<double>());
        k_lu_solve<<<SAI_GRID(1), 1024, 0, st>>>(s, C.as<double>(), g.as<double>(), z.as<double>(), cbuf.as<double>(),
                                       err.as<int>());
    }
    if (n > 0) k_smw_update<<<SAI_GRID(sai_div_up(n, 256)), 256, 0, st>>>(n, s, Y, z.as<double>(), x);
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

constexpr int NOALLOC_MAX_DEV = 64;
static unsigned char* g_noalloc_ptr[NOALLOC_MAX_DEV];
static std::mutex g_noalloc_mu;

// Device address of the scratch array for the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
sai_status noalloc_scratch(unsigned char** out)
{
    int dev = 0;
    SAI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEV) return SAI_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        SAI_CUDA(cudaGetSymbolAddress(&p, g_smw_noalloc_scratch));
        g_noalloc_ptr[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_ptr[dev];
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
    // the array keeps the previous call's contents: clear what must start at zero
    SAI_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    SAI_CUDA(cudaMemsetAsync(cval, 0, sizeof(double), st));
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
