// krylov.cu -- the s+1 right-preconditioned Krylov solves of Procedure *
// (A~ y = b, A~ w_j = u_j, eqs. (regprob), (auxi)) for k systems at once, and
// the transposed solves A~^T y = rhs with preconditioner M^T of the backward pass.
//
// Layout: inside the solver every block of k vectors is stored system-major
// (system c's vector is contiguous, leading dimension ld = n rounded up to 32),
// so each warp streams 256 contiguous bytes of one system and no lane idles.
// The caller's n x k row-major B and X are transposed on entry and exit.
//
// Work distribution: device-side lists of the systems that take part in a
// step (list[0] = count, list[1..] = system indices, ascending) are rebuilt
// by the control kernels (single-block, or one block per system with the
// last block to arrive rebuilding the list); data-parallel kernels loop over the
// items (system in the list) x (row tile or row chunk), so converged systems
// cost nothing and the host never needs to know which systems are active.
// Inner products are formed per (system, row chunk) by one warp and summed
// in a fixed order, so results do not depend on scheduling.
//
// BiCGStab: van der Vorst's recurrence on A~ M z = b with y = M z updated
// directly; stop tests after the half step (s) and the full step (r).
// GMRES(m): Arnoldi with classical Gram-Schmidt applied twice, the second
// pass delayed by one step and fused with the next step's reduction (one
// reduction and one update pass over the basis per step); Givens rotations;
// stop on the rotated residual |g_{j+1}|; restart from the true residual
// b - A~ y.
#include <math.h>

#include "internal.h"

namespace {

constexpr int CTRL = 256;      // threads of the single-block control kernels (>= k of GMRES)
constexpr int KBIG = 1 << 18;  // systems per FP64 BiCGStab call (its control kernels loop over systems)
constexpr int CHUNK = 1024;    // rows per (system, chunk) reduction item (one warp)
constexpr int CHUNK_U = 256;   // rows per item of the GMRES update (no per-vector reduction)
constexpr int TILE = 256;      // rows per SpMV item (one block)
constexpr int PJ = 16;         // basis vectors per register-tiled projection pass
constexpr int IT_WARPS = 4;    // warps per block of the item kernels (small blocks: finer occupancy)
constexpr int UP_CWARPS = 4;   // consumer warps of the ring-fed GMRES update (plus one producer warp)
constexpr int UP_PT = 2;       // 16-byte pieces per consumer thread of a vector slice (slices of 4 KB)
constexpr int UP_VPS = 2;      // vector slices per stage of its ring
constexpr int UP_STAGES = 4;   // stages of its ring

enum { ST_OK = 0, ST_MAXITER = 5, ST_BREAKDOWN = 6 };  // same values as sai_status

int g_sms = 0;
// resident blocks per SM of the GMRES dot / update kernels, [0] double, [1] float
int g_res_dots[2] = {1, 1}, g_res_upd[2] = {1, 1}, g_res_ring[2] = {1, 1}, g_res_sellp[2] = {1, 1};

// ---------------------------------------------------------------- accounting
__device__ double d_kwork[PROF_NSITES * 2];

struct Dims {
    double n, nnzA, nnzM;
    double esz;                           // bytes per vector / matrix value
    int site_spmm, site_dots, site_upd;   // profile sites of this precision
};

__device__ __forceinline__ void kwork_add(int site, double bytes, double flops)
{
    atomicAdd(&d_kwork[2 * site], bytes);
    atomicAdd(&d_kwork[2 * site + 1], flops);
}

// one SpMV launch over k_act systems: matrix once, x read once, y written
__device__ __forceinline__ void spmm_work(const Dims& D, double nnz, int kact)
{
    if (kact > 0)
        kwork_add(D.site_spmm, 8.0 * (D.n + 1) + (4.0 + D.esz) * nnz + 2.0 * D.esz * D.n * kact, 2.0 * nnz * kact);
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

// The same list built by the whole block (any k): each thread counts a
// contiguous run of systems, a block scan gives each run its offset, and the
// runs are written in order, so the list is ascending like build_list's.
// Every thread of the block calls it after a __syncthreads that makes the
// mask final; it ends with one, so list[0] is visible to the block after it.
__device__ void build_list_block(int k, const int* mask, int* list)
{
    __shared__ int wsum[32];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5, nwarps = (nt + 31) >> 5;
    const int per = (k + nt - 1) / nt;
    const int c0 = tid * per < k ? tid * per : k;
    const int c1 = c0 + per < k ? c0 + per : k;
    int cnt = 0;
    for (int c = c0; c < c1; ++c) cnt += mask[c] != 0;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(SAI_FULL, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int v = lane < nwarps ? wsum[lane] : 0;
        int w = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(SAI_FULL, w, o);
            if (lane >= o) w += u;
        }
        if (lane < nwarps) wsum[lane] = w - v;  // exclusive offset of warp `lane`
    }
    __syncthreads();
    int pos = wsum[wid] + incl - cnt;
    for (int c = c0; c < c1; ++c)
        if (mask[c]) list[1 + pos++] = c;
    if (tid == nt - 1) list[0] = pos;
    __syncthreads();
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

// The same two copies through 32 x 32 shared-memory tiles (32 x 8 threads),
// so that both the row-major and the system-major side are accessed in
// contiguous runs; used when k is at least 32.
template <bool TO_SOA>
__global__ void __launch_bounds__(256) k_soa_tiled(int64_t n, int k, int64_t ld, const double* __restrict__ src,
                                                   double* __restrict__ dst)
{
    __shared__ double tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t ti = (n + 31) / 32, tc = (k + 31) / 32;
    for (int64_t t = blockIdx.x; t < ti * tc; t += gridDim.x) {
        const int64_t i0 = (t / tc) * 32;
        const int c0 = (int)(t % tc) * 32;
        if (TO_SOA) {
            for (int j = ty; j < 32; j += 8) {  // rows i0 + j, columns c0 + tx
                const int64_t i = i0 + j;
                const int c = c0 + tx;
                if (i < n && c < k) tile[j][tx] = src[i * k + c];
            }
            __syncthreads();
            for (int j = ty; j < 32; j += 8) {  // system c0 + j, rows i0 + tx
                const int c = c0 + j;
                const int64_t i = i0 + tx;
                if (i < n && c < k) dst[(int64_t)c * ld + i] = tile[tx][j];
            }
        } else {
            for (int j = ty; j < 32; j += 8) {  // system c0 + j, rows i0 + tx
                const int c = c0 + j;
                const int64_t i = i0 + tx;
                if (i < n && c < k) tile[tx][j] = src[(int64_t)c * ld + i];
            }
            __syncthreads();
            for (int j = ty; j < 32; j += 8) {  // rows i0 + j, columns c0 + tx
                const int64_t i = i0 + j;
                const int c = c0 + tx;
                if (i < n && c < k) dst[i * k + c] = tile[j][tx];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- SpMV over a list
// When the k systems' vectors exceed what L2 holds next to the matrix, the
// SpMVs take their items system-group-major (template flag GM, chosen on the
// host from k): the warps running at one time then gather from the vectors
// of a few systems, which stay in L2, instead of from all of them. Each
// item's arithmetic is the same either way.
constexpr int64_t SPMV_GMAJ_BYTES = 64ll << 20;
inline bool spmv_group_major(int k, int64_t n, size_t esz)
{
    return (int64_t)k * n * (int64_t)esz > SPMV_GMAJ_BYTES;
}

// Y[c] = A X[c] (mode 0), B[c] - A X[c] (mode 1) or Y[c] + A X[c] (mode 2) for the systems in list, in
// the value type T (FP64, or FP32 for the inner solves of the refined GMRES).
// Items are (row tile, system), tile-major, so the systems of a tile reuse
// the tile's matrix rows from cache (system-group-major for many systems, as
// above). One thread per row (CSR).
template <class T, int MODE, bool GM>
__global__ void __launch_bounds__(TILE) k_spmv(int32_t n, int64_t ld, const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ ci, const T* __restrict__ v,
                                               const T* __restrict__ X, T* __restrict__ Y,
                                               const T* __restrict__ B, const int* __restrict__ list,
                                               const int* __restrict__ jstop, int jmax)
{
    constexpr int CT = 4;  // systems per thread: each matrix entry is loaded once for CT gathers
    if (jstop && *jstop >= jmax) return;  // the step needs no operator application
    const int cnt = list[0];
    const int groups = (cnt + CT - 1) / CT;
    const int64_t tiles = ((int64_t)n + TILE - 1) / TILE;
    for (int64_t it = blockIdx.x; it < tiles * groups; it += gridDim.x) {
        const int64_t tile = GM ? it % tiles : it / groups;
        const int g0 = (int)(GM ? it / tiles : it - tile * groups) * CT;
        const int ng = min(CT, cnt - g0);
        const int64_t row = tile * TILE + threadIdx.x;
        if (row >= n) continue;
        int64_t off[CT];
#pragma unroll
        for (int t = 0; t < CT; ++t) off[t] = t < ng ? (int64_t)list[1 + g0 + t] * ld : 0;
        T acc[CT];
#pragma unroll
        for (int t = 0; t < CT; ++t) acc[t] = 0;
        const int64_t b = rp[row], e = rp[row + 1];
        for (int64_t q0 = b; q0 < e; q0 += 8) {  // batches of 8: indices first, then the gathers
            int32_t col[8];
            T a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                col[u] = q0 + u < e ? ci[q0 + u] : 0;
                a[u] = q0 + u < e ? v[q0 + u] : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int t = 0; t < CT; ++t)
                    if (t < ng) acc[t] = fma(a[u], X[off[t] + col[u]], acc[t]);
        }
#pragma unroll
        for (int t = 0; t < CT; ++t) {
            if (t < ng) {
                if (MODE == 0) Y[off[t] + row] = acc[t];
                else if (MODE == 1) Y[off[t] + row] = B[off[t] + row] - acc[t];
                else Y[off[t] + row] += acc[t];
            }
        }
    }
}

// Sliced ELL: slices of SELL_C consecutive rows, each padded to its longest
// row and stored column-major (entry k of the slice's rows at
// sp[slice] + k*SELL_C + lane), so a warp's matrix loads are contiguous.
// Padding entries point at a valid column with value 0.
constexpr int SELL_C = 32;
constexpr int SELL_CT = 4;  // systems per pass of the sliced-ELL SpMV
constexpr int SELL_W = 8;   // slice width held in registers
constexpr int SELL_CTP = 4;  // systems per pass of the prefetching sliced-ELL SpMV

// One matrix of an operator: CSR, plus a sliced-ELL copy when sp != nullptr.
template <class T>
struct Mat {
    const int64_t* rp = nullptr;
    const int32_t* ci = nullptr;
    const T* v = nullptr;
    const int64_t* sp = nullptr;
    const int32_t* sci = nullptr;
    const T* sv = nullptr;
    int64_t nslices = 0;
};

// Sliced-ELL SpMV: one warp per slice (lane = row of the slice). A slice of
// width <= SELL_W keeps its entries in registers and loops over the listed
// systems SELL_CT at a time, so the matrix is read once for all systems and
// each system costs only its gathers; wider slices take the entries in
// batches of SELL_W per group of systems. With many systems (the
// system-group-major case above) a warp's item is one slice for a
// supergroup of SELL_SG systems, supergroup-major, which keeps the gathers
// in L2 and gives every SM enough warps; otherwise an item is a slice for
// all listed systems.
// The stop index, the list count and (without supergroups) the first pass's
// list entries are requested together, and a slice's entries before the
// stop test: the first slice of a warp waits for one round of loads less
// than it would if each waited for the one before. The list holds at least
// k + 1 entries; those past its count are loaded but not used.
constexpr int SELL_SG = 16;
template <class T, int MODE, bool GM>
__global__ void __launch_bounds__(256) k_spmv_sell(int32_t n, int64_t ld, Mat<T> Am, const T* __restrict__ X,
                                                   T* __restrict__ Y, const T* __restrict__ B,
                                                   const int* __restrict__ list, int k, const int* __restrict__ jstop,
                                                   int jmax)
{
    constexpr int CT = SELL_CT, W = SELL_W;
    const int js = jstop ? *jstop : 0;
    const int cnt = list[0];
    int l0[CT];
#pragma unroll
    for (int t = 0; t < CT; ++t) l0[t] = !GM && t < k ? list[1 + t] : 0;
    const int64_t nitems = GM ? (int64_t)((cnt + SELL_SG - 1) / SELL_SG) * Am.nslices : Am.nslices;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t itm = w0; itm < nitems; itm += nw) {
        const int64_t sgi = GM ? itm / Am.nslices : 0;
        const int64_t sl = GM ? itm - sgi * Am.nslices : itm;
        const int gb = GM ? (int)sgi * SELL_SG : 0;
        const int ge = GM ? (gb + SELL_SG < cnt ? gb + SELL_SG : cnt) : cnt;
        const int64_t b = Am.sp[sl], e = Am.sp[sl + 1];
        const int64_t row = sl * SELL_C + lane;
        if (e - b <= (int64_t)W * SELL_C) {
            int32_t col[W];
            T a[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                const int64_t q = b + (int64_t)u * SELL_C + lane;
                col[u] = q < e ? Am.sci[q] : 0;
                a[u] = q < e ? Am.sv[q] : (T)0;
            }
            if (jstop && js >= jmax) return;  // the step needs no operator application
            for (int g0 = gb; g0 < ge; g0 += CT) {
                int64_t off[CT];
#pragma unroll
                for (int t = 0; t < CT; ++t)
                    off[t] = g0 + t < ge ? (int64_t)(!GM && g0 == 0 ? l0[t] : list[1 + g0 + t]) * ld : 0;
                T acc[CT];
#pragma unroll
                for (int t = 0; t < CT; ++t) acc[t] = 0;
#pragma unroll
                for (int u = 0; u < W; ++u)
#pragma unroll
                    for (int t = 0; t < CT; ++t)
                        if (g0 + t < ge) acc[t] = fma(a[u], X[off[t] + col[u]], acc[t]);
                if (row < n) {
#pragma unroll
                    for (int t = 0; t < CT; ++t) {
                        if (g0 + t < ge) {
                            if (MODE == 0) Y[off[t] + row] = acc[t];
                            else if (MODE == 1) Y[off[t] + row] = B[off[t] + row] - acc[t];
                            else Y[off[t] + row] += acc[t];
                        }
                    }
                }
            }
        } else {
            if (jstop && js >= jmax) return;
            for (int g0 = gb; g0 < ge; g0 += CT) {
                int64_t off[CT];
#pragma unroll
                for (int t = 0; t < CT; ++t) off[t] = g0 + t < ge ? (int64_t)list[1 + g0 + t] * ld : 0;
                T acc[CT];
#pragma unroll
                for (int t = 0; t < CT; ++t) acc[t] = 0;
                for (int64_t q0 = b + lane; q0 < e; q0 += (int64_t)W * SELL_C) {
                    int32_t col[W];
                    T a[W];
#pragma unroll
                    for (int u = 0; u < W; ++u) {
                        const int64_t q = q0 + (int64_t)u * SELL_C;
                        col[u] = q < e ? Am.sci[q] : 0;
                        a[u] = q < e ? Am.sv[q] : (T)0;
                    }
#pragma unroll
                    for (int u = 0; u < W; ++u)
#pragma unroll
                        for (int t = 0; t < CT; ++t)
                            if (g0 + t < ge) acc[t] = fma(a[u], X[off[t] + col[u]], acc[t]);
                }
                if (row < n) {
#pragma unroll
                    for (int t = 0; t < CT; ++t) {
                        if (g0 + t < ge) {
                            if (MODE == 0) Y[off[t] + row] = acc[t];
                            else if (MODE == 1) Y[off[t] + row] = B[off[t] + row] - acc[t];
                            else Y[off[t] + row] += acc[t];
                        }
                    }
                }
            }
        }
    }
}

// Sliced-ELL SpMV for few systems with the slice entries prefetched: each
// warp walks its slices (grid stride; a contiguous range per block measured
// slower) and, while it gathers for one slice, copies the next slice's
// column indices and values into its own shared buffer with cp.async (16
// bytes per copy; the entry arrays start on 128-byte slice boundaries), so
// a slice waits only for its gathers. The
// block keeps the list in shared memory when it has fewer than SELL_LS
// entries. Slices wider than SELL_W are read from global memory as in
// k_spmv_sell. A system's sum runs over its row's entries in order, padding
// included, as in k_spmv_sell.
constexpr int SP_WARPS = 4;
constexpr int SELL_LS = 256;
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class T, int MODE, int CT>
__global__ void __launch_bounds__(SP_WARPS * 32) k_spmv_sellp(int32_t n, int64_t ld, Mat<T> Am, const T* __restrict__ X,
                                                             T* __restrict__ Y, const T* __restrict__ B,
                                                             const int* __restrict__ list, int k,
                                                             const int* __restrict__ jstop, int jmax)
{
    constexpr int W = SELL_W, EB = SELL_W * SELL_C;
    __shared__ alignas(16) int32_t scol[SP_WARPS][2][EB];
    __shared__ alignas(16) T sval[SP_WARPS][2][EB];
    __shared__ int ls[SELL_LS];
    if (jstop && *jstop >= jmax) return;  // the step needs no operator application
    const bool shl = k < SELL_LS;
    if (shl)
        for (int i = threadIdx.x; i <= k; i += blockDim.x) ls[i] = list[i];
    __syncthreads();
    const int* L = shl ? ls : list;
    const int cnt = L[0];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nsl = Am.nslices;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // copies the entries [b, e) of a slice (a multiple of SELL_C, at most EB) into buffer bf
    auto prefetch = [&](int bf, int64_t b, int64_t e) {
        if (e - b <= EB) {
            const int nq = (int)(e - b) / 4;  // 16-byte pieces of the column indices
            for (int q = lane; q < nq; q += 32) cp_async16(&scol[wid][bf][4 * q], Am.sci + b + 4 * q);
            constexpr int PV = 16 / (int)sizeof(T);
            const int nv = (int)(e - b) / PV;
            for (int q = lane; q < nv; q += 32) cp_async16(&sval[wid][bf][PV * q], Am.sv + b + PV * q);
        }
        cp_async_commit();
    };
    int64_t b = 0, e = 0, bn = 0, en = 0;
    if (sl < nsl) {
        b = Am.sp[sl];
        e = Am.sp[sl + 1];
    }
    if (sl + nw < nsl) {
        bn = Am.sp[sl + nw];
        en = Am.sp[sl + nw + 1];
    }
    prefetch(0, b, e);
    int bf = 0;
    for (; sl < nsl; sl += nw) {
        prefetch(bf ^ 1, bn, en);  // an empty group past the last slice
        int64_t b2 = 0, e2 = 0;
        if (sl + 2 * nw < nsl) {
            b2 = Am.sp[sl + 2 * nw];
            e2 = Am.sp[sl + 2 * nw + 1];
        }
        cp_async_wait<1>();
        __syncwarp();
        const int64_t row = sl * SELL_C + lane;
        if (e - b <= EB) {
            const int wc = (int)(e - b) / SELL_C;  // width of this slice
            const int32_t* cs = scol[wid][bf];
            const T* vs = sval[wid][bf];
            for (int g0 = 0; g0 < cnt; g0 += CT) {
                const T* xb[CT];
#pragma unroll
                for (int t = 0; t < CT; ++t) xb[t] = X + (int64_t)L[1 + (g0 + t < cnt ? g0 + t : g0)] * ld;
                T acc[CT];
#pragma unroll
                for (int t = 0; t < CT; ++t) acc[t] = 0;
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    if (u < wc) {
                        const int32_t cu = cs[u * SELL_C + lane];
                        const T au = vs[u * SELL_C + lane];
#pragma unroll
                        for (int t = 0; t < CT; ++t)
                            if (g0 + t < cnt) acc[t] = fma(au, xb[t][cu], acc[t]);
                    }
                }
                if (row < n) {
#pragma unroll
                    for (int t = 0; t < CT; ++t) {
                        if (g0 + t < cnt) {
                            const int64_t off = (int64_t)L[1 + g0 + t] * ld;
                            if (MODE == 0) Y[off + row] = acc[t];
                            else if (MODE == 1) Y[off + row] = B[off + row] - acc[t];
                            else Y[off + row] += acc[t];
                        }
                    }
                }
            }
        } else {
            for (int g0 = 0; g0 < cnt; g0 += CT) {
                int64_t off[CT];
#pragma unroll
                for (int t = 0; t < CT; ++t) off[t] = g0 + t < cnt ? (int64_t)L[1 + g0 + t] * ld : 0;
                T acc[CT];
#pragma unroll
                for (int t = 0; t < CT; ++t) acc[t] = 0;
                for (int64_t q0 = b + lane; q0 < e; q0 += (int64_t)W * SELL_C) {
                    int32_t col[W];
                    T a[W];
#pragma unroll
                    for (int u = 0; u < W; ++u) {
                        const int64_t q = q0 + (int64_t)u * SELL_C;
                        col[u] = q < e ? Am.sci[q] : 0;
                        a[u] = q < e ? Am.sv[q] : (T)0;
                    }
#pragma unroll
                    for (int u = 0; u < W; ++u)
#pragma unroll
                        for (int t = 0; t < CT; ++t)
                            if (g0 + t < cnt) acc[t] = fma(a[u], X[off[t] + col[u]], acc[t]);
                }
                if (row < n) {
#pragma unroll
                    for (int t = 0; t < CT; ++t) {
                        if (g0 + t < cnt) {
                            if (MODE == 0) Y[off[t] + row] = acc[t];
                            else if (MODE == 1) Y[off[t] + row] = B[off[t] + row] - acc[t];
                            else Y[off[t] + row] += acc[t];
                        }
                    }
                }
            }
        }
        __syncwarp();  // every lane is done with buffer bf before it is refilled
        b = bn;
        e = en;
        bn = b2;
        en = e2;
        bf ^= 1;
    }
    cp_async_wait<0>();  // no copy in flight when the warp exits
}

// slice widths (longest row of each slice) times SELL_C, one warp per slice
__global__ void k_sell_width(int32_t n, const int64_t* __restrict__ rp, int64_t nslices, int64_t* __restrict__ cnt)
{
    const int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sl >= nslices) return;
    const int64_t row = sl * SELL_C + lane;
    const unsigned len = row < n ? (unsigned)(rp[row + 1] - rp[row]) : 0u;
    const unsigned w = __reduce_max_sync(SAI_FULL, len);
    if (lane == 0) cnt[sl] = (int64_t)w * SELL_C;
}

template <class T>
__global__ void k_sell_fill(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, int64_t nslices, const int64_t* __restrict__ sp,
                            int32_t* __restrict__ sci, T* __restrict__ sv)
{
    const int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sl >= nslices) return;
    const int64_t row = sl * SELL_C + lane;
    const int64_t b = sp[sl], w = (sp[sl + 1] - b) / SELL_C;
    const int64_t r0 = row < n ? rp[row] : 0, len = row < n ? rp[row + 1] - r0 : 0;
    const int32_t pad = row < n ? (int32_t)row : 0;
    for (int64_t k = 0; k < w; ++k) {
        const int64_t q = b + k * SELL_C + lane;
        sci[q] = k < len ? ci[r0 + k] : pad;
        sv[q] = k < len ? (T)v[r0 + k] : (T)0;
    }
}

// the cp.async copies of k_spmv_sellp need 16-byte aligned entry arrays
template <class T>
bool sell_aligned(const Mat<T>& A)
{
    return (((uintptr_t)A.sci | (uintptr_t)A.sv) % 16) == 0;
}

template <class T, int MODE>
void spmv(int32_t n, int64_t ld, const Mat<T>& A, int k, const T* X, T* Y, const T* B, const int* list,
          cudaStream_t st, const int* jstop = nullptr, int jmax = 0)
{
    const bool gm = spmv_group_major(k, n, sizeof(T));
    if (A.sp) {
        // items: slices, times supergroups of SELL_SG systems when k is large
        int64_t g = (A.nslices * (gm ? (k + SELL_SG - 1) / SELL_SG : 1) + 7) / 8;
        const int64_t cap = (int64_t)g_sms * 8;
        if (g > cap) g = cap;
        if (g < 1) g = 1;
        if (gm) {
            k_spmv_sell<T, MODE, true><<<SAI_GRID(g), 256, 0, st>>>(n, ld, A, X, Y, B, list, k, jstop, jmax);
        } else if (sell_aligned(A)) {
            int64_t gp = (A.nslices + SP_WARPS - 1) / SP_WARPS;
            const int64_t pcap = (int64_t)g_sms * g_res_sellp[sizeof(T) == 4];
            if (gp > pcap) gp = pcap;
            if (gp < 1) gp = 1;
            k_spmv_sellp<T, MODE, SELL_CTP>
                <<<SAI_GRID(gp), SP_WARPS * 32, 0, st>>>(n, ld, A, X, Y, B, list, k, jstop, jmax);
        } else {
            k_spmv_sell<T, MODE, false><<<SAI_GRID(g), 256, 0, st>>>(n, ld, A, X, Y, B, list, k, jstop, jmax);
        }
        return;
    }
    const int64_t tiles = ((int64_t)n + TILE - 1) / TILE;
    int64_t g = tiles * ((k + 3) / 4);
    const int64_t cap = (int64_t)g_sms * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    if (gm) k_spmv<T, MODE, true><<<SAI_GRID(g), TILE, 0, st>>>(n, ld, A.rp, A.ci, A.v, X, Y, B, list, jstop, jmax);
    else k_spmv<T, MODE, false><<<SAI_GRID(g), TILE, 0, st>>>(n, ld, A.rp, A.ci, A.v, X, Y, B, list, jstop, jmax);
}

// Adds a sliced-ELL copy (values converted to T) of the CSR matrix (rp, ci,
// v64) to m, unless slice padding would exceed half of nnz (then m keeps
// only its CSR form). Synchronises the stream once to read the size.
template <class T>
sai_status build_sell(int32_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* v64, Buf& spb,
                      Buf& cib, Buf& vb, Mat<T>& m, cudaStream_t st)
{
    if (n <= 0) return SAI_OK;
    const int64_t ns = ((int64_t)n + SELL_C - 1) / SELL_C;
    Buf cnt;
    SAI_TRY(cnt.alloc(sizeof(int64_t) * (size_t)ns, st, true));
    SAI_TRY(spb.alloc(sizeof(int64_t) * (size_t)(ns + 1), st, true));
    const unsigned g = sai_div_up(ns * 32, 256);
    k_sell_width<<<SAI_GRID(g), 256, 0, st>>>(n, rp, ns, cnt.as<int64_t>());
    SAI_TRY(sai_scan_counts_i64(cnt.as<int64_t>(), spb.as<int64_t>(), ns, st));
    int64_t total = 0;
    SAI_CUDA(cudaMemcpyAsync(&total, spb.as<int64_t>() + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    if ((double)total > 1.5 * (double)nnz + (double)SELL_C * ns) return SAI_OK;  // too much padding: CSR
    SAI_TRY(cib.alloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1), st, true));
    SAI_TRY(vb.alloc(sizeof(T) * (size_t)(total > 0 ? total : 1), st, true));
    k_sell_fill<T><<<SAI_GRID(g), 256, 0, st>>>(n, rp, ci, v64, ns, spb.as<int64_t>(), cib.as<int32_t>(), vb.as<T>());
    SAI_CUDA(cudaGetLastError());
    m.sp = spb.as<int64_t>();
    m.sci = cib.as<int32_t>();
    m.sv = vb.as<T>();
    m.nslices = ns;
    return SAI_OK;
}

template <class T>
struct Ops {  // A~ (or A~^T) and M (or M^T) with values of type T
    Mat<T> A, M;
};

// ---------------------------------------------------------------- item kernels
// An item is (system in list, row chunk of CHUNK rows) handled by one warp.
struct Items {
    int32_t n;
    int64_t ld;
    int nch;   // CHUNK-row chunks per system
    int nchu;  // CHUNK_U-row chunks per system (GMRES update)
};

__host__ __device__ __forceinline__ int nchunks(int64_t n) { return (int)((n + CHUNK - 1) / CHUNK); }

// threads of a single-block control kernel for k systems (it loops over them)
inline int ctl_threads(int k) { return k <= CTRL ? CTRL : 1024; }

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
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
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
    build_list_block(k, S.active, S.lact);
}

// iteration start: count it, test rho, form beta
__global__ void k_bicg_start(int k, int maxit, Sys S)
{
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!S.active[c]) continue;
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
    build_list_block(k, S.active, S.lact);
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
    const int k1 = S.lact[0];
    if (threadIdx.x == 0 && k1 > 0) {
        spmm_work(D, D.nnzM, k1);
        spmm_work(D, D.nnzA, k1);
        kwork_add(PROF_BICG_VEC, 8.0 * D.n * k1 * (4 + 2), D.n * k1 * (3 + 2));  // p update, rhat^T v
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!S.active[c]) continue;
        const double rv = sum_chunks(part, 0, c, k, nch);
        if (rv == 0.0) {
            S.active[c] = 0;
            S.status[c] = ST_BREAKDOWN;
        } else {
            S.alpha[c] = S.rho[c] / rv;
        }
    }
    __syncthreads();
    build_list_block(k, S.active, S.lact);
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
    const int k2 = S.lact[0];
    if (threadIdx.x == 0 && k2 > 0) kwork_add(PROF_BICG_VEC, 8.0 * D.n * k2 * 3, D.n * k2 * 4.0);  // s, ||s||
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (S.active[c]) {
            const double ss = sum_chunks(part, 0, c, k, nch);
            S.mode[c] = sqrt(ss) < S.thr[c] ? 2 : 1;
            S.go[c] = S.mode[c] == 1;
        } else {
            S.go[c] = 0;
        }
    }
    __syncthreads();
    build_list_block(k, S.go, S.lgo);
}

__global__ void k_bicg_f3(int k, int nch, const double* part, Sys S, Dims D)
{
    const int k3 = S.lgo[0];
    if (threadIdx.x == 0 && k3 > 0) {
        spmm_work(D, D.nnzM, k3);
        spmm_work(D, D.nnzA, k3);
        kwork_add(PROF_BICG_VEC, 8.0 * D.n * k3 * 2, D.n * k3 * 4.0);  // t^T s, t^T t
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!S.go[c]) continue;
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
    build_list_block(k, S.active, S.lact);
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
    const int k4 = S.lact[0];
    if (threadIdx.x == 0 && k4 > 0) kwork_add(PROF_BICG_VEC, 8.0 * D.n * k4 * 8, D.n * k4 * 10.0);  // x, r, two dots
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!S.active[c]) continue;
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
    build_list_block(k, S.active, S.lact);
    if (threadIdx.x == 0) *any_active = S.lact[0] > 0;
}


// ---------------------------------------------------------------- panel SpMV (many systems)
// For thousands of systems the FP64 BiCGStab applies its operators in a
// panel layout: the listed systems, PNL at a time, row-major within a panel
// (P[(pc * n + row) * PNL + j] holds system list[pc * PNL + j] at row). A
// warp then reads PNL contiguous values per matrix entry instead of PNL
// scattered words, a warp per row keeps every lane busy whatever the row's
// length, and one panel (n x PNL values) stays in L2 while the warps sweep
// its rows. Each row's sum runs over its CSR entries in order from zero, as
// in k_spmv and k_spmv_sell, so a system gets the same bits as there.
constexpr int PNL = 64;

// system-major X (the systems of list) -> panels, tiles of 32 rows x PNL systems
__global__ void __launch_bounds__(256) k_pnl_gather(int32_t n, int64_t ld, const double* __restrict__ X,
                                                    const int* __restrict__ list, double* __restrict__ P)
{
    __shared__ double t[PNL][33];
    const int cnt = list[0];
    const int np = (cnt + PNL - 1) / PNL;
    const int64_t rt = ((int64_t)n + 31) / 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int64_t it = blockIdx.x; it < rt * np; it += gridDim.x) {
        const int pc = (int)(it / rt);
        const int64_t r0 = (it - (int64_t)pc * rt) * 32;
        for (int j = ty; j < PNL; j += 8) {  // system pc * PNL + j, rows r0 + tx
            const int c = pc * PNL + j;
            const int64_t row = r0 + tx;
            t[j][tx] = (c < cnt && row < n) ? X[(int64_t)list[1 + c] * ld + row] : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {  // row r0 + r: systems 2 tx, 2 tx + 1
            const int64_t row = r0 + r;
            if (row < n)
                reinterpret_cast<double2*>(P + ((int64_t)pc * n + row) * PNL)[tx] =
                    make_double2(t[2 * tx][r], t[2 * tx + 1][r]);
        }
        __syncthreads();
    }
}

// panels -> system-major Y (the systems of list)
__global__ void __launch_bounds__(256) k_pnl_scatter(int32_t n, int64_t ld, const double* __restrict__ P,
                                                     const int* __restrict__ list, double* __restrict__ Y)
{
    __shared__ double t[PNL][33];
    const int cnt = list[0];
    const int np = (cnt + PNL - 1) / PNL;
    const int64_t rt = ((int64_t)n + 31) / 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int64_t it = blockIdx.x; it < rt * np; it += gridDim.x) {
        const int pc = (int)(it / rt);
        const int64_t r0 = (it - (int64_t)pc * rt) * 32;
        for (int r = ty; r < 32; r += 8) {
            const int64_t row = r0 + r;
            if (row < n) {
                const double2 v = reinterpret_cast<const double2*>(P + ((int64_t)pc * n + row) * PNL)[tx];
                t[2 * tx][r] = v.x;
                t[2 * tx + 1][r] = v.y;
            }
        }
        __syncthreads();
        for (int j = ty; j < PNL; j += 8) {
            const int c = pc * PNL + j;
            const int64_t row = r0 + tx;
            if (c < cnt && row < n) Y[(int64_t)list[1 + c] * ld + row] = t[j][tx];
        }
        __syncthreads();
    }
}

// Pout = A Pin on the panels of the listed systems (CSR of A); one warp per
// (panel, row), panel-major; lane l holds systems 2 l and 2 l + 1
__global__ void __launch_bounds__(256) k_pnl_spmm(int32_t n, const int64_t* __restrict__ rp,
                                                  const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                  const int* __restrict__ list, const double* __restrict__ Pin,
                                                  double* __restrict__ Pout)
{
    const int cnt = list[0];
    const int np = (cnt + PNL - 1) / PNL;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = w0; it < (int64_t)np * n; it += nw) {
        const int64_t pc = it / n, row = it - pc * n;
        const double2* X = reinterpret_cast<const double2*>(Pin + pc * n * PNL);
        double a0 = 0.0, a1 = 0.0;
        const int64_t b = rp[row], e = rp[row + 1];
        for (int64_t q0 = b; q0 < e; q0 += 32) {
            const int64_t q = q0 + lane;
            const int32_t cl = q < e ? ci[q] : 0;
            const double av = q < e ? v[q] : 0.0;
            const int m = e - q0 < 32 ? (int)(e - q0) : 32;
            for (int u = 0; u < m; ++u) {
                const int32_t c = __shfl_sync(SAI_FULL, cl, u);
                const double a = __shfl_sync(SAI_FULL, av, u);
                const double2 x = X[(int64_t)c * (PNL / 2) + lane];
                a0 = fma(a, x.x, a0);
                a1 = fma(a, x.y, a1);
            }
        }
        reinterpret_cast<double2*>(Pout + (pc * n + row) * PNL)[lane] = make_double2(a0, a1);
    }
}

// Y2 = A (Y1 = M X) for the listed systems through the panels P1, P2
// (n x PNL * ceil(k / PNL) values each): gather, two SpMMs, two scatters.
void pnl_apply2(int32_t n, int64_t ld, int k, const Ops<double>& A, const double* X, double* Y1, double* Y2,
                const int* list, double* P1, double* P2, cudaStream_t st)
{
    const int64_t np = (k + PNL - 1) / PNL;
    const int64_t tiles = ((int64_t)n + 31) / 32 * np;
    const int64_t tb = tiles < (int64_t)g_sms * 16 ? (tiles > 0 ? tiles : 1) : (int64_t)g_sms * 16;
    const int64_t warps = np * n;
    int64_t sb = (warps + 7) / 8;
    if (sb > (int64_t)g_sms * 8) sb = (int64_t)g_sms * 8;
    if (sb < 1) sb = 1;
    k_pnl_gather<<<SAI_GRID(tb), 256, 0, st>>>(n, ld, X, list, P1);
    k_pnl_spmm<<<SAI_GRID(sb), 256, 0, st>>>(n, A.M.rp, A.M.ci, A.M.v, list, P1, P2);
    k_pnl_scatter<<<SAI_GRID(tb), 256, 0, st>>>(n, ld, P2, list, Y1);
    k_pnl_spmm<<<SAI_GRID(sb), 256, 0, st>>>(n, A.A.rp, A.A.ci, A.A.v, list, P2, P1);
    k_pnl_scatter<<<SAI_GRID(tb), 256, 0, st>>>(n, ld, P1, list, Y2);
}

sai_status bicgstab_run(const Items& I, int k, const Ops<double>& A, const double* Bsd, double* Xsd, Sys& S,
                        double* pt, int* fl, int maxit, const Dims& D, cudaStream_t st)
{
    const int32_t n = I.n;
    const int64_t ld = I.ld;
    const size_t blk = (size_t)ld * k;
    const int ib = item_blocks(n > 0 ? n : 1, k);
    const int nch = I.nch;
    const int check_every = 4;
    const int ct = ctl_threads(k);
    int hflag = 0;
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
    // many systems: the operators are applied in the panel layout
    const bool pnl = k > CTRL && spmv_group_major(k, n, sizeof(double));
    Buf pbuf;
    double *P1 = nullptr, *P2 = nullptr;
    if (pnl) {
        const size_t pe = (size_t)(n > 0 ? n : 1) * PNL * (size_t)((k + PNL - 1) / PNL);
        SAI_TRY(pbuf.alloc(sizeof(double) * pe * 2, st, true));
        P1 = pbuf.as<double>();
        P2 = P1 + pe;
    }
    k_bicg_init<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Bsd, Xsd, r, rh, p, v, S.lall, pt);
    k_bicg_f0<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S);
    SAI_CUDA(cudaGetLastError());
    for (int it = 0; it < maxit; ++it) {
        k_bicg_start<<<SAI_GRID(1), ct, 0, st>>>(k, maxit, S);
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_bicg_p<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, r, p, v, S);
        }
        if (pnl) {
            ProfScope ps(PROF_SPMM, st);
            pnl_apply2(n, ld, k, A, p, ph, v, S.lact, P1, P2, st);
        } else {
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<double, 0>(n, ld, A.M, k, p, ph, nullptr, S.lact, st);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<double, 0>(n, ld, A.A, k, ph, v, nullptr, S.lact, st);
            }
        }
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_dots<1><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, rh, v, nullptr, nullptr, S.lact, pt);
        }
        k_bicg_f1<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S, D);
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_bicg_s<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, r, v, s, S, pt);
        }
        k_bicg_f2<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S, D);
        if (pnl) {
            ProfScope ps(PROF_SPMM, st);
            pnl_apply2(n, ld, k, A, s, sh, t, S.lgo, P1, P2, st);
        } else {
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<double, 0>(n, ld, A.M, k, s, sh, nullptr, S.lgo, st);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<double, 0>(n, ld, A.A, k, sh, t, nullptr, S.lgo, st);
            }
        }
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_dots<2><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, t, s, t, t, S.lgo, pt);
        }
        k_bicg_f3<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S, D);
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_bicg_xr<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Xsd, r, rh, ph, sh, s, t, S, pt);
        }
        k_bicg_f4<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S, D, fl);
        SAI_CUDA(cudaGetLastError());
        if ((it + 1) % check_every == 0 || it + 1 == maxit) {
            SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            if (!hflag) break;
        }
    }
    // systems still active after maxit passes
    k_bicg_start<<<SAI_GRID(1), ct, 0, st>>>(k, maxit, S);
    SAI_CUDA(cudaGetLastError());
    return SAI_OK;
}

// ================================================================== CGS
// Conjugate gradient squared (Sonneveld) on A~ M z = b with y = M z, one
// system per entry of the list (section 5 names CGS among the other solvers
// tried). Per iteration:
//   rho = rhat^T r;  beta = rho / rho_old;  u = r + beta q;  p = u + beta (q + beta p)
//   (u = p = r in the first iteration);  phat = M p;  v = A~ phat;
//   alpha = rho / rhat^T v;  q = u - alpha v;  w = M (u + q);  y += alpha w;
//   r -= alpha A~ w
// and the recursive residual is tested after the iteration.
__global__ void k_cgs_init(Items I, int k, const double* __restrict__ Bs, double* x, double* r, double* rh,
                           double* q, double* p, const int* list, double* part)
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
            q[o + i] = 0.0;
            p[o + i] = 0.0;
            acc = fma(b, b, acc);
        }
        acc = warp_sum(acc);
        if (lane_ == 0) part[pidx(0, c, q_, k, I.nch)] = acc;
    }
}

// iteration start: count it, test rho, form beta
__global__ void k_cgs_start(int k, int maxit, Sys S)
{
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!S.active[c]) continue;
        if (S.iters[c] >= maxit) {
            S.active[c] = 0;
            S.status[c] = ST_MAXITER;
        } else {
            S.iters[c] += 1;
            if (S.rho[c] == 0.0) {
                S.active[c] = 0;
                S.status[c] = ST_BREAKDOWN;
            } else {
                S.beta[c] = S.iters[c] == 1 ? 0.0 : S.rho[c] / S.rho_old[c];
            }
        }
    }
    __syncthreads();
    build_list_block(k, S.active, S.lact);
}

__global__ void k_cgs_up(Items I, const double* __restrict__ r, double* u, double* p, const double* __restrict__ q,
                         Sys S)
{
    FOR_ITEMS(I, S.lact, c, r0, r1)
    {
        const double be = S.beta[c];
        const bool first = S.iters[c] == 1;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            const double uv = first ? r[o + i] : r[o + i] + be * q[o + i];
            u[o + i] = uv;
            p[o + i] = first ? uv : uv + be * (q[o + i] + be * p[o + i]);
        }
    }
}

__global__ void k_cgs_f1(int k, int nch, const double* part, Sys S, Dims D)
{
    const int k1 = S.lact[0];
    if (threadIdx.x == 0 && k1 > 0) {
        spmm_work(D, D.nnzM, k1);
        spmm_work(D, D.nnzA, k1);
        kwork_add(PROF_BICG_VEC, 8.0 * D.n * k1 * (5 + 2), D.n * k1 * (6 + 2));  // u, p updates, rhat^T v
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!S.active[c]) continue;
        const double sg = sum_chunks(part, 0, c, k, nch);
        if (sg == 0.0) {
            S.active[c] = 0;
            S.status[c] = ST_BREAKDOWN;
        } else {
            S.alpha[c] = S.rho[c] / sg;
        }
    }
    __syncthreads();
    build_list_block(k, S.active, S.lact);
}

__global__ void k_cgs_q(Items I, const double* __restrict__ u, const double* __restrict__ v, double* q, double* w,
                        Sys S)
{
    FOR_ITEMS(I, S.lact, c, r0, r1)
    {
        const double al = S.alpha[c];
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            const double qv = u[o + i] - al * v[o + i];
            q[o + i] = qv;
            w[o + i] = u[o + i] + qv;
        }
    }
}

__global__ void k_cgs_xr(Items I, int k, double* x, double* r, const double* __restrict__ rh,
                         const double* __restrict__ wh, const double* __restrict__ qh, Sys S, double* part)
{
    FOR_ITEMS(I, S.lact, c, r0, r1)
    {
        const double al = S.alpha[c];
        double a0 = 0.0, a1 = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            x[o + i] += al * wh[o + i];
            const double rv = r[o + i] - al * qh[o + i];
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

__global__ void k_cgs_f2(int k, int nch, const double* part, Sys S, Dims D, int* any_active)
{
    const int k2 = S.lact[0];
    if (threadIdx.x == 0 && k2 > 0) {
        spmm_work(D, D.nnzM, k2);
        spmm_work(D, D.nnzA, k2);
        kwork_add(PROF_BICG_VEC, 8.0 * D.n * k2 * (4 + 6), D.n * k2 * (3 + 8));  // q, w; x, r, two dots
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!S.active[c]) continue;
        const double rr = sum_chunks(part, 0, c, k, nch), rhr = sum_chunks(part, 1, c, k, nch);
        if (sqrt(rr) < S.thr[c]) {
            S.active[c] = 0;
            S.status[c] = ST_OK;
        } else {
            S.rho_old[c] = S.rho[c];
            S.rho[c] = rhr;
        }
    }
    __syncthreads();
    build_list_block(k, S.active, S.lact);
    if (threadIdx.x == 0) *any_active = S.lact[0] > 0;
}

sai_status cgs_run(const Items& I, int k, const Ops<double>& A, const double* Bsd, double* Xsd, Sys& S, double* pt,
                   int* fl, int maxit, const Dims& D, cudaStream_t st)
{
    const int32_t n = I.n;
    const int64_t ld = I.ld;
    const size_t blk = (size_t)ld * k;
    const int ib = item_blocks(n > 0 ? n : 1, k);
    const int nch = I.nch;
    const int check_every = 4;
    const int ct = ctl_threads(k);
    int hflag = 0;
    Buf vecs;
    SAI_TRY(vecs.alloc(sizeof(double) * blk * 9 + 8, st, true));
    SAI_CUDA(cudaMemsetAsync(vecs.p, 0, sizeof(double) * blk * 9, st));
    double* r = vecs.as<double>();
    double* rh = r + blk;
    double* u = rh + blk;
    double* p = u + blk;
    double* q = p + blk;
    double* ph = q + blk;
    double* v = ph + blk;
    double* w = v + blk;
    double* wh = w + blk;
    double* qh = ph;  // A~ M w reuses phat's block: phat is dead once v = A~ phat is formed
    const bool pnl = k > CTRL && spmv_group_major(k, n, sizeof(double));
    Buf pbuf;
    double *P1 = nullptr, *P2 = nullptr;
    if (pnl) {
        const size_t pe = (size_t)(n > 0 ? n : 1) * PNL * (size_t)((k + PNL - 1) / PNL);
        SAI_TRY(pbuf.alloc(sizeof(double) * pe * 2, st, true));
        P1 = pbuf.as<double>();
        P2 = P1 + pe;
    }
    auto apply2 = [&](const double* X, double* Y1, double* Y2) {  // Y1 = M X, Y2 = A~ Y1
        if (pnl) {
            ProfScope ps(PROF_SPMM, st);
            pnl_apply2(n, ld, k, A, X, Y1, Y2, S.lact, P1, P2, st);
        } else {
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<double, 0>(n, ld, A.M, k, X, Y1, nullptr, S.lact, st);
            }
            {
                ProfScope ps(PROF_SPMM, st);
                spmv<double, 0>(n, ld, A.A, k, Y1, Y2, nullptr, S.lact, st);
            }
        }
    };
    k_cgs_init<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Bsd, Xsd, r, rh, q, p, S.lall, pt);
    k_bicg_f0<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S);  // rho = b^T b, the first test on ||b||
    SAI_CUDA(cudaGetLastError());
    for (int it = 0; it < maxit; ++it) {
        k_cgs_start<<<SAI_GRID(1), ct, 0, st>>>(k, maxit, S);
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_cgs_up<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, r, u, p, q, S);
        }
        apply2(p, ph, v);
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_dots<1><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, rh, v, nullptr, nullptr, S.lact, pt);
        }
        k_cgs_f1<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S, D);
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_cgs_q<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, u, v, q, w, S);
        }
        apply2(w, wh, qh);
        {
            ProfScope ps(PROF_BICG_VEC, st);
            k_cgs_xr<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Xsd, r, rh, wh, qh, S, pt);
        }
        k_cgs_f2<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S, D, fl);
        SAI_CUDA(cudaGetLastError());
        if ((it + 1) % check_every == 0 || it + 1 == maxit) {
            SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            if (!hflag) break;
        }
    }
    k_cgs_start<<<SAI_GRID(1), ct, 0, st>>>(k, maxit, S);  // systems still active after maxit
    SAI_CUDA(cudaGetLastError());
    return SAI_OK;
}

// ================================================================== BiCG
// Biconjugate gradients on K z = b with K = A~ M, y = M z (section 5 names
// BiCG among the other solvers tried). The shadow sequence runs with
// K^T = M^T A~^T (the CSC arrays serve as CSR of the transposes), shadow
// residual rs = b. Per iteration:
//   rho = rs^T r;  p = r + beta p;  ps = rs + beta ps  (beta = rho / rho_old,
//   p = r, ps = rs first);  z = M p;  q = A~ z;  qs = K^T ps;
//   alpha = rho / ps^T q;  y += alpha z;  r -= alpha q;  rs -= alpha qs
// with the control kernels of CGS (same recurrences for rho, beta, alpha).
__global__ void k_bicg2_init(Items I, int k, const double* __restrict__ Bs, double* x, double* r, double* rs,
                             const int* list, double* part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        double acc = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            const double b = Bs[o + i];
            x[o + i] = 0.0;
            r[o + i] = b;
            rs[o + i] = b;
            acc = fma(b, b, acc);
        }
        acc = warp_sum(acc);
        if (lane_ == 0) part[pidx(0, c, q_, k, I.nch)] = acc;
    }
}

__global__ void k_bicg2_up(Items I, const double* __restrict__ r, const double* __restrict__ rs, double* p,
                           double* ps, Sys S)
{
    FOR_ITEMS(I, S.lact, c, r0, r1)
    {
        const double be = S.beta[c];
        const bool first = S.iters[c] == 1;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            p[o + i] = first ? r[o + i] : r[o + i] + be * p[o + i];
            ps[o + i] = first ? rs[o + i] : rs[o + i] + be * ps[o + i];
        }
    }
}

__global__ void k_bicg2_xr(Items I, int k, double* x, double* r, double* rs, const double* __restrict__ z,
                           const double* __restrict__ q, const double* __restrict__ qs, Sys S, double* part)
{
    FOR_ITEMS(I, S.lact, c, r0, r1)
    {
        const double al = S.alpha[c];
        double a0 = 0.0, a1 = 0.0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            x[o + i] += al * z[o + i];
            const double rv = r[o + i] - al * q[o + i];
            const double sv = rs[o + i] - al * qs[o + i];
            r[o + i] = rv;
            rs[o + i] = sv;
            a0 = fma(rv, rv, a0);
            a1 = fma(sv, rv, a1);
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        if (lane_ == 0) {
            part[pidx(0, c, q_, k, I.nch)] = a0;
            part[pidx(1, c, q_, k, I.nch)] = a1;
        }
    }
}

// A: the pair of K (M applied first, then A~); T: the pair of K^T (A~^T first, then M^T)
sai_status bicg_run(const Items& I, int k, const Ops<double>& A, const Ops<double>& T, const double* Bsd,
                    double* Xsd, Sys& S, double* pt, int* fl, int maxit, const Dims& D, cudaStream_t st)
{
    const int32_t n = I.n;
    const int64_t ld = I.ld;
    const size_t blk = (size_t)ld * k;
    const int ib = item_blocks(n > 0 ? n : 1, k);
    const int nch = I.nch;
    const int check_every = 4;
    const int ct = ctl_threads(k);
    int hflag = 0;
    Buf vecs;
    SAI_TRY(vecs.alloc(sizeof(double) * blk * 8 + 8, st, true));
    SAI_CUDA(cudaMemsetAsync(vecs.p, 0, sizeof(double) * blk * 8, st));
    double* r = vecs.as<double>();
    double* rs = r + blk;
    double* p = rs + blk;
    double* ps = p + blk;
    double* z = ps + blk;
    double* q = z + blk;
    double* zs = q + blk;
    double* qs = zs + blk;
    const bool pnl = k > CTRL && spmv_group_major(k, n, sizeof(double));
    Buf pbuf;
    double *P1 = nullptr, *P2 = nullptr;
    if (pnl) {
        const size_t pe = (size_t)(n > 0 ? n : 1) * PNL * (size_t)((k + PNL - 1) / PNL);
        SAI_TRY(pbuf.alloc(sizeof(double) * pe * 2, st, true));
        P1 = pbuf.as<double>();
        P2 = P1 + pe;
    }
    auto apply2 = [&](const Ops<double>& O, const double* X, double* Y1, double* Y2) {  // Y1 = O.M X, Y2 = O.A Y1
        if (pnl) {
            ProfScope ps_(PROF_SPMM, st);
            pnl_apply2(n, ld, k, O, X, Y1, Y2, S.lact, P1, P2, st);
        } else {
            {
                ProfScope ps_(PROF_SPMM, st);
                spmv<double, 0>(n, ld, O.M, k, X, Y1, nullptr, S.lact, st);
            }
            {
                ProfScope ps_(PROF_SPMM, st);
                spmv<double, 0>(n, ld, O.A, k, Y1, Y2, nullptr, S.lact, st);
            }
        }
    };
    k_bicg2_init<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Bsd, Xsd, r, rs, S.lall, pt);
    k_bicg_f0<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S);  // rho = b^T b, the first test on ||b||
    SAI_CUDA(cudaGetLastError());
    for (int it = 0; it < maxit; ++it) {
        k_cgs_start<<<SAI_GRID(1), ct, 0, st>>>(k, maxit, S);
        {
            ProfScope ps_(PROF_BICG_VEC, st);
            k_bicg2_up<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, r, rs, p, ps, S);
        }
        apply2(A, p, z, q);
        apply2(T, ps, zs, qs);
        {
            ProfScope ps_(PROF_BICG_VEC, st);
            k_dots<1><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, ps, q, nullptr, nullptr, S.lact, pt);
        }
        k_cgs_f1<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S, D);
        {
            ProfScope ps_(PROF_BICG_VEC, st);
            k_bicg2_xr<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Xsd, r, rs, z, q, qs, S, pt);
        }
        k_cgs_f2<<<SAI_GRID(1), ct, 0, st>>>(k, nch, pt, S, D, fl);
        SAI_CUDA(cudaGetLastError());
        if ((it + 1) % check_every == 0 || it + 1 == maxit) {
            SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            if (!hflag) break;
        }
    }
    k_cgs_start<<<SAI_GRID(1), ct, 0, st>>>(k, maxit, S);  // systems still active after maxit
    SAI_CUDA(cudaGetLastError());
    return SAI_OK;
}

// ================================================================== GMRES(m)
// Control state (FP64 scalars and flags), shared by the FP64 and FP32 engines.
struct Gm {
    int m;
    double* H;      // rotated columns (the triangle R): column j of system c at H[(c*m + j)*(m+1)]
    double* Hu;     // the same columns before rotation (the Hessenberg matrix of the Arnoldi relation)
    double* cs;     // k x m
    double* sn;     // k x m
    double* g;      // k x (m+1)
    double* hp;     // k x (m+1): first-pass coefficients of the newest column
    double* sco;    // k x (m+1): s = V^T u of the current step
    double* cco;    // k x (m+1): c = V^T z of the current step
    double* y;      // k x m: least-squares solution at the end of a cycle
    double* alpha;  // k: norm of u - V s
    double* dco;    // k: v_j^T (A M v_j)-part of z, see k_dc_step
    int *cyc, *adv, *jd, *done, *conv;
    int *lcyc, *ladv;  // lists
    int* jdev;         // number of finished basis vectors in the current cycle
    int* bcnt;         // arrival counter of the multi-block control kernels
    double* red;       // k x PS: a step's reduced partials per system
    int* scnt;         // k: per-system arrival counters of k_dc_step
};

constexpr int GM_MAXM = 128;             // largest restart length
constexpr int PD = 4;                    // basis vectors per pass of the fused dot kernel
constexpr int PS = 2 * GM_MAXM + 2;      // partial slots per (system, chunk)
constexpr int STEP_THREADS = 256;        // threads per block of the step kernel
constexpr int STEP_RB = 8;               // blocks per system of the step kernel
static_assert(STEP_THREADS > GM_MAXM && 2 * STEP_THREADS >= PS, "the step kernel's single-round loads");

// Krylov basis: m+1 system-major blocks of k vectors in the value type T.
template <class T>
struct Basis {
    T* V;
    int64_t vs;  // distance between V_i and V_{i+1}
};

// 16-byte vectors of T (double2 / float4) for the streaming kernels; every
// system vector starts on a 256-byte boundary (ld is a multiple of 32) and its
// padding rows [n, ld) are zero, so whole vectors can be read past n.
template <class T>
struct Vec;
template <>
struct Vec<double> {
    using type = double2;
    static constexpr int W = 2;
    __device__ static double dot(const double2& a, const double2& b) { return fma(a.x, b.x, a.y * b.y); }
    __device__ static double2 axpy(double a, const double2& x, const double2& y)
    {
        return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
    }
    __device__ static double2 lin(double a, const double2& x, double b, const double2& y)  // a x + b y
    {
        return make_double2(fma(a, x.x, b * y.x), fma(a, x.y, b * y.y));
    }
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double2 sub(const double2& a, const double2& b) { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ static double2 scale(double s, const double2& a) { return make_double2(s * a.x, s * a.y); }
};
template <>
struct Vec<float> {
    using type = float4;
    static constexpr int W = 4;
    __device__ static float dot(const float4& a, const float4& b)
    {
        return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
    }
    __device__ static float4 axpy(float a, const float4& x, const float4& y)
    {
        return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
    }
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static float4 sub(const float4& a, const float4& b)
    {
        return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    }
    __device__ static float4 scale(float s, const float4& a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }
};

template <class T>
__global__ void k_gm_init(Items I, int k, const T* __restrict__ Bs, T* x, T* r, const int* list, double* part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        T acc = 0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) {
            const T b = Bs[o + i];
            x[o + i] = 0;
            r[o + i] = b;
            acc = fma(b, b, acc);
        }
        acc = warp_sum_t(acc);
        if (lane_ == 0) part[pidx(0, c, q_, k, I.nch)] = (double)acc;
    }
}

template <class T>
__global__ void k_norm2(Items I, int k, const T* __restrict__ r, const int* list, double* part)
{
    FOR_ITEMS(I, list, c, r0, r1)
    {
        T acc = 0;
        const int64_t o = (int64_t)c * I.ld;
        for (int64_t i = r0 + lane_; i < r1; i += 32) acc = fma(r[o + i], r[o + i], acc);
        acc = warp_sum_t(acc);
        if (lane_ == 0) part[pidx(0, c, q_, k, I.nch)] = (double)acc;
    }
}

// cycle start: true residual norm, stop tests, g = beta e_1
__global__ void k_gm_cycle_start(int k, int nch, const double* part, const int* cap, Sys S, Gm G, int first,
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
        if (!G.done[c]) {
            const double beta = sqrt(sum_chunks(part, 0, c, k, nch));
            if (beta < S.thr[c]) {
                G.done[c] = 1;
                S.status[c] = ST_OK;
            } else if (S.iters[c] >= cap[c]) {
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
        *G.jdev = 0;
        *G.bcnt = 0;
        *any_cyc = G.lcyc[0] > 0;
    }
}

// ------------------------------------------------ Arnoldi with delayed re-orthogonalisation
// Classical Gram-Schmidt applied twice, with the second pass of each vector
// delayed by one step and merged into the next step's single reduction
// (the "DCGS2" Arnoldi of Swirydowicz et al. 2020 / Bielich et al. 2022).
//
// At step j the basis v_0..v_{j-1} is final and u is the candidate for v_j:
// the remainder of A M v_{j-1} after one projection (for j = 0, u = r0).
// With z = A M u, one pass over the rows forms
//     s = V^T u,  c = V^T z,  uu = u^T u,  uz = u^T z            (k_dc_dots)
// from which (k_dc_step)
//     alpha = sqrt(uu - s^T s),   v_j = (u - V s) / alpha,
//     column j-1 of the Hessenberg matrix = hp + s, with subdiagonal alpha,
//     d = (uz - s^T c) / alpha  (= v_j^T z),
//     hp(new)_i = ([c; d]_i - (Hbar s)_i) / alpha,  i = 0..j,
// using A M V_j = V_{j+1} Hbar_j, so that A M v_j = (z - V_{j+1} Hbar_j s)/alpha.
// A second pass over the rows (k_dc_update) then writes
//     v_j = (u - V s) / alpha   and   u <- (z - V c - d v_j) / alpha,
// the first-pass remainder of A M v_j against v_0..v_j. The column of the
// Hessenberg matrix, its Givens rotation and the stop test therefore run one
// step behind the operator application; a cycle of m columns takes m + 1
// steps, the last without an operator application.
// In exact arithmetic the basis, the Hessenberg matrix and the iterates are
// those of Arnoldi with modified Gram-Schmidt (Sec. 4.3's GMRES).

// Partials: slot 2i = v_i^T u, 2i+1 = v_i^T z (i < j), 2*GM_MAXM = u^T u,
// 2*GM_MAXM+1 = u^T z, stored at part[((c*PS) + slot)*ndc + q] for chunk q
// of DC_CHUNK rows. One block per item (chunk q, system, group g of PD
// basis vectors), g fastest so the items of one chunk read its rows of u and
// z from cache; the block's IT_WARPS warps take interleaved 16-byte row
// vectors of the chunk and their sums are combined in warp order through
// shared memory. (Streaming each thread's row vectors through a two-stage
// cp.async buffer in shared memory instead of registers measured slower:
// 21.5 against 18.9 ms of the 64^3 step.)
constexpr int DC_CHUNK = 2 * CHUNK;  // rows per item of the fused dot kernel (one partial per item)
inline int dc_chunks(int64_t n) { return (int)((n + DC_CHUNK - 1) / DC_CHUNK); }

template <class T>
__global__ void __launch_bounds__(IT_WARPS * 32) k_dc_dots(Items I, int ndc, const T* __restrict__ u,
                                                          const T* __restrict__ z, Basis<T> Bv, const int* list,
                                                          const int* jdev, double* __restrict__ part)
{
    using VT = typename Vec<T>::type;
    constexpr int VW = Vec<T>::W;
    constexpr int NR = 2 * PD + 2;
    __shared__ T red[IT_WARPS][NR];
    const int j = *jdev;
    const int ng = j > 0 ? (j + PD - 1) / PD : 1;  // groups of PD basis vectors
    const int cnt = list[0];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // each block takes a contiguous range of items: the groups of one
    // (chunk, system) follow one another and read u and z from cache
    const int64_t total = (int64_t)cnt * ndc * ng;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t it_end = min(total, ((int64_t)blockIdx.x + 1) * per);
    for (int64_t it = (int64_t)blockIdx.x * per; it < it_end; ++it) {
        const int g = (int)(it % ng);
        const int64_t rest = it / ng;
        const int c = list[1 + (int)(rest % cnt)];
        const int q = (int)(rest / cnt);
        const int i0 = g * PD;
        const int ni = min(PD, j - i0);
        const int64_t r0 = (int64_t)q * DC_CHUNK, r1 = min((int64_t)I.n, r0 + DC_CHUNK);
        const int64_t o = (int64_t)c * I.ld;
        const int64_t r1v = min(I.ld, (r1 + VW - 1) / VW * VW);
        const T* Vp = Bv.V + (int64_t)i0 * Bv.vs + o;
        T as[PD], ac[PD];
#pragma unroll
        for (int i = 0; i < PD; ++i) as[i] = ac[i] = 0;
        T uu = 0, uz = 0;
        for (int64_t row = r0 + (int64_t)threadIdx.x * VW; row < r1v; row += IT_WARPS * 32 * VW) {
            const VT uv = *reinterpret_cast<const VT*>(u + o + row);
            const VT zv = *reinterpret_cast<const VT*>(z + o + row);
            VT vv[PD];
#pragma unroll
            for (int i = 0; i < PD; ++i)
                if (i < ni) vv[i] = *reinterpret_cast<const VT*>(Vp + (int64_t)i * Bv.vs + row);
#pragma unroll
            for (int i = 0; i < PD; ++i)
                if (i < ni) {
                    as[i] += Vec<T>::dot(vv[i], uv);
                    ac[i] += Vec<T>::dot(vv[i], zv);
                }
            if (g == 0) {
                uu += Vec<T>::dot(uv, uv);
                uz += Vec<T>::dot(uv, zv);
            }
        }
#pragma unroll
        for (int i = 0; i < PD; ++i) {
            as[i] = warp_sum_t(as[i]);
            ac[i] = warp_sum_t(ac[i]);
        }
        uu = warp_sum_t(uu);
        uz = warp_sum_t(uz);
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < PD; ++i) {
                red[wid][2 * i] = as[i];
                red[wid][2 * i + 1] = ac[i];
            }
            red[wid][2 * PD] = uu;
            red[wid][2 * PD + 1] = uz;
        }
        __syncthreads();
        const int nsl = 2 * ni + (g == 0 ? 2 : 0);
        if ((int)threadIdx.x < nsl) {
            const int t = threadIdx.x;
            const int widx = t < 2 * ni ? t : 2 * PD + (t - 2 * ni);
            const int slot = t < 2 * ni ? 2 * i0 + t : 2 * GM_MAXM + (t - 2 * ni);
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < IT_WARPS; ++w) sum += (double)red[w][widx];
            part[((size_t)c * PS + slot) * ndc + q] = sum;
        }
        __syncthreads();
    }
}

// Arrival of one block of a multi-block control kernel: true in exactly one
// block, the last to arrive, after every other block's writes are visible.
// No block waits for another.
__device__ __forceinline__ bool last_block_arrives(int* bcnt)
{
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(bcnt, 1) == (int)gridDim.x - 1;
        if (last) __threadfence();
    }
    __syncthreads();
    return last != 0;
}

__device__ __forceinline__ void rebuild_list(int k, const int* mask, int* list)
{
    const volatile int* vm = mask;
    int q = 0;
    for (int c = 0; c < k; ++c)
        if (vm[c]) list[1 + q++] = c;
    list[0] = q;
}

// Step j for the system of block b of list ladv (grid = k blocks): reduces
// the chunk partials, finishes column j-1 (Givens rotation, residual
// estimate |g_j|, stop tests) and forms the coefficients of k_dc_update.
// tiny: relative floor of alpha^2 below which u counts as lying in span(V).
// The sums, alpha and d are FP64; the Givens rotations and the products
// with Hbar run in T, the type of the basis (FP32 for the inner solves of
// the refined GMRES, whose basis and inner products carry FP32 rounding
// already): they are the serial chain of the step, and one FP64
// instruction issues at 1/64 of the FP32 rate on this GPU.
template <class T>
__global__ void __launch_bounds__(STEP_THREADS) k_dc_step(int k, int nch, const double* __restrict__ part,
                                                         const int* cap, Sys S, Gm G, Dims D, double tiny,
                                                         int* any_adv)
{
    __shared__ double red[PS];
    __shared__ double hpS[GM_MAXM + 1];
    __shared__ T rc[GM_MAXM + 1];
    __shared__ T csS[GM_MAXM], snS[GM_MAXM];
    __shared__ double sh[3];
    __shared__ T rsT[GM_MAXM];
    __shared__ double gj1S, thrS;
    __shared__ int itS, capS;
    __shared__ int stop, mine;
    extern __shared__ double hsm[];  // columns q < j of Hbar in T (leading dimension m + 1)
    // the step index, the list count and this block's system are requested together
    const int j = *G.jdev;
    const int cnt = G.ladv[0];
    const int m = G.m;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
    const int sb = blockIdx.x / STEP_RB, rb = blockIdx.x % STEP_RB;
    const int c = G.ladv[1 + sb];  // the list holds k + 1 entries (grid: k x STEP_RB blocks)
    if (sb < cnt) {
        const int ns = 2 * j + 2;
        // the STEP_RB blocks of system c reduce its slots (one warp per slot,
        // eight independent loads in flight per lane, summed in a fixed order)
        for (int t = rb * nwarp + wid; t < ns; t += STEP_RB * nwarp) {
            const int slot = t < 2 * j ? t : 2 * GM_MAXM + (t - 2 * j);
            const double* p = part + ((size_t)c * PS + slot) * nch;
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = 0.0;
            for (int q0 = 0; q0 < nch; q0 += 8 * 32) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = q0 + u * 32 + lane;
                    if (q < nch) v[u] += p[q];
                }
            }
            double sum = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
            sum = warp_sum(sum);
            if (lane == 0) G.red[(size_t)c * PS + t] = sum;
        }
        // the last of the system's blocks to arrive does the serial part
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            mine = atomicAdd(&G.scnt[c], 1) == STEP_RB - 1;
            if (mine) {
                __threadfence();
                G.scnt[c] = 0;
            }
        }
        __syncthreads();
    }
    if (sb < cnt && mine) {
        const int ns = 2 * j + 2;
        double* Huc = G.Hu + (size_t)c * m * (m + 1);
        double* Hc = G.H + (size_t)c * m * (m + 1);
        double* hpc = G.hp + (size_t)c * (m + 1);
        double* gc = G.g + (size_t)c * (m + 1);
        // one round of independent loads: the reduced sums (through L2: the
        // other blocks of the system wrote them), the first-pass coefficients
        // of column j-1, the rotations so far, Hbar's final columns q < j-1
        // (converted to T for the products below) and the system's scalars;
        // their stores to shared memory follow them all
        const int ne = (j - 1) * (m + 1);
        const int bd = (int)blockDim.x;
        T* hsmT = reinterpret_cast<T*>(hsm);
        {
            double rv[2], hv[8];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int t = tid + u * bd;
                rv[u] = t < ns ? __ldcg(G.red + (size_t)c * PS + t) : 0.0;
            }
            const double hpv = tid < j ? hpc[tid] : 0.0;
            const double csv = tid < j - 1 ? G.cs[(size_t)c * m + tid] : 0.0;
            const double snv = tid < j - 1 ? G.sn[(size_t)c * m + tid] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = tid + u * bd;
                hv[u] = e < ne ? Huc[e] : 0.0;
            }
            double g1 = 0.0, th = 0.0;
            int itv = 0, cpv = 0;
            if (tid == 0) {
                g1 = j >= 1 ? gc[j - 1] : 0.0;
                th = S.thr[c];
                itv = S.iters[c];
                cpv = cap[c];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (tid + u * bd < ns) red[tid + u * bd] = rv[u];
            if (tid < j) hpS[tid] = hpv;
            if (tid < j - 1) {
                csS[tid] = (T)csv;
                snS[tid] = (T)snv;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (tid + u * bd < ne) hsmT[tid + u * bd] = (T)hv[u];
            if (tid == 0) {
                gj1S = g1;
                thrS = th;
                itS = itv;
                capS = cpv;
            }
            // the rest of the columns when m is large, eight loads in flight per thread
            for (int e0 = tid + 8 * bd; e0 < ne; e0 += 8 * bd) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * bd;
                    hv[u] = e < ne ? Huc[e] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (e0 + u * bd < ne) hsmT[e0 + u * bd] = (T)hv[u];
            }
        }
        __syncthreads();
        // red[2i] = s_i, red[2i+1] = c_i (i < j), red[2j] = u^T u, red[2j+1] = u^T z
        if (wid == 0) {
            double ss = 0.0, sc = 0.0;
            for (int i = lane; i < j; i += 32) {
                ss = fma(red[2 * i], red[2 * i], ss);
                sc = fma(red[2 * i], red[2 * i + 1], sc);
            }
            ss = warp_sum(ss);
            sc = warp_sum(sc);
            if (lane == 0) {
                const double uu = red[2 * j], uz = red[2 * j + 1];
                const double a2 = uu - ss;
                const double al = a2 > tiny * uu ? sqrt(a2) : 0.0;
                const double ial = al > 0.0 ? 1.0 / al : 0.0;
                sh[0] = al;
                sh[1] = (uz - sc) * ial;
                sh[2] = ial;
                stop = 0;
            }
        }
        __syncthreads();
        const double al = sh[0], d = sh[1], ial = sh[2];
        for (int i = tid; i < j; i += blockDim.x) rsT[i] = (T)red[2 * i];
        if (j >= 1) {
            // column j-1: first-pass coefficients + s, subdiagonal alpha
            for (int i = tid; i <= j; i += blockDim.x) {
                const double v = i < j ? hpS[i] + red[2 * i] : al;
                Huc[(size_t)(j - 1) * (m + 1) + i] = v;
                hsmT[(size_t)(j - 1) * (m + 1) + i] = (T)v;
                rc[i] = (T)v;
            }
            __syncthreads();
            if (tid == 0) {
                T ri = rc[0];
                for (int i = 0; i < j - 1; ++i) {
                    const T b = rc[i + 1];
                    rc[i] = csS[i] * ri + snS[i] * b;
                    ri = -snS[i] * ri + csS[i] * b;
                }
                const T a = ri, b = rc[j];
                const T den = sqrt(a * a + b * b);
                const T cn = den == (T)0 ? (T)1 : a / den, sn = den == (T)0 ? (T)0 : b / den;
                G.cs[(size_t)c * m + j - 1] = (double)cn;
                G.sn[(size_t)c * m + j - 1] = (double)sn;
                rc[j - 1] = cn * a + sn * b;
                rc[j] = (T)0;
                const T gj1 = (T)gj1S;
                const double gj = (double)(-sn * gj1);
                gc[j] = gj;
                gc[j - 1] = (double)(cn * gj1);
                const int it = itS + 1;
                S.iters[c] = it;
                G.jd[c] = j;
                if (fabs(gj) < thrS) {
                    G.conv[c] = 1;
                    stop = 1;
                } else if (al == 0.0 || it >= capS || j >= m) {
                    stop = 1;  // breakdown, iteration cap, or the cycle is full: restart
                }
            }
            __syncthreads();
            for (int i = tid; i <= j; i += blockDim.x) Hc[(size_t)(j - 1) * (m + 1) + i] = (double)rc[i];
        } else if (tid == 0) {
            // v_0 = r0 / alpha: the right-hand side of the small problem is alpha e_1
            gc[0] = al;
            if (al == 0.0) {
                G.conv[c] = 1;
                stop = 1;
            }
        }
        __syncthreads();
        if (!stop) {
            // first-pass coefficients of column j and the update coefficients;
            // (Hbar s)_i = sum_{q >= max(i-1,0)} Hbar(i,q) s_q over the final columns q < j
            // (in shared memory, in T), one thread per row i, q ascending, the column
            // loads in batches of 8 ahead of their FMAs
            for (int i = tid; i <= j; i += blockDim.x) {
                T hs = 0;
                int q = i > 0 ? i - 1 : 0;
                for (; q + 8 <= j; q += 8) {
                    T hv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) hv[u] = hsmT[(size_t)(q + u) * (m + 1) + i];
#pragma unroll
                    for (int u = 0; u < 8; ++u) hs = fma(hv[u], rsT[q + u], hs);
                }
                for (; q < j; ++q) hs = fma(hsmT[(size_t)q * (m + 1) + i], rsT[q], hs);
                const double cz = i < j ? red[2 * i + 1] : d;
                hpc[i] = (cz - (double)hs) * ial;
            }
            for (int i = tid; i < j; i += blockDim.x) {
                G.sco[(size_t)c * (m + 1) + i] = red[2 * i];
                G.cco[(size_t)c * (m + 1) + i] = red[2 * i + 1];
            }
            if (tid == 0) {
                G.alpha[c] = al;
                G.dco[c] = d;
            }
        } else if (tid == 0) {
            G.adv[c] = 0;
        }
    }
    if (last_block_arrives(G.bcnt) && wid == 0) {
        // the list of systems that advance, 32 at a time by ballot
        const volatile int* va = G.adv;
        int ku = 0;
        for (int c0 = 0; c0 < k; c0 += 32) {
            const int q = c0 + lane;
            const bool on = q < k && va[q] != 0;
            const unsigned bal = __ballot_sync(SAI_FULL, on);
            if (on) G.ladv[1 + ku + __popc(bal & ((1u << lane) - 1u))] = q;
            ku += __popc(bal);
        }
        if (lane == 0) {
            G.ladv[0] = ku;
            if (cnt > 0) {
                if (j < m) {
                    spmm_work(D, D.nnzM, cnt);
                    spmm_work(D, D.nnzA, cnt);
                }
                kwork_add(D.site_dots, D.esz * D.n * cnt * (j + 2), D.n * cnt * (4.0 * j + 4.0));
                if (ku > 0) kwork_add(D.site_upd, D.esz * D.n * ku * (j + 4), D.n * ku * (4.0 * j + 6.0));
                *G.jdev = j + 1;
            }
            *any_adv = ku > 0;
            *G.bcnt = 0;
        }
    }
}

// v_j = (u - V s)/alpha and u <- (z - V c - d v_j)/alpha for the systems of
// list; one pass over the rows, PJ basis vectors per register tile. Items
// (system, chunk of CHUNK_U rows) run system-major, each warp over a
// contiguous range of them: a warp streams consecutive rows of one system
// and loads its coefficients again only when the system changes.
template <class T>
__global__ void __launch_bounds__(IT_WARPS * 32) k_dc_update(Items I, T* __restrict__ u, const T* __restrict__ z,
                                                            Basis<T> Bv, Gm G, const int* list, const int* jdev)
{
    using VT = typename Vec<T>::type;
    constexpr int VW = Vec<T>::W;
    __shared__ T hs[IT_WARPS][GM_MAXM], hc[IT_WARPS][GM_MAXM];
    const int j = *jdev - 1;  // k_dc_step has advanced the index: write V_j
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cnt = list[0];
    const int m1 = G.m + 1;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = (int64_t)cnt * I.nchu;
    const int64_t per = (total + nw - 1) / nw;
    const int64_t it_end = min(total, (w0 + 1) * per);
    int cur = -1, c = 0;
    T ia = 0, dd = 0;
    for (int64_t it = w0 * per; it < it_end; ++it) {
        const int ci = (int)(it / I.nchu);
        const int q = (int)(it - (int64_t)ci * I.nchu);
        if (ci != cur) {
            __syncwarp();
            cur = ci;
            c = list[1 + ci];
            for (int i = lane; i < j; i += 32) {
                hs[wid][i] = (T)G.sco[(size_t)c * m1 + i];
                hc[wid][i] = (T)G.cco[(size_t)c * m1 + i];
            }
            ia = (T)(1.0 / G.alpha[c]);
            dd = (T)G.dco[c];
            __syncwarp();
        }
        const int64_t r0 = (int64_t)q * CHUNK_U, r1 = min((int64_t)I.n, r0 + CHUNK_U);
        const int64_t o = (int64_t)c * I.ld;
        const int64_t r1v = min(I.ld, (r1 + VW - 1) / VW * VW);
        T* Vj = Bv.V + (int64_t)j * Bv.vs + o;
        for (int64_t row = r0 + (int64_t)lane * VW; row < r1v; row += 32 * VW) {
            // u and z first: their loads overlap the basis loop
            const VT uv = *reinterpret_cast<const VT*>(u + o + row);
            const VT zv = *reinterpret_cast<const VT*>(z + o + row);
            VT a_s = Vec<T>::zero(), a_c = Vec<T>::zero();
            for (int i0 = 0; i0 < j; i0 += PJ) {
                const int ni = min(PJ, j - i0);
                const T* Vp = Bv.V + (int64_t)i0 * Bv.vs + o + row;
                VT vv[PJ];
#pragma unroll
                for (int i = 0; i < PJ; ++i)
                    if (i < ni) vv[i] = *reinterpret_cast<const VT*>(Vp + (int64_t)i * Bv.vs);
#pragma unroll
                for (int i = 0; i < PJ; ++i)
                    if (i < ni) {
                        a_s = Vec<T>::axpy(hs[wid][i0 + i], vv[i], a_s);
                        a_c = Vec<T>::axpy(hc[wid][i0 + i], vv[i], a_c);
                    }
            }
            const VT v = Vec<T>::scale(ia, Vec<T>::sub(uv, a_s));
            const VT un = Vec<T>::scale(ia, Vec<T>::axpy(-dd, v, Vec<T>::sub(zv, a_c)));
            *reinterpret_cast<VT*>(Vj + row) = v;
            *reinterpret_cast<VT*>(u + o + row) = un;
        }
    }
}

// ---------------------------------------------------------------- bulk-copy ring
// Shared-memory ring fed by the bulk-copy engine (cp.async.bulk, completion
// counted in bytes on an mbarrier per stage): one producer thread issues the
// copies of a block's segments in order, the consumer warps take them in the
// same order and release each stage on a second mbarrier. Every wait polls a
// bounded number of times; on running out it sets d_pipe_err and the block
// stops (the host turns the flag into SAI_CUDA_ERROR).
__device__ int d_pipe_err;
constexpr uint32_t PIPE_POLLS = 1u << 21;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

// true once the phase of parity `par` has completed; false after PIPE_POLLS polls
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t par)
{
    const uint32_t a = smem_u32(b);
    for (uint32_t it = 0; it < PIPE_POLLS; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(par)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// bytes (a multiple of 16) from src (16-byte aligned) to dst (16-byte aligned shared memory)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(UP_CWARPS * 32) : "memory"); }

// The GMRES update of k_dc_update with the basis streamed through the ring:
// items are (system, chunk of 128 UP_PT W rows) pairs, system-major, a
// contiguous range per block; an item's vector slices are V_0 .. V_{j-1}, u
// and z (the rows of its chunk, 4 KB each), UP_VPS of them per stage.
// Consumer thread t owns rows (t + 128 p) W + [0, W), p < UP_PT, of the chunk
// and forms v_j = (u - V s)/alpha and u <- (z - V c - d v_j)/alpha with the
// same per-row operation order as k_dc_update. The caller checks that V, u,
// z, the vector stride and ld give 16-byte aligned slices.
template <class T>
__global__ void __launch_bounds__((UP_CWARPS + 1) * 32) k_dc_update_ring(Items I, T* __restrict__ u,
                                                                       const T* __restrict__ z, Basis<T> Bv, Gm G,
                                                                       const int* list, const int* jdev)
{
    using VT = typename Vec<T>::type;
    constexpr int VW = Vec<T>::W;
    constexpr int NC = UP_CWARPS * 32;          // consumer threads
    constexpr int ROWS = NC * VW * UP_PT;       // rows per chunk
    constexpr uint32_t SEGB = NC * 16 * UP_PT;  // bytes per slice
    constexpr uint32_t STB = SEGB * UP_VPS;
    __shared__ alignas(128) unsigned char ring[UP_STAGES * STB];
    __shared__ alignas(8) uint64_t full[UP_STAGES], empty[UP_STAGES];
    __shared__ T hs[GM_MAXM], hc[GM_MAXM];
    __shared__ T coef[2];
    const int tid = threadIdx.x;
    const int j = *jdev - 1;  // k_dc_step has advanced the index: write V_j
    const int cnt = list[0];
    const int64_t nch = ((int64_t)I.n + ROWS - 1) / ROWS;
    const int64_t total = (int64_t)cnt * nch;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t it0 = (int64_t)blockIdx.x * per, it1 = min(total, it0 + per);
    if (tid == 0) {
        for (int s = 0; s < UP_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], UP_CWARPS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const int nseg = j + 2;  // vector slices per item
    if (tid >= UP_CWARPS * 32) {
        // producer: one thread
        if (tid != UP_CWARPS * 32) return;
        uint32_t seg = 0;  // stages filled
        bool ok = true;
        int pci = -1;
        int64_t oc = 0;
        for (int64_t it = it0; it < it1 && ok; ++it) {
            const int ci = (int)(it / nch);
            if (ci != pci) {
                pci = ci;
                oc = (int64_t)list[1 + ci] * I.ld;
            }
            const int64_t r0 = (it - (int64_t)ci * nch) * ROWS;
            const int64_t r1 = min((int64_t)I.n, r0 + ROWS);
            const int64_t r1v = min(I.ld, (r1 + VW - 1) / VW * VW);
            const uint32_t bytes = (uint32_t)((r1v - r0) * (int64_t)sizeof(T));
            const int64_t o = oc + r0;
            for (int v0 = 0; v0 < nseg; v0 += UP_VPS, ++seg) {
                const int nv = min(UP_VPS, nseg - v0);
                const uint32_t st = seg % UP_STAGES, use = seg / UP_STAGES;
                if (use > 0 && !mbar_wait(&empty[st], (use - 1) & 1)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&full[st], bytes * (uint32_t)nv);
                for (int t = 0; t < nv; ++t) {
                    const int sg = v0 + t;
                    const T* src = sg < j ? Bv.V + (int64_t)sg * Bv.vs + o : (sg == j ? u + o : z + o);
                    bulk_g2s(ring + st * STB + t * SEGB, src, bytes, &full[st]);
                }
            }
        }
        if (!ok) {
            atomicExch(&d_pipe_err, 1);
            // the copies still in flight land before the block's shared memory goes away
            const uint32_t s0 = seg > UP_STAGES ? seg - UP_STAGES : 0;
            for (uint32_t q = s0; q < seg; ++q) (void)mbar_wait(&full[q % UP_STAGES], (q / UP_STAGES) & 1);
        }
        return;
    }
    // consumers: a thread whose wait runs out stops waiting and storing but
    // keeps to the loop, so that every consumer reaches every named barrier
    const int lane = tid & 31;
    const int m1 = G.m + 1;
    uint32_t seg = 0, seg_dead = 0;
    bool dead = false;
    int cur = -1, c = 0;
    for (int64_t it = it0; it < it1; ++it) {
        const int ci = (int)(it / nch);
        const int64_t r0 = (it - (int64_t)ci * nch) * ROWS;
        const int64_t r1 = min((int64_t)I.n, r0 + ROWS);
        const int64_t r1v = min(I.ld, (r1 + VW - 1) / VW * VW);
        if (ci != cur) {
            consumer_sync();
            cur = ci;
            c = list[1 + ci];
            for (int i = tid; i < j; i += UP_CWARPS * 32) {
                hs[i] = (T)G.sco[(size_t)c * m1 + i];
                hc[i] = (T)G.cco[(size_t)c * m1 + i];
            }
            if (tid == 0) {
                coef[0] = (T)(1.0 / G.alpha[c]);
                coef[1] = (T)G.dco[c];
            }
            consumer_sync();
        }
        VT a_s[UP_PT], a_c[UP_PT], uv[UP_PT], zv[UP_PT];
#pragma unroll
        for (int p = 0; p < UP_PT; ++p) a_s[p] = a_c[p] = uv[p] = zv[p] = Vec<T>::zero();
        for (int v0 = 0; v0 < nseg; v0 += UP_VPS, ++seg) {
            const int nv = min(UP_VPS, nseg - v0);
            const uint32_t st = seg % UP_STAGES, use = seg / UP_STAGES;
            if (!dead && !mbar_wait(&full[st], use & 1)) {
                dead = true;
                seg_dead = seg;
                atomicExch(&d_pipe_err, 1);
            }
            VT v[UP_VPS][UP_PT];
#pragma unroll
            for (int t = 0; t < UP_VPS; ++t)
#pragma unroll
                for (int p = 0; p < UP_PT; ++p)
                    if (t < nv) v[t][p] = reinterpret_cast<const VT*>(ring + st * STB + t * SEGB)[tid + p * NC];
            __syncwarp();
            if (lane == 0 && !dead) mbar_arrive(&empty[st]);
#pragma unroll
            for (int t = 0; t < UP_VPS; ++t) {
                const int sg = v0 + t;
#pragma unroll
                for (int p = 0; p < UP_PT; ++p) {
                    if (sg < j) {
                        a_s[p] = Vec<T>::axpy(hs[sg], v[t][p], a_s[p]);
                        a_c[p] = Vec<T>::axpy(hc[sg], v[t][p], a_c[p]);
                    } else if (sg == j) {
                        uv[p] = v[t][p];
                    } else if (sg == j + 1) {
                        zv[p] = v[t][p];
                    }
                }
            }
        }
        if (!dead) {
            const T ia = coef[0], dd = coef[1];
            const int64_t o = (int64_t)c * I.ld;
#pragma unroll
            for (int p = 0; p < UP_PT; ++p) {
                const int64_t row = r0 + (int64_t)(tid + p * NC) * VW;
                if (row < r1v) {
                    const VT v = Vec<T>::scale(ia, Vec<T>::sub(uv[p], a_s[p]));
                    const VT un = Vec<T>::scale(ia, Vec<T>::axpy(-dd, v, Vec<T>::sub(zv[p], a_c[p])));
                    *reinterpret_cast<VT*>(Bv.V + (int64_t)j * Bv.vs + o + row) = v;
                    *reinterpret_cast<VT*>(u + o + row) = un;
                }
            }
        }
    }
    if (dead) {
        // the producer runs at most UP_STAGES stages ahead: let any of its
        // copies still in flight land (short, bounded polls)
        for (uint32_t q = seg_dead; q < seg_dead + UP_STAGES; ++q) {
            const uint32_t a = smem_u32(&full[q % UP_STAGES]);
            for (int it = 0; it < 4096; ++it) {
                uint32_t ok;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                    "selp.b32 %0, 1, 0, p;\n\t}"
                    : "=r"(ok)
                    : "r"(a), "r"((q / UP_STAGES) & 1)
                    : "memory");
                if (ok) break;
            }
        }
    }
}

// y = R(0:jd,0:jd)^{-1} g(0:jd) per system of the cycle (R upper triangular),
// by column-oriented back substitution from shared memory; grid = k blocks,
// dynamic shared memory (m*(m+1) + m) doubles.
__global__ void k_dc_trisolve(int k, Sys S, Gm G)
{
    extern __shared__ double sm[];
    __shared__ int bad;
    const int m = G.m;
    double* Rs = sm;                      // column q at Rs[q*(m+1)]
    double* t = sm + (size_t)m * (m + 1);
    const int cnt = G.lcyc[0];
    if ((int)blockIdx.x < cnt) {
        const int c = G.lcyc[1 + blockIdx.x];
        const int jd = G.jd[c];
        const double* Hc = G.H + (size_t)c * m * (m + 1);
        for (int e = threadIdx.x; e < jd * (m + 1); e += blockDim.x) Rs[e] = Hc[e];
        for (int i = threadIdx.x; i < jd; i += blockDim.x) t[i] = G.g[(size_t)c * (m + 1) + i];
        if (threadIdx.x == 0) bad = 0;
        __syncthreads();
        for (int i = jd - 1; i >= 0; --i) {
            const double dg = Rs[(size_t)i * (m + 1) + i];
            if (dg == 0.0) {
                if (threadIdx.x == 0) bad = 1;
                break;
            }
            const double yi = t[i] / dg;
            __syncthreads();
            for (int r = threadIdx.x; r < i; r += blockDim.x) t[r] = fma(-Rs[(size_t)i * (m + 1) + r], yi, t[r]);
            if (threadIdx.x == 0) t[i] = yi;
            __syncthreads();
        }
        __syncthreads();
        double* yc = G.y + (size_t)c * m;
        for (int i = threadIdx.x; i < m; i += blockDim.x) yc[i] = (bad || i >= jd) ? 0.0 : t[i];
        if (bad && threadIdx.x == 0) {
            S.status[c] = ST_BREAKDOWN;
            G.done[c] = 1;
            G.cyc[c] = 0;
        }
    }
    if (last_block_arrives(G.bcnt) && threadIdx.x == 0) {
        rebuild_list(k, G.cyc, G.lcyc);
        *G.bcnt = 0;
    }
}

// w = V y per system of the cycle (the caller adds M w to x)
template <class T>
__global__ void __launch_bounds__(IT_WARPS * 32) k_dc_combine(Items I, T* __restrict__ w, Basis<T> Bv, Gm G)
{
    using VT = typename Vec<T>::type;
    constexpr int VW = Vec<T>::W;
    __shared__ T ys[IT_WARPS][GM_MAXM];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int* list = G.lcyc;
    const int cnt = list[0];
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = w0; it < (int64_t)cnt * I.nchu; it += nw) {
        const int c = list[1 + (int)(it % cnt)];
        const int q = (int)(it / cnt);
        const int jd = G.jd[c];
        for (int i = lane; i < jd; i += 32) ys[wid][i] = (T)G.y[(size_t)c * G.m + i];
        __syncwarp();
        const int64_t r0 = (int64_t)q * CHUNK_U, r1 = min((int64_t)I.n, r0 + CHUNK_U);
        const int64_t o = (int64_t)c * I.ld;
        const int64_t r1v = min(I.ld, (r1 + VW - 1) / VW * VW);
        for (int64_t row = r0 + (int64_t)lane * VW; row < r1v; row += 32 * VW) {
            VT acc = Vec<T>::zero();
            for (int i0 = 0; i0 < jd; i0 += PJ) {
                const int ni = min(PJ, jd - i0);
                const T* Vp = Bv.V + (int64_t)i0 * Bv.vs + o + row;
                VT vv[PJ];
#pragma unroll
                for (int i = 0; i < PJ; ++i)
                    if (i < ni) vv[i] = *reinterpret_cast<const VT*>(Vp + (int64_t)i * Bv.vs);
#pragma unroll
                for (int i = 0; i < PJ; ++i)
                    if (i < ni) acc = Vec<T>::axpy(ys[wid][i0 + i], vv[i], acc);
            }
            *reinterpret_cast<VT*>(w + o + row) = acc;
        }
        __syncwarp();
    }
}

// end of a cycle: converged systems are done; a system that used its last
// iteration inside the cycle ends with MAXITER; the rest need a residual
__global__ void k_gm_cycle_end(int k, const int* cap, Sys S, Gm G, int* any_left)
{
    const int c = threadIdx.x;
    if (c < k) {
        if (G.cyc[c] && G.conv[c]) {
            G.done[c] = 1;
            S.status[c] = ST_OK;
        } else if (G.cyc[c] && S.iters[c] >= cap[c]) {
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
    for (int c = threadIdx.x; c < k; c += blockDim.x) list[1 + c] = c;
    if (threadIdx.x == 0) list[0] = k;
}

__global__ void k_fill_int(int k, int* a, int v)
{
    for (int c = threadIdx.x; c < k; c += blockDim.x) a[c] = v;
}

__global__ void k_cast_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ---------------------------------------------------------------- iterative refinement (FP64 outer)
// Outer step check: beta_c = ||b_c - A~ x_c|| (FP64). Stops a system when
// beta_c < thr_c (the FP64 stopping test) or when its inner iterations
// reach maxit; otherwise sets the inner tolerance on the normalised residual
// thr_in_c = max(tau, 0.3 thr_c / beta_c) and the inner iteration cap.
__global__ void k_ir_check(int k, int nch, const double* part, const double* thr, double tau, int maxit,
                           const int* tot, int* done, int* status, double* beta, double* thr_in, int* cap,
                           int* lir, int* any)
{
    const int c = threadIdx.x;
    if (c < k && !done[c]) {
        const double b = sqrt(sum_chunks(part, 0, c, k, nch));
        beta[c] = b;
        if (b < thr[c]) {
            done[c] = 1;
            status[c] = ST_OK;
        } else if (tot[c] >= maxit) {
            done[c] = 1;
            status[c] = ST_MAXITER;
        } else {
            thr_in[c] = fmax(tau, 0.3 * thr[c] / b);
            cap[c] = maxit - tot[c];
        }
    }
    if (c < k && done[c]) {
        thr_in[c] = INFINITY;  // a finished system takes no inner iteration
        cap[c] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int q = 0;
        for (int s = 0; s < k; ++s)
            if (!done[s]) lir[1 + q++] = s;
        lir[0] = q;
        *any = q > 0;
    }
}

// r32 = r64 / beta for the refined systems, 0 for the others
__global__ void k_ir_scale(Items I, int k, const double* __restrict__ r64, const double* beta, const int* done,
                           float* __restrict__ r32, const int* lall)
{
    FOR_ITEMS(I, lall, c, r0, r1)
    {
        const int64_t o = (int64_t)c * I.ld;
        const double s = done[c] ? 0.0 : 1.0 / beta[c];
        for (int64_t i = r0 + lane_; i < r1; i += 32) r32[o + i] = (float)(r64[o + i] * s);
    }
}

// x64 += beta * d32 for the refined systems; tot += inner iterations
__global__ void k_ir_update(Items I, double* __restrict__ x64, const float* __restrict__ d32, const double* beta,
                            const int* lir)
{
    FOR_ITEMS(I, lir, c, r0, r1)
    {
        const int64_t o = (int64_t)c * I.ld;
        const double b = beta[c];
        for (int64_t i = r0 + lane_; i < r1; i += 32) x64[o + i] = fma(b, (double)d32[o + i], x64[o + i]);
    }
}

__global__ void k_ir_total(int k, const int* lir, const int* it_in, int* tot)
{
    if (threadIdx.x == 0)
        for (int s = 0; s < lir[0]; ++s) tot[lir[1 + s]] += it_in[lir[1 + s]];
}

// final report of the refined solve: outer status and total inner iterations
__global__ void k_ir_finish(int k, const int* done, const int* status64, const int* tot, int* status, int* iters)
{
    const int c = threadIdx.x;
    if (c < k) {
        status[c] = done[c] ? status64[c] : ST_MAXITER;
        iters[c] = tot[c];
    }
}

// ---------------------------------------------------------------- GMRES engine
template <class T>
struct GmWork {  // device buffers of one GMRES engine
    Basis<T> B;
    T *r, *t, *z, *w;  // r: residual, then the candidate u of each step; t = M u; z = A~ t; w = V y
};

// One Arnoldi step (5 launches) for the advancing systems, index j on the device.
// dynamic shared memory of k_dc_step: the final columns of Hbar, m x (m+1) doubles
inline size_t step_smem(int m) { return sizeof(double) * (size_t)m * (size_t)(m + 1); }

// the bulk copies of k_dc_update_ring need 16-byte aligned segments
template <class T>
bool ring_aligned(const Items& I, const GmWork<T>& Wk)
{
    const uintptr_t p = (uintptr_t)Wk.B.V | (uintptr_t)Wk.r | (uintptr_t)Wk.z;
    return p % 16 == 0 && ((size_t)Wk.B.vs * sizeof(T)) % 16 == 0 && ((size_t)I.ld * sizeof(T)) % 16 == 0;
}

template <class T>
void arnoldi_step(const Items& I, int k, const Ops<T>& A, const GmWork<T>& Wk, Sys& S, Gm& G, const int* cap,
                  double* pt, int* fl, const Dims& D, double tiny, cudaStream_t st)
{
    const int32_t n = I.n;
    const int64_t ld = I.ld;
    // the last step of a cycle (j = m) needs no operator application
    {
        ProfScope ps(D.site_spmm, st);
        spmv<T, 0>(n, ld, A.M, k, Wk.r, Wk.t, nullptr, G.ladv, st, G.jdev, G.m);
    }
    {
        ProfScope ps(D.site_spmm, st);
        spmv<T, 0>(n, ld, A.A, k, Wk.t, Wk.z, nullptr, G.ladv, st, G.jdev, G.m);
    }
    const int fp = sizeof(T) == 4;
    const int64_t pcap = (int64_t)g_sms * g_res_dots[fp], ucap = (int64_t)g_sms * g_res_upd[fp];
    const int ndc = dc_chunks(n);
    int64_t pb = (int64_t)ndc * k * ((G.m - 1) / PD + 1);
    int64_t ub = ((int64_t)I.nchu * k + IT_WARPS - 1) / IT_WARPS;
    pb = pb < pcap ? pb : pcap;
    ub = ub < ucap ? ub : ucap;
    {
        ProfScope ps(D.site_dots, st);
        k_dc_dots<T><<<SAI_GRID(pb), IT_WARPS * 32, 0, st>>>(I, ndc, Wk.r, Wk.z, Wk.B, G.ladv, G.jdev, pt);
    }
    {
        ProfScope ps(PROF_GM_STEP, st);
        k_dc_step<T><<<SAI_GRID(k * STEP_RB), STEP_THREADS, step_smem(G.m), st>>>(k, ndc, pt, cap, S, G, D, tiny,
                                                                              fl);
    }
    {
        ProfScope ps(D.site_upd, st);
        if (ring_aligned(I, Wk)) {
            const int64_t rows = (int64_t)UP_CWARPS * 32 * Vec<T>::W * UP_PT;
            int64_t rb = ((int64_t)n + rows - 1) / rows * k;
            const int64_t rcap = (int64_t)g_sms * g_res_ring[fp];
            rb = rb < rcap ? rb : rcap;
            k_dc_update_ring<T>
                <<<SAI_GRID(rb), (UP_CWARPS + 1) * 32, 0, st>>>(I, Wk.r, Wk.z, Wk.B, G, G.ladv, G.jdev);
        } else {
            k_dc_update<T><<<SAI_GRID(ub), IT_WARPS * 32, 0, st>>>(I, Wk.r, Wk.z, Wk.B, G, G.ladv, G.jdev);
        }
    }
}

constexpr int GM_STEPS_PER_CHECK = 4;  // Arnoldi steps between host checks (one graph)
constexpr int GM_LAUNCHES_PER_STEP = 5;

// Restarted GMRES on the systems with finite thresholds: X = 0 start,
// per-system iteration caps, S.iters counts the inner steps of this call.
// Unless a profile is open, each group of GM_STEPS_PER_CHECK Arnoldi steps
// runs as one captured CUDA graph.
template <class T>
sai_status gmres_run(const Items& I, int k, int m, const Ops<T>& A, const T* Bs, T* Xs, const GmWork<T>& Wk, Sys& S,
                     Gm& G, const int* cap, double* pt, double* pt2, int* fl, const Dims& D, cudaStream_t st)
{
    const int32_t n = I.n;
    const int64_t ld = I.ld;
    const int ib = item_blocks(n > 0 ? n : 1, k);
    int64_t cb = ((int64_t)I.nchu * k + IT_WARPS - 1) / IT_WARPS;
    if (cb > (int64_t)g_sms * 8) cb = (int64_t)g_sms * 8;
    // alpha^2 below 64 unit roundoffs of u^T u: u lies in span(V) to working accuracy
    const double tiny = 64.0 * (sizeof(T) == 4 ? 5.96e-8 : 1.11e-16);
    // dynamic shared memory of the two kernels that stage Hbar / R (their
    // static shared memory counts against the same per-block limit)
    const size_t tri_smem = sizeof(double) * ((size_t)m * (m + 1) + m);
    SAI_CUDA(cudaFuncSetAttribute(k_dc_trisolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tri_smem));
    SAI_CUDA(cudaFuncSetAttribute(k_dc_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem(m)));
    int hflag = 0;
    T* r = Wk.r;
    T* w = Wk.w;
    // Graphs are captured and replayed on a library stream ordered after the
    // caller's stream (the legacy default stream cannot be captured).
    const bool use_graph = !sai_prof_on();
    cudaStream_t caller = st;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    if (use_graph) {
        cudaStream_t aux = sai_aux_stream();
        if (aux) {
            SAI_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
            SAI_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
            SAI_CUDA(cudaEventRecord(ev_in, caller));
            SAI_CUDA(cudaStreamWaitEvent(aux, ev_in, 0));
            st = aux;
        }
    }
    cudaGraphExec_t gexec = nullptr;
    if (use_graph && st != caller) {
        cudaStreamCaptureStatus cs;
        SAI_CUDA(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusNone) {
            cudaGraph_t graph = nullptr;
            SAI_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            for (int q = 0; q < GM_STEPS_PER_CHECK; ++q) arnoldi_step<T>(I, k, A, Wk, S, G, cap, pt, fl, D, tiny, st);
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                gexec = nullptr;
                (void)cudaGetLastError();
            }
            // the captured launches ran no kernel yet: count them at replay
            sai_count_grid_add(-(long long)GM_STEPS_PER_CHECK * GM_LAUNCHES_PER_STEP);
        }
    }
    k_gm_init<T><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Bs, Xs, r, S.lall, pt2);
    int first = 1;
    sai_status status = SAI_OK;
    for (;;) {
        k_gm_cycle_start<<<SAI_GRID(1), CTRL, 0, st>>>(k, I.nch, pt2, cap, S, G, first, fl);
        first = 0;
        SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        if (!hflag) break;
        // steps 0..m: every system of the cycle stops by step m
        for (int j0 = 0; j0 <= m; j0 += GM_STEPS_PER_CHECK) {
            if (gexec) {
                cudaError_t e = cudaGraphLaunch(gexec, st);
                if (e != cudaSuccess) {
                    status = SAI_CUDA_ERROR;
                    break;
                }
                sai_count_grid_add((long long)GM_STEPS_PER_CHECK * GM_LAUNCHES_PER_STEP);
            } else {
                for (int q = 0; q < GM_STEPS_PER_CHECK; ++q)
                    arnoldi_step<T>(I, k, A, Wk, S, G, cap, pt, fl, D, tiny, st);
            }
            SAI_CUDA(cudaGetLastError());
            SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            if (!hflag) break;
        }
        if (status != SAI_OK) break;
        k_dc_trisolve<<<SAI_GRID(k), 128, tri_smem, st>>>(k, S, G);
        k_dc_combine<T><<<SAI_GRID(cb), IT_WARPS * 32, 0, st>>>(I, w, Wk.B, G);
        spmv<T, 2>(n, ld, A.M, k, w, Xs, nullptr, G.lcyc, st);  // x += M V y
        k_gm_cycle_end<<<SAI_GRID(1), CTRL, 0, st>>>(k, cap, S, G, fl);
        spmv<T, 1>(n, ld, A.A, k, Xs, r, Bs, G.lcyc, st);
        k_norm2<T><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, r, G.lcyc, pt2);
        SAI_CUDA(cudaGetLastError());
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    {
        // a ring wait of k_dc_update_ring that ran out (the flag is cleared for the next call)
        int perr = 0;
        if (cudaMemcpyFromSymbolAsync(&perr, d_pipe_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess && perr != 0) {
            const int zero = 0;
            (void)cudaMemcpyToSymbolAsync(d_pipe_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
            (void)cudaStreamSynchronize(st);
            if (status == SAI_OK) status = SAI_CUDA_ERROR;
        }
    }
    if (ev_in) {
        cudaEventRecord(ev_out, st);
        cudaStreamWaitEvent(caller, ev_out, 0);
        cudaEventDestroy(ev_in);
        cudaEventDestroy(ev_out);
    }
    return status;
}

// Carves the control state of GMRES(m) for k systems out of one double and
// one int buffer.
sai_status gm_alloc(int k, int m, Buf& hb, Buf& ib, Gm& G, cudaStream_t st)
{
    G.m = m;
    const size_t km1 = (size_t)k * (m + 1);
    const size_t hsz = 2 * (size_t)k * (m + 1) * m + 2 * (size_t)k * m + 4 * km1 + (size_t)k * m + 2 * (size_t)k +
                       (size_t)k * PS;
    const size_t isz = 6 * (size_t)k + 2 * (size_t)(k + 1) + 2;
    SAI_TRY(hb.alloc(sizeof(double) * hsz, st, true));
    SAI_TRY(ib.alloc(sizeof(int) * isz, st, true));
    SAI_CUDA(cudaMemsetAsync(hb.p, 0, sizeof(double) * hsz, st));
    SAI_CUDA(cudaMemsetAsync(ib.p, 0, sizeof(int) * isz, st));
    double* hp = hb.as<double>();
    G.H = hp;
    hp += (size_t)k * (m + 1) * m;
    G.Hu = hp;
    hp += (size_t)k * (m + 1) * m;
    G.cs = hp;
    hp += (size_t)k * m;
    G.sn = hp;
    hp += (size_t)k * m;
    G.g = hp;
    hp += km1;
    G.hp = hp;
    hp += km1;
    G.sco = hp;
    hp += km1;
    G.cco = hp;
    hp += km1;
    G.y = hp;
    hp += (size_t)k * m;
    G.alpha = hp;
    G.dco = hp + k;
    G.red = hp + 2 * k;
    int* ip = ib.as<int>();
    G.cyc = ip;
    G.adv = ip + k;
    G.jd = ip + 2 * k;
    G.done = ip + 3 * k;
    G.conv = ip + 4 * k;
    G.lcyc = ip + 5 * k;
    G.ladv = G.lcyc + (k + 1);
    G.jdev = G.ladv + (k + 1);
    G.bcnt = G.jdev + 1;
    G.scnt = G.bcnt + 1;
    return SAI_OK;
}

template <class T>
sai_status gm_work_alloc(size_t blk, int m, Buf& vb, Buf& wb, GmWork<T>& Wk, cudaStream_t st)
{
    // basis blocks are vs = blk + 96 values apart (keeps the blocks off a
    // common power-of-two stride); everything starts zeroed so the padding
    // rows [n, ld) of every vector stay zero
    const int64_t vs = (int64_t)blk + 96;
    SAI_TRY(vb.alloc(sizeof(T) * (size_t)vs * (m + 1) + 16, st, true));
    SAI_TRY(wb.alloc(sizeof(T) * blk * 4 + 16, st, true));
    SAI_CUDA(cudaMemsetAsync(wb.p, 0, sizeof(T) * blk * 4, st));
    SAI_CUDA(cudaMemsetAsync(vb.p, 0, sizeof(T) * (size_t)vs * (m + 1), st));
    Wk.B.V = vb.as<T>();
    Wk.B.vs = vs;
    Wk.r = wb.as<T>();
    Wk.t = Wk.r + blk;
    Wk.z = Wk.t + blk;
    Wk.w = Wk.z + blk;
    return SAI_OK;
}

// ------------------------------------------------------------------ block GMRES(m)
// The block Krylov alternative for the s+1 systems (section 3, after
// Theorem 2): block GMRES (Vital) with right preconditioning, FP64. The kb
// systems still active at a cycle start share one block Krylov space of
// A~M; their compact positions a = 0..kb-1 map to systems lact[1+a]. The
// basis blocks V_0, V_1, .. (kb vectors each) follow one another, so basis
// vector b = j*kb + a sits at V + b*ld and any leading part of the basis is
// one contiguous range. One block step:
//   T = M V_j, W = A~ T                  (the SpMV of the other solvers)
//   H = V^T W, W -= V H, twice           (block classical Gram-Schmidt)
//   W = V_{j+1} R                        (shifted Cholesky QR, three passes:
//                                         Fukaya, Kannan, Nakatsukasa,
//                                         Yamamoto, Yanagisawa 2020)
//   one block reduces the new block column of Hbar with Householder
//   reflections on rows q..q+kb of each column q, applies them to G and
//   tests every column's least-squares residual against its threshold.
// At a cycle end Y = Rtri^{-1} G_top, X[lact] += M (V Y), R = B - A~ X.
// In exact arithmetic the iterates are those of block GMRES with block
// modified Gram-Schmidt and Householder QR.

constexpr int BG_KMAX = 32;  // largest block (systems per block)
constexpr int BG_CR = 1024;  // rows per chunk of the Gram kernel
constexpr int BG_GV = 8;     // basis vectors per Gram block (one per warp)
constexpr int BG_UT = 256;   // threads (rows) per block of the update kernels
constexpr int BG_HB = 64;    // rows of H staged at a time by the update kernel

template <class T>
struct Bg {
    T *V, *T1, *Z, *R;      // basis ((m+1)*k vectors of ld), work blocks and residuals of k vectors (type T)
    double *Hb;             // Hbar, column-major, ldh = (m+1)*k rows, m*k columns
    double *hv, *hbeta;     // reflector of column q: hv[q*(k+1) + l], l = 0..kb; its beta
    double *G;              // (m+1)*k x k, column-major (ldh)
    double *Ys;             // the cycle's solution coefficients, m*k x k, column-major (ld m*k)
    double *Rt, *Rp;        // k x k column-major: R of the QR (product of passes), one pass's R
    double *Gm;             // k x k Gram matrix of one QR pass
    double *H1, *H2;        // the two Gram-Schmidt passes' coefficients, nv x kb (ld nv)
    double *part;           // Gram partials [chunk][b][c]
    int *lact, *lid;        // active systems (count + ids); identity list (count + 0..kb-1)
    int *flags;             // [0] every column converged, [1] error, [2] kb
    int m, k;
    int64_t ldh;
};

// basis vectors per warp of the Gram kernel: W's row, held in registers,
// serves that many of them
__host__ __device__ constexpr int bg_vb(int esz, int KB)
{
    return esz == 4 ? (KB <= 12 ? 4 : (KB <= 16 ? 2 : 1)) : (KB <= 8 ? 2 : 1);
}

template <class T, int KB>
__global__ void __launch_bounds__(BG_GV * 32)
k_bg_gram(int32_t n, int64_t ld, const T* __restrict__ V, int nv, const T* __restrict__ W, int kb,
          double* __restrict__ part)
{
    constexpr int VB = bg_vb(sizeof(T), KB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b0 = (blockIdx.y * BG_GV + warp) * VB;
    if (b0 >= nv) return;
    const int64_t r0 = (int64_t)blockIdx.x * BG_CR;
    const int64_t r1 = r0 + BG_CR < n ? r0 + BG_CR : n;
    T acc[VB][KB];
#pragma unroll
    for (int u = 0; u < VB; ++u)
#pragma unroll
        for (int c = 0; c < KB; ++c) acc[u][c] = 0;
    for (int64_t r = r0 + lane; r < r1; r += 32) {
        T w[KB];
#pragma unroll
        for (int c = 0; c < KB; ++c) w[c] = c < kb ? W[(int64_t)c * ld + r] : T(0);
#pragma unroll
        for (int u = 0; u < VB; ++u)
            if (b0 + u < nv) {
                const T x = V[(int64_t)(b0 + u) * ld + r];
#pragma unroll
                for (int c = 0; c < KB; ++c) acc[u][c] = fma(x, w[c], acc[u][c]);
            }
    }
#pragma unroll
    for (int u = 0; u < VB; ++u)
        if (b0 + u < nv)
#pragma unroll
            for (int c = 0; c < KB; ++c)
                if (c < kb) {
                    const T sum = warp_sum_t(acc[u][c]);
                    if (lane == 0) part[((int64_t)blockIdx.x * nv + b0 + u) * kb + c] = (double)sum;
                }
}

// H[c*nv + b] = the sum over chunks of part[q][b][c]: a warp per (b, c), lane
// l takes chunks l, l+32, .. in order, then a fixed shuffle tree
__global__ void k_bg_reduce(int nch, int nv, int kb, const double* __restrict__ part, double* __restrict__ H)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)nv * kb) return;
    const int b = (int)(w / kb), c = (int)(w % kb);
    double s = 0.0;
    for (int q = lane; q < nch; q += 32) s += part[((int64_t)q * nv + b) * kb + c];
    s = warp_sum(s);
    if (lane == 0) H[(int64_t)c * nv + b] = s;
}

// W -= V H (overwrite = 0) or W = V H (overwrite = 1); H: nv x kb, ld ldhh
template <class T, int KB>
__global__ void __launch_bounds__(BG_UT)
k_bg_update(int32_t n, int64_t ld, const T* __restrict__ V, int nv, const double* __restrict__ H, int ldhh,
            int kb, T* __restrict__ W, int overwrite)
{
    __shared__ T hs[BG_HB * KB];
    const T sgn = overwrite ? T(1) : T(-1);
    for (int64_t base = (int64_t)blockIdx.x * BG_UT; base < n; base += (int64_t)gridDim.x * BG_UT) {
        const int64_t r = base + threadIdx.x;
        const bool ok = r < n;
        T acc[KB];
#pragma unroll
        for (int c = 0; c < KB; ++c) acc[c] = (!overwrite && ok && c < kb) ? W[(int64_t)c * ld + r] : T(0);
        for (int b0 = 0; b0 < nv; b0 += BG_HB) {
            const int bl = nv - b0 < BG_HB ? nv - b0 : BG_HB;
            __syncthreads();
            for (int e = threadIdx.x; e < bl * KB; e += BG_UT) {
                const int t = e / KB, c = e % KB;
                hs[e] = c < kb ? (T)H[(int64_t)c * ldhh + b0 + t] : T(0);
            }
            __syncthreads();
            if (ok)
                for (int t = 0; t < bl; ++t) {
                    const T x = sgn * V[(int64_t)(b0 + t) * ld + r];
#pragma unroll
                    for (int c = 0; c < KB; ++c) acc[c] = fma(x, hs[t * KB + c], acc[c]);
                }
        }
        if (ok)
#pragma unroll
            for (int c = 0; c < KB; ++c)
                if (c < kb) W[(int64_t)c * ld + r] = acc[c];
    }
}

// one QR pass's Cholesky factor: Gm (+ shift on the first pass) = Rp^T Rp,
// Rt = Rp Rt (Rt = Rp on the first pass); a pivot <= 0 sets flags[1]
__global__ void __launch_bounds__(1024) k_bg_chol(int kb, double leff, double unit, const double* __restrict__ Gm,
                                                  double* Rp, double* Rt, int first, int* flags)
{
    __shared__ double a[BG_KMAX][BG_KMAX + 1];
    __shared__ double rt[BG_KMAX][BG_KMAX + 1];
    __shared__ double sh;
    const int t = threadIdx.x;
    const int i = t / BG_KMAX, q = t % BG_KMAX;
    if (i < kb && q < kb) a[i][q] = Gm[q * kb + i];
    __syncthreads();
    if (t == 0) {
        double tr = 0.0;
        for (int c = 0; c < kb; ++c) tr += a[c][c];
        // shift of the first pass: 11 (leff kb + kb (kb + 1)) u ||W||_F^2, leff
        // the length of the summations that formed Gm, u the unit roundoff
        sh = first ? 11.0 * (leff * kb + (double)kb * (kb + 1)) * unit * tr : 0.0;
    }
    __syncthreads();
    if (i < kb && i == q) a[i][i] += sh;
    __syncthreads();
    for (int p = 0; p < kb; ++p) {
        if (t == 0) {
            double d = a[p][p];
            if (!(d > 0.0)) {
                atomicExch(&flags[1], 1);
                d = 1.0;
            }
            a[p][p] = sqrt(d);
        }
        __syncthreads();
        if (t > p && t < kb) a[p][t] /= a[p][p];
        __syncthreads();
        if (i > p && i < kb && q >= i && q < kb) a[i][q] -= a[p][i] * a[p][q];
        __syncthreads();
    }
    // a's upper triangle is Rp
    if (i < kb && q < kb) {
        const double r = q >= i ? a[i][q] : 0.0;
        Rp[q * kb + i] = r;
        if (first) Rt[q * kb + i] = r;
        else rt[i][q] = Rt[q * kb + i];
    }
    __syncthreads();
    if (!first && i < kb && q < kb) {
        double s = 0.0;
        for (int u = i; u <= q; ++u) s += a[i][u] * rt[u][q];
        Rt[q * kb + i] = q >= i ? s : 0.0;
    }
}

// W = W Rp^{-1}, row by row
template <class T, int KB>
__global__ void __launch_bounds__(BG_UT) k_bg_trsm(int32_t n, int64_t ld, T* __restrict__ W, int kb,
                                                   const double* __restrict__ Rp)
{
    __shared__ T r[KB * KB];
    for (int e = threadIdx.x; e < KB * KB; e += BG_UT) {
        const int i = e % KB, q = e / KB;
        r[e] = (i < kb && q < kb) ? (T)Rp[q * kb + i] : T(1);
    }
    __syncthreads();
    for (int64_t row = (int64_t)blockIdx.x * BG_UT + threadIdx.x; row < n; row += (int64_t)gridDim.x * BG_UT) {
        T y[KB];
#pragma unroll
        for (int c = 0; c < KB; ++c) {
            if (c < kb) {
                T s = W[(int64_t)c * ld + row];
#pragma unroll
                for (int i = 0; i < c; ++i) s -= y[i] * r[c * KB + i];
                y[c] = s / r[c * KB + c];
                W[(int64_t)c * ld + row] = y[c];
            } else {
                y[c] = 0;
            }
        }
    }
}

// the reflector of column q (rows q..q+kb, hv[0..kb], beta) applied by one
// warp to the column x (rows q..q+kb of a column-major array)
__device__ __forceinline__ void bg_reflect(const double* __restrict__ v, double beta, double* x, int kb, int lane)
{
    double d = 0.0;
    for (int l = lane; l <= kb; l += 32) d = fma(v[l], x[l], d);
    d = warp_sum(d) * beta;
    for (int l = lane; l <= kb; l += 32) x[l] -= d * v[l];
    __syncwarp();
}

// block step j: assemble the new block column of Hbar, reduce it, update G,
// test each column; one block of 32 * BG_KMAX threads, warp a owns column a
template <class T>
__global__ void __launch_bounds__(32 * BG_KMAX) k_bg_lsq(int j, Bg<T> B, Sys S, const int* __restrict__ cap)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb = B.flags[2];
    const int nv = (j + 1) * kb;
    const int64_t ldh = B.ldh;
    double* col = B.Hb + (int64_t)(j * kb + (warp < kb ? warp : 0)) * ldh;
    if (warp < kb) {
        for (int i = lane; i < nv; i += 32)
            col[i] = B.H1[(int64_t)warp * nv + i] + B.H2[(int64_t)warp * nv + i];
        for (int i = lane; i < kb; i += 32) col[nv + i] = i <= warp ? B.Rt[warp * kb + i] : 0.0;
        __syncwarp();
        // the earlier reflections, in order. Reflection q touches rows
        // q..q+kb, so for kb < 32 the kb+1 rows in play sit in the warp's
        // registers (lane l: row q+l): after reflection q, row q is final and
        // the window moves down one row; the next reflector and the row that
        // enters are loaded ahead (neither depends on the reflections so far).
        const int nq = j * kb;
        if (kb < 32 && nq > 0) {
            const int64_t hs = B.k + 1;
            double x = lane <= kb ? col[lane] : 0.0;
            double v = lane <= kb ? B.hv[lane] : 0.0;
            double be = B.hbeta[0];
            double in = lane == kb ? col[kb + 1] : 0.0;
            for (int q = 0; q < nq; ++q) {
                const bool more = q + 1 < nq;
                const double vn = (more && lane <= kb) ? B.hv[(q + 1) * hs + lane] : 0.0;
                const double bn = more ? B.hbeta[q + 1] : 0.0;
                const double inn = (more && lane == kb) ? col[q + kb + 2] : 0.0;
                const double d = warp_sum(v * x) * be;
                x -= d * v;
                if (lane == 0) col[q] = x;
                const double down = __shfl_down_sync(SAI_FULL, x, 1);
                x = lane < kb ? down : (lane == kb ? in : 0.0);
                v = vn;
                be = bn;
                in = inn;
            }
            if (lane <= kb) col[nq + lane] = x;
        } else {
            for (int q = 0; q < nq; ++q) bg_reflect(B.hv + (int64_t)q * (B.k + 1), B.hbeta[q], col + q, kb, lane);
        }
    }
    __syncthreads();
    for (int a = 0; a < kb; ++a) {
        const int q = j * kb + a;
        double* hvq = B.hv + (int64_t)q * (B.k + 1);
        if (warp == a) {
            double* x = B.Hb + (int64_t)q * ldh + q;
            double ss = 0.0;
            for (int l = lane; l <= kb; l += 32) ss = fma(x[l], x[l], ss);
            const double nrm = sqrt(warp_sum(ss));
            const double x0 = x[0];
            __syncwarp();
            if (nrm == 0.0) {
                for (int l = lane; l <= kb; l += 32) hvq[l] = 0.0;
                if (lane == 0) B.hbeta[q] = 0.0;
            } else {
                const double alpha = x0 >= 0.0 ? -nrm : nrm;
                double vv = 0.0;
                for (int l = lane; l <= kb; l += 32) {
                    const double vl = l == 0 ? x0 - alpha : x[l];
                    hvq[l] = vl;
                    vv = fma(vl, vl, vv);
                }
                vv = warp_sum(vv);
                __syncwarp();
                for (int l = lane; l <= kb; l += 32) x[l] = l == 0 ? alpha : 0.0;
                if (lane == 0) B.hbeta[q] = 2.0 / vv;
            }
        }
        __syncthreads();
        if (warp < kb) {
            const double beta = B.hbeta[q];
            if (warp > a) bg_reflect(hvq, beta, B.Hb + (int64_t)(j * kb + warp) * ldh + q, kb, lane);
            bg_reflect(hvq, beta, B.G + (int64_t)warp * ldh + q, kb, lane);
        }
        __syncthreads();
    }
    // least-squares residual of each column: G rows (j+1)kb .. (j+2)kb-1;
    // a system that used up its iterations ends the cycle too
    __shared__ int nconv, ncap;
    if (threadIdx.x == 0) {
        nconv = 0;
        ncap = 0;
    }
    __syncthreads();
    if (warp < kb) {
        const double* g = B.G + (int64_t)warp * ldh + nv;
        double e = 0.0;
        for (int l = lane; l < kb; l += 32) e = fma(g[l], g[l], e);
        e = warp_sum(e);
        if (lane == 0) {
            const int c = B.lact[1 + warp];
            S.iters[c] += 1;
            if (sqrt(e) < S.thr[c]) atomicAdd(&nconv, 1);
            if (S.iters[c] >= cap[c]) atomicAdd(&ncap, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) B.flags[0] = nconv == kb || ncap > 0;
}

// Ys = Rtri^{-1} G_top, nt = (steps) * kb rows; warp c solves column c
template <class T>
__global__ void __launch_bounds__(32 * BG_KMAX) k_bg_backsolve(int nt, Bg<T> B)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb = B.flags[2];
    if (warp >= kb) return;
    const int64_t ldh = B.ldh, ldy = (int64_t)B.m * B.k;
    double* y = B.Ys + (int64_t)warp * ldy;
    const double* g = B.G + (int64_t)warp * ldh;
    for (int i = nt - 1; i >= 0; --i) {
        double s = 0.0;
        for (int q = i + 1 + lane; q < nt; q += 32) s = fma(B.Hb[(int64_t)q * ldh + i], y[q], s);
        s = warp_sum(s);
        if (lane == 0) {
            const double d = B.Hb[(int64_t)i * ldh + i];
            if (d == 0.0) {
                atomicExch(&B.flags[1], 2);
                y[i] = 0.0;
            } else {
                y[i] = (g[i] - s) / d;
            }
        }
        __syncwarp();
    }
}

// cycle start: true residual norms (partials of the listed systems), stop
// tests, the active list and its identity list; flags[2] = kb
template <class T>
__global__ void k_bg_cycle(int k, int nch, const double* part, const int* __restrict__ cap, int first, Sys S,
                           Bg<T> B)
{
    __shared__ int act[CTRL];
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (first) {
            S.iters[c] = 0;
            S.status[c] = ST_MAXITER;
            S.active[c] = 1;
        }
        act[c] = 0;
        if (S.active[c]) {
            const double r = sqrt(sum_chunks(part, 0, c, k, nch));
            if (r < S.thr[c]) {
                S.active[c] = 0;
                S.status[c] = ST_OK;
            } else if (S.iters[c] >= cap[c] || B.flags[1]) {
                S.active[c] = 0;
                S.status[c] = B.flags[1] ? ST_BREAKDOWN : ST_MAXITER;
            } else {
                act[c] = 1;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        build_list(k, act, B.lact);
        const int kb = B.lact[0];
        B.lid[0] = kb;
        for (int a = 0; a < kb; ++a) B.lid[1 + a] = a;
        B.flags[2] = kb;
        B.flags[0] = 0;
    }
}

// V0[a] = R[lact[a]] and X[lact[a]] += T[a]
template <class T>
__global__ void k_bg_gather(int32_t n, int64_t ld, const int* __restrict__ lact, const T* __restrict__ R,
                            T* __restrict__ V0)
{
    const int kb = lact[0];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)kb * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / n);
        const int64_t r = e % n;
        V0[(int64_t)a * ld + r] = R[(int64_t)lact[1 + a] * ld + r];
    }
}

template <class T>
__global__ void k_bg_scatter_add(int32_t n, int64_t ld, const int* __restrict__ lact, const T* __restrict__ Tv,
                                 T* __restrict__ X)
{
    const int kb = lact[0];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)kb * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / n);
        const int64_t r = e % n;
        X[(int64_t)lact[1 + a] * ld + r] += Tv[(int64_t)a * ld + r];
    }
}

// algorithmic work of one block-GMRES pass, added to a profile site (only
// while a profile is open)
__global__ void k_bg_work(int site, double bytes, double flops) { kwork_add(site, bytes, flops); }

inline void bg_work(int site, double bytes, double flops, cudaStream_t st)
{
    if (sai_prof_on()) k_bg_work<<<SAI_GRID(1), 1, 0, st>>>(site, bytes, flops);
}

// the kernels specialised on the block size: KB = the smallest of 4, 8, 12,
// 16, 24, 32 that holds kb
#define BG_DISPATCH(kb, F, T, ...)                               \
    do {                                                         \
        if ((kb) <= 4) F<T, 4>__VA_ARGS__;                       \
        else if ((kb) <= 8) F<T, 8>__VA_ARGS__;                  \
        else if ((kb) <= 12) F<T, 12>__VA_ARGS__;                \
        else if ((kb) <= 16) F<T, 16>__VA_ARGS__;                \
        else if ((kb) <= 24) F<T, 24>__VA_ARGS__;                \
        else F<T, 32>__VA_ARGS__;                                \
    } while (0)

// P = V^T W (nv basis vectors from V, kb columns of W) into H (nv x kb)
template <class T>
void bg_gram(int32_t n, int64_t ld, const T* V, int nv, const T* W, int kb, double* part, double* H,
             cudaStream_t st)
{
    const int nch = (int)(((int64_t)n + BG_CR - 1) / BG_CR);
    const int KBs = kb <= 4 ? 4 : kb <= 8 ? 8 : kb <= 12 ? 12 : kb <= 16 ? 16 : kb <= 24 ? 24 : 32;
    const int per_block = BG_GV * bg_vb((int)sizeof(T), KBs);
    const dim3 grid((unsigned)nch, (unsigned)((nv + per_block - 1) / per_block));
    sai_count_grid(grid.x * grid.y);
    BG_DISPATCH(kb, k_bg_gram, T, <<<grid, BG_GV * 32, 0, st>>>(n, ld, V, nv, W, kb, part));
    k_bg_reduce<<<SAI_GRID(sai_div_up((int64_t)nv * kb * 32, 256)), 256, 0, st>>>(nch, nv, kb, part, H);
}

unsigned bg_rows_grid(int32_t n)
{
    int64_t g = ((int64_t)n + BG_UT - 1) / BG_UT;
    if (g > (int64_t)g_sms * 8) g = (int64_t)g_sms * 8;
    return (unsigned)(g > 0 ? g : 1);
}

template <class T>
void bg_update(int32_t n, int64_t ld, const T* V, int nv, const double* H, int ldhh, int kb, T* W, int overwrite,
               cudaStream_t st)
{
    const unsigned g = bg_rows_grid(n);
    sai_count_grid(g);
    BG_DISPATCH(kb, k_bg_update, T, <<<g, BG_UT, 0, st>>>(n, ld, V, nv, H, ldhh, kb, W, overwrite));
}

// W = Q R: shifted Cholesky QR in three passes, R accumulated in B.Rt. The
// Gram matrices sum BG_CR/32 products per lane and 5 shuffle levels in T,
// then the chunks in FP64 (counted too when T is FP64).
template <class T>
void bg_qr(int32_t n, int64_t ld, T* W, int kb, const Bg<T>& B, cudaStream_t st)
{
    const unsigned g = bg_rows_grid(n);
    const double unit = sizeof(T) == 4 ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
    const double leff = BG_CR / 32 + 5 + (sizeof(T) == 8 ? ((int64_t)n + BG_CR - 1) / BG_CR : 1);
    for (int pass = 0; pass < 3; ++pass) {
        bg_gram<T>(n, ld, W, kb, W, kb, B.part, B.Gm, st);
        k_bg_chol<<<SAI_GRID(1), 1024, 0, st>>>(kb, leff, unit, B.Gm, B.Rp, B.Rt, pass == 0, B.flags);
        sai_count_grid(g);
        BG_DISPATCH(kb, k_bg_trsm, T, <<<g, BG_UT, 0, st>>>(n, ld, W, kb, B.Rp));
    }
}

// Block GMRES(m) over the k systems with finite thresholds (vectors in T,
// the small matrices in FP64); system c stops at S.thr[c] or after cap[c]
// block steps; S.iters counts the block steps each system took part in.
template <class T>
sai_status bgmres_run(const Items& I, int k, int m, const Ops<T>& A, const T* Bs, T* Xs, T* R, Bg<T>& B, Sys& S,
                      const int* cap, double* pt2, const Dims& D, cudaStream_t st)
{
    const int32_t n = I.n;
    const int64_t ld = I.ld;
    const int ib = item_blocks(n > 0 ? n : 1, k);
    const unsigned gg = bg_rows_grid(n) * 4;
    k_gm_init<T><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Bs, Xs, R, S.lall, pt2);
    SAI_CUDA(cudaMemsetAsync(B.flags, 0, sizeof(int) * 4, st));
    int h[3] = {0, 0, 0};
    for (int first = 1;; first = 0) {
        k_bg_cycle<T><<<SAI_GRID(1), CTRL, 0, st>>>(k, I.nch, pt2, cap, first, S, B);
        SAI_CUDA(cudaMemcpyAsync(h, B.flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        const int kb = h[2];
        if (kb == 0) break;
        // V_0 R = the active residuals; G = [R; 0]
        k_bg_gather<T><<<SAI_GRID(gg), 256, 0, st>>>(n, ld, B.lact, R, B.V);
        bg_qr<T>(n, ld, B.V, kb, B, st);
        // a breakdown in the QR of V_0 (the active residuals are numerically
        // dependent): no step of this cycle is taken, X keeps its value and
        // the next cycle start ends the active systems with BREAKDOWN
        SAI_CUDA(cudaMemcpyAsync(h, B.flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        if (h[1]) continue;
        SAI_CUDA(cudaMemsetAsync(B.G, 0, sizeof(double) * (size_t)B.ldh * B.k, st));
        SAI_CUDA(cudaMemcpy2DAsync(B.G, sizeof(double) * B.ldh, B.Rt, sizeof(double) * kb, sizeof(double) * kb, kb,
                                   cudaMemcpyDeviceToDevice, st));
        int steps = 0;
        for (int j = 0; j < m; ++j) {
            const T* Vj = B.V + (int64_t)j * kb * ld;
            T* Vn = B.V + (int64_t)(j + 1) * kb * ld;
            const int nv = (j + 1) * kb;
            {
                ProfScope ps(D.site_spmm, st);
                spmv<T, 0>(n, ld, A.M, kb, Vj, B.T1, nullptr, B.lid, st);
            }
            {
                ProfScope ps(D.site_spmm, st);
                spmv<T, 0>(n, ld, A.A, kb, B.T1, Vn, nullptr, B.lid, st);
            }
            // SpMV: matrix values + column indices once, kb vectors in and out
            bg_work(D.site_spmm, (D.esz + 4.0) * (D.nnzM + D.nnzA) + 4.0 * D.esz * D.n * kb,
                    2.0 * (D.nnzM + D.nnzA) * kb, st);
            for (int pass = 0; pass < 2; ++pass) {
                double* H = pass ? B.H2 : B.H1;
                {
                    ProfScope ps(D.site_dots, st);
                    bg_gram<T>(n, ld, B.V, nv, Vn, kb, B.part, H, st);
                }
                {
                    ProfScope ps(D.site_upd, st);
                    bg_update<T>(n, ld, B.V, nv, H, nv, kb, Vn, 0, st);
                }
                // Gram: the nv basis vectors and W once; update: V once, W in and out
                bg_work(D.site_dots, D.esz * D.n * (nv + kb), 2.0 * D.n * nv * kb, st);
                bg_work(D.site_upd, D.esz * D.n * (nv + 2.0 * kb), 2.0 * D.n * nv * kb, st);
            }
            {
                ProfScope ps(PROF_GM_STEP, st);
                bg_qr<T>(n, ld, Vn, kb, B, st);
                k_bg_lsq<T><<<SAI_GRID(1), 32 * BG_KMAX, 0, st>>>(j, B, S, cap);
            }
            SAI_CUDA(cudaGetLastError());
            SAI_CUDA(cudaMemcpyAsync(h, B.flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            // a breakdown in this step's QR leaves the step out: the first j
            // block steps' rows of G and columns of the block Hessenberg
            // matrix are final before step j's reflections
            steps = h[1] ? j : j + 1;
            if (h[0] || h[1]) break;
        }
        if (steps == 0) continue;
        // X[lact] += M (V Ys), R = B - A~ X
        k_bg_backsolve<T><<<SAI_GRID(1), 32 * BG_KMAX, 0, st>>>(steps * kb, B);
        bg_update<T>(n, ld, B.V, steps * kb, B.Ys, m * B.k, kb, B.Z, 1, st);
        spmv<T, 0>(n, ld, A.M, kb, B.Z, B.T1, nullptr, B.lid, st);
        k_bg_scatter_add<T><<<SAI_GRID(gg), 256, 0, st>>>(n, ld, B.lact, B.T1, Xs);
        spmv<T, 1>(n, ld, A.A, k, Xs, R, Bs, B.lact, st);
        k_norm2<T><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, R, B.lact, pt2);
        SAI_CUDA(cudaGetLastError());
    }
    return SAI_OK;
}

template <class T>
sai_status bg_alloc(int k, int m, int32_t n, int64_t ld, Buf& vb, Buf& hb, Buf& ib, Bg<T>& B, cudaStream_t st)
{
    B.m = m;
    B.k = k;
    B.ldh = (int64_t)(m + 1) * k;
    const size_t blk = (size_t)ld * k;
    // basis, two work blocks and the residual block R of the caller
    SAI_TRY(vb.alloc(sizeof(T) * (blk * (size_t)(m + 1) + 3 * blk) + 64, st, true));
    SAI_CUDA(cudaMemsetAsync(vb.p, 0, sizeof(T) * (blk * (size_t)(m + 1) + 3 * blk), st));
    T* d = vb.as<T>();
    B.V = d;
    B.T1 = d + blk * (m + 1);
    B.Z = B.T1 + blk;
    B.R = B.Z + blk;
    const int nch = (int)(((int64_t)(n > 0 ? n : 1) + BG_CR - 1) / BG_CR);
    const size_t nvmax = (size_t)B.ldh;
    const size_t hsz = (size_t)B.ldh * m * k + (size_t)m * k * (k + 1) + (size_t)m * k + (size_t)B.ldh * k +
                       (size_t)m * k * k + 3 * (size_t)k * k + 2 * nvmax * k + (size_t)nch * nvmax * k;
    SAI_TRY(hb.alloc(sizeof(double) * hsz, st, true));
    SAI_CUDA(cudaMemsetAsync(hb.p, 0, sizeof(double) * hsz, st));
    double* e = hb.as<double>();
    B.Hb = e;
    e += (size_t)B.ldh * m * k;
    B.hv = e;
    e += (size_t)m * k * (k + 1);
    B.hbeta = e;
    e += (size_t)m * k;
    B.G = e;
    e += (size_t)B.ldh * k;
    B.Ys = e;
    e += (size_t)m * k * k;
    B.Rt = e;
    B.Rp = e + k * k;
    B.Gm = e + 2 * k * k;
    e += 3 * (size_t)k * k;
    B.H1 = e;
    B.H2 = e + nvmax * k;
    e += 2 * nvmax * k;
    B.part = e;
    SAI_TRY(ib.alloc(sizeof(int) * (2 * (size_t)(k + 1) + 4), st, true));
    SAI_CUDA(cudaMemsetAsync(ib.p, 0, sizeof(int) * (2 * (size_t)(k + 1) + 4), st));
    B.lact = ib.as<int>();
    B.lid = B.lact + (k + 1);
    B.flags = B.lid + (k + 1);
    return SAI_OK;
}

}  // namespace

sai_status sai_krylov_run(const sai_split_s* h, const sai_precond_s* P, int32_t k, const double* B,
                          const double* thr, const sai_krylov_params* prm, double* X, int32_t* iters,
                          int32_t* status, cudaStream_t st)
{
    if (!h || !P || !prm || !thr || !iters || !status || k < 1) return SAI_INVALID_ARG;
    const bool big_ok =
        (prm->method == SAI_BICGSTAB || prm->method == SAI_CGS || prm->method == SAI_BICG) && prm->precision == SAI_FP64;
    if (k > (big_ok ? KBIG : CTRL)) return SAI_INVALID_ARG;
    if (prm->maxit < 0 || ((prm->method == SAI_GMRES || prm->method == SAI_BGMRES) &&
                           (prm->restart < 1 || prm->restart >= GM_MAXM)))
        return SAI_INVALID_ARG;
    if (prm->method != SAI_BICGSTAB && prm->method != SAI_GMRES && prm->method != SAI_CGS && prm->method != SAI_BICG &&
        prm->method != SAI_BGMRES)
        return SAI_INVALID_ARG;
    if (prm->method == SAI_BGMRES && k > BG_KMAX) return SAI_INVALID_ARG;
    if (prm->precision != SAI_FP64 && prm->precision != SAI_FP32_REFINE64) return SAI_INVALID_ARG;
    if (prm->transpose != 0 && prm->transpose != 1) return SAI_INVALID_ARG;
    if (prm->precision == SAI_FP32_REFINE64 && prm->method != SAI_GMRES && prm->method != SAI_BGMRES)
        return SAI_NOT_IMPLEMENTED;
    const int32_t n = h->n;
    if (n > 0 && (!B || !X)) return SAI_INVALID_ARG;
    if (g_sms == 0) {
        int dev = 0;
        SAI_CUDA(cudaGetDevice(&dev));
        SAI_CUDA(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev));
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_res_dots[0], k_dc_dots<double>, IT_WARPS * 32, 0));
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_res_dots[1], k_dc_dots<float>, IT_WARPS * 32, 0));
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_res_upd[0], k_dc_update<double>, IT_WARPS * 32, 0));
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_res_upd[1], k_dc_update<float>, IT_WARPS * 32, 0));
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_res_sellp[0], k_spmv_sellp<double, 0, SELL_CTP>,
                                                               SP_WARPS * 32, 0));
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_res_sellp[1], k_spmv_sellp<float, 0, SELL_CTP>,
                                                               SP_WARPS * 32, 0));
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_res_ring[0], k_dc_update_ring<double>,
                                                               (UP_CWARPS + 1) * 32, 0));
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_res_ring[1], k_dc_update_ring<float>,
                                                               (UP_CWARPS + 1) * 32, 0));
        for (int i = 0; i < 2; ++i) {
            if (g_res_dots[i] < 1) g_res_dots[i] = 1;
            if (g_res_upd[i] < 1) g_res_upd[i] = 1;
            if (g_res_ring[i] < 1) g_res_ring[i] = 1;
            if (g_res_sellp[i] < 1) g_res_sellp[i] = 1;
        }
    }
    // leading dimension: n rounded up to 32, plus 32 so that the k system
    // vectors of a block do not all start on the same large power of two
    const int64_t ld = ((int64_t)n + 31) / 32 * 32 + 32;
    const size_t blk = (size_t)ld * k;  // one system-major block of k vectors
    Items I;
    I.n = n;
    I.ld = ld;
    I.nch = nchunks(n > 0 ? n : 1);
    I.nchu = (int)(((int64_t)(n > 0 ? n : 1) + CHUNK_U - 1) / CHUNK_U);
    const int ib = item_blocks(n > 0 ? n : 1, k);
    // CSR of A~ and M, or for the transposed solves CSR of A~^T and M^T,
    // which are the CSC arrays of A~ and M
    Ops<double> A64;
    if (!prm->transpose) {
        A64.A.rp = h->Atr_rp.as<int64_t>();
        A64.A.ci = h->Atr_ci.as<int32_t>();
        A64.A.v = h->Atr_v.as<double>();
        A64.M.rp = P->Mr_rp.as<int64_t>();
        A64.M.ci = P->Mr_ci.as<int32_t>();
        A64.M.v = P->Mr_v.as<double>();
    } else {
        A64.A.rp = h->At_cp.as<int64_t>();
        A64.A.ci = h->At_ri.as<int32_t>();
        A64.A.v = h->At_v.as<double>();
        A64.M.rp = P->M_cp.as<int64_t>();
        A64.M.ci = P->M_ri.as<int32_t>();
        A64.M.v = P->M_v.as<double>();
    }
    Buf sell[6];  // sliced-ELL copies of the two operators of the main loop
    int64_t tg = sai_div_up((int64_t)n * k > 0 ? (int64_t)n * k : 1, 256);
    if (tg > (int64_t)g_sms * 8) tg = (int64_t)g_sms * 8;
    const int tgrid = (int)tg;

    Buf sysd, sysi, part, part2, flag, Bs, Xs, capb;
    SAI_TRY(sysd.alloc(sizeof(double) * 7 * k, st, true));
    SAI_TRY(sysi.alloc(sizeof(int) * (5 * k + 3 * (k + 1)), st, true));
    const int nslot = prm->method != SAI_GMRES ? 2 : (PS > 2 ? PS : 2);  // partial sums per (system, chunk)
    SAI_TRY(part.alloc(sizeof(double) * (size_t)k * I.nch * nslot, st, true));
    SAI_TRY(part2.alloc(sizeof(double) * (size_t)k * I.nch * 2, st, true));
    SAI_TRY(flag.alloc(sizeof(int) * 4, st, true));
    SAI_TRY(Bs.alloc(sizeof(double) * blk + 8, st, true));
    SAI_TRY(Xs.alloc(sizeof(double) * blk + 8, st, true));
    SAI_TRY(capb.alloc(sizeof(int) * k, st, true));
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
    D.esz = 8.0;
    D.site_spmm = PROF_SPMM;
    D.site_dots = PROF_GM_DOTS;
    D.site_upd = PROF_GM_UPDATE;
    double* Bsd = Bs.as<double>();
    double* Xsd = Xs.as<double>();
    double* pt = part.as<double>();
    double* pt2 = part2.as<double>();
    int* cap = capb.as<int>();
    const int64_t ttiles = ((int64_t)n + 31) / 32 * ((k + 31) / 32);
    const unsigned tblk = (unsigned)(ttiles < (int64_t)g_sms * 16 ? (ttiles > 0 ? ttiles : 1) : (int64_t)g_sms * 16);
    if (n > 0 && k >= 32) k_soa_tiled<true><<<SAI_GRID(tblk), 256, 0, st>>>(n, k, ld, B, Bsd);
    else if (n > 0) k_to_soa<<<SAI_GRID(tgrid), 256, 0, st>>>(n, k, ld, B, Bsd);
    k_list_all<<<SAI_GRID(1), 256, 0, st>>>(k, S.lall);
    k_fill_int<<<SAI_GRID(1), 256, 0, st>>>(k, cap, prm->maxit);
    SAI_CUDA(cudaGetLastError());

    // sliced-ELL copies for the FP64 solvers; the refined forms build FP32
    // ones in the same buffers and keep the CSR arrays for the FP64 residual
    if (prm->precision == SAI_FP64) {
        Ops<double> S64 = A64;
        SAI_TRY(build_sell<double>(n, h->nnz_At, A64.A.rp, A64.A.ci, A64.A.v, sell[0], sell[1], sell[2], S64.A, st));
        SAI_TRY(build_sell<double>(n, P->nnz, A64.M.rp, A64.M.ci, A64.M.v, sell[3], sell[4], sell[5], S64.M, st));
        A64 = S64;
    }
    if (prm->method == SAI_BICGSTAB) {
        SAI_TRY(bicgstab_run(I, k, A64, Bsd, Xsd, S, pt, fl, prm->maxit, D, st));
    } else if (prm->method == SAI_CGS) {
        SAI_TRY(cgs_run(I, k, A64, Bsd, Xsd, S, pt, fl, prm->maxit, D, st));
    } else if (prm->method == SAI_BICG) {
        // the pair of K^T = M^T A~^T (or M A~ for the transposed solves):
        // A~'s other orientation first, then M's
        Ops<double> T64;
        if (!prm->transpose) {
            T64.M.rp = h->At_cp.as<int64_t>();
            T64.M.ci = h->At_ri.as<int32_t>();
            T64.M.v = h->At_v.as<double>();
            T64.A.rp = P->M_cp.as<int64_t>();
            T64.A.ci = P->M_ri.as<int32_t>();
            T64.A.v = P->M_v.as<double>();
        } else {
            T64.M.rp = h->Atr_rp.as<int64_t>();
            T64.M.ci = h->Atr_ci.as<int32_t>();
            T64.M.v = h->Atr_v.as<double>();
            T64.A.rp = P->Mr_rp.as<int64_t>();
            T64.A.ci = P->Mr_ci.as<int32_t>();
            T64.A.v = P->Mr_v.as<double>();
        }
        SAI_TRY(bicg_run(I, k, A64, T64, Bsd, Xsd, S, pt, fl, prm->maxit, D, st));
    } else if (prm->method == SAI_BGMRES && prm->precision == SAI_FP64) {
        Bg<double> Bgm;
        Buf vb, hb, ibuf;
        SAI_TRY(bg_alloc<double>(k, prm->restart, n, ld, vb, hb, ibuf, Bgm, st));
        SAI_TRY(bgmres_run<double>(I, k, prm->restart, A64, Bsd, Xsd, Bgm.R, Bgm, S, cap, pt2, D, st));
    } else if (prm->precision == SAI_FP64) {
        Gm G;
        Buf hb, ibuf, vb, wb;
        GmWork<double> Wk;
        SAI_TRY(gm_alloc(k, prm->restart, hb, ibuf, G, st));
        SAI_TRY(gm_work_alloc<double>(blk, prm->restart, vb, wb, Wk, st));
        SAI_TRY(gmres_run<double>(I, k, prm->restart, A64, Bsd, Xsd, Wk, S, G, cap, pt, pt2, fl, D, st));
    } else {
        // GMRES with iterative refinement: FP64 residual, correction and stop
        // tests outside; the inner solves run entirely in FP32.
        const double tau = prm->inner_tol > 0.0 ? prm->inner_tol : 1e-4;
        Gm G;
        Buf hb, ibuf, vb, wb, a32, m32, r64b, v32b, irb, ird;
        GmWork<float> Wk;
        Bg<float> Bgm;  // block GMRES inner solver
        if (prm->method == SAI_BGMRES) {
            SAI_TRY(bg_alloc<float>(k, prm->restart, n, ld, vb, hb, ibuf, Bgm, st));
        } else {
            SAI_TRY(gm_alloc(k, prm->restart, hb, ibuf, G, st));
            SAI_TRY(gm_work_alloc<float>(blk, prm->restart, vb, wb, Wk, st));
        }
        SAI_TRY(a32.alloc(sizeof(float) * (size_t)(h->nnz_At > 0 ? h->nnz_At : 1), st, true));
        SAI_TRY(m32.alloc(sizeof(float) * (size_t)(P->nnz > 0 ? P->nnz : 1), st, true));
        SAI_TRY(r64b.alloc(sizeof(double) * blk + 8, st, true));
        SAI_TRY(v32b.alloc(sizeof(float) * blk * 2 + 16, st, true));
        SAI_TRY(irb.alloc(sizeof(int) * (4 * k + (k + 1)), st, true));
        SAI_TRY(ird.alloc(sizeof(double) * 3 * k, st, true));
        SAI_CUDA(cudaMemsetAsync(v32b.p, 0, sizeof(float) * blk * 2, st));
        SAI_CUDA(cudaMemsetAsync(irb.p, 0, sizeof(int) * (4 * k + (k + 1)), st));
        int64_t cg = sai_div_up(h->nnz_At > P->nnz ? h->nnz_At : P->nnz, 256);
        if (cg > (int64_t)g_sms * 8) cg = (int64_t)g_sms * 8;
        if (cg < 1) cg = 1;
        if (h->nnz_At > 0) k_cast_f32<<<SAI_GRID(cg), 256, 0, st>>>(h->nnz_At, A64.A.v, a32.as<float>());
        if (P->nnz > 0) k_cast_f32<<<SAI_GRID(cg), 256, 0, st>>>(P->nnz, A64.M.v, m32.as<float>());
        Ops<float> A32;
        A32.A.rp = A64.A.rp;
        A32.A.ci = A64.A.ci;
        A32.A.v = a32.as<float>();
        A32.M.rp = A64.M.rp;
        A32.M.ci = A64.M.ci;
        A32.M.v = m32.as<float>();
        SAI_TRY(build_sell<float>(n, h->nnz_At, A64.A.rp, A64.A.ci, A64.A.v, sell[0], sell[1], sell[2], A32.A, st));
        SAI_TRY(build_sell<float>(n, P->nnz, A64.M.rp, A64.M.ci, A64.M.v, sell[3], sell[4], sell[5], A32.M, st));
        double* r64 = r64b.as<double>();
        float* r32 = v32b.as<float>();
        float* d32 = r32 + blk;
        int* done = irb.as<int>();
        int* status64 = done + k;
        int* tot = done + 2 * k;
        int* lir = done + 4 * k;
        double* beta = ird.as<double>();
        double* thr64 = beta + k;
        double* thr_in = S.thr;
        SAI_CUDA(cudaMemcpyAsync(thr64, thr, sizeof(double) * k, cudaMemcpyHostToDevice, st));
        Dims D32 = D;
        D32.esz = 4.0;
        D32.site_spmm = PROF_SPMM32;
        D32.site_dots = PROF_GM_DOTS32;
        D32.site_upd = PROF_GM_UPDATE32;
        // r64 = B, x64 = 0 and ||B||^2 partials
        k_gm_init<double><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, Bsd, Xsd, r64, S.lall, pt2);
        const int max_outer = 40;
        for (int outer = 0; outer < max_outer; ++outer) {
            k_ir_check<<<SAI_GRID(1), CTRL, 0, st>>>(k, I.nch, pt2, thr64, tau, prm->maxit, tot, done, status64, beta,
                                                     thr_in, cap, lir, fl);
            SAI_CUDA(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            if (!hflag) break;
            k_ir_scale<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, r64, beta, done, r32, S.lall);
            if (prm->method == SAI_BGMRES)
                SAI_TRY(bgmres_run<float>(I, k, prm->restart, A32, r32, d32, Bgm.R, Bgm, S, cap, pt2, D32, st));
            else
                SAI_TRY(gmres_run<float>(I, k, prm->restart, A32, r32, d32, Wk, S, G, cap, pt, pt2, fl, D32, st));
            k_ir_update<<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, Xsd, d32, beta, lir);
            k_ir_total<<<SAI_GRID(1), 32, 0, st>>>(k, lir, S.iters, tot);
            spmv<double, 1>(n, ld, A64.A, k, Xsd, r64, Bsd, lir, st);
            k_norm2<double><<<SAI_GRID(ib), IT_WARPS * 32, 0, st>>>(I, k, r64, lir, pt2);
            SAI_CUDA(cudaGetLastError());
        }
        // report the outer status and the total inner iterations
        k_ir_finish<<<SAI_GRID(1), CTRL, 0, st>>>(k, done, status64, tot, S.status, S.iters);
        SAI_CUDA(cudaGetLastError());
    }
    if (n > 0 && k >= 32) k_soa_tiled<false><<<SAI_GRID(tblk), 256, 0, st>>>(n, k, ld, Xsd, X);
    else if (n > 0) k_from_soa<<<SAI_GRID(tgrid), 256, 0, st>>>(n, k, ld, Xsd, X);
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
