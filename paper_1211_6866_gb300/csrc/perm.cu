// perm.cu -- zero-diagonal repair before the method (section 5): a row
// permutation p that makes the diagonal of A(p,:) zero-free (MATLAB's
// dmperm with one output: a maximum transversal), and B = A(p,:).
//
// Matching. Entries count when stored with a nonzero value. Columns whose
// diagonal counts start matched to it; the rest is found by phases of
// augmenting paths (a matching is maximum iff none exists):
//   - every unmatched column roots an alternating tree; the trees grow
//     together level by level: the frontier's columns claim their unvisited
//     rows (the smallest column wins a row, atomicMin), a claimed free row
//     ends its tree's search (the smallest such row is kept), a claimed
//     matched row brings its column into the next frontier;
//   - each tree that reached a free row flips the path back to its root.
//     Trees share no vertex, so the flips of one phase are independent.
// A tree stops growing once it has a free row, and the other trees keep
// growing, so a phase without a flip proves the matching maximum. Every
// choice is a minimum, so p does not depend on the order in which threads
// run. The host drives the levels (one small read-back per level).
//
// Frontier columns longer than CLAIM_LONG entries (the dense columns) are
// claimed by a whole block instead of one warp.
//
// Permutation. Column c of B holds the entries of column c of A with row i
// renamed pinv[i] (pinv[p[j]] = j), sorted: a warp rank sort in shared memory
// for columns up to PERM_SHORT entries, a bitmap over the n rows with a
// popcount prefix for the listed longer ones.
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int32_t NONE = 0x7f7f7f7f;  // empty atomicMin slot (memset byte 0x7f)
constexpr int PERM_SHORT = 1024;      // longest column of the warp rank sort
constexpr int PERM_WARPS = 8;         // warps per block of the rank sort
constexpr int LONG_THREADS = 512;
constexpr int CLAIM_LONG = 256;       // frontier columns longer than this are claimed by a whole block
constexpr int CLAIM_THREADS = 1024;

// counters in one small device array
enum { C_ROOTS = 0, C_CLAIMED, C_NEXT, C_LONG, C_AUG, C_ERR, C_MOVED, C_N };

__device__ __forceinline__ bool counts(const double* v, int64_t t) { return v[t] != 0.0; }

// column j starts matched to row j when A(j,j) is stored and nonzero
__global__ void k_dm_diag(int32_t n, const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
                          const double* __restrict__ v, int32_t* mcol, int32_t* mrow)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int64_t lo = cp[j], hi = cp[j + 1];  // binary search for row j in the sorted column
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ri[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    const bool d = lo < cp[j + 1] && ri[lo] == j && counts(v, lo);
    mcol[j] = d ? (int32_t)j : -1;
    if (d) mrow[j] = (int32_t)j;
}

// phase start: the unmatched columns become roots
__global__ void k_dm_roots(int32_t n, const int32_t* __restrict__ mcol, int32_t* root, int32_t* rend, int32_t* roots,
                           int32_t* cnt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || mcol[c] >= 0) return;
    root[c] = (int32_t)c;
    rend[c] = NONE;
    roots[atomicAdd(&cnt[C_ROOTS], 1)] = (int32_t)c;
}

// column c claims its unvisited rows t0, t0 + step, ...
__device__ __forceinline__ void claim_rows(int32_t c, int64_t t0, int64_t t1, int step, const int32_t* ri,
                                           const double* v, const int32_t* rlev, int32_t* pred, int32_t* claimed,
                                           int32_t* cnt)
{
    for (int64_t t = t0; t < t1; t += step) {
        const int32_t i = ri[t];
        if (!counts(v, t) || rlev[i] >= 0) continue;
        if (atomicMin(&pred[i], c) == NONE) claimed[atomicAdd(&cnt[C_CLAIMED], 1)] = i;
    }
}

// one warp per frontier column; columns longer than CLAIM_LONG are queued
// for k_dm_claim_long
__global__ void k_dm_claim(const int32_t* __restrict__ front, int32_t nf, const int64_t* __restrict__ cp,
                           const int32_t* __restrict__ ri, const double* __restrict__ v,
                           const int32_t* __restrict__ root, const int32_t* __restrict__ rend,
                           const int32_t* __restrict__ rlev, int32_t* pred, int32_t* claimed, int32_t* longq,
                           int32_t* cnt)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nf) return;
    const int32_t c = front[w];
    if (rend[root[c]] != NONE) return;  // the tree already reached a free row
    const int64_t b = cp[c], e = cp[c + 1];
    if (e - b > CLAIM_LONG) {
        if (lane == 0) longq[atomicAdd(&cnt[C_LONG], 1)] = c;
        return;
    }
    claim_rows(c, b + lane, e, 32, ri, v, rlev, pred, claimed, cnt);
}

// the queued long frontier columns, one block each (count read on the device)
__global__ void __launch_bounds__(CLAIM_THREADS)
k_dm_claim_long(const int32_t* __restrict__ longq, const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
                const double* __restrict__ v, const int32_t* __restrict__ rlev, int32_t* pred, int32_t* claimed,
                int32_t* cnt)
{
    const int32_t nl = cnt[C_LONG];
    for (int32_t q = blockIdx.x; q < nl; q += gridDim.x) {
        const int32_t c = longq[q];
        claim_rows(c, cp[c] + threadIdx.x, cp[c + 1], CLAIM_THREADS, ri, v, rlev, pred, claimed, cnt);
    }
}

// settle the rows claimed at this level (count read on the device)
__global__ void k_dm_settle(const int32_t* __restrict__ claimed, int32_t level, int32_t* rlev,
                            const int32_t* __restrict__ pred, const int32_t* __restrict__ mrow, int32_t* root,
                            int32_t* rend, int32_t* next, int32_t* cnt)
{
    const int32_t ncl = cnt[C_CLAIMED];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncl; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = claimed[t];
        rlev[i] = level;
        const int32_t r = root[pred[i]];
        const int32_t c2 = mrow[i];
        if (c2 < 0) {
            atomicMin(&rend[r], i);          // a free row: an augmenting path for tree r
        } else {
            root[c2] = r;                    // the matched column joins the tree
            next[atomicAdd(&cnt[C_NEXT], 1)] = c2;
        }
    }
}

// one thread per root: flip the path from the tree's free row back to it
__global__ void k_dm_augment(const int32_t* __restrict__ roots, int32_t nroots, const int32_t* __restrict__ rend,
                             const int32_t* __restrict__ pred, int32_t* mcol, int32_t* mrow, int32_t* cnt,
                             int32_t maxlen)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nroots) return;
    const int32_t r = roots[t];
    int32_t i = rend[r];
    if (i == NONE) return;
    for (int32_t step = 0; step < maxlen; ++step) {
        const int32_t c = pred[i];
        const int32_t inext = mcol[c];
        mcol[c] = i;
        mrow[i] = c;
        if (c == r) {
            atomicAdd(&cnt[C_AUG], 1);
            return;
        }
        i = inext;
    }
    atomicExch(&cnt[C_ERR], 1);  // a path longer than the tree's depth: internal error
}

__global__ void k_count_moved(int32_t n, const int32_t* __restrict__ p, int32_t* cnt)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool moved = j < n && p[j] != (int32_t)j;
    const unsigned m = __ballot_sync(SAI_FULL, moved);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&cnt[C_MOVED], __popc(m));
}

// the columns longer than PERM_SHORT, listed for k_perm_long
__global__ void k_long_cols(int32_t n, const int64_t* __restrict__ cp, int32_t* list, int32_t* nlong)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && cp[j + 1] - cp[j] > PERM_SHORT) list[atomicAdd(nlong, 1)] = (int32_t)j;
}

// pinv[p[j]] = j; flags p that is not a permutation of 0..n-1
__global__ void k_perm_inverse(int32_t n, const int32_t* __restrict__ p, int32_t* pinv, int32_t* bad)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int32_t i = p[j];
    if (i < 0 || i >= n || atomicExch(&pinv[i], (int32_t)j) != -1) atomicExch(bad, 1);
}

// columns of at most PERM_SHORT entries: renamed rows ranked in shared memory
__global__ void __launch_bounds__(PERM_WARPS * 32)
k_perm_short(int32_t n, const int64_t* __restrict__ cp, const int32_t* __restrict__ ri, const double* __restrict__ v,
             const int32_t* __restrict__ pinv, int32_t* __restrict__ ro, double* __restrict__ vo)
{
    __shared__ int32_t key[PERM_WARPS][PERM_SHORT];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * PERM_WARPS + wl;
    if (c >= n) return;
    const int64_t b = cp[c];
    const int32_t len = (int32_t)(cp[c + 1] - b);
    if (len > PERM_SHORT) return;
    for (int32_t t = lane; t < len; t += 32) key[wl][t] = pinv[ri[b + t]];
    __syncwarp();
    for (int32_t t = lane; t < len; t += 32) {
        const int32_t k = key[wl][t];
        int32_t rank = 0;
        for (int32_t u = 0; u < len; ++u) rank += key[wl][u] < k;  // keys are distinct
        ro[b + rank] = k;
        vo[b + rank] = v[b + t];
    }
}

// the listed longer columns, one block each: mark the renamed rows in a
// bitmap of n bits, prefix-count the words, rank = bits below the row
__global__ void __launch_bounds__(LONG_THREADS)
k_perm_long(const int32_t* __restrict__ list, int32_t nlong, const int64_t* __restrict__ cp,
            const int32_t* __restrict__ ri, const double* __restrict__ v, const int32_t* __restrict__ pinv,
            int32_t* __restrict__ ro, double* __restrict__ vo, unsigned* scratch, int64_t words)
{
    __shared__ int32_t part[LONG_THREADS];
    unsigned* bits = scratch + (size_t)blockIdx.x * 2 * words;
    int32_t* pre = (int32_t*)(bits + words);
    const int64_t chunk = (words + LONG_THREADS - 1) / LONG_THREADS;
    const int64_t w0 = (int64_t)threadIdx.x * chunk;
    const int64_t w1 = w0 + chunk < words ? w0 + chunk : words;
    for (int32_t q = blockIdx.x; q < nlong; q += gridDim.x) {
        const int32_t c = list[q];
        const int64_t b = cp[c], len = cp[c + 1] - b;
        for (int64_t w = threadIdx.x; w < words; w += LONG_THREADS) bits[w] = 0u;
        __syncthreads();
        for (int64_t t = threadIdx.x; t < len; t += LONG_THREADS) {
            const int32_t k = pinv[ri[b + t]];
            atomicOr(&bits[k >> 5], 1u << (k & 31));
        }
        __syncthreads();
        int32_t sum = 0;
        for (int64_t w = w0; w < w1; ++w) sum += __popc(bits[w]);
        part[threadIdx.x] = sum;
        __syncthreads();
        for (int off = 1; off < LONG_THREADS; off <<= 1) {  // inclusive scan of the chunk sums
            const int32_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        int32_t run = part[threadIdx.x] - sum;
        for (int64_t w = w0; w < w1; ++w) {
            pre[w] = run;
            run += __popc(bits[w]);
        }
        __syncthreads();
        for (int64_t t = threadIdx.x; t < len; t += LONG_THREADS) {
            const int32_t k = pinv[ri[b + t]];
            const int32_t rank = pre[k >> 5] + __popc(bits[k >> 5] & ((1u << (k & 31)) - 1u));
            ro[b + rank] = k;
            vo[b + rank] = v[b + t];
        }
        __syncthreads();
    }
}

__global__ void k_gather_vec(int32_t n, const int32_t* __restrict__ p, const double* __restrict__ x,
                             double* __restrict__ y)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) y[j] = x[p[j]];
}

}  // namespace

sai_status sai_dmperm_run(const sai_csc_view* A, int32_t* p, int32_t* rank_out, int32_t* moved_out, cudaStream_t st)
{
    if (!A || !rank_out || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!p || !A->col_ptr)) ||
        (A->nnz > 0 && (!A->row_idx || !A->val)) || A->n >= NONE)
        return SAI_INVALID_ARG;
    const int32_t n = A->n;
    *rank_out = 0;
    if (moved_out) *moved_out = 0;
    if (n == 0) return SAI_OK;
    SAI_TRY(sai_validate_csc(n, n, A->nnz, A->col_ptr, A->row_idx, st));
    Buf mrow, root, rend, roots, fa, fb, claimed, pred, rlev, longq, cnt;
    const size_t nb = sizeof(int32_t) * (size_t)n;
    SAI_TRY(mrow.alloc(nb, st, true));
    SAI_TRY(root.alloc(nb, st, true));
    SAI_TRY(rend.alloc(nb, st, true));
    SAI_TRY(roots.alloc(nb, st, true));
    SAI_TRY(fa.alloc(nb, st, true));
    SAI_TRY(fb.alloc(nb, st, true));
    SAI_TRY(claimed.alloc(nb, st, true));
    SAI_TRY(pred.alloc(nb, st, true));
    SAI_TRY(rlev.alloc(nb, st, true));
    SAI_TRY(longq.alloc(nb, st, true));
    SAI_TRY(cnt.alloc(sizeof(int32_t) * C_N, st, true));
    int32_t* c = cnt.as<int32_t>();
    const unsigned gn = sai_div_up(n, 256);
    SAI_CUDA(cudaMemsetAsync(mrow.p, 0xff, nb, st));
    k_dm_diag<<<SAI_GRID(gn), 256, 0, st>>>(n, A->col_ptr, A->row_idx, A->val, p, mrow.as<int32_t>());
    SAI_CUDA(cudaGetLastError());
    int32_t h[C_N] = {0};
    int32_t nroots = 0;
    for (int64_t phase = 0; phase <= n; ++phase) {
        SAI_CUDA(cudaMemsetAsync(c, 0, sizeof(int32_t) * C_N, st));
        k_dm_roots<<<SAI_GRID(gn), 256, 0, st>>>(n, p, root.as<int32_t>(), rend.as<int32_t>(), roots.as<int32_t>(), c);
        SAI_CUDA(cudaGetLastError());
        SAI_CUDA(cudaMemcpyAsync(h, c + C_ROOTS, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        nroots = h[C_ROOTS];
        if (nroots == 0) break;
        SAI_CUDA(cudaMemsetAsync(pred.p, 0x7f, nb, st));
        SAI_CUDA(cudaMemsetAsync(rlev.p, 0xff, nb, st));
        const int32_t* cur = roots.as<int32_t>();
        int32_t ncur = nroots;
        int32_t* nxt = fa.as<int32_t>();
        int32_t* spare = fb.as<int32_t>();
        for (int32_t level = 0; ncur > 0 && level <= n; ++level) {
            SAI_CUDA(cudaMemsetAsync(c + C_CLAIMED, 0, sizeof(int32_t) * 3, st));  // claimed, next, long
            k_dm_claim<<<SAI_GRID(sai_div_up((int64_t)ncur * 32, 256)), 256, 0, st>>>(
                cur, ncur, A->col_ptr, A->row_idx, A->val, root.as<int32_t>(), rend.as<int32_t>(),
                rlev.as<int32_t>(), pred.as<int32_t>(), claimed.as<int32_t>(), longq.as<int32_t>(), c);
            k_dm_claim_long<<<SAI_GRID(152), CLAIM_THREADS, 0, st>>>(longq.as<int32_t>(), A->col_ptr, A->row_idx,
                                                                    A->val, rlev.as<int32_t>(), pred.as<int32_t>(),
                                                                    claimed.as<int32_t>(), c);
            k_dm_settle<<<SAI_GRID(152 * 4), 256, 0, st>>>(claimed.as<int32_t>(), level, rlev.as<int32_t>(),
                                                          pred.as<int32_t>(), mrow.as<int32_t>(), root.as<int32_t>(),
                                                          rend.as<int32_t>(), nxt, c);
            SAI_CUDA(cudaGetLastError());
            SAI_CUDA(cudaMemcpyAsync(h + C_NEXT, c + C_NEXT, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            ncur = h[C_NEXT];
            cur = nxt;
            int32_t* t = spare;
            spare = nxt;
            nxt = t;
        }
        k_dm_augment<<<SAI_GRID(sai_div_up(nroots, 256)), 256, 0, st>>>(
            roots.as<int32_t>(), nroots, rend.as<int32_t>(), pred.as<int32_t>(), p, mrow.as<int32_t>(), c, n + 1);
        SAI_CUDA(cudaGetLastError());
        SAI_CUDA(cudaMemcpyAsync(h + C_AUG, c + C_AUG, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        if (h[C_ERR]) return SAI_CUDA_ERROR;
        if (h[C_AUG] == 0) break;  // no augmenting path: the matching is maximum
        nroots -= h[C_AUG];
        if (nroots == 0) break;
    }
    *rank_out = n - nroots;
    if (moved_out) {
        SAI_CUDA(cudaMemsetAsync(c + C_MOVED, 0, sizeof(int32_t), st));
        k_count_moved<<<SAI_GRID(gn), 256, 0, st>>>(n, p, c);
        SAI_CUDA(cudaGetLastError());
        SAI_CUDA(cudaMemcpyAsync(h + C_MOVED, c + C_MOVED, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        *moved_out = h[C_MOVED];
    }
    return SAI_OK;
}

sai_status sai_permute_rows_run(const sai_csc_view* A, const int32_t* p, int64_t* Bcp, int32_t* Bri, double* Bv,
                                cudaStream_t st)
{
    if (!A || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!p || !A->col_ptr || !Bcp)) ||
        (A->nnz > 0 && (!A->row_idx || !A->val || !Bri || !Bv)))
        return SAI_INVALID_ARG;
    const int32_t n = A->n;
    if (n == 0) {
        SAI_CUDA(cudaMemsetAsync(Bcp, 0, sizeof(int64_t), st));
        return SAI_OK;
    }
    SAI_TRY(sai_validate_csc(n, n, A->nnz, A->col_ptr, A->row_idx, st));
    Buf pinv, flags, list;
    SAI_TRY(pinv.alloc(sizeof(int32_t) * (size_t)n, st, true));
    SAI_TRY(flags.alloc(sizeof(int32_t) * 2, st, true));  // [not a permutation, long columns]
    SAI_TRY(list.alloc(sizeof(int32_t) * (size_t)n, st, true));
    SAI_CUDA(cudaMemsetAsync(pinv.p, 0xff, sizeof(int32_t) * (size_t)n, st));
    SAI_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int32_t) * 2, st));
    const unsigned gn = sai_div_up(n, 256);
    int32_t* f = flags.as<int32_t>();
    k_perm_inverse<<<SAI_GRID(gn), 256, 0, st>>>(n, p, pinv.as<int32_t>(), f);
    k_long_cols<<<SAI_GRID(gn), 256, 0, st>>>(n, A->col_ptr, list.as<int32_t>(), f + 1);
    SAI_CUDA(cudaGetLastError());
    int32_t hf[2] = {0, 0};
    SAI_CUDA(cudaMemcpyAsync(hf, f, sizeof(hf), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    if (hf[0]) return SAI_INVALID_ARG;
    const int32_t nlong = hf[1];
    SAI_CUDA(cudaMemcpyAsync(Bcp, A->col_ptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, st));
    k_perm_short<<<SAI_GRID(sai_div_up(n, PERM_WARPS)), PERM_WARPS * 32, 0, st>>>(n, A->col_ptr, A->row_idx, A->val,
                                                                                  pinv.as<int32_t>(), Bri, Bv);
    SAI_CUDA(cudaGetLastError());
    if (nlong > 0) {
        const int64_t words = ((int64_t)n + 31) / 32;
        const size_t per_block = sizeof(unsigned) * 2 * (size_t)words;
        size_t blocks = ((size_t)256 << 20) / per_block;
        if (blocks > 152) blocks = 152;
        if (blocks > (size_t)nlong) blocks = (size_t)nlong;
        if (blocks < 1) blocks = 1;
        Buf scratch;
        SAI_TRY(scratch.alloc(per_block * blocks, st, true));
        k_perm_long<<<SAI_GRID(blocks), LONG_THREADS, 0, st>>>(list.as<int32_t>(), nlong, A->col_ptr, A->row_idx,
                                                               A->val, pinv.as<int32_t>(), Bri, Bv,
                                                               scratch.as<unsigned>(), words);
        SAI_CUDA(cudaGetLastError());
    }
    return SAI_OK;
}

sai_status sai_gather_vec(int32_t n, const int32_t* p, const double* x, double* y, cudaStream_t st)
{
    if (n <= 0) return SAI_OK;
    k_gather_vec<<<SAI_GRID(sai_div_up(n, 256)), 256, 0, st>>>(n, p, x, y);
    SAI_CUDA(cudaGetLastError());
    return SAI_OK;
}
