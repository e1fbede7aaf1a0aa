// split.cu -- dense-column detection and sparsification (section 4 of the
// paper; eq. (split) A = A~ + U V^T).
//
// Kernels:
//   k_flag_dense    nnz(a_j) = col_ptr[j+1]-col_ptr[j] > tau      (one thread / column)
//   k_compact_J     J = ascending list of flagged columns           (scan + scatter)
//   k_window        for each irregular column: the kept entries are a contiguous
//                   window of its sorted rows around the diagonal (diagonal plus the
//                   p_keep-1 nearest, ties to the smaller row)      (one thread / column)
//   k_keep_largest  the other rule of section 4: the diagonal and the p_keep-1
//                   entries of largest magnitude (ties to the smaller row) of each
//                   irregular column, as per-entry keep flags      (one block / column)
//   k_copy_split    copies A into A~ (window only for irregular columns) and U
//                   (the rest)                                      (one warp / column)
//   k_colstats      ||a~_j||^2 and sum_i |a~_ij| per column, max -> ||A~||_1
#include "internal.h"

__global__ void k_flag_dense(int32_t n, const int64_t* cp, double tau, int ge, int32_t* flag)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double c = (double)(cp[j + 1] - cp[j]);
    flag[j] = ge ? (c >= tau) : (c > tau);
}

__global__ void k_compact_J(int32_t n, const int32_t* flag, const int64_t* pos, int32_t* J)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (flag[j]) J[pos[j]] = (int32_t)j;
}

// Two-pointer walk outwards from the diagonal: the kept set of an irregular
// column is [w0, w1) in its sorted entry range.
__global__ void k_window(int32_t s, const int32_t* J, const int64_t* cp, const int32_t* ri, int32_t p_keep,
                         int64_t* w0, int64_t* w1, int64_t* nkeep)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s) return;
    int32_t j = J[t];
    int64_t b = cp[j], e = cp[j + 1];
    int64_t lo = b, hi = e;  // binary search: first row >= j
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ri[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    int64_t mid = lo;
    int64_t left = mid - 1, right = mid;  // next candidates on each side
    int32_t kept = 0;
    int64_t a0 = mid, a1 = mid;           // window [a0, a1)
    if (mid < e && ri[mid] == j) {
        kept = 1;
        right = mid + 1;
        a1 = mid + 1;
    }
    while (kept < p_keep && (left >= b || right < e)) {
        bool take_left;
        if (left < b) take_left = false;
        else if (right >= e) take_left = true;
        else take_left = ((int64_t)j - ri[left]) <= ((int64_t)ri[right] - j);
        if (take_left) {
            a0 = left;
            --left;
        } else {
            a1 = right + 1;
            ++right;
        }
        ++kept;
    }
    w0[t] = a0;
    w1[t] = a1;
    nkeep[t] = a1 - a0;
}

// sum of an int over the block (blockDim.x = 256), the result in every thread
__device__ __forceinline__ long long block_sum_ll(long long x, long long* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(SAI_FULL, x, o);
    if (lane == 0) red[wid] = x;
    __syncthreads();
    long long t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ unsigned long long mag_key(double v)
{
    return (unsigned long long)__double_as_longlong(fabs(v));  // orders like |v|
}

// Keep flags of the second rule of section 4, one block (256 threads) per
// irregular column: K = p_keep-1 off-diagonal entries with the diagonal, or
// K = p_keep without one. The K-th largest key T is found bit by bit from
// the top (the largest T with #{key >= T} >= K); entries above T are kept,
// and entries equal to T in row order until K are kept.
__global__ void __launch_bounds__(256) k_keep_largest(int32_t s, const int32_t* J, const int64_t* cp,
                                                      const int32_t* ri, const double* v, int32_t p_keep,
                                                      uint8_t* keep, int64_t* nkeep)
{
    __shared__ long long red[8];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int32_t t = blockIdx.x; t < s; t += gridDim.x) {
        const int32_t j = J[t];
        const int64_t b = cp[j], e = cp[j + 1];
        long long dq = -1;
        for (int64_t q = b + tid; q < e; q += 256)
            if (ri[q] == j) dq = q;
        // the diagonal's position (rows are distinct: at most one thread finds it)
        const long long dsum = block_sum_ll(dq + 1, red) - 1;
        const int hasd = dsum >= 0;
        const long long K = hasd ? p_keep - 1 : p_keep;
        const long long off = (e - b) - hasd;
        if (off <= K || K <= 0) {
            for (int64_t q = b + tid; q < e; q += 256) keep[q] = (off <= K) || q == dsum;
            if (tid == 0) nkeep[t] = off <= K ? e - b : hasd;
            __syncthreads();
            continue;
        }
        unsigned long long T = 0;
        for (int bit = 63; bit >= 0; --bit) {
            const unsigned long long cand = T | (1ull << bit);
            long long c = 0;
            for (int64_t q = b + tid; q < e; q += 256) c += (q != dsum && mag_key(v[q]) >= cand);
            if (block_sum_ll(c, red) >= K) T = cand;
        }
        long long cg = 0;
        for (int64_t q = b + tid; q < e; q += 256) cg += (q != dsum && mag_key(v[q]) > T);
        const long long need = K - block_sum_ll(cg, red);  // >= 1 ties at T to keep
        long long carry = 0;
        for (int64_t base = b; base < e; base += 256) {
            const int64_t q = base + tid;
            const bool valid = q < e;
            const unsigned long long kq = valid ? mag_key(v[q]) : 0ull;
            const int tie = valid && q != dsum && kq == T;
            int w = tie;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(SAI_FULL, w, o);
                if (lane >= o) w += y;
            }
            if (lane == 31) red[wid] = w;
            __syncthreads();
            long long before = 0, tot = 0;
            for (int u = 0; u < 8; ++u) {
                if (u < wid) before += red[u];
                tot += red[u];
            }
            const long long rank = carry + before + w - tie;
            if (valid) keep[q] = q == dsum || (q != dsum && kq > T) || (tie && rank < need);
            carry += tot;
            __syncthreads();
        }
        if (tid == 0) nkeep[t] = K + hasd;
        __syncthreads();
    }
}

__global__ void k_count_split(int32_t n, const int64_t* cp, const int32_t* flag, const int64_t* pos,
                              const int64_t* nkeep, int64_t* cnt_At, int64_t* cnt_U)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int64_t c = cp[j + 1] - cp[j];
    if (flag[j]) {
        int64_t t = pos[j];
        int64_t kept = nkeep[t];
        cnt_At[j] = kept;
        cnt_U[t] = c - kept;
    } else {
        cnt_At[j] = c;
    }
}

__global__ void k_copy_split(int32_t n, const int64_t* cp, const int32_t* ri, const double* v,
                             const int32_t* flag, const int64_t* pos, const int64_t* w0, const int64_t* w1,
                             const uint8_t* kf, const int64_t* At_cp, int32_t* At_ri, double* At_v,
                             const int64_t* U_cp, int32_t* U_ri, double* U_v)
{
    int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (j >= n) return;
    int64_t b = cp[j], e = cp[j + 1];
    int64_t oa = At_cp[j];
    if (!flag[j]) {
        for (int64_t q = b + lane; q < e; q += 32) {
            At_ri[oa + (q - b)] = ri[q];
            At_v[oa + (q - b)] = v[q];
        }
        return;
    }
    int64_t t = pos[j];
    if (kf) {  // per-entry keep flags: kept and dropped entries each in row order
        int64_t ka = 0, ku = 0;
        const int64_t ou = U_cp[t];
        const unsigned lt = (1u << lane) - 1u;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t q = base + lane;
            const bool valid = q < e;
            const bool k = valid && kf[q];
            const unsigned mk = __ballot_sync(SAI_FULL, k), md = __ballot_sync(SAI_FULL, valid && !k);
            if (k) {
                At_ri[oa + ka + __popc(mk & lt)] = ri[q];
                At_v[oa + ka + __popc(mk & lt)] = v[q];
            } else if (valid) {
                U_ri[ou + ku + __popc(md & lt)] = ri[q];
                U_v[ou + ku + __popc(md & lt)] = v[q];
            }
            ka += __popc(mk);
            ku += __popc(md);
        }
        return;
    }
    // an irregular column can hold thousands of entries: eight in flight per lane
    int64_t a0 = w0[t], a1 = w1[t];
    int64_t ou = U_cp[t];
    for (int64_t q0 = b + lane; q0 < e; q0 += 32 * 8) {
        int32_t r[8];
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t q = q0 + 32 * u;
            r[u] = q < e ? ri[q] : 0;
            x[u] = q < e ? v[q] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t q = q0 + 32 * u;
            if (q >= e) continue;
            if (q >= a0 && q < a1) {
                At_ri[oa + (q - a0)] = r[u];
                At_v[oa + (q - a0)] = x[u];
            } else {
                int64_t d = q < a0 ? (q - b) : (q - b) - (a1 - a0);
                U_ri[ou + d] = r[u];
                U_v[ou + d] = x[u];
            }
        }
    }
}

__global__ void k_colstats(int32_t n, const int64_t* cp, const double* v, double* colnorm2,
                           unsigned long long* norm1_bits)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s1 = 0.0;
    if (j < n) {
        double s2 = 0.0;
        for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
            s2 += v[q] * v[q];
            s1 += fabs(v[q]);
        }
        colnorm2[j] = s2;
    }
    // non-negative doubles order like their bit patterns: the warp's largest, then one atomic
    unsigned long long m = (unsigned long long)__double_as_longlong(s1);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(SAI_FULL, m, o);
        m = w > m ? w : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(norm1_bits, m);
}

sai_status sai_split_build(const sai_csc_view* A, const sai_split_params* prm, cudaStream_t st, bool async,
                           sai_split_s* h)
{
    if (!A || !prm || !h || A->n < 0 || A->nnz < 0 || (prm->keep_rule != 0 && prm->keep_rule != 1))
        return SAI_INVALID_ARG;
    if (A->n > 0 && (!A->col_ptr || (A->nnz > 0 && (!A->row_idx || !A->val)))) return SAI_INVALID_ARG;
    const int32_t n = A->n;
    const int64_t nnz = A->nnz;
    SAI_TRY(sai_validate_csc(n, n, nnz, A->col_ptr, A->row_idx, st));
    cudaEvent_t e0, e1;
    SAI_CUDA(cudaEventCreate(&e0));
    SAI_CUDA(cudaEventCreate(&e1));
    SAI_CUDA(cudaEventRecord(e0, st));

    h->n = n;
    h->p = n > 0 ? (int32_t)(nnz / n) : 0;
    h->tau = prm->abs_tau >= 0.0 ? prm->abs_tau : prm->thresh_mult * (double)h->p;
    h->p_keep = prm->p_keep > 0 ? prm->p_keep : (h->p > 0 ? h->p : 1);
    const unsigned gb = sai_div_up(n > 0 ? n : 1, 256);

    Buf flag, pos;
    SAI_TRY(flag.alloc(sizeof(int32_t) * (size_t)(n + 1), st, true));
    SAI_TRY(pos.alloc(sizeof(int64_t) * (size_t)(n + 1), st, true));
    if (n > 0) k_flag_dense<<<SAI_GRID(gb), 256, 0, st>>>(n, A->col_ptr, h->tau, prm->ge, flag.as<int32_t>());
    SAI_TRY(sai_scan_counts_i32(flag.as<int32_t>(), pos.as<int64_t>(), n, st));
    int64_t s64 = 0;
    SAI_CUDA(cudaMemcpyAsync(&s64, pos.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    h->s = (int32_t)s64;
    const int32_t s = h->s;

    SAI_TRY(h->J.alloc(sizeof(int32_t) * (size_t)(s > 0 ? s : 1), st, async));
    if (n > 0) k_compact_J<<<SAI_GRID(gb), 256, 0, st>>>(n, flag.as<int32_t>(), pos.as<int64_t>(), h->J.as<int32_t>());
    Buf w0, w1, nkeep, kflag, cntA, cntU;
    SAI_TRY(w0.alloc(sizeof(int64_t) * (size_t)(s + 1), st, true));
    SAI_TRY(w1.alloc(sizeof(int64_t) * (size_t)(s + 1), st, true));
    SAI_TRY(nkeep.alloc(sizeof(int64_t) * (size_t)(s + 1), st, true));
    SAI_TRY(cntA.alloc(sizeof(int64_t) * (size_t)(n + 1), st, true));
    SAI_TRY(cntU.alloc(sizeof(int64_t) * (size_t)(s + 1), st, true));
    const bool largest = prm->keep_rule == 1;
    if (largest) SAI_TRY(kflag.alloc((size_t)(nnz > 0 ? nnz : 1), st, true));
    if (s > 0 && !largest)
        k_window<<<SAI_GRID(sai_div_up(s, 128)), 128, 0, st>>>(s, h->J.as<int32_t>(), A->col_ptr, A->row_idx, h->p_keep,
                                                     w0.as<int64_t>(), w1.as<int64_t>(), nkeep.as<int64_t>());
    if (s > 0 && largest) {
        int dev = 0, sms = 0;
        SAI_CUDA(cudaGetDevice(&dev));
        SAI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const unsigned g = (unsigned)(s < sms * 8 ? s : sms * 8);
        k_keep_largest<<<SAI_GRID(g), 256, 0, st>>>(s, h->J.as<int32_t>(), A->col_ptr, A->row_idx, A->val, h->p_keep,
                                                   kflag.as<uint8_t>(), nkeep.as<int64_t>());
    }
    if (n > 0)
        k_count_split<<<SAI_GRID(gb), 256, 0, st>>>(n, A->col_ptr, flag.as<int32_t>(), pos.as<int64_t>(),
                                          nkeep.as<int64_t>(), cntA.as<int64_t>(), cntU.as<int64_t>());
    SAI_TRY(h->At_cp.alloc(sizeof(int64_t) * (size_t)(n + 1), st, async));
    SAI_TRY(h->U_cp.alloc(sizeof(int64_t) * (size_t)(s + 1), st, async));
    SAI_TRY(sai_scan_counts_i64(cntA.as<int64_t>(), h->At_cp.as<int64_t>(), n, st));
    SAI_TRY(sai_scan_counts_i64(cntU.as<int64_t>(), h->U_cp.as<int64_t>(), s, st));
    int64_t tot[2] = {0, 0};
    SAI_CUDA(cudaMemcpyAsync(&tot[0], h->At_cp.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaMemcpyAsync(&tot[1], h->U_cp.as<int64_t>() + s, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    h->nnz_At = tot[0];
    h->nnz_U = tot[1];
    SAI_TRY(h->At_ri.alloc(sizeof(int32_t) * (size_t)(h->nnz_At > 0 ? h->nnz_At : 1), st, async));
    SAI_TRY(h->At_v.alloc(sizeof(double) * (size_t)(h->nnz_At > 0 ? h->nnz_At : 1), st, async));
    SAI_TRY(h->U_ri.alloc(sizeof(int32_t) * (size_t)(h->nnz_U > 0 ? h->nnz_U : 1), st, async));
    SAI_TRY(h->U_v.alloc(sizeof(double) * (size_t)(h->nnz_U > 0 ? h->nnz_U : 1), st, async));
    if (n > 0)
        k_copy_split<<<SAI_GRID(sai_div_up((int64_t)n * 32, 256)), 256, 0, st>>>(
            n, A->col_ptr, A->row_idx, A->val, flag.as<int32_t>(), pos.as<int64_t>(), w0.as<int64_t>(),
            w1.as<int64_t>(), largest ? kflag.as<uint8_t>() : nullptr, h->At_cp.as<int64_t>(), h->At_ri.as<int32_t>(),
            h->At_v.as<double>(),
            h->U_cp.as<int64_t>(), h->U_ri.as<int32_t>(), h->U_v.as<double>());
    SAI_CUDA(cudaGetLastError());
    SAI_TRY(sai_csc_to_csr(n, n, h->nnz_At, h->At_cp.as<int64_t>(), h->At_ri.as<int32_t>(), h->At_v.as<double>(),
                           h->Atr_rp, h->Atr_ci, h->Atr_v, st, async));
    SAI_TRY(h->colnorm2.alloc(sizeof(double) * (size_t)(n > 0 ? n : 1), st, async));
    Buf n1;
    SAI_TRY(n1.alloc(sizeof(unsigned long long), st, true));
    SAI_CUDA(cudaMemsetAsync(n1.p, 0, sizeof(unsigned long long), st));
    if (n > 0)
        k_colstats<<<SAI_GRID(gb), 256, 0, st>>>(n, h->At_cp.as<int64_t>(), h->At_v.as<double>(), h->colnorm2.as<double>(),
                                       n1.as<unsigned long long>());
    SAI_CUDA(cudaGetLastError());
    SAI_CUDA(cudaMemcpyAsync(&h->norm1, n1.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaEventRecord(e1, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    SAI_CUDA(cudaEventElapsedTime(&h->ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SAI_OK;
}
