// common.cuh -- helpers shared by the saismw CUDA sources (sm_103a only).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "saismw.h"

#define SAI_WARP 32
#define SAI_FULL 0xffffffffu

// Propagate a CUDA error as SAI_CUDA_ERROR (or SAI_OOM) from host code.
#define SAI_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) {                                         \
            sai_internal_note_cuda_error(e_, #call, __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? SAI_OOM : SAI_CUDA_ERROR; \
        }                                                                \
    } while (0)

#define SAI_TRY(expr)                        \
    do {                                     \
        sai_status s_ = (expr);              \
        if (s_ != SAI_OK) return s_;         \
    } while (0)

void sai_internal_note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

static inline unsigned sai_div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------- warp tools
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SAI_FULL, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SAI_FULL, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(SAI_FULL, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Stream-ordered device buffer owned by host code (RAII, frees on the stream).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    sai_status alloc(size_t nbytes, cudaStream_t s)
    {
        release();
        st = s;
        bytes = nbytes;
        if (nbytes == 0) return SAI_OK;
        cudaError_t e = cudaMallocAsync(&p, nbytes, s);
        if (e != cudaSuccess) {
            p = nullptr;
            sai_internal_note_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
            return e == cudaErrorMemoryAllocation ? SAI_OOM : SAI_CUDA_ERROR;
        }
        return SAI_OK;
    }
    void release()
    {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};
