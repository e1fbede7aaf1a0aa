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

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SAI_FULL, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ T warp_sum_t(T v)
{
    return warp_sum(v);
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

// ---------------------------------------------------------------- accounting
// Every kernel launch of the library passes its grid size through SAI_GRID,
// which counts the launch (the expression is only evaluated when the launch
// statement runs).
unsigned sai_count_grid(unsigned g);
#define SAI_GRID(g) sai_count_grid((unsigned)(g))
// Adjusts the count for launches replayed from a CUDA graph (counted at
// replay) or captured into one (not run at capture).
void sai_count_grid_add(long long d);

// Profiled launch sites: CUDA events around each launch (only while a
// profile is open) plus algorithmic bytes / flops accumulated on the device.
enum {
    PROF_SAI_BUILD = 0,  // k_sai, all tiers
    PROF_SPMM = 1,       // SpMM of the Krylov inner iterations
    PROF_GM_DOTS = 2,    // GMRES projections V^T w
    PROF_GM_UPDATE = 3,  // GMRES updates w -= V h
    PROF_BICG_VEC = 4,   // BiCGStab vector updates and inner products
    PROF_SPMM32 = 5,     // FP32 SpMV of the refined GMRES inner solves
    PROF_GM_DOTS32 = 6,  // FP32 projections
    PROF_GM_UPDATE32 = 7,// FP32 updates
    PROF_GM_STEP = 8,    // GMRES step control (reductions, Givens, coefficients)
    PROF_NSITES = 9
};
struct ProfScope {
    int site;
    cudaStream_t st;
    long long idx = -1;  // index of the first event of the pair in the pool
    bool all = false;    // one of the site's first launches, all of which are timed
    ProfScope(int site_, cudaStream_t st_);
    ~ProfScope();
};
bool sai_prof_on();
