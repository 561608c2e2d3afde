// Shared device helpers for the truss decomposition library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/truss.h"

#define TRUSS_WARP 32
#define FULL_MASK 0xffffffffu

// Return a TRUSS_ECUDA status from a host function when a CUDA call fails,
// remembering the CUDA error for truss_strerror / truss_last_cuda_error.
void truss_note_cuda_error(cudaError_t e);
// Process-wide count of kernels this library has launched (stats only).
void truss_note_launch(int k = 1);
long long truss_launch_count();
#define CU(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            truss_note_cuda_error(e_);             \
            return e_ == cudaErrorMemoryAllocation \
                       ? TRUSS_ENOMEM              \
                       : TRUSS_ECUDA;              \
        }                                          \
    } while (0)
#define TRY(call)                 \
    do {                          \
        int s_ = (call);          \
        if (s_ != TRUSS_OK) return s_; \
    } while (0)

static inline int grid_for(int64_t work, int block, int64_t cap = 152 * 32) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_gpu_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Warp-aggregated append: every lane with `pred` gets a distinct slot of
// `out`, using one atomic per warp on `*count`.  All 32 lanes must call.
__device__ __forceinline__ void warp_append(bool pred, int32_t value, int32_t* out, int* count) {
    unsigned b = __ballot_sync(FULL_MASK, pred);
    if (b == 0) return;
    int leader = __ffs(b) - 1;
    int base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(count, __popc(b));
    base = __shfl_sync(FULL_MASK, base, leader);
    if (pred) out[base + __popc(b & lanemask_lt())] = value;
}

// Same, for a subset of active lanes given by `active` (all of them call).
__device__ __forceinline__ void warp_append_mask(unsigned active, bool pred, int32_t value, int32_t* out,
                                                 int* count) {
    unsigned b = __ballot_sync(active, pred);
    if (b == 0) return;
    int leader = __ffs(b) - 1;
    int base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(count, __popc(b));
    base = __shfl_sync(active, base, leader);
    if (pred) out[base + __popc(b & lanemask_lt())] = value;
}

// First index i in [lo, hi) with a[i] >= key (a ascending); hi if none.
template <typename Off>
__device__ __forceinline__ Off lower_bound_dev(const int32_t* __restrict__ a, Off lo, Off hi, int32_t key) {
    while (lo < hi) {
        Off mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Index of key in a[lo, hi) (ascending), or -1.
template <typename Off>
__device__ __forceinline__ Off find_dev(const int32_t* __restrict__ a, Off lo, Off hi, int32_t key) {
    Off p = lower_bound_dev<Off>(a, lo, hi, key);
    return (p < hi && __ldg(a + p) == key) ? p : (Off)-1;
}
