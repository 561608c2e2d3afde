// Device primitives used by the graph build: exclusive scan and a stable
// LSD radix sort of 64-bit keys.  Written for this library; no external
// template library is used.
#pragma once
#include "common.cuh"

namespace prims {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Stream-ordered temporary allocation (freed by the caller with tfree).
template <typename T>
inline cudaError_t talloc(T** p, int64_t count, cudaStream_t s) {
    return cudaMallocAsync((void**)p, sizeof(T) * (size_t)(count > 0 ? count : 1), s);
}
inline void tfree(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// Block-wide exclusive scan of one value per thread; returns the block total
// in *total (shared).  blockDim.x must be SCAN_THREADS.
template <typename T>
__device__ T block_exclusive_scan(T v, T* smem_warp, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (SCAN_THREADS / 32) ? smem_warp[lane] : T(0);
        T wx = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(FULL_MASK, wx, o);
            if (lane >= o) wx += y;
        }
        if (lane < (SCAN_THREADS / 32)) smem_warp[lane] = wx - w;
        if (lane == (SCAN_THREADS / 32) - 1) *total = wx;
    }
    __syncthreads();
    return x - v + smem_warp[warp];
}

template <typename T, typename Load>
__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(Load load, int64_t n, T* block_sums) {
    __shared__ T warp_s[SCAN_THREADS / 32];
    __shared__ T total;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++)
        if (base + i < n) s += load(base + i);
    block_exclusive_scan<T>(s, warp_s, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

template <typename T, typename Load>
__global__ void __launch_bounds__(SCAN_THREADS)
    scan_down_kernel(Load load, int64_t n, const T* block_offsets, T* out, T* grand_total) {
    __shared__ T warp_s[SCAN_THREADS / 32];
    __shared__ T total;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        v[i] = (base + i < n) ? load(base + i) : T(0);
        s += v[i];
    }
    T ex = block_exclusive_scan<T>(s, warp_s, &total);
    T run = ex + (block_offsets ? block_offsets[blockIdx.x] : T(0));
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (grand_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) *grand_total = run;
}

template <typename T>
struct LoadArray {
    const T* p;
    __device__ T operator()(int64_t i) const { return p[i]; }
};

// out[i] = sum_{j<i} load(j) for i in [0, n); *d_total (device, may be
// NULL) = sum of all.  out may alias the loaded array only when load reads
// nothing but index i.
template <typename T, typename Load>
cudaError_t exclusive_scan(Load load, int64_t n, T* out, T* d_total, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(T), s);
        return cudaSuccess;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        scan_down_kernel<T, Load><<<1, SCAN_THREADS, 0, s>>>(load, n, (const T*)nullptr, out, d_total);
        return cudaGetLastError();
    }
    T* sums = nullptr;
    cudaError_t e = talloc(&sums, nb, s);
    if (e != cudaSuccess) return e;
    scan_reduce_kernel<T, Load><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(load, n, sums);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = exclusive_scan<T>(LoadArray<T>{sums}, nb, sums, (T*)nullptr, s);
    if (e == cudaSuccess) {
        scan_down_kernel<T, Load><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(load, n, sums, out, d_total);
        e = cudaGetLastError();
    }
    tfree(sums, s);
    return e;
}

// ------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                      // 32-key rounds per warp
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;    // keys per block
constexpr int RS_RADIX = 256;

static __global__ void __launch_bounds__(RS_THREADS)
    rs_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[RS_RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t k = base + i;
        if (k < n) atomicAdd(&h[(keys[k] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w of a block owns keys [w*512, (w+1)*512) of the tile
// and walks them 32 at a time in order; equal digits inside a round are
// ranked by lane (match.any), and earlier rounds / warps / blocks come first.
static __global__ void __launch_bounds__(RS_THREADS)
    rs_scatter_kernel(const uint64_t* __restrict__ keys, uint64_t* __restrict__ out, int64_t n, int shift,
                      const uint32_t* __restrict__ offsets) {
    __shared__ uint32_t cnt[RS_WARPS][RS_RADIX];
    __shared__ uint32_t goff[RS_RADIX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_THREADS) (&cnt[0][0])[i] = 0;
    goff[threadIdx.x] = offsets[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (RS_ROUNDS * 32);
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t k = wbase + r * 32 + lane;
        if (k < n) atomicAdd(&cnt[warp][(keys[k] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    {   // per digit: exclusive prefix over warps, in warp order
        uint32_t run = 0;
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = cnt[w][threadIdx.x];
            cnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t k = wbase + r * 32 + lane;
        bool valid = k < n;
        unsigned active = __ballot_sync(FULL_MASK, valid);
        if (!active) break;
        if (valid) {
            uint64_t key = keys[k];
            unsigned d = (unsigned)(key >> shift) & 0xffu;
            unsigned peers = __match_any_sync(active, d);
            unsigned rank = __popc(peers & lanemask_lt());
            uint32_t pos = goff[d] + cnt[warp][d] + rank;
            out[pos] = key;
            __syncwarp(active);
            if (rank == 0) cnt[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
}

// Sorts n keys by bits [0, bits) ascending, stable.  Ping-pongs between
// keys and tmp; *result receives whichever holds the sorted keys.
inline cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int bits, uint64_t** result,
                                  cudaStream_t s) {
    *result = keys;
    if (n <= 1 || bits <= 0) return cudaSuccess;
    int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    uint32_t* hist = nullptr;
    cudaError_t e = talloc(&hist, nb * RS_RADIX, s);
    if (e != cudaSuccess) return e;
    uint64_t *a = keys, *b = tmp;
    for (int shift = 0; shift < bits && e == cudaSuccess; shift += 8) {
        rs_hist_kernel<<<(unsigned)nb, RS_THREADS, 0, s>>>(a, n, shift, hist);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        e = exclusive_scan<uint32_t>(LoadArray<uint32_t>{hist}, nb * RS_RADIX, hist, (uint32_t*)nullptr, s);
        if (e != cudaSuccess) break;
        rs_scatter_kernel<<<(unsigned)nb, RS_THREADS, 0, s>>>(a, b, n, shift, hist);
        e = cudaGetLastError();
        uint64_t* t = a;
        a = b;
        b = t;
    }
    tfree(hist, s);
    *result = a;
    return e;
}

}  // namespace prims
