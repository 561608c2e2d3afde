// truss_support_noalloc: per-edge triangle support for a CSR the caller
// already holds on the device, with no device memory allocated by the call.
//
// Who needs this: code that must not call cudaMalloc / cudaFree -- for
// instance a process whose framework allocator owns every byte of device
// memory, a latency-critical loop with a fixed memory budget, or code that
// runs where an allocation could block on the device.  Every other entry
// point of this library allocates its workspace on first use.
//
// The only scratch it needs (the first-upper-slot index Eo of every row and
// one error word) lives in a file-scope __device__ array of fixed size,
// which every GPU that loads the library keeps until the process exits.
// Host code may not use the array's name as a device address, so the first
// call on each device looks the address up once with cudaGetSymbolAddress
// (with that device current) and caches it.
#include <mutex>

#include "common.cuh"

static __device__ __align__(256) int32_t g_noalloc_scratch[TRUSS_NOALLOC_MAX_VERTICES + 64];

namespace {

constexpr int NA_WARPS = 8;
constexpr int NA_CAP = 256;  // N+(u) staged in shared memory up to this length
constexpr int64_t NA_ERR = TRUSS_NOALLOC_MAX_VERTICES;  // error word index

// Checks the caller's row offsets before anything reads the other arrays
// through them: rowptr[0] = 0, rowptr[n] = 2m and no row ends before it
// starts, so every slot read later lies in [0, 2m).  Reads rowptr[0..n]
// only; a violation sets *err.
__global__ void k_na_check_rows(const int32_t* __restrict__ rowptr, int32_t n, int64_t m, int32_t* err) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = rowptr[u], b = rowptr[u + 1];
        bool bad = b < a;
        if (u == 0) bad |= a != 0;
        if (u == n - 1) bad |= (int64_t)b != 2 * m;
        if (bad) atomicExch(err, 1);
    }
}

__global__ void k_na_zero(int32_t* __restrict__ S, int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        S[i] = 0;
}

// Eo[u]: first slot of row u whose neighbour exceeds u
__global__ void k_na_eo(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                        int32_t* __restrict__ eo) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        eo[u] = lower_bound_dev<int32_t>(col, rowptr[u], rowptr[u + 1], (int32_t)u + 1);
}

__device__ __forceinline__ void na_add(int32_t* S, int64_t m, int32_t e, int v, int32_t* err) {
    if (e >= 0 && e < m)
        atomicAdd(S + e, v);
    else
        atomicExch(err, 1);
}

// Warp per vertex u: every triangle u < v < w is found once, at its lowest
// vertex, as w in N+(u) ∩ N+(v) (the oriented form of Algorithm 3).  Rows
// with d+(u) <= NA_CAP are staged in shared memory with one counter per
// entry; longer rows are probed in global memory.
__global__ void __launch_bounds__(NA_WARPS * 32)
    k_na_support(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ eo, const int32_t* __restrict__ col,
                 const int32_t* __restrict__ eid, int32_t n, int64_t m, int32_t* __restrict__ S, int32_t* err) {
    __shared__ int sK[NA_WARPS][NA_CAP];
    __shared__ int sC[NA_WARPS][NA_CAP];
    __shared__ int sP[NA_WARPS][NA_CAP + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *K = sK[warp], *C = sC[warp], *P = sP[warp];
    const int64_t nwarps = (int64_t)gridDim.x * NA_WARPS;
    for (int64_t u = blockIdx.x * (int64_t)NA_WARPS + warp; u < n; u += nwarps) {
        const int32_t up0 = eo[u], up1 = rowptr[u + 1];
        const int d = up1 - up0;
        if (d < 2) continue;
        if (d <= NA_CAP) {
            int carry = 0;
            for (int b = 0; b < d; b += 32) {
                const int p = b + lane;
                int dv = 0;
                if (p < d) {
                    const int v = col[up0 + p];
                    K[p] = v;
                    C[p] = 0;
                    if (v > u && v < n)
                        dv = rowptr[v + 1] - eo[v];
                    else
                        atomicExch(err, 1);
                }
                int x = dv;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(FULL_MASK, x, o);
                    if (lane >= o) x += y;
                }
                if (p < d) P[p] = carry + x - dv;
                carry += __shfl_sync(FULL_MASK, x, 31);
            }
            if (lane == 0) P[d] = carry;
            __syncwarp();
            for (int idx = lane; idx < carry; idx += 32) {
                int lo = 0, hi = d - 1;  // segment of idx: largest p with P[p] <= idx
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (P[mid] <= idx) lo = mid; else hi = mid - 1;
                }
                const int p = lo;
                const int32_t q = eo[K[p]] + (idx - P[p]);
                const int w = col[q];
                int a = p + 1, z = d;
                while (a < z) {
                    const int mid = (a + z) >> 1;
                    if (K[mid] < w) a = mid + 1; else z = mid;
                }
                if (a < d && K[a] == w) {
                    atomicAdd(&C[a], 1);
                    atomicAdd(&C[p], 1);
                    na_add(S, m, eid[q], 1, err);
                }
            }
            __syncwarp();
            for (int p = lane; p < d; p += 32)
                if (C[p]) na_add(S, m, eid[up0 + p], C[p], err);
            __syncwarp();
        } else {
            for (int32_t pv = up0; pv < up1; pv++) {
                const int v = col[pv];
                if (v <= u || v >= n) {
                    if (lane == 0) atomicExch(err, 1);
                    continue;
                }
                int cuv = 0;
                for (int32_t q = eo[v] + lane; q < rowptr[v + 1]; q += 32) {
                    const int32_t r = find_dev<int32_t>(col, pv + 1, up1, col[q]);
                    if (r >= 0) {
                        cuv++;
                        na_add(S, m, eid[r], 1, err);
                        na_add(S, m, eid[q], 1, err);
                    }
                }
                cuv = warp_sum(cuv);
                if (lane == 0 && cuv) na_add(S, m, eid[pv], cuv, err);
            }
        }
    }
}

std::mutex g_scratch_mu;
int32_t* g_scratch_ptr[64] = {};

// Device address of the scratch array on the current device (looked up
// once per device, then cached).
int scratch_address(int32_t** out) {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return TRUSS_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        CU(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = static_cast<int32_t*>(p);
    }
    *out = g_scratch_ptr[dev];
    return TRUSS_OK;
}

}  // namespace

extern "C" int truss_support_noalloc(const int32_t* d_rowptr, const int32_t* d_col, const int32_t* d_eid, int32_t n,
                                     int64_t m, int32_t* d_support, void* stream) {
    if (n < 0 || m < 0 || (n > 0 && !d_rowptr) || (m > 0 && (!d_col || !d_eid || !d_support))) return TRUSS_EINVAL;
    if (n > TRUSS_NOALLOC_MAX_VERTICES) return TRUSS_ETOOBIG;
    if (2 * m > (int64_t)INT32_MAX) return TRUSS_EOVERFLOW;  // slots are int32 row offsets
    // set-up first, so that a call with n = 0 does only the set-up
    int32_t* scratch = nullptr;
    TRY(scratch_address(&scratch));
    if (n == 0) return m == 0 ? TRUSS_OK : TRUSS_EBADGRAPH;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* eo = scratch;
    int32_t* err = scratch + NA_ERR;
    CU(cudaMemsetAsync(err, 0, sizeof(int32_t), s));  // the array keeps the last call's contents
    k_na_check_rows<<<grid_for(n, 256), 256, 0, s>>>(d_rowptr, n, m, err);
    CU(cudaGetLastError());
    int32_t h_bad = 0;
    CU(cudaMemcpyAsync(&h_bad, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h_bad) return TRUSS_EBADGRAPH;  // nothing was read through the offsets
    if (m == 0) return TRUSS_OK;
    k_na_zero<<<grid_for(m, 256), 256, 0, s>>>(d_support, m);
    k_na_eo<<<grid_for(n, 256), 256, 0, s>>>(d_rowptr, d_col, n, eo);
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    k_na_support<<<grid_for(n, NA_WARPS, (int64_t)sms * 8), NA_WARPS * 32, 0, s>>>(d_rowptr, eo, d_col, d_eid, n, m,
                                                                                    d_support, err);
    CU(cudaGetLastError());
    int32_t h_err = 0;
    CU(cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return h_err ? TRUSS_EBADGRAPH : TRUSS_OK;
}
