// Host-buffer pipeline: the whole decomposition from a host edge list to a
// host trussness array, for callers without device memory of their own.
#include <cstring>
#include <vector>

#include "graph.cuh"

// The Python binding mirrors these layouts.
static_assert(sizeof(truss_opts) == 104, "truss_opts layout");
static_assert(sizeof(truss_stats) == 128, "truss_stats layout");
static_assert(sizeof(truss_sublevel_trace) == 56, "truss_sublevel_trace layout");

extern "C" int truss_decompose_host(const int32_t* h_src, const int32_t* h_dst, int64_t n_in, int32_t n,
                                    uint32_t flags, int32_t* h_truss, int64_t m_cap, int64_t* m_out,
                                    const truss_opts* opts, truss_stats* stats, void* stream) {
    if (n_in < 0 || n < 0 || !m_out || (n_in > 0 && (!h_src || !h_dst))) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *d_src = nullptr, *d_dst = nullptr, *d_out = nullptr;
    const size_t bytes = sizeof(int32_t) * (size_t)(n_in > 0 ? n_in : 1);
    CU(cudaMallocAsync((void**)&d_src, bytes, s));
    CU(cudaMallocAsync((void**)&d_dst, bytes, s));
    if (n_in > 0) {
        CU(cudaMemcpyAsync(d_src, h_src, sizeof(int32_t) * (size_t)n_in, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(d_dst, h_dst, sizeof(int32_t) * (size_t)n_in, cudaMemcpyHostToDevice, s));
    }
    truss_graph* g = nullptr;
    int rc = truss_build_csr(d_src, d_dst, n_in, n, flags, stream, &g);
    cudaFreeAsync(d_src, s);
    cudaFreeAsync(d_dst, s);
    if (rc != TRUSS_OK) return rc;
    *m_out = g->m;
    if (g->m > m_cap || (g->m > 0 && !h_truss)) {
        truss_free(g);
        return TRUSS_EINVAL;
    }
    truss_opts o;
    if (opts)
        o = *opts;
    else
        truss_default_opts(&o);
    o.sync = 1;
    rc = cudaMallocAsync((void**)&d_out, sizeof(int32_t) * (size_t)(g->m > 0 ? g->m : 1), s) == cudaSuccess
             ? TRUSS_OK
             : TRUSS_ENOMEM;
    if (rc == TRUSS_OK) rc = truss_decompose(g, d_out, &o, stats, stream);
    if (rc == TRUSS_OK && g->m > 0) {
        cudaError_t e = cudaMemcpyAsync(h_truss, d_out, sizeof(int32_t) * (size_t)g->m, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            truss_note_cuda_error(e);
            rc = TRUSS_ECUDA;
        }
    }
    if (d_out) cudaFreeAsync(d_out, s);
    cudaStreamSynchronize(s);
    truss_free(g);
    return rc;
}

// ----------------------------------------------------------- many graphs

namespace {

// Last g with off[g] <= x (off ascending, off[0] = 0).
__device__ __forceinline__ int32_t owner_of(const int64_t* __restrict__ off, int32_t G, int64_t x) {
    int32_t lo = 0, hi = G - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// raw pairs of graph g -> union labels (ids shifted by the graph's vertex
// offset); an id outside its graph's range marks the input bad
__global__ void k_union_pairs(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t n_in,
                              const int64_t* __restrict__ eoff, const int64_t* __restrict__ voff, int32_t G,
                              int32_t* __restrict__ usrc, int32_t* __restrict__ udst, int* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_in; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = owner_of(eoff, G, i);
        const int64_t n = voff[g + 1] - voff[g];
        const int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            atomicOr(bad, 1);
            usrc[i] = udst[i] = (int32_t)voff[g];
        } else {
            usrc[i] = (int32_t)(voff[g] + a);
            udst[i] = (int32_t)(voff[g] + b);
        }
    }
}

// moff[g] = first canonical edge whose smaller endpoint lies in graph g
__global__ void k_graph_edge_offsets(const int32_t* __restrict__ u, int64_t m, const int64_t* __restrict__ voff,
                                     int32_t G, int64_t* __restrict__ moff) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g <= G; g += (int64_t)gridDim.x * blockDim.x) {
        if (g == G) {
            moff[g] = m;
            continue;
        }
        int64_t lo = 0, hi = m;
        const int64_t key = voff[g];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (u[mid] < key) lo = mid + 1; else hi = mid;
        }
        moff[g] = lo;
    }
}

}  // namespace

extern "C" int truss_decompose_batch(const int32_t* d_src, const int32_t* d_dst, const int64_t* h_eoff,
                                     const int32_t* h_nverts, int32_t G, uint32_t flags, int32_t* d_truss,
                                     int64_t capacity, int64_t* h_moff, const truss_opts* opts, truss_stats* stats,
                                     void* stream) {
    if (G < 0 || !h_moff || (G > 0 && (!h_eoff || !h_nverts))) return TRUSS_EINVAL;
    if (G == 0) {
        h_moff[0] = 0;
        return TRUSS_OK;
    }
    if (h_eoff[0] != 0) return TRUSS_EINVAL;
    std::vector<int64_t> voff((size_t)G + 1, 0);
    for (int32_t g = 0; g < G; g++) {
        if (h_nverts[g] < 0 || h_eoff[g + 1] < h_eoff[g]) return TRUSS_EINVAL;
        voff[g + 1] = voff[g] + h_nverts[g];
    }
    if (voff[G] >= INT32_MAX) return TRUSS_EOVERFLOW;
    const int64_t n_in = h_eoff[G];
    if (n_in > 0 && (!d_src || !d_dst || !d_truss)) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t *d_eoff = nullptr, *d_voff = nullptr, *d_moff = nullptr;
    int32_t *usrc = nullptr, *udst = nullptr, *tmpu = nullptr;
    int* d_bad = nullptr;
    truss_graph* g = nullptr;
    int rc = TRUSS_OK;
    auto done = [&](int r) {
        cudaStreamSynchronize(s);
        cudaFree(d_eoff); cudaFree(d_voff); cudaFree(d_moff); cudaFree(usrc); cudaFree(udst); cudaFree(tmpu); cudaFree(d_bad);
        if (g) truss_free(g);
        return r;
    };
#define BCU(call)                                   \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) {                    \
            truss_note_cuda_error(e_);              \
            return done(e_ == cudaErrorMemoryAllocation ? TRUSS_ENOMEM : TRUSS_ECUDA); \
        }                                           \
    } while (0)
    BCU(cudaMalloc((void**)&d_eoff, sizeof(int64_t) * ((size_t)G + 1)));
    BCU(cudaMalloc((void**)&d_voff, sizeof(int64_t) * ((size_t)G + 1)));
    BCU(cudaMalloc((void**)&d_moff, sizeof(int64_t) * ((size_t)G + 1)));
    BCU(cudaMalloc((void**)&usrc, sizeof(int32_t) * (size_t)(n_in > 0 ? n_in : 1)));
    BCU(cudaMalloc((void**)&udst, sizeof(int32_t) * (size_t)(n_in > 0 ? n_in : 1)));
    BCU(cudaMalloc((void**)&d_bad, sizeof(int)));
    BCU(cudaMemcpyAsync(d_eoff, h_eoff, sizeof(int64_t) * ((size_t)G + 1), cudaMemcpyHostToDevice, s));
    BCU(cudaMemcpyAsync(d_voff, voff.data(), sizeof(int64_t) * ((size_t)G + 1), cudaMemcpyHostToDevice, s));
    BCU(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
    if (n_in > 0) k_union_pairs<<<grid_for(n_in, 256), 256, 0, s>>>(d_src, d_dst, n_in, d_eoff, d_voff, G, usrc, udst, d_bad);
    BCU(cudaGetLastError());
    int bad = 0;
    BCU(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCU(cudaStreamSynchronize(s));
    if (bad) return done(TRUSS_EBADGRAPH);
    rc = truss_build_csr(usrc, udst, n_in, (int32_t)voff[G], flags, stream, &g);
    if (rc != TRUSS_OK) return done(rc);
    if (g->m > capacity) return done(TRUSS_EINVAL);
    truss_opts o;
    if (opts)
        o = *opts;
    else
        truss_default_opts(&o);
    o.sync = 1;
    rc = truss_decompose(g, d_truss, &o, stats, stream);
    if (rc != TRUSS_OK) return done(rc);
    BCU(cudaMalloc((void**)&tmpu, sizeof(int32_t) * (size_t)(2 * g->m + 2)));
    rc = truss_edge_list(g, tmpu, tmpu + g->m + 1, stream);
    if (rc != TRUSS_OK) return done(rc);
    k_graph_edge_offsets<<<grid_for((int64_t)G + 1, 256), 256, 0, s>>>(tmpu, g->m, d_voff, G, d_moff);
    BCU(cudaGetLastError());
    BCU(cudaMemcpyAsync(h_moff, d_moff, sizeof(int64_t) * ((size_t)G + 1), cudaMemcpyDeviceToHost, s));
    return done(TRUSS_OK);
#undef BCU
}
