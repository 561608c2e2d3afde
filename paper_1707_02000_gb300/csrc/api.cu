// Host-buffer pipeline: the whole decomposition from a host edge list to a
// host trussness array, for callers without device memory of their own.
#include <cstring>

#include "graph.cuh"

// The Python binding mirrors these layouts.
static_assert(sizeof(truss_opts) == 80, "truss_opts layout");
static_assert(sizeof(truss_stats) == 96, "truss_stats layout");
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
