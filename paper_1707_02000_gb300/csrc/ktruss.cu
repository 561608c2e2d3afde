// k-trusses as subgraphs (§II): a k-truss is a maximal connected subgraph in
// which every edge lies in at least k-2 of its triangles, so the k-trusses of
// a graph are the connected components of its edges of trussness >= k.  Given
// the trussness of every edge, each such edge is labelled with the smallest
// input vertex label of its component.
//
// Lock-free union-find over the internal vertex ids: a union hooks the larger
// root under the smaller with one CAS, a find halves the path as it goes.
// Every parent pointer only ever moves to a smaller id, so a find walks a
// strictly decreasing chain and ends; the loops still stop after a fixed
// number of steps and report TRUSS_EDEVICE (never reached on a consistent
// state).
#include <climits>

#include "graph.cuh"

namespace {

constexpr int UF_MAX_STEPS = 1 << 26;

__device__ __forceinline__ int32_t uf_find(int32_t* p, int32_t x, int* err) {
    volatile int32_t* vp = p;
    int32_t cur = x, nxt = vp[cur];
    for (int it = 0; nxt != cur; it++) {
        if (it >= UF_MAX_STEPS) {
            atomicExch(err, 1);
            return cur;
        }
        const int32_t nn = vp[nxt];
        if (nn != nxt) vp[cur] = nn;
        cur = nxt;
        nxt = nn;
    }
    return cur;
}

__device__ __forceinline__ void uf_union(int32_t* p, int32_t a, int32_t b, int* err) {
    for (int it = 0; it < UF_MAX_STEPS; it++) {
        a = uf_find(p, a, err);
        b = uf_find(p, b, err);
        if (a == b) return;
        if (a < b) {
            const int32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(p + a, a, b) == a) return;  // a was still a root
    }
    atomicExch(err, 1);
}

__global__ void k_uf_init(int32_t* __restrict__ p, int32_t* __restrict__ minl, int32_t n) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        p[v] = (int32_t)v;
        minl[v] = INT_MAX;
    }
}

__global__ void k_uf_union(const int2* __restrict__ el, int64_t m, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ tau, int32_t k, int32_t* p, int* err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = perm ? perm[e] : e;
        if (tau[c] >= k) {
            const int2 xy = el[e];
            uf_union(p, xy.x, xy.y, err);
        }
    }
}

// after all unions: smallest input label of each root's component
__global__ void k_uf_minlabel(const int2* __restrict__ el, int64_t m, const int32_t* __restrict__ perm,
                              const int32_t* __restrict__ tau, int32_t k, int32_t* p,
                              const int32_t* __restrict__ order, int32_t* __restrict__ minl, int* err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = perm ? perm[e] : e;
        if (tau[c] >= k) {
            const int2 xy = el[e];
            const int32_t r = uf_find(p, xy.x, err);
            atomicMin(minl + r, order ? min(order[xy.x], order[xy.y]) : min(xy.x, xy.y));
        }
    }
}

__global__ void k_uf_out(const int2* __restrict__ el, int64_t m, const int32_t* __restrict__ perm,
                         const int32_t* __restrict__ tau, int32_t k, int32_t* p, const int32_t* __restrict__ minl,
                         int32_t* __restrict__ comp, int* err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = perm ? perm[e] : e;
        comp[c] = tau[c] >= k ? minl[uf_find(p, el[e].x, err)] : -1;
    }
}

__global__ void k_uf_count(const int32_t* __restrict__ minl, int32_t n, unsigned long long* cnt) {
    unsigned long long c = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        c += minl[v] != INT_MAX;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

}  // namespace

extern "C" int truss_ktruss_components(truss_graph* g, const int32_t* d_truss, int32_t k, int32_t* d_comp,
                                       int64_t* h_ncomp, void* stream) {
    if (!g || (g->m > 0 && (!d_truss || !d_comp))) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->m == 0 || g->n == 0) {
        if (h_ncomp) *h_ncomp = 0;
        return TRUSS_OK;
    }
    const int B = 256;
    int32_t *p = nullptr, *minl = nullptr;
    int* err = nullptr;
    unsigned long long* cnt = nullptr;
    CU(cudaMallocAsync((void**)&p, sizeof(int32_t) * (size_t)g->n, s));
    CU(cudaMallocAsync((void**)&minl, sizeof(int32_t) * (size_t)g->n, s));
    CU(cudaMallocAsync((void**)&err, sizeof(int) + sizeof(unsigned long long) * 2, s));
    cnt = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(err) + sizeof(unsigned long long));
    CU(cudaMemsetAsync(err, 0, sizeof(int) + sizeof(unsigned long long) * 2, s));
    const int gv = grid_for(g->n, B), ge = grid_for(g->m, B);
    k_uf_init<<<gv, B, 0, s>>>(p, minl, g->n);
    k_uf_union<<<ge, B, 0, s>>>(g->el, g->m, g->perm, d_truss, k, p, err);
    k_uf_minlabel<<<ge, B, 0, s>>>(g->el, g->m, g->perm, d_truss, k, p, g->order, minl, err);
    k_uf_out<<<ge, B, 0, s>>>(g->el, g->m, g->perm, d_truss, k, p, minl, d_comp, err);
    int rc = TRUSS_OK;
    if (h_ncomp) {
        k_uf_count<<<gv, B, 0, s>>>(minl, g->n, cnt);
        unsigned long long hc = 0;
        int he = 0;
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(&he, err, sizeof(he), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        *h_ncomp = (int64_t)hc;
        if (he) rc = TRUSS_EDEVICE;
    }
    CU(cudaGetLastError());
    truss_note_launch(h_ncomp ? 5 : 4);
    cudaFreeAsync(p, s);
    cudaFreeAsync(minl, s);
    cudaFreeAsync(err, s);
    return rc;
}
