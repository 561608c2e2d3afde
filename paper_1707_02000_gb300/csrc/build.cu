// Device graph build: raw edge list -> the augmented CSR of §III / Fig. 2.
//
// 1. check ids, emit both orientations of every pair as one packed key
//    (a << nb | b), self-loops as a sentinel that sorts last;
// 2. stable LSD radix sort of the keys, drop repeats and sentinels;
// 3. row offsets from the sorted keys, Eo by binary search per row, the
//    upper-degree prefix (edge-id base per row), Eid and El;
// 4. with TRUSS_DEGREE_ORDER: rank vertices by (degree, label), re-emit the
//    pairs in the new labels, sort and build again, and map every internal
//    edge back to its canonical id through the first CSR.
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>

#include "graph.cuh"
#include "prims.cuh"

#include <algorithm>

using prims::talloc;
using prims::tfree;

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void truss_note_cuda_error(cudaError_t e) { g_last_cuda = e; }

static std::atomic<long long> g_launches{0};
void truss_note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long truss_launch_count() { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char* truss_strerror(int status) {
    switch (status) {
        case TRUSS_OK: return "ok";
        case TRUSS_EINVAL: return "invalid argument";
        case TRUSS_ENOMEM: return "out of memory";
        case TRUSS_ECUDA: return g_last_cuda != cudaSuccess ? cudaGetErrorString(g_last_cuda) : "CUDA error";
        case TRUSS_ETIMEOUT: return "device-side wait exceeded its time limit";
        case TRUSS_EOVERFLOW: return "edge count does not fit the index width";
        case TRUSS_EBADGRAPH: return "vertex id outside [0, n)";
        case TRUSS_EDEVICE: return "device-side consistency check failed";
        case TRUSS_ENOTSUP: return "not supported";
        case TRUSS_ETOOBIG: return "input exceeds the fixed capacity of this entry point";
        default: return "unknown status";
    }
}

namespace {

__global__ void k_check_ids(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t n_in,
                            int32_t n, int* bad) {
    bool b = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_in; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[i], c = dst[i];
        b |= (a < 0) | (a >= n) | (c < 0) | (c >= n);
    }
    if (__any_sync(FULL_MASK, b) && lane_id() == 0) atomicOr(bad, 1);
}

__global__ void k_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t n_in,
                            int32_t n, int nb, uint64_t* __restrict__ keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_in; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a = (uint32_t)src[i], b = (uint32_t)dst[i];
        if (a == b) a = b = (uint64_t)n;  // sentinel, sorts after every real pair
        keys[2 * i] = a << nb | b;
        keys[2 * i + 1] = b << nb | a;
    }
}

struct UniqueFlag {
    const uint64_t* keys;
    uint64_t sentinel;
    __device__ int64_t operator()(int64_t i) const {
        uint64_t k = keys[i];
        return (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
};

__global__ void k_compact_unique(const uint64_t* __restrict__ keys, int64_t len, uint64_t sentinel,
                                 const int64_t* __restrict__ pos, uint64_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        if (k != sentinel && (i == 0 || keys[i - 1] != k)) out[pos[i]] = k;
    }
}

// rowptr[v] = first j with row(U[j]) >= v; each entry written once.
__global__ void k_rowptr(const uint64_t* __restrict__ U, int64_t len, int nb, int32_t n, int64_t* __restrict__ rowptr) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= len; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = (j < len) ? (int64_t)(U[j] >> nb) : (int64_t)n;
        int64_t ap = (j == 0) ? -1 : (int64_t)(U[j - 1] >> nb);
        for (int64_t v = ap + 1; v <= a; v++) rowptr[v] = j;
    }
}

__global__ void k_col(const uint64_t* __restrict__ U, int64_t len, uint64_t mask, int32_t* __restrict__ col) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x)
        col[j] = (int32_t)(U[j] & mask);
}

__global__ void k_eo(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                     int64_t* __restrict__ eo) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        eo[u] = lower_bound_dev<int64_t>(col, rowptr[u], rowptr[u + 1], (int32_t)u + 1);
}

struct UpperDeg {
    const int64_t* rowptr;
    const int64_t* eo;
    __device__ int64_t operator()(int64_t u) const { return rowptr[u + 1] - eo[u]; }
};

// Eid of every slot and El of every edge.  Row of slot j = high part of U[j].
__global__ void k_eid(const uint64_t* __restrict__ U, int64_t len, int nb, const int64_t* __restrict__ rowptr,
                      const int32_t* __restrict__ col, const int64_t* __restrict__ eo,
                      const int64_t* __restrict__ ubase, int32_t* __restrict__ eid, int2* __restrict__ el) {
    const uint64_t mask = (1ull << nb) - 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = (int32_t)(U[j] >> nb), y = (int32_t)(U[j] & mask);
        int64_t e;
        if (y > x) {
            e = ubase[x] + (j - eo[x]);
            el[e] = make_int2(x, y);
        } else {
            int64_t p = lower_bound_dev<int64_t>(col, eo[y], rowptr[y + 1], x);
            e = ubase[y] + (p - eo[y]);
        }
        eid[j] = (int32_t)e;
    }
}

__global__ void k_degree_keys(const int64_t* __restrict__ rowptr, int32_t n, int nb, uint64_t* __restrict__ keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = (uint64_t)(rowptr[v + 1] - rowptr[v]) << nb | (uint64_t)v;
}

// ---- degeneracy order (TRUSS_CORE_ORDER): level-synchronous k-core peel.
// Level k: a scan removes every live vertex of degree <= k (round t); then,
// round after round, the vertices removed in the last round lower the degree
// of their live neighbours, and a neighbour whose degree falls from k + 1 to
// k is removed in the next round.  step[v] = round of v's removal (-1 while
// live); the order is by (step, label).
__global__ void k_core_init(const int64_t* __restrict__ rowptr, int32_t n, int32_t* __restrict__ deg,
                            int32_t* __restrict__ step) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        deg[v] = (int32_t)(rowptr[v + 1] - rowptr[v]);
        step[v] = -1;
    }
}

// live vertices of degree <= k join round t; the smallest live degree above
// k is reduced into *minv (for an empty scan's jump)
__global__ void k_core_scan(int32_t n, const int32_t* __restrict__ deg, int32_t* __restrict__ step, int32_t k,
                            int32_t t, int32_t* __restrict__ out, int* cnt, int* minv) {
    int mn = INT_MAX;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + threadIdx.x;
        bool take = false;
        if (v < n && step[v] < 0) {
            const int d = deg[v];
            if (d <= k) {
                step[v] = t;
                take = true;
            } else {
                mn = min(mn, d);
            }
        }
        warp_append(take, (int32_t)v, out, cnt);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(FULL_MASK, mn, o));
    if ((threadIdx.x & 31) == 0 && mn != INT_MAX) atomicMin(minv, mn);
}

// a warp per vertex removed in round t: its live neighbours lose one degree;
// one that falls to k is removed in round t + 1
__global__ void k_core_round(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ cur, int32_t ncur, int32_t* __restrict__ deg,
                             int32_t* __restrict__ step, int32_t k, int32_t t, int32_t* __restrict__ next,
                             int* nnext) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < ncur; i += nwarps) {
        const int32_t v = cur[i];
        for (int64_t j = rowptr[v] + lane; j < rowptr[v + 1]; j += 32) {
            const int32_t u = col[j];
            if (step[u] < 0 && atomicSub(deg + u, 1) == k + 1) {
                step[u] = t + 1;
                next[atomicAdd(nnext, 1)] = u;
            }
        }
    }
}

__global__ void k_core_keys(const int32_t* __restrict__ step, int32_t n, int nb, uint64_t* __restrict__ keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = (uint64_t)step[v] << nb | (uint64_t)v;
}

__global__ void k_order(const uint64_t* __restrict__ keys, int32_t n, uint64_t mask, int32_t* __restrict__ order,
                        int32_t* __restrict__ newid) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = (int32_t)(keys[i] & mask);
        order[i] = v;
        newid[v] = (int32_t)i;
    }
}

__global__ void k_relabel(const uint64_t* __restrict__ U, int64_t len, int nb, const int32_t* __restrict__ newid,
                          uint64_t* __restrict__ out) {
    const uint64_t mask = (1ull << nb) - 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a = (uint32_t)newid[U[j] >> nb], b = (uint32_t)newid[U[j] & mask];
        out[j] = a << nb | b;
    }
}

// perm[e]: canonical id of internal edge e, found in the input-label CSR.
__global__ void k_perm(const int2* __restrict__ el, int64_t m, const int32_t* __restrict__ order,
                       const int64_t* __restrict__ rowptr0, const int32_t* __restrict__ col0,
                       const int64_t* __restrict__ eo0, const int64_t* __restrict__ ubase0, int32_t* __restrict__ perm) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int2 xy = el[e];
        int32_t p = order[xy.x], q = order[xy.y];
        int32_t lo = min(p, q), hi = max(p, q);
        int64_t pos = lower_bound_dev<int64_t>(col0, eo0[lo], rowptr0[lo + 1], hi);
        perm[e] = (int32_t)(ubase0[lo] + (pos - eo0[lo]));
    }
}

template <typename Off>
__global__ void k_narrow(const int64_t* __restrict__ in, int64_t len, Off* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (Off)in[i];
}

__global__ void k_classify_vertices(const int64_t* __restrict__ rowptr, const int64_t* __restrict__ eo, int32_t n,
                                    int32_t* __restrict__ big, int* nbig, int32_t* __restrict__ huge, int* nhuge,
                                    unsigned long long* __restrict__ maxes) {
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = base + threadIdx.x;
        int64_t up = 0, d = 0;
        if (u < n) {
            up = rowptr[u + 1] - eo[u];
            d = rowptr[u + 1] - rowptr[u];
        }
        const bool isbig = up > TRUSS_SUP_WARP_CAP && up <= TRUSS_SUP_BLOCK_CAP;
        warp_append(isbig, (int32_t)u, big, nbig);
        warp_append(up > TRUSS_SUP_BLOCK_CAP, (int32_t)u, huge, nhuge);
        // over the block-kernel vertices: the longest N+(u) and the widest
        // label window above u (n - 1 - u), which size that kernel's
        // shared-memory bitmap
        int64_t bup = isbig ? up : 0, bwin = isbig ? (int64_t)n - 1 - u : 0;
        // one atomic per warp for each maximum (same-address atomics from
        // every vertex cost more than the rest of the kernel)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            d = max(d, (int64_t)__shfl_xor_sync(FULL_MASK, (long long)d, o));
            up = max(up, (int64_t)__shfl_xor_sync(FULL_MASK, (long long)up, o));
            bup = max(bup, (int64_t)__shfl_xor_sync(FULL_MASK, (long long)bup, o));
            bwin = max(bwin, (int64_t)__shfl_xor_sync(FULL_MASK, (long long)bwin, o));
        }
        if ((threadIdx.x & 31) == 0) {
            if (d) atomicMax(&maxes[0], (unsigned long long)d);
            if (up) atomicMax(&maxes[1], (unsigned long long)up);
            if (bup) atomicMax(&maxes[2], (unsigned long long)bup);
            if (bwin) atomicMax(&maxes[3], (unsigned long long)bwin);
        }
    }
}

// W+ = sum_v d-(v) d+(v) and sum over edges of min(d(u), d(v)).
__global__ void k_work_stats(const int64_t* __restrict__ rowptr, const int64_t* __restrict__ eo, int32_t n,
                             const int2* __restrict__ el, int64_t m, unsigned long long* __restrict__ out) {
    unsigned long long w = 0, d = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        w += (unsigned long long)(eo[u] - rowptr[u]) * (unsigned long long)(rowptr[u + 1] - eo[u]);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int2 xy = el[e];
        d += (unsigned long long)min(rowptr[xy.x + 1] - rowptr[xy.x], rowptr[xy.y + 1] - rowptr[xy.y]);
    }
    w = warp_sum(w);
    d = warp_sum(d);
    if (lane_id() == 0) {
        atomicAdd(out, w);
        atomicAdd(out + 1, d);
    }
}

struct Csr64 {
    int64_t* rowptr = nullptr;
    int64_t* eo = nullptr;
    int64_t* ubase = nullptr;
    int32_t* col = nullptr;
};

void free_csr(Csr64& c, cudaStream_t s) {
    tfree(c.rowptr, s);
    tfree(c.eo, s);
    tfree(c.ubase, s);
    tfree(c.col, s);
    c = Csr64();
}

// Removal rounds of the k-core peel (see k_core_round) as sort keys
// (round << nb | v); *rounds receives the number of rounds.
static int core_steps(const Csr64& c, int32_t n, int nb, uint64_t* keys, int32_t* rounds, cudaStream_t s) {
    const int B = 256;
    int32_t *deg = nullptr, *step = nullptr, *fa = nullptr, *fb = nullptr;
    int* ctr = nullptr;
    CU(talloc(&deg, n, s));
    CU(talloc(&step, n, s));
    CU(talloc(&fa, n, s));
    CU(talloc(&fb, n, s));
    CU(talloc(&ctr, 2, s));
    k_core_init<<<grid_for(n, B), B, 0, s>>>(c.rowptr, n, deg, step);
    CU(cudaGetLastError());
    int h[2];
    int64_t removed = 0;
    int32_t k = 0, t = 0;
    const int rblocks = grid_for((int64_t)n * 32, B, (int64_t)152 * 16);
    while (removed < n) {
        const int init[2] = {0, INT_MAX};
        CU(cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, s));
        k_core_scan<<<grid_for(n, B), B, 0, s>>>(n, deg, step, k, t, fa, ctr, ctr + 1);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (h[0] == 0) {
            if (h[1] == INT_MAX) break;  // nothing live (cannot happen while removed < n)
            k = h[1];
            continue;
        }
        removed += h[0];
        int32_t* cur = fa;
        int32_t* nxt = fb;
        int32_t ncur = h[0];
        for (;;) {
            CU(cudaMemsetAsync(ctr, 0, sizeof(int), s));
            k_core_round<<<rblocks, B, 0, s>>>(c.rowptr, c.col, cur, ncur, deg, step, k, t, nxt, ctr);
            CU(cudaGetLastError());
            CU(cudaMemcpyAsync(h, ctr, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            t++;
            if (h[0] == 0) break;
            removed += h[0];
            ncur = h[0];
            std::swap(cur, nxt);
        }
        k++;
    }
    k_core_keys<<<grid_for(n, B), B, 0, s>>>(step, n, nb, keys);
    CU(cudaGetLastError());
    *rounds = t;
    tfree(deg, s);
    tfree(step, s);
    tfree(fa, s);
    tfree(fb, s);
    tfree(ctr, s);
    return TRUSS_OK;
}

// ---------------------------------------------------- locality (RCM) order
//
// A reverse Cuthill-McKee order (TRUSS_LOCALITY_ORDER): a breadth-first
// search from the vertex of highest degree (lowest label among ties) ranks
// each new level by (rank of its first-ranked neighbour in the level
// before, label), so vertices close in the graph get close labels; the
// ranks are then reversed.  Vertices the search does not reach (other
// components, isolated vertices) follow in label order.  On mesh-like
// graphs this keeps a vertex's rows, and the edges of its triangles, near
// each other in memory (geometric 2^21 workload: peel 24.8 -> 22.4 ms,
// support 2.57 -> 2.84 ms as W+ grows from 4.0e8 to 5.3e8 without the
// degree orientation).

// max over v of deg(v) << nb | (mask - v): the highest degree, then the
// lowest label
__global__ void k_rcm_start(const int64_t* __restrict__ rowptr, int32_t n, int nb, unsigned long long* best) {
    const uint64_t mask = (1ull << nb) - 1;
    unsigned long long b = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t d = (uint64_t)(rowptr[v + 1] - rowptr[v]);
        if (d) b = max(b, (unsigned long long)(d << nb | (mask - (uint64_t)v)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(FULL_MASK, b, o));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

__global__ void k_rcm_init(int32_t n, int nb, const unsigned long long* __restrict__ best, int32_t* __restrict__ rank,
                           int32_t* __restrict__ par, int32_t* __restrict__ level) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        rank[v] = -1;
        par[v] = INT_MAX;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && *best) {
        const uint64_t mask = (1ull << nb) - 1;
        level[0] = (int32_t)(mask - (*best & mask));
    }
}

__global__ void k_rcm_seed(const int32_t* __restrict__ level, int32_t* __restrict__ rank) { rank[level[0]] = 0; }

// A warp per vertex u of the current level: each unranked neighbour w keeps
// the lowest rank among its neighbours in this level (par) and is appended
// to the next level by the first of them.
__global__ void k_rcm_expand(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ level, int32_t nlev, const int32_t* __restrict__ rank,
                             int32_t* __restrict__ par, int32_t* __restrict__ cand, int* ncand) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nlev; i += nwarps) {
        const int32_t u = level[i];
        const int32_t ru = rank[u];
        for (int64_t j = rowptr[u] + lane; j < rowptr[u + 1]; j += 32) {
            const int32_t w = col[j];
            if (rank[w] < 0 && atomicMin(par + w, ru) == INT_MAX) cand[atomicAdd(ncand, 1)] = w;
        }
    }
}

__global__ void k_rcm_keys(const int32_t* __restrict__ cand, int32_t k, const int32_t* __restrict__ par, int nb,
                           uint64_t* __restrict__ keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t w = cand[i];
        keys[i] = (uint64_t)par[w] << nb | (uint64_t)w;
    }
}

__global__ void k_rcm_assign(const uint64_t* __restrict__ sorted, int32_t k, uint64_t mask, int32_t base,
                             int32_t* __restrict__ rank, int32_t* __restrict__ level) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t w = (int32_t)(sorted[i] & mask);
        rank[w] = base + (int32_t)i;
        level[i] = w;
    }
}

struct Unranked {
    const int32_t* rank;
    __device__ int64_t operator()(int64_t v) const { return rank[v] < 0 ? 1 : 0; }
};

// Sort keys (n - 1 - rank) << nb | v, the unreached vertices ranked after
// the search's in label order.
__global__ void k_rcm_keys_final(const int32_t* __restrict__ rank, const int64_t* __restrict__ before, int32_t n,
                                 int32_t reached, int nb, uint64_t* __restrict__ keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = rank[v] >= 0 ? rank[v] : (int64_t)reached + before[v];
        keys[v] = (uint64_t)((int64_t)n - 1 - r) << nb | (uint64_t)v;
    }
}

// RCM ranks as sort keys (key_bits 2 nb).  One host round trip per level.
static int locality_keys(const Csr64& c, int32_t n, int nb, uint64_t* keys, cudaStream_t s) {
    const int B = 256;
    const uint64_t mask = (1ull << nb) - 1;
    int32_t *rank = nullptr, *par = nullptr, *la = nullptr, *lb = nullptr;
    uint64_t *kk = nullptr, *kt = nullptr;
    int64_t* before = nullptr;
    unsigned long long* best = nullptr;
    int* cnt = nullptr;
    CU(talloc(&rank, n, s));
    CU(talloc(&par, n, s));
    CU(talloc(&la, n, s));
    CU(talloc(&lb, n, s));
    CU(talloc(&kk, n, s));
    CU(talloc(&kt, n, s));
    CU(talloc(&before, (int64_t)n + 1, s));
    CU(talloc(&best, 1, s));
    CU(talloc(&cnt, 1, s));
    CU(cudaMemsetAsync(best, 0, sizeof(unsigned long long), s));
    k_rcm_start<<<grid_for(n, B), B, 0, s>>>(c.rowptr, n, nb, best);
    k_rcm_init<<<grid_for(n, B), B, 0, s>>>(n, nb, best, rank, par, la);
    CU(cudaGetLastError());
    unsigned long long hb = 0;
    CU(cudaMemcpyAsync(&hb, best, sizeof(hb), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    int32_t reached = 0;
    if (hb) {
        k_rcm_seed<<<1, 1, 0, s>>>(la, rank);
        CU(cudaGetLastError());
        int32_t nlev = 1;
        reached = 1;
        const int eblocks = grid_for((int64_t)n * 32, B, (int64_t)152 * 16);
        while (nlev > 0) {
            CU(cudaMemsetAsync(cnt, 0, sizeof(int), s));
            k_rcm_expand<<<eblocks, B, 0, s>>>(c.rowptr, c.col, la, nlev, rank, par, lb, cnt);
            CU(cudaGetLastError());
            int k = 0;
            CU(cudaMemcpyAsync(&k, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            if (k == 0) break;
            k_rcm_keys<<<grid_for(k, B), B, 0, s>>>(lb, k, par, nb, kk);
            CU(cudaGetLastError());
            uint64_t* sorted = nullptr;
            CU(prims::radix_sort_u64(kk, kt, k, 2 * nb, &sorted, s));
            k_rcm_assign<<<grid_for(k, B), B, 0, s>>>(sorted, k, mask, reached, rank, la);
            CU(cudaGetLastError());
            reached += k;
            nlev = k;
        }
    }
    CU(prims::exclusive_scan<int64_t>(Unranked{rank}, n, before, before + n, s));
    k_rcm_keys_final<<<grid_for(n, B), B, 0, s>>>(rank, before, n, reached, nb, keys);
    CU(cudaGetLastError());
    tfree(rank, s);
    tfree(par, s);
    tfree(la, s);
    tfree(lb, s);
    tfree(kk, s);
    tfree(kt, s);
    tfree(before, s);
    tfree(best, s);
    tfree(cnt, s);
    return TRUSS_OK;
}

// CSR (64-bit offsets) from 2m sorted unique directed keys.
int csr_from_keys(const uint64_t* U, int64_t len, int32_t n, int nb, Csr64& c, cudaStream_t s) {
    const int B = 256;
    CU(talloc(&c.rowptr, (int64_t)n + 1, s));
    CU(talloc(&c.eo, (int64_t)n + 1, s));
    CU(talloc(&c.ubase, (int64_t)n + 1, s));
    CU(talloc(&c.col, len, s));
    k_rowptr<<<grid_for(len + 1, B), B, 0, s>>>(U, len, nb, n, c.rowptr);
    k_col<<<grid_for(len, B), B, 0, s>>>(U, len, (1ull << nb) - 1, c.col);
    k_eo<<<grid_for(n, B), B, 0, s>>>(c.rowptr, c.col, n, c.eo);
    CU(cudaGetLastError());
    CU(prims::exclusive_scan<int64_t>(UpperDeg{c.rowptr, c.eo}, n, c.ubase, c.ubase + n, s));
    return TRUSS_OK;
}

int build_impl(const int32_t* d_src, const int32_t* d_dst, int64_t n_in, int32_t n, uint32_t flags,
               cudaStream_t s, truss_graph* g) {
    const int B = 256;
    int nb = 1;
    while (nb < 32 && (1ll << nb) <= (int64_t)n) nb++;
    const uint64_t mask = (1ull << nb) - 1;
    const uint64_t sentinel = ((uint64_t)n << nb) | (uint64_t)n;
    int* d_flag = nullptr;
    CU(talloc(&d_flag, 4, s));
    CU(cudaMemsetAsync(d_flag, 0, 4 * sizeof(int), s));
    if (n_in > 0) {
        k_check_ids<<<grid_for(n_in, B), B, 0, s>>>(d_src, d_dst, n_in, n, d_flag);
        CU(cudaGetLastError());
        int bad = 0;
        CU(cudaMemcpyAsync(&bad, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (bad) {
            tfree(d_flag, s);
            return TRUSS_EBADGRAPH;
        }
    }
    // 1-2: packed keys, sort, unique
    const int64_t K = 2 * n_in;
    uint64_t *keys = nullptr, *tmp = nullptr, *sorted = nullptr, *U = nullptr;
    int64_t* pos = nullptr;
    CU(talloc(&keys, K, s));
    CU(talloc(&tmp, K, s));
    if (n_in > 0) k_make_keys<<<grid_for(n_in, B), B, 0, s>>>(d_src, d_dst, n_in, n, nb, keys);
    CU(cudaGetLastError());
    CU(prims::radix_sort_u64(keys, tmp, K, 2 * nb, &sorted, s));
    CU(talloc(&pos, K + 1, s));
    CU(prims::exclusive_scan<int64_t>(UniqueFlag{sorted, sentinel}, K, pos, pos + K, s));
    int64_t two_m = 0;
    CU(cudaMemcpyAsync(&two_m, pos + K, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (two_m / 2 >= (int64_t)INT32_MAX - 1) {
        tfree(keys, s); tfree(tmp, s); tfree(pos, s); tfree(d_flag, s);
        return TRUSS_EOVERFLOW;
    }
    const int64_t m = two_m / 2;
    uint64_t* other = (sorted == keys) ? tmp : keys;  // free half of the ping-pong pair
    U = other;
    if (K > 0) k_compact_unique<<<grid_for(K, B), B, 0, s>>>(sorted, K, sentinel, pos, U);
    CU(cudaGetLastError());
    tfree(pos, s);
    pos = nullptr;

    g->n = n;
    g->m = m;
    g->off64 = ((flags & TRUSS_OFFSETS64) || two_m > (int64_t)INT32_MAX) ? 1 : 0;

    // 3: CSR in input labels
    Csr64 c0;
    TRY(csr_from_keys(U, two_m, n, nb, c0, s));
    Csr64 c1;
    uint64_t* U1 = U;
    const bool locality_order = (flags & TRUSS_LOCALITY_ORDER) && n > 1;
    const bool core_order = (flags & TRUSS_CORE_ORDER) && !locality_order && n > 1;
    const bool relabel = ((flags & TRUSS_DEGREE_ORDER) || core_order || locality_order) && n > 1;
    int32_t* newid = nullptr;
    if (relabel) {
        // 4: rank by (degree, label); a degree is below 2^nb
        uint64_t *dk = nullptr, *dtmp = nullptr, *dsorted = nullptr;
        CU(talloc(&dk, n, s));
        CU(talloc(&dtmp, n, s));
        int key_bits = 2 * nb;
        if (locality_order) {
            TRY(locality_keys(c0, n, nb, dk, s));
        } else if (core_order) {
            int32_t rounds = 0;
            TRY(core_steps(c0, n, nb, dk, &rounds, s));
            int rb = 1;
            while (rb < 31 && (1ll << rb) <= (int64_t)rounds) rb++;
            key_bits = nb + rb;
        } else {
            k_degree_keys<<<grid_for(n, B), B, 0, s>>>(c0.rowptr, n, nb, dk);
        }
        CU(cudaGetLastError());
        CU(prims::radix_sort_u64(dk, dtmp, n, key_bits, &dsorted, s));
        CU(cudaMallocAsync((void**)&g->order, sizeof(int32_t) * (size_t)n, s));
        CU(talloc(&newid, n, s));
        k_order<<<grid_for(n, B), B, 0, s>>>(dsorted, n, mask, g->order, newid);
        CU(cudaGetLastError());
        tfree(dk, s);
        tfree(dtmp, s);
        // pairs in the new labels go to the free half of the key buffers;
        // U is no longer needed afterwards and serves as the sort temp
        k_relabel<<<grid_for(two_m, B), B, 0, s>>>(U, two_m, nb, newid, sorted);
        CU(cudaGetLastError());
        CU(prims::radix_sort_u64(sorted, U, two_m, 2 * nb, &U1, s));
        TRY(csr_from_keys(U1, two_m, n, nb, c1, s));
        tfree(newid, s);
    } else {
        c1 = c0;
    }

    // Eid, El in internal labels
    CU(cudaMallocAsync((void**)&g->col, sizeof(int32_t) * (size_t)(two_m > 0 ? two_m : 1), s));
    CU(cudaMallocAsync((void**)&g->eid, sizeof(int32_t) * (size_t)(two_m > 0 ? two_m : 1), s));
    CU(cudaMallocAsync((void**)&g->el, sizeof(int2) * (size_t)(m > 0 ? m : 1), s));
    CU(cudaMemcpyAsync(g->col, c1.col, sizeof(int32_t) * (size_t)two_m, cudaMemcpyDeviceToDevice, s));
    if (two_m > 0)
        k_eid<<<grid_for(two_m, B), B, 0, s>>>(U1, two_m, nb, c1.rowptr, c1.col, c1.eo, c1.ubase, g->eid, g->el);
    CU(cudaGetLastError());
    if (relabel) {
        CU(cudaMallocAsync((void**)&g->perm, sizeof(int32_t) * (size_t)(m > 0 ? m : 1), s));
        if (m > 0)
            k_perm<<<grid_for(m, B), B, 0, s>>>(g->el, m, g->order, c0.rowptr, c0.col, c0.eo, c0.ubase, g->perm);
        CU(cudaGetLastError());
    }
    // final offsets in the chosen width
    const size_t osz = g->off64 ? sizeof(int64_t) : sizeof(int32_t);
    CU(cudaMallocAsync(&g->rowptr, osz * ((size_t)n + 1), s));
    CU(cudaMallocAsync(&g->eo, osz * ((size_t)n + 1), s));
    if (g->off64) {
        CU(cudaMemcpyAsync(g->rowptr, c1.rowptr, osz * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s));
        CU(cudaMemcpyAsync(g->eo, c1.eo, osz * ((size_t)n), cudaMemcpyDeviceToDevice, s));
    } else {
        k_narrow<int32_t><<<grid_for((int64_t)n + 1, B), B, 0, s>>>(c1.rowptr, (int64_t)n + 1, (int32_t*)g->rowptr);
        if (n > 0) k_narrow<int32_t><<<grid_for(n, B), B, 0, s>>>(c1.eo, n, (int32_t*)g->eo);
        CU(cudaGetLastError());
    }
    // work statistics (reported by truss_decompose)
    {
        unsigned long long* ws = nullptr;
        CU(talloc(&ws, 2, s));
        CU(cudaMemsetAsync(ws, 0, 2 * sizeof(unsigned long long), s));
        k_work_stats<<<grid_for(std::max<int64_t>(n, m), B), B, 0, s>>>(c1.rowptr, c1.eo, n, g->el, m, ws);
        CU(cudaGetLastError());
        unsigned long long h[2];
        CU(cudaMemcpyAsync(h, ws, sizeof(h), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        g->wedges_up = (int64_t)h[0];
        g->dmin_sum = (int64_t)h[1];
        tfree(ws, s);
    }
    // vertex classes for the support kernels
    {
        int32_t *big = nullptr, *huge = nullptr;
        unsigned long long* maxes = nullptr;
        CU(talloc(&big, n, s));
        CU(talloc(&huge, n, s));
        CU(talloc(&maxes, 4, s));
        CU(cudaMemsetAsync(maxes, 0, 4 * sizeof(unsigned long long), s));
        CU(cudaMemsetAsync(d_flag, 0, 4 * sizeof(int), s));
        if (n > 0)
            k_classify_vertices<<<grid_for(n, B), B, 0, s>>>(c1.rowptr, c1.eo, n, big, d_flag, huge, d_flag + 1, maxes);
        CU(cudaGetLastError());
        int h_cnt[2];
        unsigned long long h_max[4];
        CU(cudaMemcpyAsync(h_cnt, d_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(h_max, maxes, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        g->n_sup_big = h_cnt[0];
        g->n_sup_huge = h_cnt[1];
        g->max_deg = (int64_t)h_max[0];
        g->max_updeg = (int64_t)h_max[1];
        g->sup_big_maxup = (int64_t)h_max[2];
        g->sup_big_maxwin = (int64_t)h_max[3];
        CU(cudaMallocAsync((void**)&g->sup_big, sizeof(int32_t) * (size_t)(h_cnt[0] + 1), s));
        CU(cudaMallocAsync((void**)&g->sup_huge, sizeof(int32_t) * (size_t)(h_cnt[1] + 1), s));
        CU(cudaMemcpyAsync(g->sup_big, big, sizeof(int32_t) * (size_t)h_cnt[0], cudaMemcpyDeviceToDevice, s));
        CU(cudaMemcpyAsync(g->sup_huge, huge, sizeof(int32_t) * (size_t)h_cnt[1], cudaMemcpyDeviceToDevice, s));
        tfree(big, s);
        tfree(huge, s);
        tfree(maxes, s);
    }
    if (relabel) free_csr(c1, s);
    free_csr(c0, s);
    tfree(keys, s);
    tfree(tmp, s);
    tfree(d_flag, s);
    CU(cudaStreamSynchronize(s));
    return TRUSS_OK;
}

// canonical edge list: (min, max) of the input labels of internal edge e
__global__ void k_edge_list(const int2* __restrict__ el, int64_t m, const int32_t* __restrict__ order,
                            const int32_t* __restrict__ perm, int32_t* __restrict__ u, int32_t* __restrict__ v) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int2 xy = el[e];
        int32_t p = order ? order[xy.x] : xy.x, q = order ? order[xy.y] : xy.y;
        int64_t c = perm ? perm[e] : e;
        u[c] = min(p, q);
        v[c] = max(p, q);
    }
}

template <typename Off>
__global__ void k_csr_copy(const Off* __restrict__ rowptr, const Off* __restrict__ eo, int32_t n,
                           int64_t* __restrict__ r64, int64_t* __restrict__ eo64) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        if (r64) r64[i] = (int64_t)rowptr[i];
        if (eo64 && i < n) eo64[i] = (int64_t)eo[i];
    }
}

__global__ void k_eid_canon(const int32_t* __restrict__ eid, int64_t len, const int32_t* __restrict__ perm,
                            int32_t* __restrict__ out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = perm ? perm[eid[j]] : eid[j];
}

__global__ void k_iota(int32_t* __restrict__ out, int32_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)i;
}

}  // namespace

void truss_free_device(truss_graph* g) {
    cudaFree(g->rowptr);
    cudaFree(g->eo);
    cudaFree(g->col);
    cudaFree(g->eid);
    cudaFree(g->el);
    cudaFree(g->perm);
    cudaFree(g->order);
    cudaFree(g->sup_big);
    cudaFree(g->sup_huge);
    truss_release_workspace(g);
}

// The library allocates from this process's default stream-ordered pool.
// Its release threshold (default 0) returns freed memory to the driver at
// every synchronisation, so each new graph would map its buffers again; keep
// up to 16 GiB of freed pool memory for reuse instead (truss_pool_keep sets
// another amount).  The attribute belongs to this process's pool and ends
// with it.
static bool g_pool_set[64] = {};

static void keep_pool_memory(int device) {
    if (device < 0 || device >= 64 || g_pool_set[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = (uint64_t)16 << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    g_pool_set[device] = true;
}

extern "C" int truss_pool_keep(int64_t bytes) {
    if (bytes < 0) return TRUSS_EINVAL;
    int device = 0;
    CU(cudaGetDevice(&device));
    cudaMemPool_t pool;
    CU(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t keep = (uint64_t)bytes;
    CU(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    if (bytes == 0) CU(cudaMemPoolTrimTo(pool, 0));
    if (device >= 0 && device < 64) g_pool_set[device] = true;
    return TRUSS_OK;
}

extern "C" int truss_build_csr(const int32_t* d_src, const int32_t* d_dst, int64_t n_in, int32_t n, uint32_t flags,
                               void* stream, truss_graph** out) {
    if (!out) return TRUSS_EINVAL;
    *out = nullptr;
    if (n_in < 0 || n < 0 || (n_in > 0 && (!d_src || !d_dst))) return TRUSS_EINVAL;
    if (n_in > ((int64_t)1 << 31)) return TRUSS_EOVERFLOW;
    cudaStream_t s = (cudaStream_t)stream;
    truss_graph* g = new (std::nothrow) truss_graph();
    if (!g) return TRUSS_ENOMEM;
    CU(cudaGetDevice(&g->device));
    CU(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device));
    keep_pool_memory(g->device);
    int rc = build_impl(d_src, d_dst, n_in, n, flags, s, g);
    if (rc != TRUSS_OK) {
        cudaStreamSynchronize(s);
        truss_free_device(g);
        delete g;
        return rc;
    }
    *out = g;
    return TRUSS_OK;
}

extern "C" void truss_free(truss_graph* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    truss_free_device(g);
    delete g;
}

extern "C" int truss_num_edges(const truss_graph* g, int64_t* m) {
    if (!g || !m) return TRUSS_EINVAL;
    *m = g->m;
    return TRUSS_OK;
}

extern "C" int truss_num_vertices(const truss_graph* g, int32_t* n) {
    if (!g || !n) return TRUSS_EINVAL;
    *n = g->n;
    return TRUSS_OK;
}

extern "C" int truss_edge_list(const truss_graph* g, int32_t* d_u, int32_t* d_v, void* stream) {
    if (!g || (g->m > 0 && (!d_u || !d_v))) return TRUSS_EINVAL;
    if (g->m == 0) return TRUSS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_edge_list<<<grid_for(g->m, 256), 256, 0, s>>>(g->el, g->m, g->order, g->perm, d_u, d_v);
    CU(cudaGetLastError());
    return TRUSS_OK;
}

extern "C" int truss_csr_copy(const truss_graph* g, int64_t* d_rowptr, int32_t* d_col, int32_t* d_eid, int64_t* d_eo,
                              int32_t* d_order, void* stream) {
    if (!g) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t two_m = 2 * g->m;
    if (d_rowptr || d_eo) {
        if (g->off64)
            k_csr_copy<int64_t><<<grid_for((int64_t)g->n + 1, 256), 256, 0, s>>>((const int64_t*)g->rowptr,
                                                                               (const int64_t*)g->eo, g->n, d_rowptr, d_eo);
        else
            k_csr_copy<int32_t><<<grid_for((int64_t)g->n + 1, 256), 256, 0, s>>>((const int32_t*)g->rowptr,
                                                                               (const int32_t*)g->eo, g->n, d_rowptr, d_eo);
    }
    if (d_col && two_m) CU(cudaMemcpyAsync(d_col, g->col, sizeof(int32_t) * (size_t)two_m, cudaMemcpyDeviceToDevice, s));
    if (d_eid && two_m) k_eid_canon<<<grid_for(two_m, 256), 256, 0, s>>>(g->eid, two_m, g->perm, d_eid);
    if (d_order && g->n) {
        if (g->order)
            CU(cudaMemcpyAsync(d_order, g->order, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToDevice, s));
        else
            k_iota<<<grid_for(g->n, 256), 256, 0, s>>>(d_order, g->n);
    }
    CU(cudaGetLastError());
    return TRUSS_OK;
}
