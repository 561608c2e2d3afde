// Asynchronous local truss decomposition: the h-index iteration.
//
// The paper contrasts its level-synchronous peel with local algorithms that
// repeat one update rule at every edge until nothing changes (the MPM-style
// k-core iteration and its nucleus/truss generalisation, §II).  For trusses
// the rule is: given current values tau (upper bounds of the trussness),
//     tau(e) <- 2 + min(tau(e) - 2, h),
//     h = the largest k with at least k triangles {e, e2, e3} of e whose
//         value min(tau(e2), tau(e3)) - 2 is >= k   (an h-index),
// started from tau(e) = S(e) + 2.  Every update keeps tau an upper bound of
// the trussness and never raises it, and a state where no update changes
// anything is the trussness: the same answer as the peel, reached with no
// level or sub-level barriers -- updates happen in place while other edges
// read them (any value read is a valid upper bound), and only edges that
// share a triangle with an edge changed in the previous sweep are evaluated
// again.
//
// A warp takes an edge: it walks the shorter row, searches the longer one
// (hub bitmap or binary search), and adds each triangle's value into a
// per-warp histogram in shared memory (values from min(tau(e) - 2, HB - 1)
// up share the top bucket); a suffix scan from the top gives h.  When the
// top bucket decides (h >= HB - 1 and tau(e) - 2 > HB - 1), h is found by
// binary search over [HB - 1, tau(e) - 2] with one counting walk per step.
#include <algorithm>
#include <climits>

#include "graph.cuh"
#include "rows.cuh"

namespace {

constexpr int LT = 256;     // threads per block
constexpr int LW = LT / 32;
constexpr int HB = 512;     // histogram buckets per warp
constexpr int LBATCH = 8;   // edges a warp takes from the work counter at once

template <typename Off>
Graph<Off> local_view(truss_graph* g) {
    return Graph<Off>{(const Off*)g->rowptr, g->col, g->eid, g->el, g->dmin, (const Off*)g->rows, g->lhub,
                      g->hub_bits, g->hub_words, g->eid, g->ss, g->m, g->hc, g->ocap};
}

// Calls f(e2, e3) for every triangle {e, e2, e3} of the edge whose rows are
// r: lanes take slots a0 + lane, a0 + lane + 32, ... of the shorter row, two
// at a time.  Warp-uniform.
template <typename Off, typename F>
__device__ __forceinline__ void for_triangles(const Graph<Off>& G, const Rows<Off>& r, int lane, F& f) {
    const int32_t* ye = r.hub >= 0 ? G.oeid : G.eid;
    for (Off j = r.a0 + lane; j < r.a1; j += 64) {
        const Off j2 = j + 32;
        const bool two = j2 < r.a1;
        const int32_t w1 = __ldg(G.col + j), x1 = __ldg(G.eid + j);
        const int32_t w2 = two ? __ldg(G.col + j2) : w1, x2 = two ? __ldg(G.eid + j2) : x1;
        Off q1, q2;
        if (r.hub >= 0) {
            q1 = hub_find<Off>(G, r.hub, r.b0, w1);
            q2 = hub_find<Off>(G, r.hub, r.b0, w2);
        } else {
            find2<Off>(G.col, r.b0, r.b1 - r.b0, w1, w2, q1, q2);
        }
        if (q1 >= 0) f(x1, __ldg(ye + q1));
        if (two && q2 >= 0) f(x2, __ldg(ye + q2));
    }
}

// value of a triangle for the h-index: min(tau(e2), tau(e3)) - 2, read
// through L2 (other warps update tau during the sweep)
__device__ __forceinline__ int tri_value(const int32_t* tau, int32_t e2, int32_t e3) {
    return min(__ldcg(tau + e2), __ldcg(tau + e3)) - 2;
}

// values above `top` (= min(tau(e) - 2, HB - 1)) are counted at top
struct HistF {
    int* H;
    const int32_t* tau;
    int top;
    __device__ __forceinline__ void operator()(int32_t e2, int32_t e3) {
        atomicAdd(H + min(tri_value(tau, e2, e3), top), 1);
    }
};

struct CountF {
    const int32_t* tau;
    int k;
    int c;
    __device__ __forceinline__ void operator()(int32_t e2, int32_t e3) { c += tri_value(tau, e2, e3) >= k; }
};

struct MarkF {
    uint8_t* nxt;
    __device__ __forceinline__ void operator()(int32_t e2, int32_t e3) {
        nxt[e2] = 1;
        nxt[e3] = 1;
    }
};

// One sweep over the active edges.  changed[0] counts the edges whose value
// dropped; each of them marks the edges of its triangles active in nxt.
template <typename Off>
__global__ void __launch_bounds__(LT) k_local_sweep(Graph<Off> G, int32_t* tau, const uint8_t* __restrict__ act,
                                                    uint8_t* nxt, unsigned long long* ctr) {
    __shared__ int hist[LW][HB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* H = hist[warp];
    unsigned long long* next = ctr;
    unsigned long long* changed = ctr + 1;
    for (;;) {
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(next, (unsigned long long)LBATCH);
        b0 = __shfl_sync(FULL_MASK, b0, 0);
        if ((int64_t)b0 >= G.m) break;
        const int64_t b1 = min((int64_t)b0 + LBATCH, G.m);
        for (int64_t e = (int64_t)b0; e < b1; e++) {
            if (!act[e]) continue;
            const int cap = __ldcg(tau + e) - 2;
            if (cap <= 0) continue;  // trussness 2 cannot drop
            const Rows<Off> r = rows_of<Off>(G, (int32_t)e);
            const int top = min(cap, HB - 1);
            for (int i = lane; i <= top; i += 32) H[i] = 0;
            __syncwarp();
            HistF hf{H, tau, top};
            for_triangles<Off>(G, r, lane, hf);
            __syncwarp();
            // h = the largest k <= top with #{value >= k} >= k (values above
            // top count as top); scan 32 buckets a round from the top down
            int h = 0, carry = 0;
            for (int base = top; base > 0; base -= 32) {
                const int k = base - lane;
                int c = k > 0 ? H[k] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL_MASK, c, o);
                    if (lane >= o) c += y;
                }
                const bool ok = k > 0 && carry + c >= k;
                const unsigned b = __ballot_sync(FULL_MASK, ok);
                if (b) {
                    h = base - (__ffs(b) - 1);
                    break;
                }
                carry += __shfl_sync(FULL_MASK, c, 31);
            }
            __syncwarp();
            if (h == HB - 1 && cap > HB - 1) {
                // the top bucket decided: binary search for h in [HB-1, cap]
                int lo = HB - 1, hi = cap;
                while (lo < hi) {
                    const int mid = lo + (hi - lo + 1) / 2;
                    CountF cf{tau, mid, 0};
                    for_triangles<Off>(G, r, lane, cf);
                    if (warp_sum(cf.c) >= mid) lo = mid; else hi = mid - 1;
                }
                h = lo;
            }
            if (h < cap) {
                if (lane == 0) {
                    tau[e] = h + 2;
                    atomicAdd(changed, 1ull);
                }
                MarkF mf{nxt};
                for_triangles<Off>(G, r, lane, mf);
            }
        }
    }
}

__global__ void k_local_init(const int2* __restrict__ ss, int64_t m, int32_t* __restrict__ tau,
                             uint8_t* __restrict__ act) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        tau[e] = ss[e].x + 2;
        act[e] = 1;
    }
}

__global__ void k_local_out(const int32_t* __restrict__ tau, int64_t m, const int32_t* __restrict__ perm,
                            int32_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[perm ? perm[e] : e] = tau[e];
}

template <typename Off>
int local_impl(truss_graph* g, int32_t* d_truss, int64_t max_sweeps, int64_t* h_sweeps, int64_t* h_updates,
               cudaStream_t s) {
    const int64_t m = g->m;
    int32_t* tau = nullptr;
    uint8_t* flags = nullptr;
    unsigned long long* ctr = nullptr;
    int rc = TRUSS_OK;
    auto done = [&](int r) {
        cudaStreamSynchronize(s);
        cudaFree(tau);
        cudaFree(flags);
        cudaFree(ctr);
        return r;
    };
#define LCU(call)                                                               \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            truss_note_cuda_error(e_);                                          \
            return done(e_ == cudaErrorMemoryAllocation ? TRUSS_ENOMEM : TRUSS_ECUDA); \
        }                                                                       \
    } while (0)
    LCU(cudaMalloc((void**)&tau, sizeof(int32_t) * (size_t)m));
    LCU(cudaMalloc((void**)&flags, 2 * (size_t)m));
    LCU(cudaMalloc((void**)&ctr, 2 * sizeof(unsigned long long)));
    rc = truss_support_internal(g, g->ss, s);
    if (rc != TRUSS_OK) return done(rc);
    uint8_t* act = flags;
    uint8_t* nxt = flags + m;
    k_local_init<<<grid_for(m, 256), 256, 0, s>>>(g->ss, m, tau, act);
    LCU(cudaGetLastError());
    truss_note_launch();
    int per_sm = 0;
    LCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_local_sweep<Off>, LT, 0));
    const int blocks = std::max(1, per_sm) * g->sms;
    const Graph<Off> G = local_view<Off>(g);
    int64_t sweeps = 0, updates = 0;
    unsigned long long h[2] = {0, 0};
    for (;;) {
        if (max_sweeps > 0 && sweeps >= max_sweeps) {
            rc = TRUSS_ETIMEOUT;  // not converged within the allowed sweeps
            break;
        }
        LCU(cudaMemsetAsync(nxt, 0, (size_t)m, s));
        LCU(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), s));
        k_local_sweep<Off><<<blocks, LT, 0, s>>>(G, tau, act, nxt, ctr);
        LCU(cudaGetLastError());
        truss_note_launch();
        LCU(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
        LCU(cudaStreamSynchronize(s));
        sweeps++;
        updates += (int64_t)h[1];
        if (h[1] == 0) break;
        std::swap(act, nxt);
    }
    if (rc == TRUSS_OK) {
        k_local_out<<<grid_for(m, 256), 256, 0, s>>>(tau, m, g->perm, d_truss);
        LCU(cudaGetLastError());
        truss_note_launch();
    }
    if (h_sweeps) *h_sweeps = sweeps;
    if (h_updates) *h_updates = updates;
    return done(rc);
#undef LCU
}

}  // namespace

extern "C" int truss_decompose_local(truss_graph* g, int32_t* d_truss, int64_t max_sweeps, int64_t* h_sweeps,
                                     int64_t* h_updates, void* stream) {
    if (!g || (g->m > 0 && !d_truss)) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    TRY(truss_ensure_workspace(g, s));
    if (h_sweeps) *h_sweeps = 0;
    if (h_updates) *h_updates = 0;
    if (g->m == 0) return TRUSS_OK;
    return g->off64 ? local_impl<int64_t>(g, d_truss, max_sweeps, h_sweeps, h_updates, s)
                    : local_impl<int32_t>(g, d_truss, max_sweeps, h_sweeps, h_updates, s);
}
