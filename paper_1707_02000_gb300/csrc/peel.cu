// Level-synchronous peeling (Algorithms 4 and 5, §III) on the device.
//
// Scan (K2): one coalesced pass over the {S, stamp} words, 16 bytes (two
// edges) per thread per step; edges with S = l join curr (warp ballot +
// one atomic per warp), and the minimum support above l is reduced on the
// side so that an empty level can jump straight to the next live one.
//
// ProcessSubLevel (K3): for every e1 = {u, v} in curr, the common
// neighbours w of u and v are found by binary search of each entry of the
// shorter row in the longer one.  Each triangle {e1, e2, e3} whose other two
// edges are unprocessed lowers e2 (resp. e3) by one when its support is
// above l and e3 (resp. e2) is not in curr or has a larger id than e1: the
// two-sided reading of Algorithm 5, which prints only the e2 case.  The
// decrement is atomicSub; an edge whose old value was l+1 joins next; a
// thread that pushed an edge below l adds the 1 back (the clamp-and-restore
// of Algorithm 5), so the final value is max(l, S - #triangles removed).
// The rule is symmetric in e2 and e3, so which of them is {u,w} or {v,w}
// does not matter.
//
// Three ways to map a frontier edge onto the GPU, all exact:
//   thread  one thread walks the shorter row (short rows),
//   warp    32 lanes split the shorter row (the common case),
//   block   the whole block splits it (hubs).
// The default picks per edge by the length of the shorter row.
//
// Loop forms: PLAIN launches Scan / ProcessSubLevel from the host and reads
// the frontier size back after every phase (the direct transcription of
// Algorithm 4's loop); PERSISTENT runs the whole loop in one cooperative
// kernel whose phases are separated by a grid barrier with a time limit.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "graph.cuh"

namespace {

enum {
    C_CNT = 0,   // [0..3] frontier size produced by phase p, slot p & 3
    C_MIN = 4,   // [4..7] minimum live support above l found by phase p, slot p & 3
    C_BAR_COUNT = 8,
    C_BAR_GEN = 9,
    C_ERR = 10,
    C_NSUB = 11,
    C_NSCAN = 12,
    C_NLEVEL = 13,
    C_LAST_L = 14,
    C_TRI_LO = 16,  // triangle count (int64 at 16..17)
    C_TOTAL = 32
};

constexpr int PT = 256;              // threads per block in the peel kernels
constexpr int APPEND_CAP = 2048;     // per-block staging for next-frontier appends

struct PeelSmem {
    int32_t buf[APPEND_CAP];
    int bufcnt;
    int qcnt;
    int base;
    int32_t q[PT][3];  // block-path queue: e1, shorter endpoint a, other b
};

template <typename Off>
struct Graph {
    const Off* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const int32_t* __restrict__ eid;
    const int2* __restrict__ el;
    int2* ss;
    int64_t m;
};

// Block-staged append to the next frontier: shared-memory slot first, the
// global list directly when the staging buffer is full.
struct Appender {
    PeelSmem* sm;
    int32_t* out;
    int* count;
    __device__ __forceinline__ void push(int32_t f) const {
        int p = atomicAdd(&sm->bufcnt, 1);
        if (p < APPEND_CAP) {
            sm->buf[p] = f;
        } else {
            int q = atomicAdd(count, 1);
            out[q] = f;
        }
    }
    // whole block; ends with the buffer empty
    __device__ __forceinline__ void flush() const {
        __syncthreads();
        int k = min(sm->bufcnt, APPEND_CAP);
        if (threadIdx.x == 0) sm->base = k ? atomicAdd(count, k) : 0;
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += blockDim.x) out[sm->base + i] = sm->buf[i];
        __syncthreads();
        if (threadIdx.x == 0) sm->bufcnt = 0;
        __syncthreads();
    }
};

__device__ __forceinline__ void relax(int2* ss, int32_t f, int32_t l, int32_t g, const Appender& ap) {
    int a = atomicSub(&ss[f].x, 1);
    if (a == l + 1) {
        ss[f].y = g + 1;  // f enters the next sub-level
        ap.push(f);
    } else if (a <= l) {
        atomicAdd(&ss[f].x, 1);  // pushed below l by a racing thread: restore
    }
}

// Triangle {e1, x, y} seen while processing e1 in sub-level g at level l.
__device__ __forceinline__ void on_triangle(int2* ss, int32_t e1, int32_t x, int32_t y, int32_t l, int32_t g,
                                            const Appender& ap) {
    int2 sx = __ldcg(ss + x);
    int2 sy = __ldcg(ss + y);
    if (sx.y < g || sy.y < g) return;  // an edge of it is processed: the triangle is gone
    const bool inx = sx.y == g, iny = sy.y == g;
    if (sx.x > l && (!iny || e1 < y)) relax(ss, x, l, g, ap);
    if (sy.x > l && (!inx || e1 < x)) relax(ss, y, l, g, ap);
}

// All triangles through e1 whose apex comes from slots j = start, start+step,
// ... of the shorter row [a0, a1), probed in the longer row [b0, b1).
template <typename Off>
__device__ __forceinline__ void walk_rows(const Graph<Off>& G, int32_t e1, Off a0, Off a1, Off b0, Off b1, int start,
                                          int step, int32_t l, int32_t g, const Appender& ap) {
    for (Off j = a0 + start; j < a1; j += step) {
        int32_t w = __ldg(G.col + j);
        Off q = find_dev<Off>(G.col, b0, b1, w);
        if (q >= 0) on_triangle(G.ss, e1, __ldg(G.eid + j), __ldg(G.eid + q), l, g, ap);
    }
}

// One frontier, all blocks of the grid.  Blocks take tiles of PT frontier
// edges in turn; inside a tile each edge goes to the thread, warp or block
// path.  The per-block trip count is uniform, so __syncthreads is safe.
template <typename Off>
__device__ void process_frontier(const Graph<Off>& G, const int32_t* curr, int ncurr, int32_t l, int32_t g,
                                 int32_t* next, int* next_count, int variant, int thr_thread, int thr_block,
                                 PeelSmem* sm) {
    const int lane = threadIdx.x & 31;
    const Appender ap{sm, next, next_count};
    const int ntiles = (ncurr + PT - 1) / PT;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int i = t * PT + threadIdx.x;
        int cls = -1;
        int32_t e1 = 0, a = 0, b = 0;
        Off a0 = 0, a1 = 0, b0 = 0, b1 = 0;
        if (i < ncurr) {
            e1 = __ldcg(curr + i);
            int2 uv = __ldg(G.el + e1);
            Off u0 = __ldg(G.rowptr + uv.x), u1 = __ldg(G.rowptr + uv.x + 1);
            Off v0 = __ldg(G.rowptr + uv.y), v1 = __ldg(G.rowptr + uv.y + 1);
            if (u1 - u0 <= v1 - v0) {
                a = uv.x; b = uv.y; a0 = u0; a1 = u1; b0 = v0; b1 = v1;
            } else {
                a = uv.y; b = uv.x; a0 = v0; a1 = v1; b0 = u0; b1 = u1;
            }
            const int64_t da = (int64_t)(a1 - a0);
            cls = variant >= 0 ? variant : (da <= thr_thread ? 0 : (da <= thr_block ? 1 : 2));
        }
        // thread path
        if (cls == 0) walk_rows<Off>(G, e1, a0, a1, b0, b1, 0, 1, l, g, ap);
        // warp path: the warp serves its warp-class lanes one after another
        unsigned wm = __ballot_sync(FULL_MASK, cls == 1);
        while (wm) {
            const int src = __ffs(wm) - 1;
            wm &= wm - 1;
            int32_t e = __shfl_sync(FULL_MASK, e1, src);
            Off x0 = __shfl_sync(FULL_MASK, a0, src), x1 = __shfl_sync(FULL_MASK, a1, src);
            Off y0 = __shfl_sync(FULL_MASK, b0, src), y1 = __shfl_sync(FULL_MASK, b1, src);
            walk_rows<Off>(G, e, x0, x1, y0, y1, lane, 32, l, g, ap);
        }
        // block path: queue, then the whole block per queued edge
        if (cls == 2) {
            int p = atomicAdd(&sm->qcnt, 1);
            sm->q[p][0] = e1;
            sm->q[p][1] = a;
            sm->q[p][2] = b;
        }
        __syncthreads();
        const int nq = sm->qcnt;
        for (int k = 0; k < nq; k++) {
            const int32_t e = sm->q[k][0], x = sm->q[k][1], y = sm->q[k][2];
            walk_rows<Off>(G, e, __ldg(G.rowptr + x), __ldg(G.rowptr + x + 1), __ldg(G.rowptr + y),
                           __ldg(G.rowptr + y + 1), threadIdx.x, PT, l, g, ap);
        }
        __syncthreads();
        if (threadIdx.x == 0) sm->qcnt = 0;
        ap.flush();
    }
}

// Scan at level l: curr <- {e : S[e] = l}, their stamps <- g; *minslot <-
// min(*minslot, min{S[e] : S[e] > l}).  Two edges per 16-byte load.
__device__ void scan_level(int2* ss, int64_t m, int32_t l, int32_t g, int32_t* curr, int* count, int* minslot) {
    const int64_t npair = (m + 1) / 2;
    const int4* ss4 = reinterpret_cast<const int4*>(ss);
    int mn = INT_MAX;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npair; base += stride) {
        const int64_t p = base + threadIdx.x;
        int s0 = INT_MIN, s1 = INT_MIN;
        if (p < npair) {
            if (2 * p + 1 < m) {
                int4 v = __ldcg(ss4 + p);
                s0 = v.x;
                s1 = v.z;
            } else {
                s0 = __ldcg(ss + 2 * p).x;
            }
        }
        const bool h0 = s0 == l, h1 = s1 == l;
        if (h0) ss[2 * p].y = g;
        if (h1) ss[2 * p + 1].y = g;
        if (s0 > l) mn = min(mn, s0);
        if (s1 > l) mn = min(mn, s1);
        warp_append(h0, (int32_t)(2 * p), curr, count);
        warp_append(h1, (int32_t)(2 * p + 1), curr, count);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(FULL_MASK, mn, o));
    if (lane_id() == 0 && mn != INT_MAX) atomicMin(minslot, mn);
}

// ------------------------------------------------------- standalone kernels

__global__ void __launch_bounds__(PT) k_scan(int2* ss, int64_t m, int32_t l, int32_t g, int32_t* curr, int* count,
                                              int* minslot) {
    scan_level(ss, m, l, g, curr, count, minslot);
}

template <typename Off>
__global__ void __launch_bounds__(PT) k_process(Graph<Off> G, const int32_t* curr, int ncurr, int32_t l, int32_t g,
                                                int32_t* next, int* next_count, int variant, int thr_thread,
                                                int thr_block) {
    __shared__ PeelSmem sm;
    if (threadIdx.x == 0) {
        sm.bufcnt = 0;
        sm.qcnt = 0;
    }
    __syncthreads();
    process_frontier<Off>(G, curr, ncurr, l, g, next, next_count, variant, thr_thread, thr_block, &sm);
}

// ------------------------------------------------------------ grid barrier

// Sense-free generation barrier over all blocks of a cooperative launch.
// Every wait is bounded: past timeout_ns the block records TRUSS_ETIMEOUT
// and returns false; a block that sees an error recorded also returns false.
__device__ bool grid_barrier(int* ctr, unsigned nblocks, uint64_t timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* count = reinterpret_cast<unsigned*>(ctr + C_BAR_COUNT);
        unsigned* gen = reinterpret_cast<unsigned*>(ctr + C_BAR_GEN);
        int ok = 1;
        const unsigned my_gen = ld_acquire_gpu_u32(gen);
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            st_release_gpu_u32(gen, my_gen + 1);
        } else {
            const uint64_t t0 = global_ns();
            while (ld_acquire_gpu_u32(gen) == my_gen) {
                if (ld_acquire_gpu(ctr + C_ERR) != 0) { ok = 0; break; }
                if (global_ns() - t0 > timeout_ns) {
                    atomicCAS(ctr + C_ERR, 0, TRUSS_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok && ld_acquire_gpu(ctr + C_ERR) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole of Algorithm 4 in one cooperative launch.  Every thread follows
// the same (l, g, scan#) sequence because every branch depends only on
// counters read after a barrier.
template <typename Off>
__global__ void __launch_bounds__(PT)
    k_persistent(Graph<Off> G, int32_t* fr0, int32_t* fr1, int* ctr, int variant, int thr_thread, int thr_block,
                 int level_jump, uint64_t timeout_ns, int32_t* rec_level, int64_t* rec_size, int64_t max_rec) {
    __shared__ PeelSmem sm;
    if (threadIdx.x == 0) {
        sm.bufcnt = 0;
        sm.qcnt = 0;
    }
    __syncthreads();
    const unsigned nblocks = gridDim.x;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    // Phase p (every Scan and every sub-level is one phase) writes its
    // counters to slot p & 3.  Slot (p+2) & 3 is cleared during phase p: its
    // last readers read it right after the barrier that ended phase p-2, and
    // the barrier ending phase p-1 lies in between.
    int32_t l = 0, g = 0;
    int64_t processed = 0, nsub = 0, sc = 0, nlevel = 0, p = 0;
    while (processed < G.m) {
        if (leader) {
            ctr[C_CNT + ((p + 2) & 3)] = 0;
            ctr[C_MIN + ((p + 2) & 3)] = INT_MAX;
        }
        int32_t* curr = (g & 1) ? fr1 : fr0;
        scan_level(G.ss, G.m, l, g, curr, ctr + C_CNT + (p & 3), ctr + C_MIN + (p & 3));
        if (!grid_barrier(ctr, nblocks, timeout_ns)) return;
        int c = ld_acquire_gpu(ctr + C_CNT + (p & 3));
        const int mn = ld_acquire_gpu(ctr + C_MIN + (p & 3));
        p++;
        sc++;
        if (c == 0) {
            if (mn == INT_MAX) break;
            l = level_jump ? mn : l + 1;
            continue;
        }
        nlevel++;
        while (c > 0) {
            processed += c;
            if (leader) {
                if (nsub < max_rec) {
                    rec_level[nsub] = l;
                    rec_size[nsub] = c;
                }
                ctr[C_CNT + ((p + 2) & 3)] = 0;
                ctr[C_MIN + ((p + 2) & 3)] = INT_MAX;
            }
            int32_t* cu = (g & 1) ? fr1 : fr0;
            int32_t* nx = (g & 1) ? fr0 : fr1;
            process_frontier<Off>(G, cu, c, l, g, nx, ctr + C_CNT + (p & 3), variant, thr_thread, thr_block, &sm);
            if (!grid_barrier(ctr, nblocks, timeout_ns)) return;
            c = ld_acquire_gpu(ctr + C_CNT + (p & 3));
            p++;
            g++;
            nsub++;
        }
        l++;
    }
    if (leader) {
        ctr[C_NSUB] = (int)nsub;
        ctr[C_NSCAN] = (int)sc;
        ctr[C_NLEVEL] = (int)nlevel;
        ctr[C_LAST_L] = l;
    }
}

// --------------------------------------------------------------- helpers

__global__ void k_truss_out(const int2* __restrict__ ss, int64_t m, const int32_t* __restrict__ perm,
                            int32_t* __restrict__ out, int add) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[perm ? perm[e] : e] = ss[e].x + add;
}

__global__ void k_sum_support(const int2* __restrict__ ss, int64_t m, unsigned long long* out, int* smax) {
    unsigned long long s = 0;
    int mx = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int v = ss[e].x;
        s += (unsigned long long)v;
        mx = max(mx, v);
    }
    s = warp_sum(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
    if (lane_id() == 0) {
        atomicAdd(out, s);
        atomicMax(smax, mx);
    }
}

__global__ void k_init_counters(int* ctr) {
    int i = threadIdx.x;
    if (i < C_TOTAL) ctr[i] = (i >= C_MIN && i < C_MIN + 4) ? INT_MAX : 0;
}

// state import for truss_peel_sublevel: canonical (S, flags) -> internal ss
__global__ void k_import_state(const int32_t* __restrict__ S, const uint8_t* __restrict__ flags,
                               const int32_t* __restrict__ perm, int64_t m, int2* __restrict__ ss) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = perm ? perm[e] : e;
        uint8_t f = flags[c];
        // sub-level number 1: processed -> stamp 0, in curr -> 1, else none
        int st = (f & 1) ? 0 : ((f & 2) ? 1 : TRUSS_STAMP_NONE);
        ss[e] = make_int2(S[c], st);
    }
}

__global__ void k_export_state(const int2* __restrict__ ss, const int32_t* __restrict__ perm, int64_t m,
                               int32_t* __restrict__ S, uint8_t* __restrict__ flags) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = perm ? perm[e] : e;
        int2 v = ss[e];
        S[c] = v.x;
        flags[c] = (uint8_t)((v.y < 2 ? 1 : 0) | (v.y == 2 ? 2 : 0));
    }
}

__global__ void k_mark_curr(const int32_t* __restrict__ curr, int64_t k, int2* __restrict__ ss) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        ss[curr[i]].y = 1;
}

__global__ void k_inverse_perm(const int32_t* __restrict__ perm, int64_t m, int32_t* __restrict__ inv) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        inv[perm[e]] = (int32_t)e;
}

__global__ void k_map_ids(const int32_t* __restrict__ in, int64_t k, const int32_t* __restrict__ map,
                          int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = map ? map[in[i]] : in[i];
}

// heuristic split of frontier edges by the length of the shorter row
constexpr int THR_THREAD = 8;
constexpr int THR_BLOCK = 2048;

template <typename Off>
int process_blocks(const truss_graph* g) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_process<Off>, PT, 0);
    return std::max(1, per_sm) * g->sms;
}

template <typename Off>
Graph<Off> graph_view(truss_graph* g) {
    return Graph<Off>{(const Off*)g->rowptr, g->col, g->eid, g->el, g->ss, g->m};
}

struct RunOut {
    int64_t nsub = 0, nscan = 0, nlevel = 0;
    int32_t last_l = 0;
};

// Algorithm 4's loop driven from the host: one Scan launch per level, one
// ProcessSubLevel launch per sub-level, the frontier size read back after each.
template <typename Off>
int run_plain(truss_graph* g, const truss_opts& o, cudaStream_t s, std::vector<int32_t>* rl,
              std::vector<int64_t>* rs, RunOut* out) {
    Graph<Off> G = graph_view<Off>(g);
    int* ctr = g->ctr;
    int* h = g->h_ctr;
    const int sblocks = grid_for((g->m + 1) / 2, PT, (int64_t)g->sms * 8);
    const int pmax = process_blocks<Off>(g);
    int32_t l = 0, gs = 0;
    int64_t processed = 0;
    while (processed < g->m) {
        // counters: [0] curr size, [4] min above
        k_init_counters<<<1, 32, 0, s>>>(ctr);
        k_scan<<<sblocks, PT, 0, s>>>(g->ss, g->m, l, gs, g->fr[gs & 1], ctr + C_CNT, ctr + C_MIN);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(h, ctr, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        out->nscan++;
        int c = h[C_CNT];
        if (c == 0) {
            if (h[C_MIN] == INT_MAX) break;
            l = o.level_jump ? h[C_MIN] : l + 1;
            continue;
        }
        out->nlevel++;
        while (c > 0) {
            processed += c;
            if (rl) {
                rl->push_back(l);
                rs->push_back(c);
            }
            CU(cudaMemsetAsync(ctr + C_CNT + 1, 0, sizeof(int), s));
            const int blocks = std::min(pmax, (c + PT - 1) / PT);
            k_process<Off><<<blocks, PT, 0, s>>>(G, g->fr[gs & 1], c, l, gs, g->fr[(gs + 1) & 1], ctr + C_CNT + 1,
                                                 o.variant, THR_THREAD, THR_BLOCK);
            CU(cudaGetLastError());
            CU(cudaMemcpyAsync(h + 1, ctr + C_CNT + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            c = h[1];
            gs++;
            out->nsub++;
        }
        l++;
    }
    out->last_l = l;
    return TRUSS_OK;
}

template <typename Off>
int run_persistent(truss_graph* g, const truss_opts& o, cudaStream_t s, int32_t* d_rl, int64_t* d_rs, int64_t max_rec) {
    Graph<Off> G = graph_view<Off>(g);
    int per_sm = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<Off>, PT, 0));
    if (per_sm < 1) return TRUSS_ENOTSUP;
    int blocks = per_sm * g->sms;
    k_init_counters<<<1, 32, 0, s>>>(g->ctr);
    CU(cudaGetLastError());
    int variant = o.variant;
    int thr_t = THR_THREAD, thr_b = THR_BLOCK, jump = o.level_jump;
    uint64_t tmo = o.timeout_ns > 0 ? (uint64_t)o.timeout_ns : 10000000000ull;
    int32_t* fr0 = g->fr[0];
    int32_t* fr1 = g->fr[1];
    int* ctr = g->ctr;
    void* args[] = {&G, &fr0, &fr1, &ctr, &variant, &thr_t, &thr_b, &jump, &tmo, &d_rl, &d_rs, &max_rec};
    CU(cudaLaunchCooperativeKernel((const void*)k_persistent<Off>, dim3(blocks), dim3(PT), args, 0, s));
    return TRUSS_OK;
}

int check_opts(const truss_opts& o) {
    if (o.loop != TRUSS_LOOP_PLAIN && o.loop != TRUSS_LOOP_PERSISTENT) return TRUSS_EINVAL;
    if (o.variant < TRUSS_VAR_AUTO || o.variant > TRUSS_VAR_BLOCK) return TRUSS_EINVAL;
    if ((o.h_sub_level || o.h_sub_size) && (!o.h_sub_level || !o.h_sub_size || o.max_sub < 0 || !o.sync))
        return TRUSS_EINVAL;
    return TRUSS_OK;
}

template <typename Off>
int decompose_impl(truss_graph* g, int32_t* d_truss, const truss_opts& o, truss_stats* st, cudaStream_t s) {
    TRY(truss_ensure_workspace(g));
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    const bool timed = o.sync && st;
    if (timed)
        for (auto& e : ev) CU(cudaEventCreate(&e));
    if (timed) CU(cudaEventRecord(ev[0], s));
    TRY(truss_support_internal(g, g->ss, s));
    unsigned long long* d_tri = reinterpret_cast<unsigned long long*>(g->ctr + C_TRI_LO);
    if (st) {
        CU(cudaMemsetAsync(g->ctr + C_TRI_LO, 0, 4 * sizeof(int), s));
        k_sum_support<<<grid_for(g->m, 256, (int64_t)g->sms * 4), 256, 0, s>>>(g->ss, g->m, d_tri, g->ctr + C_TRI_LO + 2);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(g->h_ctr + C_TRI_LO, g->ctr + C_TRI_LO, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    if (timed) CU(cudaEventRecord(ev[1], s));
    RunOut ro;
    std::vector<int32_t> rl;
    std::vector<int64_t> rs;
    const bool rec = o.h_sub_level && o.max_sub > 0;
    if (o.loop == TRUSS_LOOP_PLAIN) {
        TRY(run_plain<Off>(g, o, s, rec ? &rl : nullptr, rec ? &rs : nullptr, &ro));
    } else {
        int32_t* d_rl = nullptr;
        int64_t* d_rs = nullptr;
        if (rec) {
            CU(cudaMallocAsync((void**)&d_rl, sizeof(int32_t) * (size_t)o.max_sub, s));
            CU(cudaMallocAsync((void**)&d_rs, sizeof(int64_t) * (size_t)o.max_sub, s));
        }
        int rc = run_persistent<Off>(g, o, s, d_rl, d_rs, rec ? o.max_sub : 0);
        if (rc == TRUSS_OK && o.sync) {
            CU(cudaMemcpyAsync(g->h_ctr, g->ctr, sizeof(int) * C_TRI_LO, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            if (g->h_ctr[C_ERR]) rc = g->h_ctr[C_ERR];
            ro.nsub = g->h_ctr[C_NSUB];
            ro.nscan = g->h_ctr[C_NSCAN];
            ro.nlevel = g->h_ctr[C_NLEVEL];
            ro.last_l = g->h_ctr[C_LAST_L];
            if (rec && rc == TRUSS_OK) {
                int64_t k = std::min<int64_t>(ro.nsub, o.max_sub);
                CU(cudaMemcpyAsync(o.h_sub_level, d_rl, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, s));
                CU(cudaMemcpyAsync(o.h_sub_size, d_rs, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost, s));
            }
        }
        if (d_rl) cudaFreeAsync(d_rl, s);
        if (d_rs) cudaFreeAsync(d_rs, s);
        if (rc != TRUSS_OK) {
            if (timed)
                for (auto& e : ev) cudaEventDestroy(e);
            return rc;
        }
    }
    if (timed) CU(cudaEventRecord(ev[2], s));
    if (g->m > 0) k_truss_out<<<grid_for(g->m, 256), 256, 0, s>>>(g->ss, g->m, g->perm, d_truss, 2);
    CU(cudaGetLastError());
    if (o.sync) {
        CU(cudaStreamSynchronize(s));
        if (rec && o.loop == TRUSS_LOOP_PLAIN) {
            int64_t k = std::min<int64_t>((int64_t)rl.size(), o.max_sub);
            std::copy(rl.begin(), rl.begin() + k, o.h_sub_level);
            std::copy(rs.begin(), rs.begin() + k, o.h_sub_size);
        }
    }
    if (st) {
        memset(st, 0, sizeof(*st));
        st->m = g->m;
        st->sublevels = ro.nsub;
        st->scans = ro.nscan;
        st->levels = (int32_t)ro.nlevel;
        if (o.sync) {
            unsigned long long tri = 0;
            memcpy(&tri, g->h_ctr + C_TRI_LO, sizeof(tri));
            st->triangles = (int64_t)(tri / 3);
            // largest level that held edges: the last l before the loop ended
            st->t_max = g->m > 0 ? ro.last_l - 1 + 2 : 0;
        }
        if (timed) {
            cudaEventElapsedTime(&st->ms_support, ev[0], ev[1]);
            cudaEventElapsedTime(&st->ms_peel, ev[1], ev[2]);
        }
    }
    if (timed)
        for (auto& e : ev) cudaEventDestroy(e);
    return TRUSS_OK;
}

template <typename Off>
int peel_sublevel_impl(truss_graph* g, int32_t* d_S, uint8_t* d_flags, const int32_t* d_curr, int64_t ncurr,
                       int32_t l, int32_t* d_next, int64_t* h_nnext, int32_t variant, cudaStream_t s) {
    TRY(truss_ensure_workspace(g));
    const int64_t m = g->m;
    int32_t* inv = nullptr;
    if (g->perm) {
        CU(cudaMallocAsync((void**)&inv, sizeof(int32_t) * (size_t)m, s));
        k_inverse_perm<<<grid_for(m, 256), 256, 0, s>>>(g->perm, m, inv);
    }
    k_import_state<<<grid_for(m, 256), 256, 0, s>>>(d_S, d_flags, g->perm, m, g->ss);
    if (ncurr > 0) {
        k_map_ids<<<grid_for(ncurr, 256), 256, 0, s>>>(d_curr, ncurr, inv, g->fr[0]);
        k_mark_curr<<<grid_for(ncurr, 256), 256, 0, s>>>(g->fr[0], ncurr, g->ss);
    }
    CU(cudaMemsetAsync(g->ctr, 0, sizeof(int) * 2, s));
    CU(cudaGetLastError());
    if (ncurr > 0) {
        Graph<Off> G = graph_view<Off>(g);
        const int blocks = std::min<int64_t>(process_blocks<Off>(g), (ncurr + PT - 1) / PT);
        k_process<Off><<<blocks, PT, 0, s>>>(G, g->fr[0], (int)ncurr, l, 1, g->fr[1], g->ctr + 1, variant, THR_THREAD,
                                             THR_BLOCK);
        CU(cudaGetLastError());
    }
    int nn = 0;
    CU(cudaMemcpyAsync(&nn, g->ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (nn > 0) k_map_ids<<<grid_for(nn, 256), 256, 0, s>>>(g->fr[1], nn, g->perm, d_next);
    k_export_state<<<grid_for(m, 256), 256, 0, s>>>(g->ss, g->perm, m, d_S, d_flags);
    CU(cudaGetLastError());
    if (inv) cudaFreeAsync(inv, s);
    CU(cudaStreamSynchronize(s));
    *h_nnext = nn;
    return TRUSS_OK;
}

}  // namespace

int truss_ensure_workspace(truss_graph* g) {
    if (g->ctr) return TRUSS_OK;
    const size_t m = (size_t)(g->m > 0 ? g->m : 1);
    CU(cudaMalloc((void**)&g->ss, sizeof(int2) * (m + 1)));
    CU(cudaMalloc((void**)&g->fr[0], sizeof(int32_t) * m));
    CU(cudaMalloc((void**)&g->fr[1], sizeof(int32_t) * m));
    CU(cudaMalloc((void**)&g->ctr, sizeof(int) * C_TOTAL));
    CU(cudaMallocHost((void**)&g->h_ctr, sizeof(int) * C_TOTAL));
    return TRUSS_OK;
}

void truss_release_workspace(truss_graph* g) {
    cudaFree(g->ss);
    cudaFree(g->fr[0]);
    cudaFree(g->fr[1]);
    cudaFree(g->ctr);
    cudaFreeHost(g->h_ctr);
    g->ss = nullptr;
    g->fr[0] = g->fr[1] = nullptr;
    g->ctr = nullptr;
    g->h_ctr = nullptr;
}

extern "C" void truss_default_opts(truss_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->loop = TRUSS_LOOP_PERSISTENT;
    o->variant = TRUSS_VAR_AUTO;
    o->sync = 0;
    o->level_jump = 1;
    o->timeout_ns = 10000000000ll;
}

extern "C" int truss_support(truss_graph* g, int32_t* d_support, void* stream) {
    if (!g || (g->m > 0 && !d_support)) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    TRY(truss_ensure_workspace(g));
    TRY(truss_support_internal(g, g->ss, s));
    if (g->m > 0) k_truss_out<<<grid_for(g->m, 256), 256, 0, s>>>(g->ss, g->m, g->perm, d_support, 0);
    CU(cudaGetLastError());
    return TRUSS_OK;
}

extern "C" int truss_decompose(truss_graph* g, int32_t* d_truss, const truss_opts* opts, truss_stats* stats,
                               void* stream) {
    if (!g || (g->m > 0 && !d_truss)) return TRUSS_EINVAL;
    truss_opts o;
    if (opts)
        o = *opts;
    else
        truss_default_opts(&o);
    TRY(check_opts(o));
    if (g->latched) {
        int e = g->latched;
        g->latched = 0;
        return e;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (g->m == 0) {
        if (stats) {
            memset(stats, 0, sizeof(*stats));
        }
        return TRUSS_OK;
    }
    return g->off64 ? decompose_impl<int64_t>(g, d_truss, o, stats, s) : decompose_impl<int32_t>(g, d_truss, o, stats, s);
}

extern "C" int truss_sync(truss_graph* g, void* stream) {
    if (!g) return TRUSS_EINVAL;
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    int e = g->latched;
    if (g->ctr) {
        int err = 0;
        CU(cudaMemcpy(&err, g->ctr + C_ERR, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) {
            e = err;
            int zero = 0;
            CU(cudaMemcpy(g->ctr + C_ERR, &zero, sizeof(int), cudaMemcpyHostToDevice));
        }
    }
    g->latched = 0;
    return e;
}

extern "C" int truss_peel_sublevel(truss_graph* g, int32_t* d_S, uint8_t* d_flags, const int32_t* d_curr,
                                   int64_t ncurr, int32_t l, int32_t* d_next, int64_t* h_nnext, int32_t variant,
                                   void* stream) {
    if (!g || !h_nnext || ncurr < 0 || ncurr > g->m || variant < TRUSS_VAR_AUTO || variant > TRUSS_VAR_BLOCK)
        return TRUSS_EINVAL;
    if (g->m > 0 && (!d_S || !d_flags || !d_next)) return TRUSS_EINVAL;
    if (ncurr > 0 && !d_curr) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->m == 0) {
        *h_nnext = 0;
        return TRUSS_OK;
    }
    return g->off64 ? peel_sublevel_impl<int64_t>(g, d_S, d_flags, d_curr, ncurr, l, d_next, h_nnext, variant, s)
                    : peel_sublevel_impl<int32_t>(g, d_S, d_flags, d_curr, ncurr, l, d_next, h_nnext, variant, s);
}
