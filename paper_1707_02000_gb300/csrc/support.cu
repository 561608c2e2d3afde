// K1: per-edge triangle support (Algorithm 3, §III "Parallel support
// computation").
//
// Vertices carry the library's internal order (ascending degree when the
// graph was built with TRUSS_DEGREE_ORDER), and N+(u) is the part of row u
// above u (slots [Eo[u], Es[u+1])).  Each triangle u < v < w is found exactly
// once, at its lowest vertex u: for every v in N+(u) and every w in N+(v),
// w closes a triangle iff w is in N+(u).  This is Algorithm 3's mark-and-
// probe with X held in shared memory (the paper visits the middle vertex;
// visiting the lowest one finds the same set of triangles, each once).
//
// GB300 mapping:
//  - warp per vertex (d+(u) <= TRUSS_SUP_WARP_CAP): N+(u) is staged in shared
//    memory with a counter per entry, the start of each N+(v) and the prefix
//    of d+(v) over v in N+(u).  Two instances of different capacity: when
//    no N+(u) exceeds 128 entries, the 128-entry one (16 KB of shared memory
//    a block, so 8 blocks of 8 warps fit an SM: a quarter less support time
//    on the geometric workload than the 256-entry one at 6 blocks an SM);
//    else the 256-entry one;
//    the 32 lanes then walk the concatenation of all N+(v) lists as one flat
//    range (balanced within the warp, coalesced reads of each N+(v); a
//    lane's segment only moves forward, see seg_advance), and probe each w
//    by binary search in the staged N+(u);
//  - block per vertex for larger d+(u) (listed at build time), same scheme
//    with the block's shared memory, its warps taking chunks of the flat
//    range; when the label windows above the listed vertices fit shared
//    memory (degree order puts these vertices at the top), N+(u) is also a
//    bitmap over its window and a probe is one word read;
//  - global-memory fallback for d+(u) beyond the shared-memory capacity.
// Every grid-stride launch is sized to the blocks that fit the GPU at once
// (resident_blocks).
// Supports of the edges {u, x}, x in N+(u), are accumulated in shared
// counters and added once per edge; only the {v, w} edges take one global
// atomic per triangle.
#include <algorithm>

#include "graph.cuh"

namespace {

constexpr int SW_WARPS = 8;  // warps per block, warp-per-vertex kernel
constexpr int SW_SPLIT = TRUSS_SUP_SPLIT;  // rows up to here go to the smaller instance
// Switch sides at a hub v when N+(v) is longer than SUP_SWITCH_FACTOR times
// u's entries above v (R-MAT scale 24 support: 1.07 s at 1, 1.08 at 2, 1.10
// at 4, 1.15 at 8; Chung-Lu 2^20: 3.65 / 3.89 / 4.08 / 4.33 ms).
constexpr int SUP_SWITCH_FACTOR = 1;
// The switching instances hold more registers (fewer warps an SM), so a
// graph uses them only when the switch saves at least 1/SUP_SWITCH_MIN_GAIN
// of W+ (the 4096-graph batch saves 0.3 % and runs 40 % slower with them).
constexpr int SUP_SWITCH_MIN_GAIN = 10;

// S accumulates in a plain int32[m] array (half the footprint of the
// {S, stamp} pairs, so more of the random per-triangle atomics hit L2); the
// pairs are written from it once at the end.  When that array takes more
// than half of L2 (beside the rows it would not stay there) but 16-bit
// counters would take at most three quarters, and no support can exceed
// 65535 (every degree at most 65536), two 16-bit counters share each word:
// the geometric 2^21 graph's 134 MB become 67 MB (support 2.60 -> 2.56
// ms; graphs whose int32 array already fits, or whose 16-bit one still
// does not, ran 2-3 % slower with the packed adds, so they keep int32).  An add to the
// upper half cannot carry out of the word, and one to the lower half
// cannot carry into the upper, since neither count passes 65535.
struct Acc {
    int* S;
    int s16;
};

__device__ __forceinline__ void add_support(const Acc& a, int32_t e, int v) {
    if (a.s16)
        atomicAdd(reinterpret_cast<unsigned*>(a.S) + (e >> 1), (unsigned)v << ((e & 1) << 4));
    else
        atomicAdd(a.S + e, v);
}

// Largest index p in [0, d) with P[p] <= idx (P ascending, P[0] = 0).
__device__ __forceinline__ int seg_of(const int* P, int d, int idx) {
    int lo = 0, hi = d - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P[mid] <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Segment of idx given the segment p of an earlier index of the same flat
// range (P[p] <= idx, segments only move forward): the largest q >= p with
// P[q] <= idx, found by steps of 1, 2, 4, ... from p and a binary search in
// the last step, so a lane that moves a few segments pays a few reads
// instead of a full search.  P[d] is the range's length, above idx.
__device__ __forceinline__ int seg_advance(const int* P, int d, int p, int idx) {
    if (P[p + 1] > idx) return p;
    int lo = p + 1, hi = d - 1;  // P[lo] <= idx
    for (int step = 1;; step <<= 1) {
        const int probe = lo + step;
        if (probe >= d) break;
        if (P[probe] > idx) {
            hi = probe - 1;
            break;
        }
        lo = probe;
    }
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P[mid] <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// First position in [lo, hi) with K[pos] >= w (K ascending); hi if none.
__device__ __forceinline__ int lower_bound_smem(const int* K, int lo, int hi, int w) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (K[mid] < w) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The peel's hub bitmaps (full rows of the highest-degree vertices, 32-byte
// blocks of 192 vertex ids led by the count of neighbours before the block),
// used by the support kernels to switch sides; hub_of == nullptr: no hubs.
struct HubView {
    const int32_t* hub_of;
    const unsigned long long* bits;
    int64_t hw;
    int factor;  // switch when N+(v) is longer than factor x u's entries above v
};

// Rank of w among the neighbours of the hub h's vertex, or -1 when w is not
// one of them (one 32-byte block read).
__device__ __forceinline__ int64_t hub_rank(const HubView& hv, int32_t h, int32_t w) {
    const int32_t b = w / 192, r = w - b * 192;
    const ulonglong2* B = reinterpret_cast<const ulonglong2*>(hv.bits + (int64_t)h * hv.hw + 4 * (int64_t)b);
    const ulonglong2 lo = __ldg(B), hi = __ldg(B + 1);
    const int k = r >> 6, bit = r & 63;
    const unsigned long long word = k == 0 ? lo.y : (k == 1 ? hi.x : hi.y);
    if (!((word >> bit) & 1ull)) return -1;
    int64_t rank = (int64_t)(uint32_t)lo.x;
    if (k > 0) rank += __popcll(lo.y);
    if (k > 1) rank += __popcll(hi.x);
    return rank + __popcll(word & ((1ull << bit) - 1ull));
}

// Vertices u with d+(u) <= CAP (longer rows go to the block kernels).  With
// COUNT the kernels only count triangles into *tri (no edge ids, no
// per-edge atomics).
//
// Switching sides at hubs: for a pair u < v (v in N+(u), at position p),
// the triangles u < v < w are the w in N+(v) that are also in N+(u) above
// position p.  When v is a hub and N+(v) is longer than those d - 1 - p
// entries, the kernel walks the entries instead (they are staged) and asks
// v's bitmap about each -- one block read -- so the pair costs
// min(d+(v), d - 1 - p) probes instead of d+(v).  Such pairs are marked by a
// negative E[p] = -(hub index + 1) and get length 0 in the N+(v) walk.
// HUB: the instance that switches sides at hubs (graphs with hub bitmaps);
// graphs without hubs run the instance without that code (fewer registers,
// so the 128-entry one keeps 8 blocks an SM).
template <typename Off, int CAP, bool COUNT = false, bool HUB = false>
__global__ void __launch_bounds__(SW_WARPS * 32)
    k_support_warp(const Off* __restrict__ rowptr, const Off* __restrict__ eo, const int32_t* __restrict__ col,
                   const int32_t* __restrict__ eid, int32_t n, Acc S,
                   unsigned long long* __restrict__ tri = nullptr, HubView hv = HubView{nullptr, nullptr, 0, 1},
                   unsigned long long* work = nullptr) {
    __shared__ int sK[SW_WARPS][CAP];
    __shared__ int sC[SW_WARPS][CAP];
    __shared__ int sP[SW_WARPS][CAP + 1];
    __shared__ Off sE[SW_WARPS][CAP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* K = sK[warp];
    int* C = sC[warp];
    int* P = sP[warp];
    Off* E = sE[warp];
    unsigned long long ntri = 0, wv = 0, wh = 0;  // triangles; N+(v) entries walked, bitmap probes
    const int64_t nwarps = (int64_t)gridDim.x * SW_WARPS;
    for (int64_t u = blockIdx.x * (int64_t)SW_WARPS + warp; u < n; u += nwarps) {
        const Off up0 = eo[u], up1 = rowptr[u + 1];
        const int d = (int)(up1 - up0);
        if (d < 2 || d > CAP) continue;  // no triangle at u / handled by the block kernels
        // stage N+(u), zero counters, prefix of d+(v)
        int carry = 0;
        for (int b = 0; b < d; b += 32) {
            int p = b + lane;
            int dv = 0;
            if (p < d) {
                int v = __ldg(col + up0 + p);
                K[p] = v;
                C[p] = 0;
                const Off v0 = __ldg(eo + v);
                E[p] = v0;
                dv = (int)(__ldg(rowptr + v + 1) - v0);
                if constexpr (!COUNT && HUB) {
                    const int32_t h = __ldg(hv.hub_of + v);
                    if (h >= 0 && (d - 1 - p) * hv.factor < dv) {  // walk u's entries above v instead
                        E[p] = -(Off)h - 1;
                        dv = 0;
                    }
                }
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
        const int total = carry;
        // two entries per lane (idx and idx + 32) with independent chains;
        // a lane's segment only moves forward
        int ps = 0;
        for (int idx = lane; idx < total; idx += 64) {
            const int i2 = idx + 32;
            const bool two = i2 < total;
            const int p1 = ps = seg_advance(P, d, ps, idx);
            const int p2 = two ? (ps = seg_advance(P, d, ps, i2)) : p1;
            const Off q1 = E[p1] + (idx - P[p1]);  // N+(v) starts at E[p] (staged)
            const Off q2 = two ? E[p2] + (i2 - P[p2]) : q1;
            const int w1 = __ldg(col + q1), x1 = COUNT ? 0 : __ldg(eid + q1);
            const int w2 = __ldg(col + q2), x2 = COUNT ? 0 : __ldg(eid + q2);
            const int r1 = lower_bound_smem(K, p1 + 1, d, w1);
            const int r2 = lower_bound_smem(K, p2 + 1, d, w2);
            const bool t1 = r1 < d && K[r1] == w1, t2 = two && r2 < d && K[r2] == w2;
            if constexpr (COUNT) {
                ntri += (unsigned)t1 + (unsigned)t2;
            } else {
                if (t1) {
                    atomicAdd(&C[r1], 1);  // edge {u, w}
                    atomicAdd(&C[p1], 1);  // edge {u, v}
                    add_support(S, x1, 1);  // edge {v, w}
                }
                if (t2) {
                    atomicAdd(&C[r2], 1);
                    atomicAdd(&C[p2], 1);
                    add_support(S, x2, 1);
                }
            }
        }
        __syncwarp();
        if constexpr (!COUNT) {
            if constexpr (HUB) {
                // the switched pairs: P <- prefix of their d - 1 - p entries
                int carry2 = 0;
                for (int b = 0; b < d; b += 32) {
                    const int p = b + lane;
                    const int a = (p < d && E[p] < 0) ? d - 1 - p : 0;
                    int x = a;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(FULL_MASK, x, o);
                        if (lane >= o) x += y;
                    }
                    if (p < d) P[p] = carry2 + x - a;
                    carry2 += __shfl_sync(FULL_MASK, x, 31);
                }
                if (lane == 0) P[d] = carry2;
                __syncwarp();
                int ps2 = 0;
                for (int idx = lane; idx < carry2; idx += 32) {
                    const int p = ps2 = seg_advance(P, d, ps2, idx);
                    const int r = p + 1 + (idx - P[p]);
                    const int32_t h = (int32_t)(-E[p] - 1);
                    const int64_t k = hub_rank(hv, h, K[r]);
                    if (k >= 0) {
                        atomicAdd(&C[r], 1);  // edge {u, w}
                        atomicAdd(&C[p], 1);  // edge {u, v}
                        add_support(S, __ldg(eid + __ldg(rowptr + K[p]) + k), 1);  // edge {v, w}
                    }
                }
                __syncwarp();
            }
            for (int p = lane; p < d; p += 32)
                if (C[p]) add_support(S, __ldg(eid + up0 + p), C[p]);
            if constexpr (HUB) {
                wv += (unsigned long long)total;
                wh += (unsigned long long)P[d];
            }
        }
        __syncwarp();
    }
    if constexpr (COUNT) {
        ntri = warp_sum(ntri);
        if (lane == 0 && ntri) atomicAdd(tri, ntri);
    } else if constexpr (HUB) {
        if (work && lane == 0 && (wv | wh)) {
            atomicAdd(work, wv);
            atomicAdd(work + 1, wh);
        }
    }
}

constexpr int SB_THREADS = 1024;  // one block an SM (shared memory); 512 left it latency-bound
constexpr int SB_WARPS = SB_THREADS / 32;

// Chunk of the flat range a warp of the block kernel takes at a time: about
// a quarter of the range per warp (so the warps finish together), between
// 64 and 1024 indices (a lane finds its first segment by binary search once
// per chunk and then only advances).
__device__ __forceinline__ int sb_chunk(int total) {
    const int c = ((total / (SB_WARPS * 4)) + 63) & ~63;
    return c < 64 ? 64 : (c > 1024 ? 1024 : c);
}

// Block-wide inclusive scan helper for the prefix of d+(v).
__device__ int block_scan_incl(int x, int* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < SB_THREADS / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL_MASK, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SB_THREADS / 32) wsum[lane] = w;
    }
    __syncthreads();
    int r = x + (warp ? wsum[warp - 1] : 0);
    __syncthreads();
    return r;
}

// One block per listed vertex; cap entries of K, C, P, Hs in dynamic shared
// memory.
//
// WIN: N+(u) is also held as a bitmap over the labels above u (bit w - u - 1;
// nwcap 32-bit words, enough for the widest window of the listed vertices),
// with the count of entries before each word, so a probe of w is one word
// read (the rank only on a hit) instead of a binary search in K.  The
// launch uses this instance when the bitmap fits shared memory, which it
// does for degree-ordered graphs: the vertices with long N+(u) have the
// highest labels (R-MAT scale 24: windows of at most 190,050 labels).
template <typename Off, bool COUNT = false, bool WIN = false>
__global__ void __launch_bounds__(SB_THREADS, WIN ? 2 : 1)
    k_support_block(const Off* __restrict__ rowptr, const Off* __restrict__ eo, const int32_t* __restrict__ col,
                    const int32_t* __restrict__ eid, const int32_t* __restrict__ verts, int32_t nverts, int cap,
                    Acc S, unsigned long long* __restrict__ tri = nullptr,
                    HubView hv = HubView{nullptr, nullptr, 0, 1}, unsigned long long* work = nullptr,
                    int32_t n = 0, int nwcap = 0) {
    extern __shared__ int smem[];
    unsigned long long ntri = 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* K = smem;
    int* C = smem + cap;
    int* P = smem + 2 * cap;      // cap + 1 entries
    int* Hs = smem + 3 * cap + 1;  // hub index of a switched pair, else -1 (support only)
    uint32_t* F = reinterpret_cast<uint32_t*>(smem + 4 * cap + 1);  // WIN: window bitmap, nwcap words
    unsigned short* R = reinterpret_cast<unsigned short*>(F + nwcap);  // WIN: entries before each word
    __shared__ int wsum[SB_THREADS / 32];
    __shared__ int s_carry;
    for (int32_t i = blockIdx.x; i < nverts; i += gridDim.x) {
        const int32_t u = verts[i];
        const Off up0 = eo[u], up1 = rowptr[u + 1];
        const int d = (int)(up1 - up0);
        const int nw = WIN ? (int)(((int64_t)n - 1 - u + 31) >> 5) : 0;  // <= nwcap
        if constexpr (WIN)
            for (int j = threadIdx.x; j < nw; j += SB_THREADS) F[j] = 0u;
        if (threadIdx.x == 0) s_carry = 0;
        __syncthreads();
        for (int b = 0; b < d; b += SB_THREADS) {
            int p = b + threadIdx.x;
            int dv = 0;
            if (p < d) {
                int v = __ldg(col + up0 + p);
                K[p] = v;
                C[p] = 0;
                if constexpr (WIN) {
                    const uint32_t b = (uint32_t)(v - u - 1);
                    atomicOr(F + (b >> 5), 1u << (b & 31));
                }
                dv = (int)(__ldg(rowptr + v + 1) - __ldg(eo + v));
                if constexpr (!COUNT) {
                    int32_t h = hv.hub_of ? __ldg(hv.hub_of + v) : -1;
                    if (h >= 0 && (d - 1 - p) * hv.factor < dv)
                        dv = 0;  // walk u's entries above v in v's bitmap instead
                    else
                        h = -1;
                    Hs[p] = h;
                }
            }
            int incl = block_scan_incl(dv, wsum);
            int carry = s_carry;
            if (p < d) P[p] = carry + incl - dv;
            __syncthreads();
            if (threadIdx.x == SB_THREADS - 1) s_carry = carry + incl;
            __syncthreads();
        }
        const int total = s_carry;
        if (threadIdx.x == 0) P[d] = total;
        if constexpr (WIN) {
            // R[j] = entries in the words before j: a block scan over
            // consecutive runs of words per thread
            const int per = (nw + SB_THREADS - 1) / SB_THREADS;
            const int j0 = min(nw, (int)threadIdx.x * per), j1 = min(nw, j0 + per);
            int cnt = 0;
            for (int j = j0; j < j1; ++j) cnt += __popc(F[j]);
            int run = block_scan_incl(cnt, wsum) - cnt;
            for (int j = j0; j < j1; ++j) {
                R[j] = (unsigned short)run;
                run += __popc(F[j]);
            }
        }
        __syncthreads();
        // Warps take chunks of consecutive indices (lanes 32 apart, two
        // entries a lane in flight); a lane's segment, and the start of its
        // N+(v) in col, change only when it crosses into the next one.
        const int ch = sb_chunk(total);
        for (int c0 = warp * ch; c0 < total; c0 += SB_WARPS * ch) {
            const int cend = min(c0 + ch, total);
            int idx = c0 + lane;
            if (idx >= cend) continue;
            int p = seg_of(P, d, idx);
            Off qb = __ldg(eo + K[p]) - P[p];  // N+(v) of segment p at qb + idx
            for (; idx < cend; idx += 64) {
                int np = seg_advance(P, d, p, idx);
                if (np != p) {
                    p = np;
                    qb = __ldg(eo + K[p]) - P[p];
                }
                const int p1 = p;
                const Off q1 = qb + idx;
                const int i2 = idx + 32;
                const bool two = i2 < cend;
                if (two) {
                    np = seg_advance(P, d, p, i2);
                    if (np != p) {
                        p = np;
                        qb = __ldg(eo + K[p]) - P[p];
                    }
                }
                const int p2 = p;
                const Off q2 = two ? qb + i2 : q1;
                const int w1 = __ldg(col + q1), x1 = COUNT ? 0 : __ldg(eid + q1);
                const int w2 = __ldg(col + q2), x2 = COUNT ? 0 : __ldg(eid + q2);
                int r1, r2;
                bool t1, t2;
                if constexpr (WIN) {
                    // w > v > u, so w - u - 1 lies in the window
                    const uint32_t b1 = (uint32_t)(w1 - u - 1), b2 = (uint32_t)(w2 - u - 1);
                    const uint32_t f1 = F[b1 >> 5], f2 = F[b2 >> 5];
                    t1 = (f1 >> (b1 & 31)) & 1u;
                    t2 = two && ((f2 >> (b2 & 31)) & 1u);
                    r1 = t1 ? (int)R[b1 >> 5] + __popc(f1 & ((1u << (b1 & 31)) - 1u)) : 0;
                    r2 = t2 ? (int)R[b2 >> 5] + __popc(f2 & ((1u << (b2 & 31)) - 1u)) : 0;
                } else {
                    r1 = lower_bound_smem(K, p1 + 1, d, w1);
                    r2 = lower_bound_smem(K, p2 + 1, d, w2);
                    t1 = r1 < d && K[r1] == w1;
                    t2 = two && r2 < d && K[r2] == w2;
                }
                if constexpr (COUNT) {
                    ntri += (unsigned)t1 + (unsigned)t2;
                } else {
                    if (t1) {
                        atomicAdd(&C[r1], 1);
                        atomicAdd(&C[p1], 1);
                        add_support(S, x1, 1);
                    }
                    if (t2) {
                        atomicAdd(&C[r2], 1);
                        atomicAdd(&C[p2], 1);
                        add_support(S, x2, 1);
                    }
                }
            }
        }
        __syncthreads();
        if constexpr (!COUNT) {
            int total2 = 0;
            if (hv.hub_of) {
                // switched pairs: P <- prefix of their d - 1 - p entries
                if (threadIdx.x == 0) s_carry = 0;
                __syncthreads();
                for (int b = 0; b < d; b += SB_THREADS) {
                    const int p = b + threadIdx.x;
                    const int a = (p < d && Hs[p] >= 0) ? d - 1 - p : 0;
                    const int incl = block_scan_incl(a, wsum);
                    const int carry = s_carry;
                    if (p < d) P[p] = carry + incl - a;
                    __syncthreads();
                    if (threadIdx.x == SB_THREADS - 1) s_carry = carry + incl;
                    __syncthreads();
                }
                total2 = s_carry;
                if (threadIdx.x == 0) P[d] = total2;
                __syncthreads();
                const int ch2 = sb_chunk(total2);
                for (int c0 = warp * ch2; c0 < total2; c0 += SB_WARPS * ch2) {
                    const int cend = min(c0 + ch2, total2);
                    int idx = c0 + lane;
                    if (idx >= cend) continue;
                    int p = seg_of(P, d, idx);
                    for (; idx < cend; idx += 32) {
                        p = seg_advance(P, d, p, idx);
                        const int r = p + 1 + (idx - P[p]);
                        const int64_t k = hub_rank(hv, Hs[p], K[r]);
                        if (k >= 0) {
                            atomicAdd(&C[r], 1);  // edge {u, w}
                            atomicAdd(&C[p], 1);  // edge {u, v}
                            add_support(S, __ldg(eid + __ldg(rowptr + K[p]) + k), 1);  // edge {v, w}
                        }
                    }
                }
                __syncthreads();
            }
            for (int p = threadIdx.x; p < d; p += SB_THREADS)
                if (C[p]) add_support(S, __ldg(eid + up0 + p), C[p]);
            if (work && threadIdx.x == 0) {
                atomicAdd(work, (unsigned long long)total);
                atomicAdd(work + 1, (unsigned long long)total2);
            }
        }
        __syncthreads();
    }
    if constexpr (COUNT) {
        ntri = warp_sum(ntri);
        if ((threadIdx.x & 31) == 0 && ntri) atomicAdd(tri, ntri);
    }
}

// Vertices whose N+(u) exceeds shared memory: one block per vertex, one warp
// per v in N+(u), probes by binary search in the global row of u.
template <typename Off, bool COUNT = false>
__global__ void __launch_bounds__(SB_THREADS)
    k_support_global(const Off* __restrict__ rowptr, const Off* __restrict__ eo, const int32_t* __restrict__ col,
                     const int32_t* __restrict__ eid, const int32_t* __restrict__ verts, int32_t nverts,
                     Acc S, unsigned long long* __restrict__ tri = nullptr,
                     unsigned long long* work = nullptr) {
    unsigned long long ntri = 0, wv = 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int32_t i = blockIdx.x; i < nverts; i += gridDim.x) {
        const int32_t u = verts[i];
        const Off up0 = eo[u], up1 = rowptr[u + 1];
        for (Off pv = up0 + warp; pv < up1; pv += SB_THREADS / 32) {
            const int v = __ldg(col + pv);
            const Off v0 = __ldg(eo + v), v1 = __ldg(rowptr + v + 1);
            wv += (unsigned long long)(v1 - v0);
            int cuv = 0;
            for (Off q = v0 + lane; q < v1; q += 32) {
                int w = __ldg(col + q);
                Off r = find_dev<Off>(col, pv + 1, up1, w);
                if (r >= 0) {
                    cuv++;
                    if constexpr (!COUNT) {
                        add_support(S, __ldg(eid + r), 1);
                        add_support(S, __ldg(eid + q), 1);
                    }
                }
            }
            if constexpr (COUNT) {
                ntri += (unsigned)cuv;
            } else {
                cuv = warp_sum(cuv);
                if (lane == 0 && cuv) add_support(S, __ldg(eid + pv), cuv);
            }
        }
    }
    if constexpr (COUNT) {
        ntri = warp_sum(ntri);
        if (lane == 0 && ntri) atomicAdd(tri, ntri);
    } else if (work && lane == 0 && wv) {
        atomicAdd(work, wv);
    }
}

// N+(v) entries the side switch saves: over pairs u < v (v at slot p of
// N+(u)) whose v is a hub and whose N+(v) is longer than u's entries above
// v, d+(v) minus those entries.  A warp per vertex.
template <typename Off>
__global__ void k_switch_gain(const Off* __restrict__ rowptr, const Off* __restrict__ eo,
                              const int32_t* __restrict__ col, const int32_t* __restrict__ hub_of, int32_t n,
                              unsigned long long* __restrict__ gain) {
    const int lane = threadIdx.x & 31;
    unsigned long long s = 0;
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n;
         u += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const Off p0 = eo[u], p1 = rowptr[u + 1];
        for (Off p = p0 + lane; p < p1; p += 32) {
            const int32_t v = col[p];
            if (hub_of[v] < 0) continue;
            const int64_t above = (int64_t)(p1 - 1 - p), dv = (int64_t)(rowptr[v + 1] - eo[v]);
            if (above * SUP_SWITCH_FACTOR < dv) s += (unsigned long long)(dv - above);
        }
    }
    s = warp_sum(s);
    if (lane == 0 && s) atomicAdd(gain, s);
}

__global__ void k_pack_ss(Acc S, int2* __restrict__ ss, int64_t m) {
    const unsigned short* S16 = reinterpret_cast<const unsigned short*>(S.S);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        ss[e] = make_int2(S.s16 ? (int)S16[e] : S.S[e], TRUSS_STAMP_NONE);
}

// Blocks for a grid-stride kernel: no more than fit the GPU at once.  A
// block beyond those would start only when a resident block had finished
// its whole share, and run its own share on an emptier SM (R-MAT scale 21:
// the 256-entry warp kernel launched 8 blocks an SM where 6 fit, and its
// warps were active 54 % of the time against 75 % possible).
template <typename K>
int resident_blocks(K kern, int threads, size_t smem, int sms, int64_t want) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess || per < 1) per = 1;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per * sms));
}

// The warp-per-vertex kernel over all vertices (those beyond CAP are left
// to the block kernels).
template <typename Off, int CAP, bool COUNT, bool HUB>
int launch_warp(truss_graph* g, Acc S, unsigned long long* tri, HubView hv, unsigned long long* work,
                cudaStream_t s) {
    const int blocks = resident_blocks(k_support_warp<Off, CAP, COUNT, HUB>, SW_WARPS * 32, 0, g->sms,
                                       ((int64_t)g->n + SW_WARPS - 1) / SW_WARPS);
    k_support_warp<Off, CAP, COUNT, HUB><<<blocks, SW_WARPS * 32, 0, s>>>(
        (const Off*)g->rowptr, (const Off*)g->eo, g->col, g->eid, g->n, S, tri, hv, work);
    CU(cudaGetLastError());
    truss_note_launch();
    return TRUSS_OK;
}

// Dynamic shared memory of the block kernel's window instance for this graph
// (K, C, P, Hs for the longest listed N+(u), the bitmap and its word
// counts for the widest window), or 0 when it does not fit a block.
template <typename Off, bool COUNT>
size_t block_win_smem(const truss_graph* g) {
    if (g->n_sup_big <= 0 || g->sup_big_maxup <= 0 || g->sup_big_maxup > TRUSS_SUP_BLOCK_CAP) return 0;
    const int64_t nw = (g->sup_big_maxwin + 31) >> 5;
    const size_t bytes = sizeof(int) * (size_t)(4 * g->sup_big_maxup + 1) + 6 * (size_t)nw;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device) != cudaSuccess) return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_support_block<Off, COUNT, true>) != cudaSuccess) return 0;
    return bytes + fa.sharedSizeBytes <= (size_t)optin ? bytes : 0;
}

// Launches the block kernel on the listed vertices: the window instance when
// its bitmap fits, else the binary-search one.
template <typename Off, bool COUNT>
int launch_block(truss_graph* g, Acc S, unsigned long long* tri, HubView hv, unsigned long long* work,
                 cudaStream_t s) {
    const Off* rowptr = (const Off*)g->rowptr;
    const Off* eo = (const Off*)g->eo;
    const size_t wsm = block_win_smem<Off, COUNT>(g);
    if (wsm) {
        const int cap = (int)g->sup_big_maxup, nwcap = (int)((g->sup_big_maxwin + 31) >> 5);
        CU(cudaFuncSetAttribute(k_support_block<Off, COUNT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)wsm));
        const int blocks = resident_blocks(k_support_block<Off, COUNT, true>, SB_THREADS, wsm, g->sms,
                                           (int64_t)g->n_sup_big);
        k_support_block<Off, COUNT, true><<<blocks, SB_THREADS, wsm, s>>>(
            rowptr, eo, g->col, g->eid, g->sup_big, g->n_sup_big, cap, S, tri, hv, work, g->n, nwcap);
    } else {
        const int cap = TRUSS_SUP_BLOCK_CAP;
        const size_t smem = sizeof(int) * (size_t)(4 * cap + 1);
        CU(cudaFuncSetAttribute(k_support_block<Off, COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
        const int blocks = (int)std::min<int64_t>(g->n_sup_big, (int64_t)g->sms);
        k_support_block<Off, COUNT><<<blocks, SB_THREADS, smem, s>>>(rowptr, eo, g->col, g->eid, g->sup_big,
                                                                     g->n_sup_big, cap, S, tri, hv, work);
    }
    CU(cudaGetLastError());
    truss_note_launch();
    return TRUSS_OK;
}

template <typename Off>
int support_impl(truss_graph* g, int2* ss, cudaStream_t s) {
    const Off* rowptr = (const Off*)g->rowptr;
    const Off* eo = (const Off*)g->eo;
    // accumulator: the first light-frontier buffer (int32[m], idle until the
    // peel starts)
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device) != cudaSuccess) l2 = 0;
    const bool s16 = g->max_deg <= 65536 && 4 * g->m > (int64_t)l2 / 2 && 2 * g->m <= (int64_t)l2 * 3 / 4;
    const Acc S{g->fq[0][0], s16 ? 1 : 0};
    const size_t words = S.s16 ? ((size_t)g->m + 1) / 2 : (size_t)g->m;
    CU(cudaMemsetAsync(S.S, 0, sizeof(int) * (words > 0 ? words : 1), s));
    // the hub bitmaps, when the peeling workspace has built them
    HubView hv{nullptr, nullptr, 0, 1};
    if (g->sup_switch && g->n_hub > 0 && g->hub_of && g->hub_bits)
        hv = HubView{g->hub_of, g->hub_bits, g->hub_words, SUP_SWITCH_FACTOR};
    // work counters: without hubs every kernel walks exactly W+ = sum_v
    // d-(v) d+(v) entries (known from the build), so only the switching
    // instances count
    unsigned long long* work = nullptr;
    if (g->ctr && hv.hub_of) {
        work = reinterpret_cast<unsigned long long*>(g->ctr + TRUSS_CTR_SUPPORT_WORK);
        CU(cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), s));
    }
    if (g->n > 0 && g->m > 0) {
        // one warp-per-vertex instance: the 128-entry one when no N+(u) is
        // longer (8 blocks an SM), else the 256-entry one (6 blocks an SM);
        // two instances run one after the other cost more than either
        const bool hub = hv.hub_of != nullptr;
        int rc;
        if (g->max_updeg <= SW_SPLIT && hub)
            rc = launch_warp<Off, SW_SPLIT, false, true>(g, S, nullptr, hv, work, s);
        else if (g->max_updeg <= SW_SPLIT)
            rc = launch_warp<Off, SW_SPLIT, false, false>(g, S, nullptr, hv, work, s);
        else if (hub)
            rc = launch_warp<Off, TRUSS_SUP_WARP_CAP, false, true>(g, S, nullptr, hv, work, s);
        else
            rc = launch_warp<Off, TRUSS_SUP_WARP_CAP, false, false>(g, S, nullptr, hv, work, s);
        if (rc != TRUSS_OK) return rc;
    }
    if (g->n_sup_big > 0) {
        const int rc = launch_block<Off, false>(g, S, nullptr, hv, work, s);
        if (rc != TRUSS_OK) return rc;
    }
    if (g->n_sup_huge > 0) {
        int blocks = (int)std::min<int64_t>(g->n_sup_huge, (int64_t)g->sms * 2);
        k_support_global<Off>
            <<<blocks, SB_THREADS, 0, s>>>(rowptr, eo, g->col, g->eid, g->sup_huge, g->n_sup_huge, S, nullptr, work);
        CU(cudaGetLastError());
        truss_note_launch();
    }
    if (g->m > 0) {
        k_pack_ss<<<grid_for(g->m, 256), 256, 0, s>>>(S, ss, g->m);
        CU(cudaGetLastError());
        truss_note_launch();
    }
    return TRUSS_OK;
}

// Triangle count: the support kernels' walk without edge ids or per-edge
// atomics (each triangle u < v < w counted once at u).
template <typename Off>
int count_impl(truss_graph* g, unsigned long long* d_tri, cudaStream_t s) {
    const Off* rowptr = (const Off*)g->rowptr;
    const Off* eo = (const Off*)g->eo;
    CU(cudaMemsetAsync(d_tri, 0, sizeof(unsigned long long), s));
    if (g->n > 0 && g->m > 0) {
        const HubView none{nullptr, nullptr, 0, 1};
        const Acc no{nullptr, 0};
        const int rc = g->max_updeg <= SW_SPLIT
                           ? launch_warp<Off, SW_SPLIT, true, false>(g, no, d_tri, none, nullptr, s)
                           : launch_warp<Off, TRUSS_SUP_WARP_CAP, true, false>(g, no, d_tri, none, nullptr, s);
        if (rc != TRUSS_OK) return rc;
    }
    if (g->n_sup_big > 0) {
        const int rc =
            launch_block<Off, true>(g, Acc{nullptr, 0}, d_tri, HubView{nullptr, nullptr, 0, 1}, nullptr, s);
        if (rc != TRUSS_OK) return rc;
    }
    if (g->n_sup_huge > 0) {
        int blocks = (int)std::min<int64_t>(g->n_sup_huge, (int64_t)g->sms * 2);
        k_support_global<Off, true><<<blocks, SB_THREADS, 0, s>>>(rowptr, eo, g->col, g->eid, g->sup_huge,
                                                                  g->n_sup_huge, Acc{nullptr, 0}, d_tri);
        CU(cudaGetLastError());
        truss_note_launch();
    }
    return TRUSS_OK;
}

}  // namespace

extern "C" int truss_triangle_count(truss_graph* g, int64_t* h_count, void* stream) {
    if (!g || !h_count) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* d_tri = nullptr;
    CU(cudaMallocAsync((void**)&d_tri, sizeof(unsigned long long), s));
    int rc = g->off64 ? count_impl<int64_t>(g, d_tri, s) : count_impl<int32_t>(g, d_tri, s);
    unsigned long long h = 0;
    if (rc == TRUSS_OK) {
        CU(cudaMemcpyAsync(&h, d_tri, sizeof(h), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        *h_count = (int64_t)h;
    }
    cudaFreeAsync(d_tri, s);
    return rc;
}

// Decides, once the hub bitmaps exist, whether the support kernels switch
// sides at hubs for this graph (sets g->sup_switch).
int truss_support_plan(truss_graph* g, cudaStream_t s) {
    g->sup_switch = 0;
    if (g->n_hub <= 0 || !g->hub_of || g->n <= 0 || g->wedges_up <= 0) return TRUSS_OK;
    unsigned long long* d_gain = nullptr;
    CU(cudaMallocAsync((void**)&d_gain, sizeof(unsigned long long), s));
    CU(cudaMemsetAsync(d_gain, 0, sizeof(unsigned long long), s));
    const int blocks = grid_for((int64_t)g->n, 8, (int64_t)g->sms * 8);
    if (g->off64)
        k_switch_gain<int64_t><<<blocks, 256, 0, s>>>((const int64_t*)g->rowptr, (const int64_t*)g->eo, g->col,
                                                      g->hub_of, g->n, d_gain);
    else
        k_switch_gain<int32_t><<<blocks, 256, 0, s>>>((const int32_t*)g->rowptr, (const int32_t*)g->eo, g->col,
                                                      g->hub_of, g->n, d_gain);
    CU(cudaGetLastError());
    unsigned long long gain = 0;
    CU(cudaMemcpyAsync(&gain, d_gain, sizeof(gain), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    cudaFreeAsync(d_gain, s);
    g->sup_gain = (int64_t)gain;
    g->sup_switch = (int64_t)gain * SUP_SWITCH_MIN_GAIN >= g->wedges_up;
    return TRUSS_OK;
}

int truss_support_internal(truss_graph* g, int2* ss, cudaStream_t s) {
    return g->off64 ? support_impl<int64_t>(g, ss, s) : support_impl<int32_t>(g, ss, s);
}
