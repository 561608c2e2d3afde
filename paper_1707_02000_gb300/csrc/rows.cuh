// The peel's view of a graph, and the searches every edge-wise kernel uses:
// the per-edge row records (shorter row walked, longer row searched), the
// lockstep binary search and the hub-bitmap probe.  Shared by the level-
// synchronous peel (peel.cu) and the local h-index iteration (local.cu).
#pragma once
#include "graph.cuh"

namespace {

template <typename Off>
struct Graph {
    const Off* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const int32_t* __restrict__ eid;
    const int2* __restrict__ el;
    const int32_t* __restrict__ dmin;  // min(d(u), d(v)) per edge
    const Off* __restrict__ rows;      // per edge: shorter row [a0, a1), longer row [b0, b1)
    const int32_t* __restrict__ lhub;  // per edge: hub index of the longer row's vertex, -1 if none
    const unsigned long long* __restrict__ hbits;  // per hub: 32-byte blocks {count before, 3 x 64 ids}
    int64_t hw;                                    // words per hub (4 per block)
    const int32_t* __restrict__ oeid;  // edge ids of the rows as built: a hub probe gives a slot there
    int2* ss;
    int64_t m;
    int hc;  // heavy chunk length (entries of the shorter row)
    uint32_t ocap;                     // capacity of each side's chunk owner map
};

template <typename Off>
struct Rows {
    Off a0, a1, b0, b1;  // shorter row [a0, a1), longer row [b0, b1)
    int32_t hub;         // hub index of the longer row's vertex, -1 if none
};

// The rows of edge e from its precomputed record (one 16-byte load for
// int32 offsets, two for int64): no endpoint -> row-pointer round trip.
template <typename Off>
__device__ __forceinline__ Rows<Off> rows_of(const Graph<Off>& G, int32_t e) {
    const int32_t hub = __ldg(G.lhub + e);
    if constexpr (sizeof(Off) == 4) {
        const int4 v = __ldg(reinterpret_cast<const int4*>(G.rows) + e);
        return Rows<Off>{v.x, v.y, v.z, v.w, hub};
    } else {
        const longlong2* p = reinterpret_cast<const longlong2*>(G.rows) + 2 * (int64_t)e;
        const longlong2 a = __ldg(p), b = __ldg(p + 1);
        return Rows<Off>{a.x, a.y, b.x, b.y, hub};
    }
}

// Slots of k1 and k2 in the ascending row a[lo, lo + n) (n >= 1), or -1.
// Both searches run in lockstep (the step count depends on n only), so each
// step issues two independent loads.  Each search keeps the last slot whose
// value is <= its key, with that value, so no load follows the loop.
template <typename Off>
__device__ __forceinline__ void find2(const int32_t* __restrict__ a, Off lo, Off n, int32_t k1, int32_t k2, Off& p1,
                                      Off& p2) {
    Off b1 = lo, b2 = lo;
    int32_t v1 = __ldg(a + lo), v2 = v1;
    while (n > 1) {
        const Off h = n >> 1;
        const int32_t t1 = __ldg(a + b1 + h), t2 = __ldg(a + b2 + h);
        if (t1 <= k1) {
            b1 += h;
            v1 = t1;
        }
        if (t2 <= k2) {
            b2 += h;
            v2 = t2;
        }
        n -= h;
    }
    p1 = v1 == k1 ? b1 : (Off)-1;
    p2 = v2 == k2 ? b2 : (Off)-1;
}

// Slot of w in the row (starting at slot b0) of the vertex that owns hub h,
// or -1.  The hub's bitmap is cut into 32-byte blocks of 192 ids: word 0
// holds the number of neighbours before the block, words 1-3 the bits.  One
// probe reads one block (one sector): the bit of w, and its rank = the count
// before the block + the bits of the block's earlier words + the bits below
// w in its word.
template <typename Off>
__device__ __forceinline__ Off hub_find(const Graph<Off>& G, int32_t h, Off b0, int32_t w) {
    const int32_t b = w / 192, r = w - b * 192;
    const ulonglong2* B = reinterpret_cast<const ulonglong2*>(G.hbits + (int64_t)h * G.hw + 4 * (int64_t)b);
    const ulonglong2 lo = __ldg(B), hi = __ldg(B + 1);
    const int k = r >> 6, bit = r & 63;
    const unsigned long long word = k == 0 ? lo.y : (k == 1 ? hi.x : hi.y);
    uint32_t rank = (uint32_t)lo.x;
    if (k > 0) rank += (uint32_t)__popcll(lo.y);
    if (k > 1) rank += (uint32_t)__popcll(hi.x);
    rank += (uint32_t)__popcll(word & ((1ull << bit) - 1ull));
    return ((word >> bit) & 1ull) ? b0 + (Off)rank : (Off)-1;
}

}  // namespace
