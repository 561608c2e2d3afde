// Level-synchronous peeling (Algorithms 4 and 5, §III) on the device.
//
// Scan (K2): the first Scan reads all {S, stamp} words (16 bytes, two edges,
// per load); every Scan writes the edges above its level to a live list that
// the next Scan reads instead of all m edges.  Edges with S = l join curr,
// split into light and heavy lists; a block step places its appends with one
// block prefix sum and at most three atomics.  The minimum support above l
// is reduced on the side, so an empty level jumps straight to the next live
// one.
//
// ProcessSubLevel (K3): for every e1 = {u, v} in curr, the common neighbours
// w of u and v are found by searching each entry of the shorter row in the
// longer one: through registers when the longer row is short, through the
// neighbour bitmap when its vertex is a hub, else by binary search (two keys
// per lane in lockstep).  Each triangle {e1, e2, e3} whose other two edges
// are unprocessed lowers e2 (resp. e3) by one when its support is above l
// and e3 (resp. e2) is not in curr or has a larger id than e1: the two-sided
// reading of Algorithm 5, which prints only the e2 case.  The decrement is
// atomicSub; an edge whose old value was l+1 joins next; a thread that
// pushed an edge below l adds the 1 back (the clamp-and-restore of Algorithm
// 5), so the final value is max(l, S - #triangles removed).  The rule is
// symmetric in e2 and e3, so which of them is {u,w} or {v,w} does not matter.
//
// Work mapping.  A frontier is kept as two lists:
//   light  edges whose shorter row has <= LIGHT entries; each is walked by a
//          group of G lanes, G in {1, 16, 32} chosen per sub-level (the
//          "variant": one thread per edge, half a warp per edge with the
//          longer row in registers, or a whole warp per edge);
//   heavy  longer rows, cut into chunks of hc entries.  Appending a heavy
//          edge reserves its chunk range with one 64-bit atomic on
//          (edge count << 32 | chunk total), so the chunk bases are monotone
//          in list order; the owner map records each chunk's edge and place
//          in the row (beyond its capacity a warp finds the edge by binary
//          search over the chunk bases).  All warps of the grid share all
//          chunks, so the few huge rows of a small late frontier spread over
//          the whole GPU.
//
// Loop forms: PLAIN launches Scan / ProcessSubLevel from the host and reads
// the frontier size back after every phase (the direct transcription of
// Algorithm 4's loop); PERSISTENT runs the whole loop in one cooperative
// kernel whose phases are separated by a grid barrier with a time limit (in
// two register budgets); GRAPH runs it as one CUDA graph whose control
// kernel picks each next phase on the device.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "graph.cuh"
#include "rows.cuh"
#include "sched.cuh"

namespace {

enum {
    C_SLOTS = 0,  // [0..31]  four SlotVals: what phase p produced, slot p & 3
    C_BAR_COUNT = 32,  // grid-barrier arrivals since the launch began
    C_ERR = 34,
    C_NSUB = 35,
    C_NSCAN = 36,
    C_NLEVEL = 37,
    C_LAST_L = 38,
    C_TRI = 40,   // [40..41] triangle count (u64), [42] max support
    C_SCANNED = 44,  // [44..45] entries all Scans visited (i64)
    C_WALKED = 46,   // [46..47] shorter-row entries of all frontiers (i64)
    C_ROS = 48,      // [48..49] next edge batch of the edge-centric support (u64)
    // [50..53] the support kernels' work counters (TRUSS_CTR_SUPPORT_WORK)
    C_ST = 64,       // [64..95] loop state a persistent launch leaves (PState)
    C_TOTAL = 96
};

// Where a persistent launch stopped: at the end of the peel (stop = 0), or
// before the Scan of level l when the rows are due for compaction (stop = 1;
// the next launch resumes from here).
struct PState {
    int32_t l, g, stop, pad;
    long long processed, nsub, sc, nlevel, nlive, scanned, walked, scan_ns;
};
static_assert(sizeof(PState) <= sizeof(int) * (C_TOTAL - C_ST), "PState fits the counter block");

// A compaction runs once the live (unprocessed) edges are at most this
// share (in %) of the edges the rows hold: 80 % while the rows hold at
// least 2^25 edges (the walk saved outweighs the passes), 50 % below (each
// compaction also costs a stop of the persistent launch and a host round
// trip).  Measured: R-MAT scale 24 peel 1.51 s at 50 %, 1.32 s at 65 %,
// 1.21 s at 80 %, 1.22 s at 90 %; Chung-Lu 2^20 and the geometric 2^21
// graph are fastest at 50 % (80 %: +3 % and +7 %).
constexpr int64_t CMP_BIG_HELD = (int64_t)1 << 25;
__host__ __device__ __forceinline__ int cmp_live_pct(int64_t held) { return held >= CMP_BIG_HELD ? 80 : 50; }

constexpr int PT = 256;      // threads per block in the peel kernels
constexpr int PW = PT / 32;
constexpr int LIGHT = 32;    // shorter row <= LIGHT entries: light edge
constexpr int LCAP = 1024;   // per-block staging of light next-frontier appends
constexpr int HPT = 1;       // staged heavy appends per thread at flush
constexpr int HCAP = PT * HPT;  // per-block staging of heavy appends

// One side of the frontier ping-pong.
struct Frontier {
    int32_t* light;
    int32_t* heavy;
    uint32_t* cbase;  // first chunk number of each heavy edge (monotone)
    int2* owner;      // per chunk: {owning edge, chunk index within its row} (if the total fits ocap)
};

struct PeelSmem {
    int32_t lbuf[LCAP];
    int32_t hbuf[HCAP];
    int lcnt, hcnt, lbase, hq0;
    uint32_t hb0;
    uint32_t wsum[PT / 32];
    unsigned long long wtot[PW];  // per-warp packed counts / sums, then offsets
    unsigned long long dsum;  // shorter-row lengths appended by this block
    int dmax;
    int wcnt[PW];             // per-warp maxima
    int bbase;
    int bmin[PW];
};

// Counters a phase fills in for the frontier it produces (32 bytes, read
// back in one piece after the barrier that ends the phase).
struct SlotVals {
    int nl;                  // light-list size
    int dmax;                // longest shorter row in the frontier
    unsigned long long hc;   // heavy count << 32 | heavy chunk total
    unsigned long long dsum; // sum of shorter-row lengths
    int minv;                // minimum live support above l (Scan)
    int nlive;               // live edges kept for the next Scan
};
static_assert(sizeof(SlotVals) == 32, "SlotVals is read as two 16-byte words");

struct Slot {
    int* nl;
    unsigned long long* hc;
    unsigned long long* dsum;
    int* dmax;
    int* minv;
    int* nlive;
};

__host__ __device__ __forceinline__ SlotVals* slots(int* ctr) { return reinterpret_cast<SlotVals*>(ctr + C_SLOTS); }

__host__ __device__ __forceinline__ Slot slot_of(int* ctr, int s) {
    SlotVals* v = slots(ctr) + s;
    return Slot{&v->nl, &v->hc, &v->dsum, &v->dmax, &v->minv, &v->nlive};
}

__host__ __device__ __forceinline__ void clear_slot_vals(SlotVals* v) {
    v->nl = 0;
    v->dmax = 0;
    v->hc = 0ull;
    v->dsum = 0ull;
    v->minv = INT_MAX;
    v->nlive = 0;
}


__device__ __forceinline__ uint32_t nchunks_of(int d, int hc) { return (uint32_t)((d + hc - 1) / hc); }

// owner[base + k] = {f, k} for the n chunks of heavy edge f, when that
// range fits the map
__device__ __forceinline__ void write_owner(const Frontier& out, uint32_t ocap, uint32_t base, uint32_t n,
                                            int32_t f) {
    if ((uint64_t)base + n <= ocap)
        for (uint32_t k = 0; k < n; k++) out.owner[base + k] = make_int2(f, (int)k);
}

// Next-frontier appends of one block during a sub-level: staged in shared
// memory and placed by flush() at the end of the phase with one block prefix
// sum and one atomic per list; entries beyond the stage go to the lists
// directly.  The shorter-row sum and maximum of the block's appends are kept
// in shared memory as they arrive, so flush() reads no global memory for
// light entries.
struct Appender {
    PeelSmem* sm;
    Frontier out;
    Slot cnt;
    const int32_t* dmin;
    int hc;
    uint32_t ocap;
    __device__ __forceinline__ void push(int32_t f) const {
        const int d = __ldg(dmin + f);
        atomicAdd(&sm->dsum, (unsigned long long)d);
        atomicMax(&sm->dmax, d);
        if (d <= LIGHT) {
            const int p = atomicAdd(&sm->lcnt, 1);
            if (p < LCAP) {
                sm->lbuf[p] = f;
                return;
            }
            out.light[atomicAdd(cnt.nl, 1)] = f;
        } else {
            const int p = atomicAdd(&sm->hcnt, 1);
            if (p < HCAP) {
                sm->hbuf[p] = f;
                return;
            }
            const uint32_t nch = nchunks_of(d, hc);
            const unsigned long long old = atomicAdd(cnt.hc, (1ull << 32) | nch);
            const int q = (int)(old >> 32);
            out.heavy[q] = f;
            out.cbase[q] = (uint32_t)old;
            write_owner(out, ocap, (uint32_t)old, nch, f);
        }
    }
    // whole block; leaves the stage empty
    __device__ void flush() const {
        __syncthreads();
        const int kl = min(sm->lcnt, LCAP), kh = min(sm->hcnt, HCAP);
        const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
        // thread t owns staged heavy entries [t * HPT, (t + 1) * HPT)
        uint32_t c[HPT];
        uint32_t ct = 0;
#pragma unroll
        for (int k = 0; k < HPT; k++) {
            const int i = t * HPT + k;
            c[k] = 0;
            if (i < kh) {
                c[k] = nchunks_of(__ldg(dmin + sm->hbuf[i]), hc);
                ct += c[k];
            }
        }
        uint32_t x = ct;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm->wsum[warp] = x;
        __syncthreads();
        if (t == 0) {
            uint32_t run = 0;
            for (int w = 0; w < PW; w++) {
                const uint32_t v = sm->wsum[w];
                sm->wsum[w] = run;
                run += v;
            }
            if (sm->dsum) {
                atomicAdd(cnt.dsum, sm->dsum);
                atomicMax(cnt.dmax, sm->dmax);
            }
            // both reservations in flight before either result is used
            const int lb = kl ? atomicAdd(cnt.nl, kl) : 0;
            const unsigned long long old = kh ? atomicAdd(cnt.hc, ((unsigned long long)kh << 32) | run) : 0ull;
            sm->lbase = lb;
            sm->hq0 = (int)(old >> 32);
            sm->hb0 = (uint32_t)old;
        }
        __syncthreads();
        for (int i = t; i < kl; i += PT) out.light[sm->lbase + i] = sm->lbuf[i];
        uint32_t pc = sm->hb0 + sm->wsum[warp] + x - ct;
#pragma unroll
        for (int k = 0; k < HPT; k++) {
            const int i = t * HPT + k;
            if (i < kh) {
                out.heavy[sm->hq0 + i] = sm->hbuf[i];
                out.cbase[sm->hq0 + i] = pc;
                write_owner(out, ocap, pc, c[k], sm->hbuf[i]);
                pc += c[k];
            }
        }
        __syncthreads();
        if (t == 0) {
            sm->lcnt = 0;
            sm->hcnt = 0;
            sm->dsum = 0;
            sm->dmax = 0;
        }
        __syncthreads();
    }
};

__device__ __forceinline__ void smem_init(PeelSmem* sm) {
    if (threadIdx.x == 0) {
        sm->lcnt = 0;
        sm->hcnt = 0;
        sm->dsum = 0;
        sm->dmax = 0;
    }
    __syncthreads();
}

// After the decrement of f's support returned a: f enters the next
// sub-level when it reached l; a value at or below l (pushed there by a racing
// thread) is restored.
__device__ __forceinline__ void settle(int2* ss, int32_t f, int a, int32_t l, int32_t g, const Appender& ap) {
    if (a == l + 1) {
        ss[f].y = g + 1;  // f enters the next sub-level
        ap.push(f);
    } else if (a <= l) {
        atomicAdd(&ss[f].x, 1);
    }
}

// Which edges of triangle {e1, x, y} (seen while processing e1 in sub-level g
// at level l, with x's and y's (S, stamp) pairs sx, sy) lose one support:
// none when an edge of it is processed; x when S[x] > l and y is not in curr
// or e1 < y; y likewise.
__device__ __forceinline__ void decide(int32_t e1, int32_t x, int32_t y, int2 sx, int2 sy, int32_t l, int32_t g,
                                       bool& dx, bool& dy) {
    if (sx.y < g || sy.y < g) {
        dx = dy = false;
        return;
    }
    const bool inx = sx.y == g, iny = sy.y == g;
    dx = sx.x > l && (!iny || e1 < y);
    dy = sy.x > l && (!inx || e1 < x);
}

// Two candidate triangles {e1, x1, y1} (ok1) and {e1, x2, y2} (ok2) of one
// lane; the four edges are distinct, so their loads and decrements are
// issued together and the round trips overlap.
__device__ __forceinline__ void on_triangles(int2* ss, int32_t e1, bool ok1, int32_t x1, int32_t y1, bool ok2,
                                             int32_t x2, int32_t y2, int32_t l, int32_t g, const Appender& ap) {
    const int2 none = make_int2(0, 0);
    const int2 sx1 = ok1 ? __ldcg(ss + x1) : none, sy1 = ok1 ? __ldcg(ss + y1) : none;
    const int2 sx2 = ok2 ? __ldcg(ss + x2) : none, sy2 = ok2 ? __ldcg(ss + y2) : none;
    bool d1x = false, d1y = false, d2x = false, d2y = false;
    if (ok1) decide(e1, x1, y1, sx1, sy1, l, g, d1x, d1y);
    if (ok2) decide(e1, x2, y2, sx2, sy2, l, g, d2x, d2y);
    const int a1x = d1x ? atomicSub(&ss[x1].x, 1) : 0;
    const int a1y = d1y ? atomicSub(&ss[y1].x, 1) : 0;
    const int a2x = d2x ? atomicSub(&ss[x2].x, 1) : 0;
    const int a2y = d2y ? atomicSub(&ss[y2].x, 1) : 0;
    if (d1x) settle(ss, x1, a1x, l, g, ap);
    if (d1y) settle(ss, y1, a1y, l, g, ap);
    if (d2x) settle(ss, x2, a2x, l, g, ap);
    if (d2y) settle(ss, y2, a2y, l, g, ap);
}

// All triangles through e1 whose apex is one of the slots start, start+step,
// ... of [a0, a1) (part of the shorter row), each probed in the longer row;
// a lane takes two slots at a time (j and j + step) and searches for both
// at once.
template <typename Off>
__device__ __forceinline__ void walk_rows(const Graph<Off>& G, int32_t e1, Off a0, Off a1, const Rows<Off>& r,
                                          int start, int step, int32_t l, int32_t g, const Appender& ap) {
    for (Off j = a0 + start; j < a1; j += 2 * step) {
        const Off j2 = j + step;
        const bool two = j2 < a1;
        // the edge ids of the walked entries are read only for the entries
        // that close a triangle (R-MAT scale 24 peel 2.4 % faster than
        // reading them beside the neighbour ids)
        const int32_t w1 = __ldg(G.col + j), w2 = two ? __ldg(G.col + j2) : w1;
        Off q1, q2;
        if (r.hub >= 0) {
            q1 = hub_find<Off>(G, r.hub, r.b0, w1);
            q2 = hub_find<Off>(G, r.hub, r.b0, w2);
        } else {
            find2<Off>(G.col, r.b0, r.b1 - r.b0, w1, w2, q1, q2);
        }
        const bool ok1 = q1 >= 0, ok2 = two && q2 >= 0;
        // a hub probe gives a slot of the row as built (the bitmaps are not
        // rebuilt when rows are compacted; a stale bit finds a processed
        // edge, whose triangle is skipped like any other)
        const int32_t* ye = r.hub >= 0 ? G.oeid : G.eid;
        const int32_t y1 = ok1 ? __ldg(ye + q1) : 0, y2 = ok2 ? __ldg(ye + q2) : 0;
        const int32_t x1 = ok1 ? __ldg(G.eid + j) : 0, x2 = ok2 ? __ldg(G.eid + j2) : 0;
        on_triangles(G.ss, e1, ok1, x1, y1, ok2, x2, y2, l, g, ap);
    }
}

// The same walk for a whole warp on one edge (lanes 0..31 take slots a0 +
// lane, a0 + lane + 32, ...) when the longer row has at most 32 R entries:
// the row is loaded once into R registers per lane (coalesced) and each lane
// binary-searches it through warp shuffles, so a probe costs no memory round
// trip.  Slot i of the row lives in lane i % 32, register i / 32; slots past
// the end read as INT_MAX (no vertex id).  Warp-uniform: every lane must call
// it with the same arguments.
template <typename Off, int R>
__device__ __forceinline__ void walk_rows_warp(const Graph<Off>& G, int32_t e1, Off a0, Off a1, const Rows<Off>& r,
                                               int lane, int32_t l, int32_t g, const Appender& ap) {
    const int nb = (int)(r.b1 - r.b0);
    int32_t L[R];
#pragma unroll
    for (int k = 0; k < R; k++) L[k] = k * 32 + lane < nb ? __ldg(G.col + r.b0 + k * 32 + lane) : INT_MAX;
    const int32_t v0 = __shfl_sync(FULL_MASK, L[0], 0);
    const int rounds = (int)((a1 - a0 + 31) >> 5);
    for (int t = 0; t < rounds; t++) {
        const Off j = a0 + (Off)t * 32 + lane;
        const bool act = j < a1;
        const int32_t w = act ? __ldg(G.col + j) : INT_MIN;
        // last slot whose value is <= w (slot 0 when none is)
        int lo = 0;
        int32_t vlo = v0;
#pragma unroll
        for (int h = R * 16; h >= 1; h >>= 1) {
            const int p = lo + h;
            int32_t v = __shfl_sync(FULL_MASK, L[0], p & 31);
#pragma unroll
            for (int k = 1; k < R; k++) {
                const int32_t vk = __shfl_sync(FULL_MASK, L[k], p & 31);
                if ((p >> 5) == k) v = vk;
            }
            if (v <= w) {
                lo = p;
                vlo = v;
            }
        }
        const bool ok = act && vlo == w;
        const int32_t x = ok ? __ldg(G.eid + j) : 0;
        const int32_t y = ok ? __ldg(G.eid + r.b0 + lo) : 0;
        on_triangles(G.ss, e1, ok, x, y, false, 0, 0, l, g, ap);
    }
}

// A warp's walk over [a0, a1) of e1's shorter row: through registers when
// the longer row is short, else by searches in global memory.  Warp-uniform.
template <typename Off>
__device__ __forceinline__ void walk_warp(const Graph<Off>& G, int32_t e1, Off a0, Off a1, const Rows<Off>& r,
                                          int lane, int32_t l, int32_t g, const Appender& ap) {
    const Off nb = r.b1 - r.b0;
    if (nb <= 32)
        walk_rows_warp<Off, 1>(G, e1, a0, a1, r, lane, l, g, ap);
    else if (nb <= 64)
        walk_rows_warp<Off, 2>(G, e1, a0, a1, r, lane, l, g, ap);
    else if (nb <= 128)
        walk_rows_warp<Off, 4>(G, e1, a0, a1, r, lane, l, g, ap);
    else
        walk_rows<Off>(G, e1, a0, a1, r, lane, 32, l, g, ap);
}

// Two light edges per warp: lanes 0-15 walk the shorter row of one, lanes
// 16-31 of the other (sub = lane % 16).  When both longer rows have at most
// 64 entries each half holds its row in 4 registers a lane and searches it
// through 16-lane shuffles; the trip counts are the warp's maximum, so the
// shuffles always run with the full warp.  Warp-uniform call.
template <typename Off>
__device__ __forceinline__ void walk_half_reg(const Graph<Off>& G, bool valid, int32_t e1, const Rows<Off>& r,
                                              int sub, int32_t l, int32_t g, const Appender& ap) {
    const int nb = valid ? (int)(r.b1 - r.b0) : 0;
    int32_t L[4];
#pragma unroll
    for (int k = 0; k < 4; k++) L[k] = k * 16 + sub < nb ? __ldg(G.col + r.b0 + k * 16 + sub) : INT_MAX;
    const int32_t v0 = __shfl_sync(FULL_MASK, L[0], 0, 16);
    int rounds = valid ? (int)((r.a1 - r.a0 + 15) >> 4) : 0;
    rounds = max(rounds, __shfl_xor_sync(FULL_MASK, rounds, 16));
    for (int t = 0; t < rounds; t++) {
        const Off j = r.a0 + (Off)t * 16 + sub;
        const bool act = valid && j < r.a1;
        const int32_t w = act ? __ldg(G.col + j) : INT_MIN;
        int lo = 0;
        int32_t vlo = v0;
#pragma unroll
        for (int h = 32; h >= 1; h >>= 1) {
            const int p = lo + h;
            int32_t v = __shfl_sync(FULL_MASK, L[0], p & 15, 16);
#pragma unroll
            for (int k = 1; k < 4; k++) {
                const int32_t vk = __shfl_sync(FULL_MASK, L[k], p & 15, 16);
                if ((p >> 4) == k) v = vk;
            }
            if (v <= w) {
                lo = p;
                vlo = v;
            }
        }
        const bool ok = act && vlo == w;
        const int32_t x = ok ? __ldg(G.eid + j) : 0;
        const int32_t y = ok ? __ldg(G.eid + r.b0 + lo) : 0;
        on_triangles(G.ss, e1, ok, x, y, false, 0, 0, l, g, ap);
    }
}

// Largest q in [0, nh) with cb[q] <= w (cb ascending, cb[0] = 0).
__device__ __forceinline__ int chunk_owner(const uint32_t* cb, int nh, uint32_t w) {
    int lo = 0, hi = nh - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldcg(cb + mid) <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One sub-level over the whole grid (ProcessSubLevel).  gsz = lanes per
// light edge (1, 16 or 32); heavy chunks go one per warp.
template <typename Off>
__device__ void process_frontier(const Graph<Off>& G, const Frontier cur, int nl, int nh, uint32_t nchunk, int gsz,
                                 int32_t l, int32_t g, const Appender& ap) {
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    if (gsz == 16) {
        const int lane = threadIdx.x & 31;
        for (int64_t pw = gtid / 32; 2 * pw < nl; pw += nth / 32) {
            const int64_t i = 2 * pw + (lane >> 4);
            const bool valid = i < nl;
            const int32_t e1 = valid ? __ldcg(cur.light + i) : 0;
            Rows<Off> r{0, 0, 0, 0, -1};
            if (valid) r = rows_of<Off>(G, e1);
            if (__all_sync(FULL_MASK, !valid || r.b1 - r.b0 <= 64))
                walk_half_reg<Off>(G, valid, e1, r, lane & 15, l, g, ap);
            else if (valid)
                walk_rows<Off>(G, e1, r.a0, r.a1, r, lane & 15, 16, l, g, ap);
        }
    } else {
        const int64_t ngrp = nth / gsz;
        const int sub = (int)(gtid % gsz);
        for (int64_t i = gtid / gsz; i < nl; i += ngrp) {
            const int32_t e1 = __ldcg(cur.light + i);
            const Rows<Off> r = rows_of<Off>(G, e1);
            if (gsz == 32)
                walk_warp<Off>(G, e1, r.a0, r.a1, r, sub, l, g, ap);
            else
                walk_rows<Off>(G, e1, r.a0, r.a1, r, sub, gsz, l, g, ap);
        }
    }
    // heavy chunks: warp w takes the contiguous chunk range [c0, c1).  With
    // the owner map, one load gives a chunk's edge and its place in the row
    // (the next chunk's entry is fetched during the current walk); without
    // it, the owning edge is found once by search and the warp walks forward
    // through the list.
    const int lane = threadIdx.x & 31;
    const uint64_t nw = (uint64_t)(nth / 32), w = (uint64_t)(gtid / 32);
    const uint32_t c0 = (uint32_t)((uint64_t)nchunk * w / nw), c1 = (uint32_t)((uint64_t)nchunk * (w + 1) / nw);
    if (c0 < c1 && nchunk <= G.ocap) {
        int2 o = __ldcg(cur.owner + c0);
        int32_t e1 = o.x;
        Rows<Off> r = rows_of<Off>(G, e1);
        for (uint32_t c = c0; c < c1; c++) {
            const int2 on = c + 1 < c1 ? __ldcg(cur.owner + c + 1) : o;
            const int64_t s0 = (int64_t)r.a0 + (int64_t)o.y * G.hc;
            const int64_t s1 = min((int64_t)r.a1, s0 + (int64_t)G.hc);
            walk_warp<Off>(G, e1, (Off)s0, (Off)s1, r, lane, l, g, ap);
            if (on.x != e1) {
                e1 = on.x;
                r = rows_of<Off>(G, e1);
            }
            o = on;
        }
    } else if (c0 < c1) {
        int q = chunk_owner(cur.cbase, nh, c0);
        uint32_t qb = __ldcg(cur.cbase + q);
        uint32_t qn = q + 1 < nh ? __ldcg(cur.cbase + q + 1) : nchunk;
        int32_t e1 = __ldcg(cur.heavy + q);
        Rows<Off> r = rows_of<Off>(G, e1);
        for (uint32_t c = c0; c < c1; c++) {
            while (c >= qn) {  // every heavy edge owns at least one chunk
                q++;
                qb = qn;
                qn = q + 1 < nh ? __ldcg(cur.cbase + q + 1) : nchunk;
                e1 = __ldcg(cur.heavy + q);
                r = rows_of<Off>(G, e1);
            }
            const int64_t s0 = (int64_t)r.a0 + (int64_t)(c - qb) * G.hc;
            const int64_t s1 = min((int64_t)r.a1, s0 + (int64_t)G.hc);
            walk_warp<Off>(G, e1, (Off)s0, (Off)s1, r, lane, l, g, ap);
        }
    }
}

// Lanes per light edge for each variant.
__host__ __device__ __forceinline__ int group_of(int v) {
    return v == TRUSS_VAR_THREAD ? 1 : (v == TRUSS_VAR_GROUP ? 16 : 32);
}

struct TuneTable {
    int8_t v[TRUSS_TUNE_CLASSES];
};

__host__ __device__ __forceinline__ int ilog2_floor(int64_t x) {
    int r = 0;
    while (x > 1) {
        x >>= 1;
        r++;
    }
    return r;
}

// class of a sub-level in the autotuned table (see truss.h)
__host__ __device__ __forceinline__ int tune_class(int64_t nl, int64_t dsum, int64_t size) {
    const int a = min(15, ilog2_floor(1 + nl));
    const int b = min(7, ilog2_floor(1 + dsum / (size > 0 ? size : 1)));
    return 8 * a + b;
}

// Lanes per light edge for a sub-level under a fixed or table-driven
// policy.  Default: half a warp per light edge -- on the power-law and
// geometric workloads it peels 3 % faster than a warp per edge and far
// faster than a thread per edge.
__host__ __device__ __forceinline__ int pick_group(int variant, int64_t nl, int64_t dsum, int64_t size,
                                                   const TuneTable& tt) {
    if (variant >= TRUSS_VAR_THREAD && variant <= TRUSS_VAR_WARP) return group_of(variant);
    const int t = tt.v[tune_class(nl, dsum, size)];
    return t >= 0 ? group_of(t) : 16;
}

// the learned policy is consulted only when a sub-level has this many light
// edges (below it the light-edge mapping barely matters)
constexpr int LEARN_MIN_LIGHT = 64;

// Warp-aggregated append of matched edges to the light or heavy list.
__device__ __forceinline__ void warp_classify_append(bool hit, int32_t e, const int32_t* dmin, int hc, uint32_t ocap,
                                                     const Frontier& out, const Slot& cnt) {
    if (!__any_sync(FULL_MASK, hit)) return;
    const int d = hit ? __ldg(dmin + e) : 0;
    {
        unsigned long long sd = warp_sum((unsigned long long)d);
        int md = d;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) md = max(md, __shfl_xor_sync(FULL_MASK, md, o));
        if (lane_id() == 0) {
            atomicAdd(cnt.dsum, sd);
            atomicMax(cnt.dmax, md);
        }
    }
    int* nl = cnt.nl;
    unsigned long long* hcp = cnt.hc;
    const bool light = hit && d <= LIGHT;
    warp_append(light, e, out.light, nl);
    const bool heavy = hit && !light;
    const unsigned b = __ballot_sync(FULL_MASK, heavy);
    if (b) {
        const int lane = (int)lane_id();
        const uint32_t c = heavy ? nchunks_of(d, hc) : 0u;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        const uint32_t total = __shfl_sync(FULL_MASK, x, 31);
        unsigned long long old = 0;
        if (lane == 0) old = atomicAdd(hcp, ((unsigned long long)__popc(b) << 32) | total);
        old = __shfl_sync(FULL_MASK, old, 0);
        if (heavy) {
            const int q = (int)(old >> 32) + __popc(b & lanemask_lt());
            out.heavy[q] = e;
            out.cbase[q] = (uint32_t)old + x - c;
            write_owner(out, ocap, (uint32_t)old + x - c, c, e);
        }
    }
}


// Scan at level l over the live edges: `in` lists them (nullptr: all m
// edges, in id order).  curr <- {e : S[e] = l}, split into light / heavy
// lists, their stamps <- g; edges with S > l are the live list of the next
// Scan (`keep`); cnt.minv <- min(cnt.minv, min{S[e] : S[e] > l}).  Edges
// below l are processed and drop out for good.  Each thread takes SI
// consecutive list entries per step (16-byte loads where aligned).  A whole
// block step places its light, heavy and surviving edges with one block
// prefix sum and at most three atomics (light count; heavy count and chunk
// total packed in one 64-bit word, which keeps heavy positions and chunk
// bases in the same order; survivors); the shorter-row sum and maximum are
// kept per thread and added once per block at the end.
constexpr int SI = 4;

__device__ void scan_level(int2* ss, const int32_t* in, int64_t nin, int32_t* keep, int32_t l, int32_t g,
                           const Frontier out, const Slot& cnt, const int32_t* dmin, int hc, uint32_t ocap,
                           PeelSmem* sm) {
    int mn = INT_MAX;
    unsigned long long dsum = 0;
    int dmax = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * SI;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * SI; base < nin; base += step) {
        const int64_t i0 = base + (int64_t)threadIdx.x * SI;
        int32_t e[SI];
        int sv[SI];
        if (i0 + SI <= nin) {
            if (in) {
                const int4 a = __ldcg(reinterpret_cast<const int4*>(in + i0));
                e[0] = a.x; e[1] = a.y; e[2] = a.z; e[3] = a.w;
#pragma unroll
                for (int k = 0; k < SI; k++) sv[k] = __ldcg(&ss[e[k]].x);
            } else {
                const int4* p = reinterpret_cast<const int4*>(ss + i0);
                const int4 a = __ldcg(p), b = __ldcg(p + 1);
                sv[0] = a.x; sv[1] = a.z; sv[2] = b.x; sv[3] = b.z;
#pragma unroll
                for (int k = 0; k < SI; k++) e[k] = (int32_t)(i0 + k);
            }
        } else {
#pragma unroll
            for (int k = 0; k < SI; k++) {
                const bool ok = i0 + k < nin;
                e[k] = ok ? (in ? __ldcg(in + i0 + k) : (int32_t)(i0 + k)) : 0;
                sv[k] = ok ? __ldcg(&ss[e[k]].x) : INT_MIN;
            }
        }
        // per thread: light / heavy / survivor counts (SI bits each) and
        // the heavy edges' chunk total
        uint32_t c[SI];
        unsigned nlt = 0, nht = 0, nlv = 0;
        uint32_t ct = 0;
#pragma unroll
        for (int k = 0; k < SI; k++) {
            c[k] = 0;
            if (sv[k] == l) {
                ss[e[k]].y = g;
                const int d = __ldg(dmin + e[k]);
                dsum += (unsigned)d;
                dmax = max(dmax, d);
                if (d <= LIGHT) {
                    nlt++;
                } else {
                    c[k] = nchunks_of(d, hc);
                    ct += c[k];
                    nht++;
                }
            } else if (sv[k] > l) {
                mn = min(mn, sv[k]);
                nlv++;
            }
        }
        // block exclusive prefix of (light, heavy, survivors) packed 16 bits
        // apiece (a block step holds PT * SI < 2^16 entries) and of chunks
        unsigned long long x = (unsigned long long)nlt | ((unsigned long long)nht << 16) |
                               ((unsigned long long)nlv << 32);
        uint32_t xc = ct;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL_MASK, x, o);
            const uint32_t yc = __shfl_up_sync(FULL_MASK, xc, o);
            if (lane >= o) {
                x += y;
                xc += yc;
            }
        }
        if (lane == 31) {
            sm->wtot[warp] = x;
            sm->wsum[warp] = xc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long run = 0;
            uint32_t runc = 0;
            for (int w = 0; w < PW; w++) {
                const unsigned long long t = sm->wtot[w];
                const uint32_t tc = sm->wsum[w];
                sm->wtot[w] = run;
                sm->wsum[w] = runc;
                run += t;
                runc += tc;
            }
            const int tl = (int)(run & 0xffff), th = (int)((run >> 16) & 0xffff), tv = (int)(run >> 32);
            // the three reservations in flight before any result is used
            const int lb = tl ? atomicAdd(cnt.nl, tl) : 0;
            const unsigned long long old = th ? atomicAdd(cnt.hc, ((unsigned long long)th << 32) | runc) : 0ull;
            const int vb = tv ? atomicAdd(cnt.nlive, tv) : 0;
            sm->lbase = lb;
            sm->hq0 = (int)(old >> 32);
            sm->hb0 = (uint32_t)old;
            sm->bbase = vb;
        }
        __syncthreads();
        const unsigned long long ex = sm->wtot[warp] + x -
                                      ((unsigned long long)nlt | ((unsigned long long)nht << 16) |
                                       ((unsigned long long)nlv << 32));
        int pl = sm->lbase + (int)(ex & 0xffff);
        int ph = sm->hq0 + (int)((ex >> 16) & 0xffff);
        int pv = sm->bbase + (int)(ex >> 32);
        uint32_t pc = sm->hb0 + sm->wsum[warp] + xc - ct;
#pragma unroll
        for (int k = 0; k < SI; k++) {
            if (sv[k] == l) {
                if (c[k] == 0) {
                    out.light[pl++] = e[k];
                } else {
                    out.heavy[ph] = e[k];
                    out.cbase[ph] = pc;
                    write_owner(out, ocap, pc, c[k], e[k]);
                    ph++;
                    pc += c[k];
                }
            } else if (sv[k] > l) {
                keep[pv++] = e[k];
            }
        }
        // no barrier needed here: a warp's shuffles in the next step (or
        // below) come after all its lanes read their offsets, and thread 0
        // rewrites the shared offsets only after the next step's barrier
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(FULL_MASK, mn, o));
        dmax = max(dmax, __shfl_xor_sync(FULL_MASK, dmax, o));
    }
    dsum = warp_sum(dsum);
    if (lane == 0) {
        sm->bmin[warp] = mn;
        sm->wtot[warp] = dsum;
        sm->wcnt[warp] = dmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = INT_MAX, bm = 0;
        unsigned long long bs = 0;
        for (int w = 0; w < PW; w++) {
            b = min(b, sm->bmin[w]);
            bm = max(bm, sm->wcnt[w]);
            bs += sm->wtot[w];
        }
        if (b != INT_MAX) atomicMin(cnt.minv, b);
        if (bs) {
            atomicAdd(cnt.dsum, bs);
            atomicMax(cnt.dmax, bm);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------- standalone kernels

__global__ void __launch_bounds__(PT) k_scan(int2* ss, const int32_t* in, int64_t nin, int32_t* keep, int32_t l,
                                              int32_t g, Frontier out, int* ctr, const int32_t* dmin, int hc,
                                              uint32_t ocap) {
    __shared__ PeelSmem sm;
    smem_init(&sm);
    scan_level(ss, in, nin, keep, l, g, out, slot_of(ctr, 0), dmin, hc, ocap, &sm);
}

// split a given edge list into light / heavy lists (state-level entry point)
__global__ void k_classify(const int32_t* __restrict__ edges, int64_t k, const int32_t* dmin, int hc, uint32_t ocap,
                           Frontier out, int* ctr) {
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < k; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool hit = i < k;
        warp_classify_append(hit, hit ? edges[i] : 0, dmin, hc, ocap, out, slot_of(ctr, 0));
    }
}

// one sub-level: lists of side `cur` with the counts given, next lists into
// side `nxt` counted in slot 1
// In a decomposition run (in_run) level 0 is the first level, so its edges
// have had support 0 from the start: they lie in no triangle and there is
// nothing to walk.  A caller-set state (truss_peel_sublevel) may differ.
__device__ __forceinline__ bool walk_needed(int32_t l, int in_run) { return l > 0 || !in_run; }

template <typename Off>
__global__ void __launch_bounds__(PT) k_process(Graph<Off> G, Frontier cur, int nl, int nh, uint32_t nchunk, int gsz,
                                                int32_t l, int32_t g, Frontier nxt, int* ctr, int in_run) {
    __shared__ PeelSmem sm;
    smem_init(&sm);
    const Appender ap{&sm, nxt, slot_of(ctr, 1), G.dmin, G.hc, G.ocap};
    if (walk_needed(l, in_run)) process_frontier<Off>(G, cur, nl, nh, nchunk, gsz, l, g, ap);
    ap.flush();
}

// ------------------------------------------------------------ grid barrier

// Barrier over all blocks of a cooperative launch.  One counter counts
// arrivals since the launch began (never reset): the k-th barrier is passed
// once it reaches k * nblocks.  Thread 0 arrives with one acq_rel atomic and
// spins with acquire loads; it also copies the counter slot the next phase
// needs into shared memory, so the block reads it without further round
// trips.  Every wait is bounded: past timeout_ns the block records
// TRUSS_ETIMEOUT and returns false; a block that sees an error recorded
// also returns false.
__device__ bool grid_barrier(int* ctr, unsigned nblocks, uint64_t timeout_ns, unsigned& epoch, int read_slot,
                             SlotVals* sv) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* count = reinterpret_cast<unsigned*>(ctr + C_BAR_COUNT);
        epoch += 1;
        const unsigned target = epoch * nblocks;
        unsigned v;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(v) : "l"(count) : "memory");
        v += 1;
        int ok = 1;
        if ((int)(v - target) < 0) {
            // tight poll; the error word and the clock are read at polls
            // 1, 2, 4, ..., 256 and then every 256 (each read is another L2
            // round trip; the early reads let short limits take effect)
            const uint64_t t0 = global_ns();
            for (unsigned spin = 1;; spin++) {
                v = ld_acquire_gpu_u32(count);
                if ((int)(v - target) >= 0) break;
                if ((spin & (spin - 1)) == 0 || (spin & 255u) == 0) {
                    if (ld_acquire_gpu(ctr + C_ERR) != 0) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > timeout_ns) {
                        atomicCAS(ctr + C_ERR, 0, TRUSS_ETIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (ok && read_slot >= 0) {
            const int4* src = reinterpret_cast<const int4*>(slots(ctr) + read_slot);
            int4* dst = reinterpret_cast<int4*>(sv);
            dst[0] = __ldcg(src);
            dst[1] = __ldcg(src + 1);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole of Algorithm 4 in one cooperative launch.  Every thread follows
// the same (l, g, phase) sequence because every branch depends only on
// counters read after a barrier.  Phase p (each Scan and each sub-level)
// writes its counters to slot p & 3; slot (p+2) & 3 is cleared during phase
// p: its last readers read it right after the barrier that ended phase p-2,
// and the barrier ending phase p-1 lies in between.
// MINB blocks per SM: 6 (at most 40 registers a thread) gives the warps that
// large frontiers of short rows need; 4 (64 registers, no spills) runs the
// dependent-load chains of many small sub-levels of long rows fastest.
// Measured on the power-law and geometric workloads against 5 and 7.
// With `held` >= 0 the launch also stops (stop = 1) at the top of a level
// once at most cmp_live_pct(held) % of the `held` edges its rows hold are
// unprocessed (and held >= min_held): the host then compacts the rows and
// resumes the loop with `resume` set, from the state in the counter block.
template <typename Off, int MINB>
__global__ void __launch_bounds__(PT, MINB)
    k_persistent(Graph<Off> G, Frontier f0, Frontier f1, int32_t* live0, int32_t* live1, int* ctr, int variant,
                 int level_jump, uint64_t timeout_ns, truss_sublevel_trace* trace, int64_t max_trace,
                 const float* sched, TuneTable tt, int64_t held, int64_t min_held, int resume) {
    __shared__ PeelSmem sm;
    __shared__ __align__(16) SlotVals sv;
    __shared__ int s_choice;
    smem_init(&sm);
    const unsigned nblocks = gridDim.x;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    PState* st = reinterpret_cast<PState*>(ctr + C_ST);
    unsigned epoch = 0;
    int32_t l = 0, g = 0;
    int64_t processed = 0, nsub = 0, sc = 0, nlevel = 0, p = 0;
    int64_t nlive = G.m;  // edges the next Scan visits
    int64_t scanned = 0, walked = 0;
    uint64_t scan_ns = 0;
    if (resume) {
        l = st->l;
        g = st->g;
        processed = st->processed;
        nsub = st->nsub;
        sc = st->sc;
        nlevel = st->nlevel;
        nlive = st->nlive;
        scanned = st->scanned;
        walked = st->walked;
        scan_ns = (uint64_t)st->scan_ns;
    }
    int stop = 0;
    while (processed < G.m) {
        if (held >= min_held && (G.m - processed) * 100 <= held * cmp_live_pct(held) && processed > 0) {
            stop = 1;  // the rows are due for compaction
            break;
        }
        uint64_t ts = 0;
        if (leader) {
            clear_slot_vals(slots(ctr) + ((p + 2) & 3));
            ts = global_ns();
        }
        const Frontier cur = (g & 1) ? f1 : f0;
        int s = (int)(p & 3);
        const int32_t* lin = sc == 0 ? nullptr : ((sc & 1) ? live0 : live1);
        int32_t* lout = (sc & 1) ? live1 : live0;
        scanned += nlive;
        scan_level(G.ss, lin, nlive, lout, l, g, cur, slot_of(ctr, s), G.dmin, G.hc, G.ocap, &sm);
        if (!grid_barrier(ctr, nblocks, timeout_ns, epoch, s, &sv)) return;
        if (leader) scan_ns += global_ns() - ts;
        SlotVals v = sv;
        nlive = v.nlive;
        p++;
        sc++;
        if (v.nl + (int)(v.hc >> 32) == 0) {
            if (v.minv == INT_MAX) break;
            l = level_jump ? v.minv : l + 1;
            continue;
        }
        nlevel++;
        while (v.nl + (int)(v.hc >> 32) > 0) {
            const int nl = v.nl;
            const int nh = (int)(v.hc >> 32);
            const uint32_t nchunk = (uint32_t)v.hc;
            int gsz = pick_group(variant, nl, (int64_t)v.dsum, (int64_t)nl + nh, tt);
            if (variant == TRUSS_VAR_LEARNED && sched && nl >= LEARN_MIN_LIGHT) {
                // warp 0 of every block evaluates the model on the same
                // inputs, so every block takes the same decision
                if (threadIdx.x < 32) {
                    float x[SF];
                    sched_features((int64_t)nl + nh, (int64_t)v.dsum, v.dmax, l, G.m - processed, x);
                    const int c = sched_pick(sched, x);
                    if (threadIdx.x == 0) s_choice = c;
                }
                __syncthreads();
                if (s_choice >= 0) gsz = group_of(s_choice);
            }
            const int q = (int)(p & 3);
            uint64_t t0 = 0;
            if (leader) {
                if (nsub < max_trace) {
                    truss_sublevel_trace& r = trace[nsub];
                    r.level = l;
                    r.group = gsz;
                    r.n_light = nl;
                    r.n_heavy = nh;
                    r.n_chunks = nchunk;
                    r.dmax = v.dmax;
                    r.dsum = (int64_t)v.dsum;
                    r.todo = G.m - processed;
                    r.scan_ns = (int64_t)scan_ns;
                }
                scan_ns = 0;
                clear_slot_vals(slots(ctr) + ((p + 2) & 3));
                t0 = global_ns();
            }
            processed += nl + nh;
            if (l > 0) walked += (int64_t)v.dsum;
            const Frontier cu = (g & 1) ? f1 : f0;
            const Frontier nx = (g & 1) ? f0 : f1;
            const Appender ap{&sm, nx, slot_of(ctr, q), G.dmin, G.hc, G.ocap};
            if (walk_needed(l, 1)) process_frontier<Off>(G, cu, nl, nh, nchunk, gsz, l, g, ap);
            ap.flush();
            if (!grid_barrier(ctr, nblocks, timeout_ns, epoch, q, &sv)) return;
            if (leader && nsub < max_trace) trace[nsub].t_ns = (int64_t)(global_ns() - t0);
            v = sv;
            p++;
            g++;
            nsub++;
        }
        l++;
    }
    if (leader) {
        st->l = l;
        st->g = g;
        st->stop = stop;
        st->processed = processed;
        st->nsub = nsub;
        st->sc = sc;
        st->nlevel = nlevel;
        st->nlive = nlive;
        st->scanned = scanned;
        st->walked = walked;
        st->scan_ns = (long long)scan_ns;
        ctr[C_NSUB] = (int)nsub;
        ctr[C_NSCAN] = (int)sc;
        ctr[C_NLEVEL] = (int)nlevel;
        ctr[C_LAST_L] = l;
        *reinterpret_cast<long long*>(ctr + C_SCANNED) = scanned;
        *reinterpret_cast<long long*>(ctr + C_WALKED) = walked;
    }
}

// ------------------------------------------------------- row compaction
//
// A processed edge never takes part in a triangle again (Algorithm 5 skips
// every triangle with a processed edge), so its two row entries can leave
// the rows.  Between levels, once few enough of the edges the rows hold are
// unprocessed (cmp_live_pct), the live entries are packed into a second buffer (rows
// keep their order and follow one another), every vertex gets its new row
// bounds, and every live edge new records: its shorter live row (walked),
// its longer live row (searched) and the walk length dmin, which also sets
// its light / heavy class.  So ProcessSubLevel walks min(live d(u), live
// d(v)) entries instead of min(d(u), d(v)), and searches shorter rows.
// Four or five launches, A-D over the same grid:
//   L  (graphs of 2^25 edges or more) one bit per edge: unprocessed (a
//      sequential pass over the pairs, so the per-slot test below reads
//      L2-resident bits, not a random pair);
//   A  per tile of CT slots: the live bits, and the tile's offset within its
//      block's contiguous range of tiles; per block, its live total;
//   B  one block: exclusive prefix of the block totals;
//   C  scatter the live entries; map each vertex's bounds through P(s), the
//      number of live slots before slot s;
//   D  the records of the live edges.
// The hub bitmaps keep describing the rows as built: a longer row of a hub
// that still holds more than 128 live entries is probed there, and the
// probe's slot is read in the edge ids as built (a stale bit leads to a
// processed edge, whose triangle is skipped).

constexpr int CT = PT;        // slots per compaction tile (one per thread)
constexpr int CTW = CT / 32;  // bit words per tile
constexpr int CUN = 4;        // tiles per block step in phase A (loads in flight)

template <typename Off>
struct Compactor {
    const int32_t* col;  // source rows (the rows as built, or the last compaction's)
    const int32_t* eid;
    int64_t nslots;      // source slots in use
    int32_t* tcol;       // target rows
    int32_t* teid;
    Off* vstart;         // per vertex: row bounds in the target (updated in place)
    Off* vend;
    int first;           // the source is the rows as built (bounds from rowptr)
    const Off* rowptr;
    const int32_t* hub_of;  // per vertex: hub index, -1; nullptr without hubs
    const int2* el;
    const int2* ss;
    int32_t g;           // sub-level number: processed <=> stamp < g
    int32_t n;
    Off* rows;           // working records
    int32_t* dmin;
    int32_t* lhub;
    const uint32_t* live;  // one bit per edge: unprocessed (k_cmp_live); nullptr: read the pairs
    uint32_t* bits;      // one bit per source slot: its edge is live
    int32_t* toff;       // per tile: live slots before it within its block's range
    long long* bsum;     // per block: live total [0, B), then its offset [B, 2B)
    int64_t live_slots;  // 2 x unprocessed edges: slots in the target
    int64_t hub_min;     // a hub's longer row is probed in its bitmap above this many live entries
};

// block b of B takes tiles [nt b / B, nt (b + 1) / B)
__host__ __device__ __forceinline__ int64_t tile_lo(int64_t nt, int64_t b, int64_t B) { return nt * b / B; }
// the block whose range holds tile t
__device__ __forceinline__ int64_t tile_owner(int64_t nt, int64_t t, int64_t B) { return ((t + 1) * B - 1) / nt; }

// live[e / 32] bit e % 32: edge e is unprocessed (stamp >= g).  One
// sequential pass over the (S, stamp) pairs; the bits (m / 8 bytes: 33 MB
// for R-MAT scale 24) stay in L2 for the count below, which would otherwise
// gather a random pair -- one 32-byte sector -- for every row slot.
__global__ void k_cmp_live(const int2* __restrict__ ss, int64_t m, int32_t g, uint32_t* __restrict__ live) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of 32
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; base < m; base += stride) {
        const int64_t e = base + lane;
        const unsigned w = __ballot_sync(FULL_MASK, e < m && __ldg(ss + e).y >= g);
        if (lane == 0) live[base >> 5] = w;
    }
}

template <typename Off>
__global__ void __launch_bounds__(PT) k_cmp_count(Compactor<Off> C) {
    __shared__ int wc[CUN][PW];
    const int64_t nt = (C.nslots + CT - 1) / CT, B = gridDim.x;
    const int64_t t0 = tile_lo(nt, blockIdx.x, B), t1 = tile_lo(nt, blockIdx.x + 1, B);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long carry = 0;  // thread 0's running total
    for (int64_t t = t0; t < t1; t += CUN) {
        int32_t e[CUN];
#pragma unroll
        for (int k = 0; k < CUN; k++) {
            const int64_t s = (t + k) * CT + threadIdx.x;
            e[k] = (t + k < t1 && s < C.nslots) ? __ldg(C.eid + s) : -1;
        }
        bool lv[CUN];
#pragma unroll
        for (int k = 0; k < CUN; k++)
            lv[k] = e[k] >= 0 && (C.live ? ((__ldg(C.live + (e[k] >> 5)) >> (e[k] & 31)) & 1u)
                                         : __ldg(&C.ss[e[k]].y) >= C.g);
#pragma unroll
        for (int k = 0; k < CUN; k++) {
            const unsigned b = __ballot_sync(FULL_MASK, lv[k]);
            if (t + k < t1) {
                if (lane == 0) {
                    C.bits[(t + k) * CTW + warp] = b;
                    wc[k][warp] = __popc(b);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 0; k < CUN && t + k < t1; k++) {
                C.toff[t + k] = (int32_t)carry;
                for (int w = 0; w < PW; w++) carry += wc[k][w];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) C.bsum[blockIdx.x] = carry;
}

// one block: bsum[B + b] = sum of bsum[0, b)
__global__ void k_cmp_blocks(long long* bsum, int B) {
    __shared__ long long part[PT];
    const int per = (B + PT - 1) / PT;
    const int lo = min(B, (int)threadIdx.x * per), hi = min(B, lo + per);
    long long s = 0;
    for (int i = lo; i < hi; i++) s += bsum[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int i = 0; i < PT; i++) {
            const long long v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    long long run = part[threadIdx.x];
    for (int i = lo; i < hi; i++) {
        const long long v = bsum[i];
        bsum[B + i] = run;
        run += v;
    }
}

// live slots before source slot s (0 <= s <= nslots)
template <typename Off>
__device__ __forceinline__ long long live_before(const Compactor<Off>& C, int64_t s, int64_t nt, int64_t B) {
    if (s >= C.nslots) return C.live_slots;
    const int64_t t = s / CT;
    const int r = (int)(s - t * CT), w = r >> 5, bit = r & 31;
    long long p = C.bsum[B + tile_owner(nt, t, B)] + C.toff[t];
    const uint32_t* bw = C.bits + t * CTW;
    for (int k = 0; k < w; k++) p += __popc(bw[k]);
    return p + __popc(bw[w] & ((1u << bit) - 1u));
}

template <typename Off>
__global__ void __launch_bounds__(PT) k_cmp_scatter(Compactor<Off> C) {
    __shared__ long long base;
    const int64_t nt = (C.nslots + CT - 1) / CT, B = gridDim.x;
    const int64_t t0 = tile_lo(nt, blockIdx.x, B), t1 = tile_lo(nt, blockIdx.x + 1, B);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = C.bsum[B + blockIdx.x];
    __syncthreads();
    for (int64_t t = t0; t < t1; t++) {
        const uint32_t* bw = C.bits + t * CTW;
        const uint32_t mine = bw[warp];
        if (!((mine >> lane) & 1u)) continue;
        int before = 0;
        for (int k = 0; k < warp; k++) before += __popc(bw[k]);
        const long long pos = base + C.toff[t] + before + __popc(mine & ((1u << lane) - 1u));
        const int64_t s = t * CT + threadIdx.x;
        C.tcol[pos] = __ldg(C.col + s);
        C.teid[pos] = __ldg(C.eid + s);
    }
    // new row bounds of every vertex
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < C.n; v += (int64_t)gridDim.x * blockDim.x) {
        const Off a = C.first ? C.rowptr[v] : C.vstart[v];
        const Off b = C.first ? C.rowptr[v + 1] : C.vend[v];
        C.vstart[v] = (Off)live_before(C, (int64_t)a, nt, B);
        C.vend[v] = (Off)live_before(C, (int64_t)b, nt, B);
    }
}

// records of the live edges of `list` (the last Scan's survivors: every
// unprocessed edge is among them)
template <typename Off>
__global__ void k_cmp_records(Compactor<Off> C, const int32_t* __restrict__ list, int64_t k) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = list[i];
        if (C.ss[e].y < C.g) continue;  // processed
        const int2 xy = C.el[e];
        const Off u0 = C.vstart[xy.x], u1 = C.vend[xy.x], v0 = C.vstart[xy.y], v1 = C.vend[xy.y];
        const bool ushort = u1 - u0 <= v1 - v0;
        const int32_t lv = ushort ? xy.y : xy.x;
        const Off llen = ushort ? v1 - v0 : u1 - u0;
        const int32_t h = C.hub_of ? C.hub_of[lv] : -1;
        Off* r = C.rows + 4 * (int64_t)e;
        r[0] = ushort ? u0 : v0;
        r[1] = ushort ? u1 : v1;
        if (h >= 0 && llen > (Off)C.hub_min) {
            // probed in the hub's bitmap of the row as built
            r[2] = C.rowptr[lv];
            r[3] = C.rowptr[lv] + llen;
            C.lhub[e] = h;
        } else {
            r[2] = ushort ? v0 : u0;
            r[3] = ushort ? v1 : u1;
            C.lhub[e] = -1;
        }
        C.dmin[e] = (int32_t)(ushort ? u1 - u0 : v1 - v0);
    }
}

// before a resumed persistent launch: clear the phase slots and the barrier
// count, keep everything else
__global__ void k_resume_counters(int* ctr) {
    for (int i = threadIdx.x; i < C_ERR; i += blockDim.x) ctr[i] = 0;
    __syncthreads();
    if (threadIdx.x < 4) clear_slot_vals(slots(ctr) + threadIdx.x);
}

// --------------------------------------------------------------- helpers

__global__ void k_truss_out(const int2* __restrict__ ss, int64_t m, const int32_t* __restrict__ perm,
                            int32_t* __restrict__ out, int add) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[perm ? perm[e] : e] = ss[e].x + add;
}

__global__ void k_step_out(const int2* __restrict__ ss, int64_t m, const int32_t* __restrict__ perm,
                           int32_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[perm ? perm[e] : e] = ss[e].y;
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

__global__ void k_clear_slot(int* ctr, int q) {
    if (threadIdx.x == 0) clear_slot_vals(slots(ctr) + q);
}

__global__ void k_init_counters(int* ctr) {
    for (int i = threadIdx.x; i < C_TOTAL; i += blockDim.x) ctr[i] = 0;
    __syncthreads();
    if (threadIdx.x < 4) clear_slot_vals(slots(ctr) + threadIdx.x);
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

// Validates a caller's frontier before any kernel indexes with it: every id
// in [0, m) and none twice (seen: a zeroed bitmap of m bits).  Only curr[0,
// k) and the bitmap are touched; a bad id sets bit 0 of *err, a repeat bit 1.
__global__ void k_check_curr(const int32_t* __restrict__ curr, int64_t k, int64_t m, uint32_t* __restrict__ seen,
                             int* __restrict__ err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = curr[i];
        if (e < 0 || (int64_t)e >= m) {
            atomicOr(err, 1);
            continue;
        }
        const uint32_t bit = 1u << (e & 31);
        if (atomicOr(&seen[e >> 5], bit) & bit) atomicOr(err, 2);
    }
}

__global__ void k_map_ids(const int32_t* __restrict__ in, int64_t k, const int32_t* __restrict__ map,
                          int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = map ? map[in[i]] : in[i];
}

template <typename Off>
__global__ void k_dmin(const Off* __restrict__ rowptr, const int2* __restrict__ el, int64_t m, int32_t* __restrict__ dmin,
                       Off* __restrict__ rows, const int32_t* __restrict__ hub_of, int32_t* __restrict__ lhub) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int2 xy = el[e];
        const Off u0 = rowptr[xy.x], u1 = rowptr[xy.x + 1], v0 = rowptr[xy.y], v1 = rowptr[xy.y + 1];
        const bool ushort = u1 - u0 <= v1 - v0;
        dmin[e] = (int32_t)(ushort ? u1 - u0 : v1 - v0);
        lhub[e] = hub_of ? hub_of[ushort ? xy.y : xy.x] : -1;
        Off* r = rows + 4 * e;
        r[0] = ushort ? u0 : v0;
        r[1] = ushort ? u1 : v1;
        r[2] = ushort ? v0 : u0;
        r[3] = ushort ? v1 : u1;
    }
}

// Hub bitmaps: for each vertex of degree >= the hub threshold, its
// neighbours as bits over vertex ids in 32-byte blocks of 192 ids, each
// block led by the number of neighbours before it; ProcessSubLevel probes
// these rows through hub_find instead of a binary search.
template <typename Off>
__global__ void k_count_deg(const Off* __restrict__ rowptr, int32_t n, int64_t thr, int* cnt) {
    int c = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        c += (rowptr[v + 1] - rowptr[v]) >= thr;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

template <typename Off>
__global__ void k_hub_list(const Off* __restrict__ rowptr, int32_t n, int64_t thr, int32_t* __restrict__ hub_of,
                           int32_t* __restrict__ hub_vert, int* cnt) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int h = -1;
        if (rowptr[v + 1] - rowptr[v] >= thr) {
            h = atomicAdd(cnt, 1);
            hub_vert[h] = (int32_t)v;
        }
        hub_of[v] = h;
    }
}

template <typename Off>
__global__ void k_hub_fill(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ hub_vert, int32_t nhub, int64_t hw,
                           unsigned long long* __restrict__ bits) {
    for (int32_t h = blockIdx.x; h < nhub; h += gridDim.x) {
        const int32_t v = hub_vert[h];
        unsigned long long* B = bits + (int64_t)h * hw;
        for (Off j = rowptr[v] + threadIdx.x; j < rowptr[v + 1]; j += blockDim.x) {
            const int32_t w = col[j];
            const int32_t b = w / 192, r = w - b * 192;
            atomicOr(B + 4 * (int64_t)b + 1 + (r >> 6), 1ull << (r & 63));
        }
    }
}

// per hub: word 0 of each block <- neighbours in the blocks before it.  A
// block takes a hub; each thread owns HPRE consecutive 32-byte blocks a
// round (their counts kept in registers), one block-wide scan a round.
constexpr int HPRE = 8;

__global__ void k_hub_pre(unsigned long long* __restrict__ bits, int32_t nhub, int64_t hw) {
    __shared__ uint32_t wsum[32];
    const int64_t nb = hw >> 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int32_t h = blockIdx.x; h < nhub; h += gridDim.x) {
        unsigned long long* B = bits + (int64_t)h * hw;
        uint32_t carry = 0;
        for (int64_t base = 0; base < nb; base += (int64_t)blockDim.x * HPRE) {
            const int64_t b0 = base + (int64_t)threadIdx.x * HPRE;
            uint32_t c[HPRE];
            uint32_t tot = 0;
#pragma unroll
            for (int k = 0; k < HPRE; k++) {
                const int64_t b = b0 + k;
                c[k] = b < nb ? (uint32_t)(__popcll(B[4 * b + 1]) + __popcll(B[4 * b + 2]) + __popcll(B[4 * b + 3]))
                              : 0u;
                tot += c[k];
            }
            uint32_t x = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL_MASK, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            if (warp == 0) {
                uint32_t w = lane < nwarp ? wsum[lane] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(FULL_MASK, w, o);
                    if (lane >= o) w += y;
                }
                if (lane < nwarp) wsum[lane] = w;
            }
            __syncthreads();
            uint32_t before = carry + (warp ? wsum[warp - 1] : 0u) + x - tot;
#pragma unroll
            for (int k = 0; k < HPRE; k++) {
                const int64_t b = b0 + k;
                if (b < nb) B[4 * b] = before;
                before += c[k];
            }
            carry += wsum[nwarp - 1];
            __syncthreads();  // wsum is rewritten next round
        }
    }
}

// ------------------------------------------------------------- host side

template <typename Off>
int process_blocks(const truss_graph* g) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_process<Off>, PT, 0);
    return std::max(1, per_sm) * g->sms;
}

template <typename Off>
Graph<Off> graph_view(truss_graph* g) {
    return Graph<Off>{(const Off*)g->rowptr, g->col, g->eid, g->el, g->dmin, (const Off*)g->rows, g->lhub,
                      g->hub_bits, g->hub_words, g->eid, g->ss, g->m, g->hc, g->ocap};
}

// ---------------------------------------------------- row compaction (host)


// Compaction of one run: whether it is on, the smallest row set worth
// compacting, and what it did.
struct CmpRun {
    int enabled = 0;
    int64_t min_held = 0;
    int buf = -1;             // rows the peel reads: -1 as built, 0 (wcol) or 1 (tcol)
    int64_t held = 0;         // edges the current rows hold
    int count = 0;            // compactions run
    int64_t slots = 0;        // source slots they visited
};

constexpr int CMP_MAX_BLOCKS = 2048;
// After a compaction a hub's longer row is probed in its bitmap only while
// it holds more than this many live entries; shorter rows are searched (128
// entries and fewer fit the register-resident warp search).  Measured on
// R-MAT scale 24: peel 1.22 s at 128 and 1024, 1.32 s at 8192, 1.43 s with
// no bitmap after the first compaction (Chung-Lu 2^20: 32.9 / 35.8 / 37.7 /
// 37.8 ms): the bitmaps keep paying on compacted rows.
constexpr int64_t CMP_HUB_MIN_LIVE = 128;

int cmp_blocks(const truss_graph* g) { return std::min(CMP_MAX_BLOCKS, std::max(1, g->sms * 4)); }

// Slots each row buffer holds: the live entries of the first compaction,
// at most 2 m cmp_live_pct(m) / 100 (later ones hold fewer).
size_t cmp_slots(const truss_graph* g) { return (size_t)(2 * g->m * cmp_live_pct(g->m) / 100) + 1; }

void truss_release_compaction(truss_graph* g) {
    cudaFree(g->wcol);
    cudaFree(g->weid);
    cudaFree(g->tcol);
    cudaFree(g->teid);
    cudaFree(g->wrows);
    cudaFree(g->wdmin);
    cudaFree(g->wlhub);
    cudaFree(g->vstart);
    cudaFree(g->vend);
    cudaFree(g->cbits);
    cudaFree(g->clive);
    cudaFree(g->ctoff);
    cudaFree(g->cbsum);
    g->wcol = g->weid = g->tcol = g->teid = nullptr;
    g->wrows = g->vstart = g->vend = nullptr;
    g->wdmin = g->wlhub = nullptr;
    g->cbits = nullptr;
    g->clive = nullptr;
    g->ctoff = nullptr;
    g->cbsum = nullptr;
    g->cmp_ready = 0;
}

// The compaction buffers (about 16 + 4 * sizeof(Off) + 8 bytes per edge, 2
// Off per vertex).  A graph whose buffers do not fit runs without
// compaction (TRUSS_ENOMEM is not returned for it).
int ensure_compaction(truss_graph* g, cudaStream_t s) {
    if (g->cmp_ready) return TRUSS_OK;
    const size_t m = (size_t)g->m + 1, osz = g->off64 ? sizeof(int64_t) : sizeof(int32_t);
    const size_t slots = cmp_slots(g);
    const size_t ntile = (size_t)((2 * g->m + CT - 1) / CT) + 1;
    bool ok = true;
    auto get = [&](void** p, size_t bytes) {
        if (ok && cudaMallocAsync(p, bytes, s) != cudaSuccess) {
            *p = nullptr;
            ok = false;
        }
    };
    get((void**)&g->wcol, sizeof(int32_t) * slots);
    get((void**)&g->weid, sizeof(int32_t) * slots);
    get((void**)&g->tcol, sizeof(int32_t) * slots);
    get((void**)&g->teid, sizeof(int32_t) * slots);
    get(&g->wrows, osz * 4 * m);
    get((void**)&g->wdmin, sizeof(int32_t) * m);
    get((void**)&g->wlhub, sizeof(int32_t) * m);
    get(&g->vstart, osz * ((size_t)g->n + 1));
    get(&g->vend, osz * ((size_t)g->n + 1));
    get((void**)&g->cbits, sizeof(uint32_t) * CTW * ntile);
    get((void**)&g->clive, sizeof(uint32_t) * (m / 32 + 1));
    get((void**)&g->ctoff, sizeof(int32_t) * ntile);
    get((void**)&g->cbsum, sizeof(long long) * 2 * CMP_MAX_BLOCKS);
    if (!ok) {
        cudaGetLastError();  // clear the failed allocation
        cudaStreamSynchronize(s);
        truss_release_compaction(g);
        return TRUSS_ENOMEM;
    }
    g->cmp_ready = 1;
    return TRUSS_OK;
}

// Compaction settings of a run (TRUSS_LOOP_GRAPH never compacts).
CmpRun compact_policy(truss_graph* g, const truss_opts& o, cudaStream_t s) {
    CmpRun c;
    if (o.loop == TRUSS_LOOP_GRAPH || o.compact == 0 || g->m <= 0) return c;
    if (o.compact < 0 && g->m < TRUSS_COMPACT_MIN_EDGES) return c;
    if (ensure_compaction(g, s) != TRUSS_OK) return c;
    c.enabled = 1;
    c.min_held = o.compact < 0 ? TRUSS_COMPACT_MIN_EDGES : 0;
    c.held = g->m;
    return c;
}

// The peel's view of compacted rows in buffer `buf` with the working records.
template <typename Off>
Graph<Off> view_compacted(truss_graph* g, int buf) {
    Graph<Off> G = graph_view<Off>(g);
    G.col = buf == 0 ? g->wcol : g->tcol;
    G.eid = buf == 0 ? g->weid : g->teid;
    G.rows = (const Off*)g->wrows;
    G.dmin = g->wdmin;
    G.lhub = g->wlhub;
    return G;
}

// One compaction before the Scan of a level, at sub-level number gsub, with
// `list` (k entries) holding every unprocessed edge and `processed` edges
// peeled so far.  Moves the rows to the other buffer and returns the view.
template <typename Off>
int run_compaction(truss_graph* g, CmpRun& c, int32_t gsub, int64_t processed, const int32_t* list, int64_t k,
                   cudaStream_t s, Graph<Off>* view) {
    Compactor<Off> C;
    const int dst = c.buf == 0 ? 1 : 0;
    C.col = c.buf < 0 ? g->col : (c.buf == 0 ? g->wcol : g->tcol);
    C.eid = c.buf < 0 ? g->eid : (c.buf == 0 ? g->weid : g->teid);
    C.nslots = 2 * c.held;
    C.tcol = dst == 0 ? g->wcol : g->tcol;
    C.teid = dst == 0 ? g->weid : g->teid;
    C.vstart = (Off*)g->vstart;
    C.vend = (Off*)g->vend;
    C.first = c.buf < 0;
    C.rowptr = (const Off*)g->rowptr;
    C.hub_of = g->n_hub > 0 ? g->hub_of : nullptr;
    C.el = g->el;
    C.ss = g->ss;
    C.g = gsub;
    C.n = g->n;
    C.rows = (Off*)g->wrows;
    C.dmin = g->wdmin;
    C.lhub = g->wlhub;
    // graphs whose pairs outgrow L2 test the slots against live bits
    // (R-MAT scale 24 peel 843 -> 832 ms); smaller ones read the pairs,
    // which stay in L2 (Chung-Lu 2^20: the extra pass cost 0.15 ms)
    const bool bits = g->m >= CMP_BIG_HELD;
    C.live = bits ? g->clive : nullptr;
    C.bits = g->cbits;
    C.toff = g->ctoff;
    C.bsum = g->cbsum;
    C.live_slots = 2 * (g->m - processed);
    C.hub_min = CMP_HUB_MIN_LIVE;
    if ((size_t)C.live_slots > cmp_slots(g)) return TRUSS_EINVAL;  // beyond the target's capacity
    const int B = cmp_blocks(g);
    if (bits) k_cmp_live<<<grid_for(g->m, PT, (int64_t)g->sms * 8), PT, 0, s>>>(g->ss, g->m, gsub, g->clive);
    k_cmp_count<Off><<<B, PT, 0, s>>>(C);
    k_cmp_blocks<<<1, PT, 0, s>>>(g->cbsum, B);
    k_cmp_scatter<Off><<<B, PT, 0, s>>>(C);
    if (k > 0) k_cmp_records<Off><<<grid_for(k, 256), 256, 0, s>>>(C, list, k);
    CU(cudaGetLastError());
    truss_note_launch((k > 0 ? 4 : 3) + (bits ? 1 : 0));
    c.count++;
    c.slots += C.nslots;
    c.buf = dst;
    c.held = g->m - processed;
    *view = view_compacted<Off>(g, dst);
    return TRUSS_OK;
}

TuneTable tune_table_of(const truss_opts& o) {
    TuneTable t;
    for (int i = 0; i < TRUSS_TUNE_CLASSES; i++) t.v[i] = o.tune_table ? o.tune_table[i] : (int8_t)-1;
    return t;
}

Frontier side(truss_graph* g, int k) {
    return Frontier{g->fq[k][0], g->fq[k][1], reinterpret_cast<uint32_t*>(g->fq[k][2]), g->owner[k]};
}

struct RunOut {
    int64_t nsub = 0, nscan = 0, nlevel = 0, scanned = 0, walked = 0;
    int32_t last_l = 0;
};

// Algorithm 4's loop driven from the host: one Scan launch per level, one
// ProcessSubLevel launch per sub-level, the frontier sizes read back after
// each.  trace (host, may be NULL) receives max_trace sub-level records.
template <typename Off>
int run_plain(truss_graph* g, const truss_opts& o, cudaStream_t s, truss_sublevel_trace* trace, int64_t max_trace,
              RunOut* out, CmpRun& cmp) {
    Graph<Off> G = graph_view<Off>(g);
    int* ctr = g->ctr;
    int* h = g->h_ctr;
    const int sblocks = grid_for((g->m + 1) / 2, PT, (int64_t)g->sms * 8);
    const int pmax = process_blocks<Off>(g);
    int32_t l = 0, gs = 0;
    int64_t processed = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (trace) {
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
    }
    auto read_slot = [&](int slot, int* nl, int* nh, uint32_t* nc, int64_t* dsum, int* dmax) {
        SlotVals v;
        memcpy(&v, slots(h) + slot, sizeof(v));
        *nl = v.nl;
        *nh = (int)(v.hc >> 32);
        *nc = (uint32_t)v.hc;
        *dsum = (int64_t)v.dsum;
        *dmax = v.dmax;
    };
    int rc = TRUSS_OK;
    int64_t nlive = g->m, scan_ns = 0;
    while (processed < g->m && rc == TRUSS_OK) {
        const int32_t* lin = out->nscan == 0 ? nullptr : g->live[(out->nscan + 1) & 1];
        int32_t* lout = g->live[out->nscan & 1];
        if (cmp.enabled && cmp.held >= cmp.min_held && (g->m - processed) * 100 <= cmp.held * cmp_live_pct(cmp.held) &&
            processed > 0)
            TRY(run_compaction<Off>(g, cmp, gs, processed, lin, nlive, s, &G));
        k_init_counters<<<1, 64, 0, s>>>(ctr);
        if (trace) CU(cudaEventRecord(e0, s));
        k_scan<<<sblocks, PT, 0, s>>>(g->ss, lin, nlive, lout, l, gs, side(g, gs & 1), ctr, G.dmin, g->hc, g->ocap);
        out->scanned += nlive;
        if (trace) CU(cudaEventRecord(e1, s));
        CU(cudaGetLastError());
        truss_note_launch(2);
        CU(cudaMemcpyAsync(h, ctr, sizeof(int) * C_BAR_COUNT, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (trace) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            scan_ns += (int64_t)(ms * 1e6);
        }
        nlive = slots(h)[0].nlive;
        out->nscan++;
        int nl, nh, dmax;
        uint32_t nc;
        int64_t dsum;
        read_slot(0, &nl, &nh, &nc, &dsum, &dmax);
        if (nl + nh == 0) {
            const int mn = slots(h)[0].minv;
            if (mn == INT_MAX) break;
            l = o.level_jump ? mn : l + 1;
            continue;
        }
        out->nlevel++;
        while (nl + nh > 0) {
            const int gsz = pick_group(o.variant, nl, dsum, (int64_t)nl + nh, tune_table_of(o));
            truss_sublevel_trace* r = (trace && out->nsub < max_trace) ? trace + out->nsub : nullptr;
            if (r) *r = truss_sublevel_trace{l, gsz, nl, nh, nc, dmax, dsum, g->m - processed, 0, scan_ns};
            scan_ns = 0;
            processed += nl + nh;
            if (l > 0) out->walked += dsum;
            // the next frontier is counted in slot 1
            k_clear_slot<<<1, 32, 0, s>>>(ctr, 1);
            const int64_t want = std::max<int64_t>(((int64_t)nl * gsz + PT - 1) / PT, ((int64_t)nc * 32 + PT - 1) / PT);
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(pmax, want));
            if (r) CU(cudaEventRecord(e0, s));
            k_process<Off><<<blocks, PT, 0, s>>>(G, side(g, gs & 1), nl, nh, nc, gsz, l, gs, side(g, (gs + 1) & 1), ctr,
                                                 1);
            if (r) CU(cudaEventRecord(e1, s));
            CU(cudaGetLastError());
            truss_note_launch(2);
            CU(cudaMemcpyAsync(h, ctr, sizeof(int) * C_BAR_COUNT, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            if (r) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                r->t_ns = (int64_t)(ms * 1e6);
            }
            read_slot(1, &nl, &nh, &nc, &dsum, &dmax);
            gs++;
            out->nsub++;
        }
        l++;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    out->last_l = l;
    return rc;
}

// ------------------------------------------------- graph-driven level loop

// Algorithm 4's loop as one CUDA graph: a while node whose body runs a
// one-block control kernel and then a switch node holding the Scan kernel
// (case 0) and the ProcessSubLevel kernel (case 1).  The control kernel
// reads the counters of the phase that just ran, decides the next phase
// exactly as the host loop and the persistent kernel do, and sets both
// conditions; no host round trip and no grid barrier between phases.  Every
// phase is a separate kernel, so the state lives in device memory (GCtl).
enum { PH_SCAN = 0, PH_SUB = 1, PH_DONE = 2, PH_FIRST = -1 };

struct GCtl {
    int32_t type;      // phase the body runs now (PH_*)
    int32_t l, g;      // level, sub-level number (the stamp of curr)
    int32_t nl, nh;    // frontier of the sub-level
    int32_t gsz;       // lanes per light edge
    int32_t slot;      // counter slot the phase writes (0 or 1)
    int32_t err;
    int32_t dmax;
    uint32_t nchunk;
    int64_t dsum;
    int64_t processed, nsub, nscan, nlevel;
    int64_t nlive;     // entries the next Scan visits
    int64_t scanned;
    int64_t walked;    // shorter-row entries of all frontiers
    int64_t phases, cap;  // phases run, and the bound on them
    uint64_t t_phase;  // start of the phase that is running
    uint64_t scan_ns;  // Scan time since the last sub-level
    uint64_t timeout;  // limit on one phase
};

__global__ void k_ginit(GCtl* c, int* ctr, int64_t m, int64_t cap, uint64_t timeout) {
    for (int i = threadIdx.x; i < C_TOTAL; i += blockDim.x) ctr[i] = 0;
    __syncthreads();
    if (threadIdx.x < 4) clear_slot_vals(slots(ctr) + threadIdx.x);
    if (threadIdx.x == 0) {
        GCtl s;
        memset(&s, 0, sizeof(s));
        s.type = PH_FIRST;
        s.slot = 1;
        s.nlive = m;
        s.cap = cap;
        s.timeout = timeout;
        *c = s;
    }
}

// One warp.  Thread 0 runs the state machine; the whole warp evaluates the
// learned model when it is consulted.
__global__ void __launch_bounds__(32) k_gctl(GCtl* c, int* ctr, int64_t m, int variant, int level_jump,
                                             truss_sublevel_trace* trace, int64_t max_trace, const float* sched,
                                             TuneTable tt, cudaGraphConditionalHandle wh,
                                             cudaGraphConditionalHandle sh) {
    __shared__ GCtl s;
    if (threadIdx.x == 0) {
        const uint64_t now = global_ns();
        s = *c;
        if (s.type == PH_FIRST) {
            s.type = m > 0 ? PH_SCAN : PH_DONE;
        } else {
            SlotVals v;
            memcpy(&v, slots(ctr) + s.slot, sizeof(v));
            const int vnh = (int)(v.hc >> 32);
            if (now - s.t_phase > s.timeout) s.err = TRUSS_ETIMEOUT;
            if (s.type == PH_SCAN) {
                s.nscan++;
                s.scanned += s.nlive;
                s.nlive = v.nlive;
                s.scan_ns += now - s.t_phase;
                if (v.nl + vnh == 0) {
                    if (v.minv == INT_MAX) {
                        s.type = PH_DONE;
                    } else {
                        s.l = level_jump ? v.minv : s.l + 1;
                    }
                } else {
                    s.nlevel++;
                    s.type = PH_SUB;
                }
            } else {  // a sub-level just ran
                if (trace && s.nsub - 1 < max_trace) trace[s.nsub - 1].t_ns = (int64_t)(now - s.t_phase);
                s.g++;
                if (v.nl + vnh == 0) {
                    s.l++;
                    s.type = s.processed < m ? PH_SCAN : PH_DONE;
                }
            }
            if (s.type == PH_SUB) {
                s.nl = v.nl;
                s.nh = vnh;
                s.nchunk = (uint32_t)v.hc;
                s.dsum = (int64_t)v.dsum;
                s.dmax = v.dmax;
            }
        }
        s.phases++;
        if (s.type != PH_DONE && s.phases > s.cap) s.err = TRUSS_ETIMEOUT;
        if (s.err) s.type = PH_DONE;
        s.gsz = s.type == PH_SUB ? pick_group(variant, s.nl, s.dsum, (int64_t)s.nl + s.nh, tt) : 0;
    }
    __syncwarp();
    if (s.type == PH_SUB && variant == TRUSS_VAR_LEARNED && sched && s.nl >= LEARN_MIN_LIGHT) {
        float x[SF];
        sched_features((int64_t)s.nl + s.nh, s.dsum, s.dmax, s.l, m - s.processed, x);
        const int ch = sched_pick(sched, x);
        if (threadIdx.x == 0 && ch >= 0) s.gsz = group_of(ch);
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        if (s.type == PH_SUB) {
            if (trace && s.nsub < max_trace) {
                truss_sublevel_trace& r = trace[s.nsub];
                r.level = s.l;
                r.group = s.gsz;
                r.n_light = s.nl;
                r.n_heavy = s.nh;
                r.n_chunks = s.nchunk;
                r.dmax = s.dmax;
                r.dsum = s.dsum;
                r.todo = m - s.processed;
                r.t_ns = 0;
                r.scan_ns = (int64_t)s.scan_ns;
            }
            s.scan_ns = 0;
            s.processed += (int64_t)s.nl + s.nh;
            if (s.l > 0) s.walked += s.dsum;
            s.nsub++;
        }
        s.slot ^= 1;
        clear_slot_vals(slots(ctr) + s.slot);
        if (s.type == PH_DONE) {
            ctr[C_NSUB] = (int)s.nsub;
            ctr[C_NSCAN] = (int)s.nscan;
            ctr[C_NLEVEL] = (int)s.nlevel;
            ctr[C_LAST_L] = s.l;
            *reinterpret_cast<long long*>(ctr + C_SCANNED) = s.scanned;
            *reinterpret_cast<long long*>(ctr + C_WALKED) = s.walked;
            if (s.err) ctr[C_ERR] = s.err;
        }
        s.t_phase = global_ns();
        *c = s;
        cudaGraphSetConditional(sh, (unsigned)s.type);  // PH_DONE (2) runs no case
        cudaGraphSetConditional(wh, s.type != PH_DONE ? 1u : 0u);
    }
}

template <typename Off>
__global__ void __launch_bounds__(PT) k_gscan(Graph<Off> G, const GCtl* c, Frontier f0, Frontier f1,
                                              int32_t* live0, int32_t* live1, int* ctr) {
    __shared__ PeelSmem sm;
    smem_init(&sm);
    const int64_t sc = c->nscan, nin = c->nlive;
    const int32_t l = c->l, g = c->g;
    const int slot = c->slot;
    const int32_t* lin = sc == 0 ? nullptr : ((sc & 1) ? live0 : live1);
    int32_t* lout = (sc & 1) ? live1 : live0;
    scan_level(G.ss, lin, nin, lout, l, g, (g & 1) ? f1 : f0, slot_of(ctr, slot), G.dmin, G.hc, G.ocap, &sm);
}

template <typename Off>
__global__ void __launch_bounds__(PT) k_gprocess(Graph<Off> G, const GCtl* c, Frontier f0, Frontier f1, int* ctr) {
    __shared__ PeelSmem sm;
    smem_init(&sm);
    const int nl = c->nl, nh = c->nh, gsz = c->gsz, slot = c->slot;
    const uint32_t nchunk = c->nchunk;
    const int32_t l = c->l, g = c->g;
    const Frontier cu = (g & 1) ? f1 : f0, nx = (g & 1) ? f0 : f1;
    const Appender ap{&sm, nx, slot_of(ctr, slot), G.dmin, G.hc, G.ocap};
    if (walk_needed(l, 1)) process_frontier<Off>(G, cu, nl, nh, nchunk, gsz, l, g, ap);
    ap.flush();
}

// Builds, launches and releases the graph of one decomposition's peel (the
// executable graph is freed by the runtime once it has run).
template <typename Off>
int run_graph(truss_graph* g, const truss_opts& o, cudaStream_t s, truss_sublevel_trace* d_trace,
              int64_t max_trace) {
    Graph<Off> G = graph_view<Off>(g);
    GCtl* c = reinterpret_cast<GCtl*>(g->gctl);
    int* ctr = g->ctr;
    int64_t m = g->m;
    const int sblocks = grid_for((g->m + 1) / 2, PT, (int64_t)g->sms * 8);
    int per_sm = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gprocess<Off>, PT, 0));
    const int pblocks = std::max(1, per_sm) * g->sms;
    g->last_grid = pblocks;
    g->last_per_sm = std::max(1, per_sm);
    // a bound on the phases: at most m sub-levels, m non-empty Scans and one
    // empty Scan per support level
    const int64_t cap = 2 * g->m + g->max_deg + 64;
    const uint64_t tmo = o.timeout_ns > 0 ? (uint64_t)o.timeout_ns : 10000000000ull;
    k_ginit<<<1, 64, 0, s>>>(c, ctr, m, cap, tmo);
    CU(cudaGetLastError());
    truss_note_launch();

    int variant = o.variant;
    int jump = o.level_jump;
    const float* sched = o.sched_params;
    TuneTable tt = tune_table_of(o);
    Frontier f0 = side(g, 0), f1 = side(g, 1);
    int32_t* live0 = g->live[0];
    int32_t* live1 = g->live[1];
    cudaGraph_t top = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = TRUSS_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TRUSS_OK) {
            truss_note_cuda_error(e);
            rc = e == cudaErrorMemoryAllocation ? TRUSS_ENOMEM : TRUSS_ECUDA;
        }
        return rc == TRUSS_OK;
    };
    do {
        if (!ok(cudaGraphCreate(&top, 0))) break;
        cudaGraphConditionalHandle wh, sh;
        if (!ok(cudaGraphConditionalHandleCreate(&wh, top, 1, cudaGraphCondAssignDefault))) break;
        cudaGraphNodeParams wp = {};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = wh;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wn;
        if (!ok(cudaGraphAddNode(&wn, top, nullptr, nullptr, 0, &wp))) break;
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        if (!ok(cudaGraphConditionalHandleCreate(&sh, body, PH_DONE, cudaGraphCondAssignDefault))) break;
        void* cargs[] = {&c, &ctr, &m, &variant, &jump, &d_trace, &max_trace, &sched, &tt, &wh, &sh};
        cudaKernelNodeParams kp = {};
        kp.func = (void*)k_gctl;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = cargs;
        cudaGraphNode_t cn;
        if (!ok(cudaGraphAddKernelNode(&cn, body, nullptr, 0, &kp))) break;
        cudaGraphNodeParams sp = {};
        sp.type = cudaGraphNodeTypeConditional;
        sp.conditional.handle = sh;
        sp.conditional.type = cudaGraphCondTypeSwitch;
        sp.conditional.size = 2;
        cudaGraphNode_t sn;
        if (!ok(cudaGraphAddNode(&sn, body, &cn, nullptr, 1, &sp))) break;
        const GCtl* cc = c;
        void* sargs[] = {&G, &cc, &f0, &f1, &live0, &live1, &ctr};
        cudaKernelNodeParams kscan = {};
        kscan.func = (void*)k_gscan<Off>;
        kscan.gridDim = dim3(sblocks);
        kscan.blockDim = dim3(PT);
        kscan.kernelParams = sargs;
        cudaGraphNode_t n0, n1;
        if (!ok(cudaGraphAddKernelNode(&n0, sp.conditional.phGraph_out[0], nullptr, 0, &kscan))) break;
        void* pargs[] = {&G, &cc, &f0, &f1, &ctr};
        cudaKernelNodeParams kproc = {};
        kproc.func = (void*)k_gprocess<Off>;
        kproc.gridDim = dim3(pblocks);
        kproc.blockDim = dim3(PT);
        kproc.kernelParams = pargs;
        if (!ok(cudaGraphAddKernelNode(&n1, sp.conditional.phGraph_out[1], nullptr, 0, &kproc))) break;
        if (!ok(cudaGraphInstantiate(&exec, top, 0))) break;
        if (!ok(cudaGraphLaunch(exec, s))) break;
    } while (false);
    if (exec) cudaGraphExecDestroy(exec);
    if (top) cudaGraphDestroy(top);
    return rc;
}

// Blocks per SM of the persistent form for options o on graph g whose
// largest support is smax.  The automatic form takes 6 (throughput) when the
// walk is large against the number of phases: when the shorter-row entries
// all sub-levels walk (W = sum of min(d(u), d(v))) reach 2^24 per support
// level, or 2^34 in all (at about 4.5e10 entries/s that is 0.4 s of walking,
// far above the latency of a few thousand phases; large skewed graphs have
// far fewer non-empty levels than their largest support).  Measured on
// GB300: R-MAT scale 10 (W 1.6e5) and Chung-Lu 2^20 (W 1.8e9, 7.7e6 a
// level) run fastest at 4 blocks per SM, the geometric graph 2^21 (3.3e7 a
// level) and R-MAT scale 24 (W 2.7e11) at 6.
inline int persistent_minb(const truss_graph* g, const truss_opts& o, int32_t smax) {
    if (o.loop == TRUSS_LOOP_PERSISTENT_LAT) return 4;
    if (o.loop == TRUSS_LOOP_PERSISTENT_OCC) return 6;
    const int64_t per_level = g->dmin_sum / ((int64_t)(smax > 0 ? smax : 0) + 1);
    return (per_level >= ((int64_t)1 << 24) || g->dmin_sum >= ((int64_t)1 << 34)) ? 6 : 4;
}

// The persistent loop: one cooperative launch, or, with compaction on, one
// launch per stretch between compactions -- each launch stops before the
// Scan of the level whose rows are due, the host compacts them (four or five
// launches) and resumes the loop from the state the launch left.  Each stop
// reads that state back (one synchronisation per compaction).
template <typename Off, int MINB>
int launch_persistent(truss_graph* g, const truss_opts& o, cudaStream_t s, truss_sublevel_trace* d_trace,
                      int64_t max_trace, CmpRun& cmp) {
    Graph<Off> G = graph_view<Off>(g);
    int per_sm = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<Off, MINB>, PT, 0));
    if (per_sm < 1) return TRUSS_ENOTSUP;
    int blocks = per_sm * g->sms;
    g->last_grid = blocks;
    g->last_per_sm = per_sm;
    k_init_counters<<<1, 64, 0, s>>>(g->ctr);
    CU(cudaGetLastError());
    int variant = o.variant;
    int jump = o.level_jump;
    uint64_t tmo = o.timeout_ns > 0 ? (uint64_t)o.timeout_ns : 10000000000ull;
    Frontier f0 = side(g, 0), f1 = side(g, 1);
    int32_t* live0 = g->live[0];
    int32_t* live1 = g->live[1];
    int* ctr = g->ctr;
    const float* sched = o.sched_params;
    TuneTable tt = tune_table_of(o);
    int64_t held = cmp.enabled ? cmp.held : -1;  // -1: the launch never stops early
    int64_t min_held = cmp.min_held;
    int resume = 0;
    for (;;) {
        void* args[] = {&G,   &f0,        &f1,    &live0, &live1, &ctr,      &variant,  &jump,
                        &tmo, &d_trace, &max_trace, &sched, &tt,   &held, &min_held, &resume};
        CU(cudaLaunchCooperativeKernel((const void*)k_persistent<Off, MINB>, dim3(blocks), dim3(PT), args, 0, s));
        truss_note_launch(resume ? 1 : 2);
        if (!cmp.enabled) break;
        int* h = g->h_ctr;
        CU(cudaMemcpyAsync(h + C_ERR, ctr + C_ERR, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(h + C_ST, ctr + C_ST, sizeof(PState), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        PState ps;
        memcpy(&ps, h + C_ST, sizeof(ps));
        if (h[C_ERR] != 0 || !ps.stop) break;
        const int32_t* lin = (ps.sc & 1) ? live0 : live1;
        TRY(run_compaction<Off>(g, cmp, ps.g, ps.processed, lin, ps.nlive, s, &G));
        k_resume_counters<<<1, 64, 0, s>>>(ctr);
        truss_note_launch();
        held = cmp.held;
        resume = 1;
    }
    return TRUSS_OK;
}

template <typename Off>
int run_persistent(truss_graph* g, const truss_opts& o, cudaStream_t s, truss_sublevel_trace* d_trace,
                   int64_t max_trace, int32_t smax, CmpRun& cmp) {
    if (persistent_minb(g, o, smax) == 4) return launch_persistent<Off, 4>(g, o, s, d_trace, max_trace, cmp);
    return launch_persistent<Off, 6>(g, o, s, d_trace, max_trace, cmp);
}

int check_opts(const truss_opts& o) {
    if (o.loop < TRUSS_LOOP_PLAIN || o.loop > TRUSS_LOOP_GRAPH) return TRUSS_EINVAL;
    if (o.variant < TRUSS_VAR_AUTO || o.variant > TRUSS_VAR_LEARNED) return TRUSS_EINVAL;
    if ((o.h_sub_level || o.h_sub_size) && (!o.h_sub_level || !o.h_sub_size)) return TRUSS_EINVAL;
    if ((o.h_sub_level || o.h_trace) && (o.max_sub < 0 || !o.sync)) return TRUSS_EINVAL;
    if ((o.h_level_edges || o.h_level_ns) && (o.max_level <= 0 || !o.sync)) return TRUSS_EINVAL;
    if (o.compact < -1 || o.compact > 1) return TRUSS_EINVAL;
    return TRUSS_OK;
}

// sub-level records kept for the per-level distribution when the caller
// asked for no trace of its own
constexpr int64_t LEVEL_TRACE_CAP = (int64_t)1 << 20;

template <typename Off>
int decompose_impl(truss_graph* g, int32_t* d_truss, const truss_opts& o, truss_stats* st, cudaStream_t s) {
    TRY(truss_ensure_workspace(g, s));
    const long long launches0 = truss_launch_count();
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    const bool timed = o.sync && st;
    if (timed)
        for (auto& e : ev) CU(cudaEventCreate(&e));
    if (timed) CU(cudaEventRecord(ev[0], s));
    TRY(truss_support_internal(g, g->ss, s));
    unsigned long long* d_tri = reinterpret_cast<unsigned long long*>(g->ctr + C_TRI);
    // the automatic persistent form needs the largest support on the host
    // (it waits for the support phase); the other forms stay asynchronous
    const bool pick = o.loop == TRUSS_LOOP_PERSISTENT;
    int32_t smax = 0;
    if (st || pick) {
        CU(cudaMemsetAsync(g->ctr + C_TRI, 0, 4 * sizeof(int), s));
        k_sum_support<<<grid_for(g->m, 256, (int64_t)g->sms * 4), 256, 0, s>>>(g->ss, g->m, d_tri, g->ctr + C_TRI + 2);
        CU(cudaGetLastError());
        truss_note_launch();
        CU(cudaMemcpyAsync(g->h_ctr + C_TRI, g->ctr + C_TRI, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(g->h_ctr + TRUSS_CTR_SUPPORT_WORK, g->ctr + TRUSS_CTR_SUPPORT_WORK,
                           2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        if (pick) {
            CU(cudaStreamSynchronize(s));
            smax = g->h_ctr[C_TRI + 2];
        }
    }
    CmpRun cmp = compact_policy(g, o, s);
    if (timed) CU(cudaEventRecord(ev[1], s));
    RunOut ro;
    const bool lvl = (o.h_level_edges || o.h_level_ns) && o.max_level > 0;
    const bool rec = ((o.h_sub_level || o.h_trace) && o.max_sub > 0) || lvl;
    const int64_t tcap = std::max<int64_t>(o.max_sub, lvl ? LEVEL_TRACE_CAP : 0);
    std::vector<truss_sublevel_trace> htr(rec ? (size_t)tcap : 0);
    int rc = TRUSS_OK;
    if (o.loop == TRUSS_LOOP_PLAIN) {
        rc = run_plain<Off>(g, o, s, rec ? htr.data() : nullptr, rec ? tcap : 0, &ro, cmp);
    } else {
        truss_sublevel_trace* d_tr = nullptr;
        if (rec) CU(cudaMallocAsync((void**)&d_tr, sizeof(truss_sublevel_trace) * (size_t)tcap, s));
        if (o.loop == TRUSS_LOOP_GRAPH)
            rc = run_graph<Off>(g, o, s, d_tr, rec ? tcap : 0);
        else
            rc = run_persistent<Off>(g, o, s, d_tr, rec ? tcap : 0, smax, cmp);
        if (rc == TRUSS_OK && o.sync) {
            // the triangle words (C_TRI on) keep the support phase's count on
            // the host side; the peel cleared them on the device
            CU(cudaMemcpyAsync(g->h_ctr, g->ctr, sizeof(int) * C_TRI, cudaMemcpyDeviceToHost, s));
            CU(cudaMemcpyAsync(g->h_ctr + C_SCANNED, g->ctr + C_SCANNED, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost,
                               s));
            CU(cudaStreamSynchronize(s));
            if (g->h_ctr[C_ERR]) rc = g->h_ctr[C_ERR];
            ro.nsub = g->h_ctr[C_NSUB];
            ro.nscan = g->h_ctr[C_NSCAN];
            ro.nlevel = g->h_ctr[C_NLEVEL];
            ro.last_l = g->h_ctr[C_LAST_L];
            memcpy(&ro.scanned, g->h_ctr + C_SCANNED, sizeof(ro.scanned));
            memcpy(&ro.walked, g->h_ctr + C_WALKED, sizeof(ro.walked));
            // the graph ran a control kernel per phase, a Scan or sub-level
            // kernel in every phase but the last
            if (o.loop == TRUSS_LOOP_GRAPH) truss_note_launch((int)(2 * (ro.nsub + ro.nscan) + 1));
            if (rec && rc == TRUSS_OK) {
                const int64_t k = std::min<int64_t>(ro.nsub, tcap);
                CU(cudaMemcpyAsync(htr.data(), d_tr, sizeof(truss_sublevel_trace) * (size_t)k, cudaMemcpyDeviceToHost, s));
            }
        }
        if (d_tr) cudaFreeAsync(d_tr, s);
    }
    if (rc != TRUSS_OK) {
        if (timed)
            for (auto& e : ev) cudaEventDestroy(e);
        return rc;
    }
    if (timed) CU(cudaEventRecord(ev[2], s));
    if (g->m > 0) {
        k_truss_out<<<grid_for(g->m, 256), 256, 0, s>>>(g->ss, g->m, g->perm, d_truss, 2);
        truss_note_launch();
        if (o.d_peel_step) {
            k_step_out<<<grid_for(g->m, 256), 256, 0, s>>>(g->ss, g->m, g->perm, o.d_peel_step);
            truss_note_launch();
        }
    }
    CU(cudaGetLastError());
    if (o.sync) {
        CU(cudaStreamSynchronize(s));
        if (rec) {
            const int64_t k = std::min<int64_t>(ro.nsub, o.max_sub);
            for (int64_t i = 0; i < k; i++) {
                if (o.h_sub_level) {
                    o.h_sub_level[i] = htr[i].level;
                    o.h_sub_size[i] = (int64_t)htr[i].n_light + htr[i].n_heavy;
                }
                if (o.h_trace) o.h_trace[i] = htr[i];
            }
        }
        if (lvl) {
            // Fig. 6: edges and device time per support level (a level's
            // time is its sub-levels and the Scans that opened it)
            for (int32_t i = 0; i < o.max_level; i++) {
                if (o.h_level_edges) o.h_level_edges[i] = 0;
                if (o.h_level_ns) o.h_level_ns[i] = 0;
            }
            const int64_t k = std::min<int64_t>(ro.nsub, tcap);
            for (int64_t i = 0; i < k; i++) {
                const truss_sublevel_trace& r = htr[i];
                if (r.level < 0 || r.level >= o.max_level) continue;
                if (o.h_level_edges) o.h_level_edges[r.level] += (int64_t)r.n_light + r.n_heavy;
                if (o.h_level_ns) o.h_level_ns[r.level] += r.t_ns + r.scan_ns;
            }
        }
    }
    if (st) {
        memset(st, 0, sizeof(*st));
        st->m = g->m;
        st->sublevels = ro.nsub;
        st->scans = ro.nscan;
        st->levels = (int32_t)ro.nlevel;
        st->launches = truss_launch_count() - launches0;
        st->wedges_up = g->wedges_up;
        st->dmin_sum = g->dmin_sum;
        st->scanned = ro.scanned;
        st->walked = ro.walked;
        if (o.sync && g->sup_switch) {
            unsigned long long sw[2];
            memcpy(sw, g->h_ctr + TRUSS_CTR_SUPPORT_WORK, sizeof(sw));
            st->support_walked = (int64_t)sw[0];
            st->support_hub_probes = (int64_t)sw[1];
        } else {
            st->support_walked = g->wedges_up;  // no side switch: the walk is exactly W+
        }
        st->compactions = cmp.count;
        st->compacted_slots = cmp.slots;
        st->grid_blocks = o.loop == TRUSS_LOOP_PLAIN ? 0 : g->last_grid;
        st->blocks_per_sm = o.loop == TRUSS_LOOP_PLAIN ? 0 : g->last_per_sm;
        if (o.sync) {
            unsigned long long tri = 0;
            memcpy(&tri, g->h_ctr + C_TRI, sizeof(tri));
            st->triangles = (int64_t)(tri / 3);
            st->max_support = g->h_ctr[C_TRI + 2];
            // the last level that held edges is the final l minus one
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
    const int64_t m = g->m;
    if (ncurr > 0) {
        // reject out-of-range or repeated ids before any kernel indexes with them
        const int64_t words = (m + 31) / 32;
        uint32_t* seen = nullptr;
        CU(cudaMallocAsync((void**)&seen, sizeof(uint32_t) * (size_t)words + sizeof(int), s));
        int* d_err = (int*)(seen + words);
        CU(cudaMemsetAsync(seen, 0, sizeof(uint32_t) * (size_t)words + sizeof(int), s));
        k_check_curr<<<grid_for(ncurr, 256), 256, 0, s>>>(d_curr, ncurr, m, seen, d_err);
        int h_err = 0;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(seen, s);
        if (e != cudaSuccess) {
            truss_note_cuda_error(e);
            return TRUSS_ECUDA;
        }
        if (h_err) return TRUSS_EBADGRAPH;
    }
    TRY(truss_ensure_workspace(g, s));
    int32_t *inv = nullptr, *cur = nullptr;
    CU(cudaMallocAsync((void**)&cur, sizeof(int32_t) * (size_t)(ncurr > 0 ? ncurr : 1), s));
    if (g->perm) {
        CU(cudaMallocAsync((void**)&inv, sizeof(int32_t) * (size_t)m, s));
        k_inverse_perm<<<grid_for(m, 256), 256, 0, s>>>(g->perm, m, inv);
    }
    k_import_state<<<grid_for(m, 256), 256, 0, s>>>(d_S, d_flags, g->perm, m, g->ss);
    k_init_counters<<<1, 64, 0, s>>>(g->ctr);
    if (ncurr > 0) {
        k_map_ids<<<grid_for(ncurr, 256), 256, 0, s>>>(d_curr, ncurr, inv, cur);
        k_mark_curr<<<grid_for(ncurr, 256), 256, 0, s>>>(cur, ncurr, g->ss);
        k_classify<<<grid_for(ncurr, 256), 256, 0, s>>>(cur, ncurr, g->dmin, g->hc, g->ocap, side(g, 0), g->ctr);
    }
    CU(cudaGetLastError());
    int* h = g->h_ctr;
    CU(cudaMemcpyAsync(h, g->ctr, sizeof(int) * C_BAR_COUNT, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    SlotVals v0;
    memcpy(&v0, slots(h), sizeof(v0));
    const int nl = v0.nl, nh = (int)(v0.hc >> 32);
    const uint32_t nc = (uint32_t)v0.hc;
    if (nl + nh > 0) {
        Graph<Off> G = graph_view<Off>(g);
        const int blocks = process_blocks<Off>(g);
        k_process<Off><<<blocks, PT, 0, s>>>(G, side(g, 0), nl, nh, nc, pick_group(variant, nl, 0, nl + nh, tune_table_of(truss_opts{})), l,
                                             1, side(g, 1), g->ctr, 0);
        CU(cudaGetLastError());
    }
    CU(cudaMemcpyAsync(h, g->ctr, sizeof(int) * C_BAR_COUNT, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    SlotVals v1;
    memcpy(&v1, slots(h) + 1, sizeof(v1));
    const int nl1 = v1.nl, nh1 = (int)(v1.hc >> 32);
    if (nl1 > 0) k_map_ids<<<grid_for(nl1, 256), 256, 0, s>>>(g->fq[1][0], nl1, g->perm, d_next);
    if (nh1 > 0) k_map_ids<<<grid_for(nh1, 256), 256, 0, s>>>(g->fq[1][1], nh1, g->perm, d_next + nl1);
    k_export_state<<<grid_for(m, 256), 256, 0, s>>>(g->ss, g->perm, m, d_S, d_flags);
    CU(cudaGetLastError());
    if (inv) cudaFreeAsync(inv, s);
    cudaFreeAsync(cur, s);
    CU(cudaStreamSynchronize(s));
    *h_nnext = nl1 + nh1;
    return TRUSS_OK;
}

}  // namespace

// Hub bitmaps for the vertices of degree >= thr, thr = HUB_MIN_DEG doubled
// until they fit the budget: 32 bytes per 192 vertex ids for each hub, at
// most HUB_BYTES_PER_EDGE per edge and HUB_FREE_SHARE of the device memory
// free when the workspace is built; when their allocation fails all the
// same, thr doubles again.  The bitmaps serve the peel's probes of long rows
// and the support's side switch.  R-MAT scale 24 (hubs of degree >= 8192 /
// 4096 / 2048: 6 / 34 / 144 GiB of bitmaps): support 1.07 / 0.70 / 0.49 s,
// peel 1.21 / 0.98 / 0.84 s; Chung-Lu 2^20 (1602 hubs of degree >= 1024,
// 0.3 GiB) and the batch are fastest with HUB_MIN_DEG = 1024.
constexpr int64_t HUB_MIN_DEG = 1024;
constexpr int64_t HUB_BYTES_PER_EDGE = 1024;
constexpr double HUB_FREE_SHARE = 0.75;

template <typename Off>
int build_hubs(truss_graph* g, cudaStream_t s) {
    const Off* rowptr = (const Off*)g->rowptr;
    const int64_t hw = (((int64_t)g->n + 191) / 192) * 4;
    const int64_t per_hub = hw * 8;
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    const int64_t budget = std::min<int64_t>(HUB_BYTES_PER_EDGE * g->m, (int64_t)((double)free_b * HUB_FREE_SHARE));
    int* d_cnt = nullptr;
    CU(cudaMallocAsync((void**)&d_cnt, sizeof(int), s));
    int64_t thr = HUB_MIN_DEG;
    int cnt = 0;
    for (;;) {
        CU(cudaMemsetAsync(d_cnt, 0, sizeof(int), s));
        k_count_deg<Off><<<grid_for(g->n, 256), 256, 0, s>>>(rowptr, g->n, thr, d_cnt);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(&cnt, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if ((int64_t)cnt * per_hub <= budget) {
            if (cnt == 0) break;
            // reserve the bitmaps now; when the device cannot hold them, fewer hubs
            if (cudaMallocAsync((void**)&g->hub_bits, sizeof(unsigned long long) * (size_t)(cnt * hw), s) ==
                cudaSuccess)
                break;
            cudaGetLastError();  // clear the failed allocation
            g->hub_bits = nullptr;
        }
        thr *= 2;
    }
    g->n_hub = cnt;
    g->hub_words = hw;
    if (cnt > 0) {
        int32_t* hub_vert = nullptr;
        CU(cudaMallocAsync((void**)&g->hub_of, sizeof(int32_t) * (size_t)g->n, s));
        CU(cudaMallocAsync((void**)&hub_vert, sizeof(int32_t) * (size_t)cnt, s));
        CU(cudaMemsetAsync(d_cnt, 0, sizeof(int), s));
        CU(cudaMemsetAsync(g->hub_bits, 0, sizeof(unsigned long long) * (size_t)(cnt * hw), s));
        k_hub_list<Off><<<grid_for(g->n, 256), 256, 0, s>>>(rowptr, g->n, thr, g->hub_of, hub_vert, d_cnt);
        CU(cudaGetLastError());
        k_hub_fill<Off><<<std::min<int64_t>(cnt, (int64_t)g->sms * 8), 256, 0, s>>>(rowptr, g->col, hub_vert, cnt, hw,
                                                                               g->hub_bits);
        CU(cudaGetLastError());
        k_hub_pre<<<std::min<int64_t>(cnt, (int64_t)g->sms * 8), 256, 0, s>>>(g->hub_bits, cnt, hw);
        CU(cudaGetLastError());
        cudaFreeAsync(hub_vert, s);
    }
    cudaFreeAsync(d_cnt, s);
    return TRUSS_OK;
}

// Allocations come from the stream-ordered pool and the setup kernels run on
// stream s (one synchronisation at the end).
int truss_ensure_workspace(truss_graph* g, cudaStream_t s) {
    if (g->ctr) return TRUSS_OK;
    const size_t m = (size_t)(g->m > 0 ? g->m : 1);
    // heavy chunk length: 64 entries (two per lane), longer when the graph is
    // so large that a sub-level's chunk total could leave 32 bits
    int64_t hc = 64;
    while ((int64_t)g->m + g->dmin_sum / hc >= ((int64_t)1 << 32) - 1) hc *= 2;
    g->hc = (int)hc;
    CU(cudaMallocAsync((void**)&g->ss, sizeof(int2) * (m + 1), s));
    CU(cudaMallocAsync((void**)&g->dmin, sizeof(int32_t) * m, s));
    CU(cudaMallocAsync(&g->rows, (g->off64 ? sizeof(int64_t) : sizeof(int32_t)) * 4 * m, s));
    for (int k = 0; k < 2; k++) {
        for (int j = 0; j < 3; j++) CU(cudaMallocAsync((void**)&g->fq[k][j], sizeof(int32_t) * m, s));
        CU(cudaMallocAsync((void**)&g->live[k], sizeof(int32_t) * m, s));
    }
    CU(cudaMallocAsync(&g->gctl, sizeof(GCtl), s));
    CU(cudaMallocHost((void**)&g->h_ctr, sizeof(int) * C_TOTAL));
    // chunk owner maps: enough for any sub-level of graphs up to moderate
    // size; larger chunk totals fall back to a search
    {
        const int64_t want = (int64_t)g->m + g->dmin_sum / hc + 1;
        const int64_t cap = std::min<int64_t>(want, std::min<int64_t>(4 * (int64_t)g->m + 1024, (int64_t)UINT32_MAX));
        g->ocap = (uint32_t)cap;
        for (int k = 0; k < 2; k++) CU(cudaMallocAsync((void**)&g->owner[k], sizeof(int2) * (size_t)cap, s));
    }
    CU(cudaMallocAsync((void**)&g->lhub, sizeof(int32_t) * m, s));
    if (g->m > 0) {
        TRY(g->off64 ? build_hubs<int64_t>(g, s) : build_hubs<int32_t>(g, s));
        TRY(truss_support_plan(g, s));
        if (g->off64)
            k_dmin<int64_t><<<grid_for(g->m, 256), 256, 0, s>>>((const int64_t*)g->rowptr, g->el, g->m, g->dmin,
                                                                 (int64_t*)g->rows, g->hub_of, g->lhub);
        else
            k_dmin<int32_t><<<grid_for(g->m, 256), 256, 0, s>>>((const int32_t*)g->rowptr, g->el, g->m, g->dmin,
                                                                 (int32_t*)g->rows, g->hub_of, g->lhub);
        CU(cudaGetLastError());
    }
    // the counter block last: a workspace with ctr set is complete
    int* ctr = nullptr;
    CU(cudaMallocAsync((void**)&ctr, sizeof(int) * C_TOTAL, s));
    CU(cudaStreamSynchronize(s));
    g->ctr = ctr;
    return TRUSS_OK;
}

void truss_release_workspace(truss_graph* g) {
    truss_release_compaction(g);
    cudaFree(g->ss);
    cudaFree(g->dmin);
    cudaFree(g->rows);
    g->rows = nullptr;
    cudaFree(g->lhub);
    cudaFree(g->hub_of);
    cudaFree(g->hub_bits);
    g->lhub = g->hub_of = nullptr;
    g->hub_bits = nullptr;
    g->n_hub = 0;
    g->sup_switch = 0;
    for (int k = 0; k < 2; k++) {
        for (int j = 0; j < 3; j++) {
            cudaFree(g->fq[k][j]);
            g->fq[k][j] = nullptr;
        }
        cudaFree(g->live[k]);
        g->live[k] = nullptr;
    }
    cudaFree(g->ctr);
    cudaFree(g->gctl);
    cudaFreeHost(g->h_ctr);
    for (int k = 0; k < 2; k++) {
        cudaFree(g->owner[k]);
        g->owner[k] = nullptr;
    }
    g->ss = nullptr;
    g->dmin = nullptr;
    g->ctr = nullptr;
    g->gctl = nullptr;
    g->h_ctr = nullptr;
}

extern "C" int truss_autotune(truss_graph* g, int8_t* h_table, int32_t repeats, void* stream) {
    if (!g || !h_table || repeats < 1) return TRUSS_EINVAL;
    for (int i = 0; i < TRUSS_TUNE_CLASSES; i++) h_table[i] = -1;
    if (g->m == 0) return TRUSS_OK;
    int32_t* d_out = nullptr;
    CU(cudaMalloc((void**)&d_out, sizeof(int32_t) * (size_t)g->m));
    truss_opts o;
    truss_default_opts(&o);
    o.sync = 1;
    truss_stats st;
    int rc = truss_decompose(g, d_out, &o, &st, stream);
    std::vector<truss_sublevel_trace> tr((size_t)std::max<int64_t>(1, st.sublevels));
    std::vector<double> tot((size_t)3 * TRUSS_TUNE_CLASSES, 0.0);
    std::vector<int> seen(TRUSS_TUNE_CLASSES, 0);
    const int vars[3] = {TRUSS_VAR_THREAD, TRUSS_VAR_GROUP, TRUSS_VAR_WARP};
    for (int k = 0; k < 3 && rc == TRUSS_OK; k++)
        for (int r = 0; r < repeats && rc == TRUSS_OK; r++) {
            o.variant = vars[k];
            o.h_trace = tr.data();
            o.max_sub = (int64_t)tr.size();
            rc = truss_decompose(g, d_out, &o, &st, stream);
            const int64_t n = std::min<int64_t>(st.sublevels, (int64_t)tr.size());
            for (int64_t i = 0; i < n && rc == TRUSS_OK; i++) {
                if (tr[i].n_light == 0) continue;  // the variant only maps light edges
                const int c = tune_class(tr[i].n_light, tr[i].dsum, (int64_t)tr[i].n_light + tr[i].n_heavy);
                tot[(size_t)k * TRUSS_TUNE_CLASSES + c] += (double)tr[i].t_ns;
                seen[c] = 1;
            }
        }
    cudaFree(d_out);
    if (rc != TRUSS_OK) return rc;
    for (int c = 0; c < TRUSS_TUNE_CLASSES; c++) {
        if (!seen[c]) continue;
        int best = 0;
        for (int k = 1; k < 3; k++)
            if (tot[(size_t)k * TRUSS_TUNE_CLASSES + c] < tot[(size_t)best * TRUSS_TUNE_CLASSES + c]) best = k;
        h_table[c] = (int8_t)vars[best];
    }
    return TRUSS_OK;
}

extern "C" void truss_default_opts(truss_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->loop = TRUSS_LOOP_PERSISTENT;
    o->variant = TRUSS_VAR_AUTO;
    o->sync = 0;
    o->level_jump = 1;
    o->timeout_ns = 10000000000ll;
    o->compact = -1;
}

// ------------------------------------------- edge-centric support (Alg. 2)

// Ros's support step as Algorithm 2 gives it: every edge {u, v} on its own
// counts the neighbours of v that are neighbours of u.  Here a warp takes an
// edge, walks its shorter row (32 entries per round, two per lane) and
// searches each entry in the longer row -- through the hub bitmap when that
// row belongs to a hub, else by binary search -- in place of the per-thread
// marker array X; the count is written once, without atomics.  Warps take
// edges in batches of ROS_BATCH from a counter, so the few edges with very
// long rows do not hold up a fixed share of the grid.
constexpr int ROS_BATCH = 8;

template <typename Off>
__global__ void __launch_bounds__(PT) k_support_ros(Graph<Off> G, const int32_t* __restrict__ perm,
                                                    int32_t* __restrict__ out, unsigned long long* next) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(next, (unsigned long long)ROS_BATCH);
        b0 = __shfl_sync(FULL_MASK, b0, 0);
        if ((int64_t)b0 >= G.m) break;
        const int64_t b1 = min((int64_t)b0 + ROS_BATCH, G.m);
        for (int64_t e = (int64_t)b0; e < b1; e++) {
            const Rows<Off> r = rows_of<Off>(G, (int32_t)e);
            int c = 0;
            for (Off j = r.a0 + lane; j < r.a1; j += 64) {
                const Off j2 = j + 32;
                const bool two = j2 < r.a1;
                const int32_t w1 = __ldg(G.col + j), w2 = two ? __ldg(G.col + j2) : w1;
                Off q1, q2;
                if (r.hub >= 0) {
                    q1 = hub_find<Off>(G, r.hub, r.b0, w1);
                    q2 = hub_find<Off>(G, r.hub, r.b0, w2);
                } else {
                    find2<Off>(G.col, r.b0, r.b1 - r.b0, w1, w2, q1, q2);
                }
                c += (q1 >= 0) + (two && q2 >= 0);
            }
            c = warp_sum(c);
            if (lane == 0) out[perm ? perm[e] : e] = c;
        }
    }
}

template <typename Off>
int support_ros_impl(truss_graph* g, int32_t* d_support, cudaStream_t s) {
    unsigned long long* next = reinterpret_cast<unsigned long long*>(g->ctr + C_ROS);
    CU(cudaMemsetAsync(next, 0, sizeof(unsigned long long), s));
    int per_sm = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_support_ros<Off>, PT, 0));
    const int blocks = std::max(1, per_sm) * g->sms;
    k_support_ros<Off><<<blocks, PT, 0, s>>>(graph_view<Off>(g), g->perm, d_support, next);
    CU(cudaGetLastError());
    truss_note_launch();
    return TRUSS_OK;
}

extern "C" int truss_support_ros(truss_graph* g, int32_t* d_support, void* stream) {
    if (!g || (g->m > 0 && !d_support)) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    TRY(truss_ensure_workspace(g, s));
    if (g->m == 0) return TRUSS_OK;
    return g->off64 ? support_ros_impl<int64_t>(g, d_support, s) : support_ros_impl<int32_t>(g, d_support, s);
}

extern "C" int truss_support(truss_graph* g, int32_t* d_support, void* stream) {
    if (!g || (g->m > 0 && !d_support)) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    TRY(truss_ensure_workspace(g, s));
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
        if (stats) memset(stats, 0, sizeof(*stats));
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
    if (!g || !h_nnext || ncurr < 0 || ncurr > g->m || variant < TRUSS_VAR_AUTO || variant > TRUSS_VAR_LEARNED)
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
