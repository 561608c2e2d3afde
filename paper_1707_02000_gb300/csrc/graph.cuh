// Device-resident graph handle shared by the build, support and peel units.
//
// HBM layout (internal vertex labels; with TRUSS_DEGREE_ORDER a vertex's
// label is its rank by (degree, input label)):
//   rowptr Off[n+1]   Es of Fig. 2: row offsets of the symmetric adjacency
//   eo     Off[n]     Eo of Fig. 2: first slot of row u whose neighbour > u
//   col    int32[2m]  N of Fig. 2: neighbours, every row ascending
//   eid    int32[2m]  Eid of Fig. 2: internal edge id of every slot
//   el     int2[m]    El of Fig. 2: endpoints (x < y) of internal edge e;
//                     internal ids are the lexicographic order of (x, y)
//   perm   int32[m]   internal edge id -> canonical (input-label) edge id;
//                     NULL when no relabelling is done (identity)
//   order  int32[n]   internal vertex -> input label; NULL = identity
// Peeling state (allocated on first decomposition):
//   ss     int2[m]    {S, stamp} per internal edge.  S is the live support;
//                     stamp is the number of the sub-level whose frontier
//                     the edge entered (INT32_MAX while it has entered none).
//                     During sub-level g: processed <=> stamp < g, in curr
//                     <=> stamp == g (the processed / inCurr / inNext arrays
//                     of Algorithms 4-5 folded into one word, so finishing a
//                     sub-level needs no pass over curr: g+1 flips them all).
//   dmin   int32[m]   min(d(u), d(v)) of each edge: length of the shorter
//                     row ProcessSubLevel walks, which sets its light/heavy
//                     class
//   fq[2]  3 x int32[m] per side of the curr/next ping-pong: light edges,
//                     heavy edges, first chunk number of each heavy edge
//   live[2] int32[m]  edges each Scan found above its level: the only edges
//                     the next Scan visits (a list that shrinks level by level)
//   owner[2] int2     chunk -> {edge, chunk index in its row}, each side
//   rows   Off[4m]    per edge: shorter row [a0, a1), longer row [b0, b1)
//   lhub   int32[m]   per edge: hub index of the longer row's vertex, -1
//   hub_of int32[n]   per vertex: hub index, -1 (degree below the threshold)
//   hub_bits          per hub: 32-byte blocks of 192 vertex ids, {count of
//                     neighbours before the block, 3 x 64 neighbour bits}
//   ctr    int[...]   device counters (see peel.cu)
// Row compaction (peel.cu; allocated on the first decomposition that uses it):
//   wcol, weid int32[.]   rows after a compaction; between levels the
//                     entries of processed edges are dropped from it, so the
//                     rows the peel walks and searches shrink as it goes
//   tcol, teid int32[.]   scatter target of a compaction (a compaction runs
//                     once at most 80 % (2^25 edges held or more) or 50 % of
//                     the held edges are live, so the live entries of the
//                     first one fit in 1.6 m or m slots; both buffers take
//                     that many)
//   wrows, wdmin, wlhub   working copies of rows / dmin / lhub, rewritten
//                     for the live edges by each compaction
//   vstart, vend Off[n]  current row bounds of every vertex in wcol
//   clive uint32[m/32]  live bit per edge at a compaction
//   cbits, ctoff, cbsum  live bits per slot, per-tile and per-block offsets
#pragma once
#include "common.cuh"

#define TRUSS_STAMP_NONE 0x7fffffff

// Words of the counter block (int index) where the support kernels count
// their work: u64 N+(v) entries walked, u64 hub-bitmap probes.
#define TRUSS_CTR_SUPPORT_WORK 50

// Support-kernel classes by upper degree d+(u): the warp-per-vertex kernel
// takes d+(u) <= TRUSS_SUP_WARP_CAP (its 128-entry instance when no d+(u)
// exceeds TRUSS_SUP_SPLIT), the block-per-vertex kernel up to
// TRUSS_SUP_BLOCK_CAP, a global-memory kernel beyond.
#define TRUSS_SUP_SPLIT 128
#define TRUSS_SUP_WARP_CAP 256
#define TRUSS_SUP_BLOCK_CAP 12288

struct truss_graph {
    int32_t n = 0;
    int64_t m = 0;
    int off64 = 0;
    int device = 0;
    int sms = 0;
    void* rowptr = nullptr;
    void* eo = nullptr;
    int32_t* col = nullptr;
    int32_t* eid = nullptr;
    int2* el = nullptr;
    int32_t* perm = nullptr;
    int32_t* order = nullptr;
    // vertices by upper degree for the support kernels
    int32_t* sup_big = nullptr;   // d+ in (WARP_CAP, BLOCK_CAP]
    int32_t n_sup_big = 0;
    int32_t* sup_huge = nullptr;  // d+ > BLOCK_CAP
    int32_t n_sup_huge = 0;
    int64_t sup_big_maxup = 0;   // over sup_big: the largest d+(u)
    int64_t sup_big_maxwin = 0;  // over sup_big: the largest n - 1 - u
    int64_t max_deg = 0;
    int last_grid = 0, last_per_sm = 0;  // blocks of the last persistent launch
    void* gctl = nullptr;   // state of the graph-driven level loop
    void* rows = nullptr;   // per edge: shorter row bounds, longer row bounds (Off x 4)
    int32_t* lhub = nullptr;     // per edge: hub index of the longer row's vertex, -1 if none
    int32_t* hub_of = nullptr;   // per vertex: hub index, -1 if none
    unsigned long long* hub_bits = nullptr;  // per hub: hub_words words, blocks of {count before, 3 x 64 ids}
    int32_t n_hub = 0;
    int64_t hub_words = 0;
    int64_t max_updeg = 0;
    int64_t wedges_up = 0;  // sum_v d-(v) d+(v)
    int64_t dmin_sum = 0;   // sum_e min(d(u), d(v))
    int sup_switch = 0;     // support kernels switch sides at hubs (truss_support_plan)
    int64_t sup_gain = 0;   // N+(v) entries the switch saves
    int hc = 64;            // heavy-edge chunk length used by ProcessSubLevel
    // peeling workspace
    int2* ss = nullptr;
    int32_t* dmin = nullptr;
    int32_t* fq[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    int32_t* live[2] = {nullptr, nullptr};  // live-edge lists of consecutive Scans
    int2* owner[2] = {nullptr, nullptr};     // chunk -> {edge, chunk index in its row}, per side
    uint32_t ocap = 0;
    // row compaction (see peel.cu)
    int32_t *wcol = nullptr, *weid = nullptr, *tcol = nullptr, *teid = nullptr;
    void* wrows = nullptr;
    int32_t *wdmin = nullptr, *wlhub = nullptr;
    void *vstart = nullptr, *vend = nullptr;
    uint32_t* cbits = nullptr;
    uint32_t* clive = nullptr;  // one bit per edge: unprocessed at the compaction
    int32_t* ctoff = nullptr;
    long long* cbsum = nullptr;
    int cmp_ready = 0;  // compaction workspace allocated
    int cmp_dirty = 0;  // working copies may differ from the pristine arrays
    int* ctr = nullptr;
    int* h_ctr = nullptr;  // pinned host mirror
    int latched = 0;       // latched device-side error status
};

// Implemented in support.cu: fills ss[e].x = S(e) for every internal edge;
// truss_support_plan decides the hub side switch once the bitmaps exist.
int truss_support_internal(truss_graph* g, int2* ss, cudaStream_t s);
int truss_support_plan(truss_graph* g, cudaStream_t s);
// Implemented in peel.cu.
int truss_ensure_workspace(truss_graph* g, cudaStream_t s);
void truss_release_workspace(truss_graph* g);
