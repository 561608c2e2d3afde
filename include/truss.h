/*
 * truss.h -- C ABI of the GB300 truss decomposition library (libtruss.so).
 *
 * The library computes, for every undirected edge of a simple graph, its
 * trussness: the largest k such that the edge belongs to a k-truss, a
 * subgraph in which every edge lies in at least k-2 triangles of the
 * subgraph (Kabir & Madduri, "Shared-memory Graph Truss Decomposition",
 * §II).  Edges in no triangle have trussness 2.  The method is PKT (§III):
 * per-edge triangle support (Algorithm 3), then level-synchronous peeling
 * (Algorithm 4: Scan; Algorithm 5: ProcessSubLevel), run as CUDA kernels.
 *
 * Conventions for every entry point:
 *  - Pointers prefixed d_ are device pointers, h_ host pointers.  The caller
 *    owns every buffer it passes; the library owns the opaque truss_graph and
 *    its device workspace, released by truss_free.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered: device work is enqueued on `stream`
 *    and may still be running when the call returns, unless stated otherwise.
 *  - Every call returns an int status (TRUSS_OK or a negative TRUSS_E*).
 *    Nothing is thrown across the ABI; no kernel traps.  Errors found on
 *    the device (a grid-barrier wait that exceeded its limit, an index out
 *    of range) are latched in the graph handle and returned by the next call
 *    that synchronises (truss_decompose with opts->sync = 1, truss_sync,
 *    truss_num_edges after a build, and every host-buffer call).
 *  - Canonical edge order: edge i is the i-th pair (min(u,v), max(u,v)) in
 *    ascending lexicographic order of the INPUT vertex labels, after
 *    self-loops and repeated pairs are dropped (§IV-A).  Every per-edge
 *    output is in that order, whatever internal relabelling is used.
 */
#ifndef TRUSS_H
#define TRUSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TRUSS_API __attribute__((visibility("default")))
#else
#define TRUSS_API
#endif

/* ------------------------------------------------------------- statuses */
#define TRUSS_OK 0
#define TRUSS_EINVAL (-1)    /* bad argument (null pointer, negative size)   */
#define TRUSS_ENOMEM (-2)    /* device or host allocation failed             */
#define TRUSS_ECUDA (-3)     /* a CUDA runtime call failed                   */
#define TRUSS_ETIMEOUT (-4)  /* a device-side wait gave up (grid barrier)    */
#define TRUSS_EOVERFLOW (-5) /* m or 2m does not fit the index width         */
#define TRUSS_EBADGRAPH (-6) /* a vertex id outside [0, n)                   */
#define TRUSS_EDEVICE (-7)   /* a device-side consistency check failed       */
#define TRUSS_ENOTSUP (-8)   /* the requested form is not available here     */
#define TRUSS_ETOOBIG (-9)   /* input larger than a fixed-capacity entry
                                point accepts                               */

/* Human-readable text for a status.  Never NULL; static storage. */
TRUSS_API const char* truss_strerror(int status);

/* ---------------------------------------------------------------- graph */
typedef struct truss_graph truss_graph;

/* truss_build_csr flags */
#define TRUSS_DEGREE_ORDER 1u /* relabel vertices by ascending degree inside
                                 the library (results stay in input labels) */
#define TRUSS_OFFSETS64 2u    /* store row offsets as int64 (else int32,
                                 switched to int64 automatically when 2m
                                 exceeds INT32_MAX)                          */
#define TRUSS_CORE_ORDER 4u   /* relabel vertices in a degeneracy order (§IV-B:
                                 vertices ordered by k-core): the order in
                                 which a level-synchronous k-core peel on the
                                 device removes them, ties by label, so each
                                 vertex has at most its coreness of
                                 neighbours after it.  Costs one host round
                                 trip per peel round at build time.  Takes
                                 precedence over TRUSS_DEGREE_ORDER.         */
#define TRUSS_LOCALITY_ORDER 8u /* relabel vertices in a reverse Cuthill-McKee
                                 order: a breadth-first search from the
                                 vertex of highest degree (lowest label among
                                 ties) ranks each new level by (rank of its
                                 first-ranked neighbour in the level before,
                                 label); the ranks are then reversed, and
                                 vertices the search does not reach follow
                                 in label order.  Close vertices get close
                                 labels, so rows and the edges of a
                                 triangle lie near each other in memory: for
                                 mesh-like graphs (the paper orders vertices
                                 for the same reason, §IV-B).  The support's
                                 orientation then follows this order, not
                                 the degree.  One host round trip per
                                 search level at build time.  Takes
                                 precedence over the other two orders.      */

/*
 * truss_build_csr -- build the device graph of §III / Fig. 2 from a raw edge
 * list: undirect, drop self-loops and repeated pairs (§IV-A), sort every
 * adjacency row ascending (N, row offsets Es), give each slot its edge id
 * (Eid), record the first slot whose neighbour exceeds the row vertex (Eo),
 * and the endpoint pair of every edge (El).  With TRUSS_DEGREE_ORDER the
 * vertices are relabelled by ascending degree first (the paper orders
 * vertices by k-core number for the same purpose, §IV-B; trussness does not
 * depend on the labelling).
 *   d_src, d_dst : device int32[n_in], endpoint pairs; may hold self-loops,
 *                  repeats and both orientations.  Read only; the caller may
 *                  free them once the call has synchronised.
 *   n_in         : number of pairs (>= 0).
 *   n            : number of vertices; ids must lie in [0, n).
 *   flags        : TRUSS_DEGREE_ORDER | TRUSS_CORE_ORDER | TRUSS_LOCALITY_ORDER
 *                  | TRUSS_OFFSETS64.
 *   out          : receives the handle (NULL on failure).
 * Synchronises `stream` before returning (the edge count sizes later
 * buffers).  Returns TRUSS_EBADGRAPH for an id outside [0, n),
 * TRUSS_EOVERFLOW if m >= 2^31-1, TRUSS_ENOMEM / TRUSS_ECUDA otherwise.
 * m = 0 is valid.
 */
TRUSS_API int truss_build_csr(const int32_t* d_src, const int32_t* d_dst, int64_t n_in, int32_t n, uint32_t flags,
                    void* stream, truss_graph** out);

/* Release the handle and all its device memory (NULL is ignored). */
TRUSS_API void truss_free(truss_graph* g);

/* Number of undirected edges m / vertices n of the built graph. */
TRUSS_API int truss_num_edges(const truss_graph* g, int64_t* m);
TRUSS_API int truss_num_vertices(const truss_graph* g, int32_t* n);

/* Canonical edge list: d_u[i] < d_v[i], input labels, int32[m] each. */
TRUSS_API int truss_edge_list(const truss_graph* g, int32_t* d_u, int32_t* d_v, void* stream);

/*
 * truss_csr_copy -- copy the internal augmented CSR (Fig. 2) for inspection:
 * d_rowptr int64[n+1] (Es), d_col int32[2m] (N), d_eid int32[2m] (Eid, in
 * canonical edge ids), d_eo int64[n] (Eo).  Internal vertex labels: with
 * TRUSS_DEGREE_ORDER they differ from the input labels, and d_order (int32[n],
 * may be NULL) receives the input label of each internal vertex.
 */
TRUSS_API int truss_csr_copy(const truss_graph* g, int64_t* d_rowptr, int32_t* d_col, int32_t* d_eid, int64_t* d_eo,
                   int32_t* d_order, void* stream);

/*
 * truss_support -- per-edge triangle count S(e), the number of triangles
 * containing e (§II), computed by the oriented vertex-iterator of
 * Algorithm 3 (each triangle u < v < w found once, +1 on its three edges).
 *   d_support : device int32[m], canonical order (written).
 */
TRUSS_API int truss_support(truss_graph* g, int32_t* d_support, void* stream);

/*
 * truss_support_ros -- the same S(e) by the edge-centric scheme of
 * Algorithm 2 (Ros's support step, §II): each edge {u, v} counts, on its
 * own, the neighbours of v that are also neighbours of u -- here by walking
 * the shorter of the two rows and searching each entry in the longer one
 * (the hub bitmap of a high-degree vertex stands in for the marker array X).
 * No orientation and no atomics: every edge writes its own count, at the
 * cost of min(d(u), d(v)) searches per edge instead of the oriented
 * scheme's one search per wedge of N+ lists.
 *   d_support : device int32[m], canonical order (written).
 * Allocates the graph's peeling workspace on first use, like truss_decompose.
 */
TRUSS_API int truss_support_ros(truss_graph* g, int32_t* d_support, void* stream);

/* ------------------------------------------------------- decomposition */

/* level-loop forms (how the sub-levels of Algorithm 4 are driven) */
#define TRUSS_LOOP_PLAIN 0      /* host loop, one launch per phase; the host
                                   reads the frontier size every sub-level */
#define TRUSS_LOOP_PERSISTENT 1 /* one cooperative kernel, grid barriers with
                                   a time limit between phases; its
                                   register budget is chosen from the graph:
                                   the _OCC form when the shorter-row entries
                                   the peel walks, W = sum_e min(d(u), d(v)),
                                   reach 2^24 per support level (W over the
                                   largest support + 1) or 2^34 in all, else
                                   the _LAT form.  The call waits for the
                                   support phase to read the largest support
                                   (the forced forms below do not wait)    */
#define TRUSS_LOOP_PERSISTENT_LAT 2 /* the persistent kernel at 4 blocks of
                                   256 threads per SM, 64 registers a thread
                                   (latency-bound peels: many small
                                   sub-levels of long rows)               */
#define TRUSS_LOOP_PERSISTENT_OCC 3 /* the persistent kernel at 6 blocks of
                                   256 threads per SM, 40 registers a thread
                                   (throughput-bound peels: few large
                                   sub-levels of short rows)              */
#define TRUSS_LOOP_GRAPH 4      /* one CUDA graph: a conditional while node
                                   whose body runs a one-block control
                                   kernel that picks the next phase on the
                                   device, then a switch node with the Scan
                                   or the ProcessSubLevel kernel; no host
                                   round trip between phases.  The limit
                                   (timeout_ns) applies to each phase, and
                                   the phases are bounded by 2m + dmax + 64 */

/* ProcessSubLevel work mappings (all exact).  Frontier edges whose shorter
 * adjacency row has more than 32 entries are always cut into fixed-size
 * chunks shared by every warp of the grid; the variant chooses how many
 * lanes walk each of the other ("light") edges. */
#define TRUSS_VAR_AUTO (-1)   /* chosen per sub-level from the frontier size */
#define TRUSS_VAR_THREAD 0    /* one thread per light edge                   */
#define TRUSS_VAR_GROUP 1     /* half a warp (16 lanes) per light edge; a
                                 longer row of at most 64 entries is held in
                                 registers and searched by shuffles; the
                                 default                                     */
#define TRUSS_VAR_WARP 2      /* one warp per light edge                     */
#define TRUSS_VAR_LEARNED 3   /* chosen per sub-level by the learned cost
                                 model (opts->sched_params); falls back to
                                 TRUSS_VAR_AUTO when it is absent, when the
                                 frontier has few light edges, or when the
                                 model's output is not finite              */

/* Learned scheduler (project addition): an FP32 MLP 5 -> 32 -> 32 -> 3 that
 * predicts the log2 device time of a sub-level under each of the three light-
 * edge variants (THREAD, GROUP, WARP) from the sub-level's features.
 * Parameters: TRUSS_SCHED_PARAMS floats, in this order: feature means [5],
 * inverse standard deviations [5], W1 [32][5], b1 [32], W2 [32][32], b2 [32],
 * W3 [3][32], b3 [3]; ReLU after the two hidden layers. */
#define TRUSS_SCHED_FEATURES 5
#define TRUSS_SCHED_VARIANTS 3
#define TRUSS_SCHED_PARAMS 1357

/* Autotuned variant table (project addition): TRUSS_TUNE_CLASSES entries,
 * indexed by 8 * min(15, floor(log2(1 + light edges))) +
 * min(7, floor(log2(1 + shorter-row sum / frontier size))); each entry is a
 * TRUSS_VAR_THREAD / GROUP / WARP, or -1 for the default. */
#define TRUSS_TUNE_CLASSES 128

/* One record per non-empty sub-level (see truss_opts.h_trace). */
typedef struct truss_sublevel_trace {
    int32_t level;     /* support level l                                     */
    int32_t group;     /* lanes per light edge used (1, 16 or 32)             */
    int32_t n_light;   /* frontier edges with shorter row <= 32 entries       */
    int32_t n_heavy;   /* the other frontier edges                            */
    uint32_t n_chunks; /* heavy-row chunks shared out to warps                */
    int32_t dmax;      /* longest shorter row in the frontier                 */
    int64_t dsum;      /* sum of shorter-row lengths over the frontier        */
    int64_t todo;      /* edges not yet peeled when the sub-level starts      */
    int64_t t_ns;      /* device time of the sub-level, barrier to barrier    */
    int64_t scan_ns;   /* device time of the Scans since the previous record
                          (the Scan, or empty Scans, that opened this level) */
} truss_sublevel_trace;

typedef struct truss_opts {
    int32_t loop;        /* TRUSS_LOOP_*                                      */
    int32_t variant;     /* TRUSS_VAR_*                                       */
    int32_t sync;        /* nonzero: synchronise before returning and report
                            device-side errors                                */
    int32_t level_jump;  /* nonzero: after an empty Scan, continue at the
                            smallest live support instead of l+1 (same result,
                            fewer empty scans)                                */
    int64_t timeout_ns;  /* limit on each device-side wait (0: 10 s)          */
    int32_t* h_sub_level; /* optional host arrays: level l and frontier size */
    int64_t* h_sub_size;  /* |curr| of every non-empty sub-level, in order   */
    int64_t max_sub;      /* their capacity (entries); needs sync = 1        */
    int32_t* d_peel_step; /* optional device int32[m], canonical order: the
                             number of the sub-level (0, 1, ...) in which each
                             edge was peeled -- a peeling order that lets a
                             checker certify the result (see truss_decompose) */
    truss_sublevel_trace* h_trace; /* optional host array of max_sub records,
                             one per sub-level; needs sync = 1               */
    const float* sched_params; /* device float[TRUSS_SCHED_PARAMS] for
                             TRUSS_VAR_LEARNED, or NULL                      */
    const int8_t* tune_table;  /* host int8[TRUSS_TUNE_CLASSES] consulted by
                             TRUSS_VAR_AUTO, or NULL (built-in default)      */
    int32_t compact;      /* row compaction between levels (persistent and
                             plain loops): -1 automatic (graphs of at least
                             TRUSS_COMPACT_MIN_EDGES edges), 0 off, 1 on for
                             any size.  Once at most 50 % (80 % while the
                             rows hold 2^25 edges or more) of the edges the
                             rows hold are unprocessed, the entries of
                             processed edges are dropped from the rows, so
                             ProcessSubLevel walks and searches only live
                             rows (the triangles it skips are those through
                             processed edges, §III); results are identical */
    int32_t max_level;    /* capacity (levels) of the two arrays below        */
    int64_t* h_level_edges; /* optional host int64[max_level]: edges peeled at
                             support level l, i.e. of trussness l + 2 (the
                             trussness distribution of Fig. 6); needs sync  */
    int64_t* h_level_ns;  /* optional host int64[max_level]: device time of
                             level l -- its Scans and sub-levels (the time
                             distribution of Fig. 6); needs sync = 1        */
} truss_opts;

/* Graphs with at least this many edges compact their rows by default. */
#define TRUSS_COMPACT_MIN_EDGES 65536

typedef struct truss_stats {
    int64_t m;           /* undirected edges                                 */
    int64_t sublevels;   /* non-empty sub-levels (frontiers) processed       */
    int64_t scans;       /* Scan passes over the support array               */
    int64_t triangles;   /* number of triangles (sum of support / 3)         */
    int32_t t_max;       /* largest trussness (0 when m = 0)                 */
    int32_t levels;      /* levels with at least one edge                    */
    float ms_support;    /* device time of the support phase (sync = 1)      */
    float ms_peel;       /* device time of the peeling phase (sync = 1)      */
    int64_t launches;    /* kernels this call launched                        */
    int64_t wedges_up;   /* W+ = sum over v of d-(v) * d+(v): N+ entries the
                            support kernel reads (internal vertex order)      */
    int64_t dmin_sum;    /* sum over edges of min(d(u), d(v)): entries of the
                            shorter row that ProcessSubLevel reads            */
    int64_t scanned;     /* entries all Scans visited: m for the first Scan,
                            then the live (unpeeled) edges each later Scan
                            reads from the compacted list (sync = 1)         */
    int32_t grid_blocks; /* blocks of the persistent launch (0: plain loop)  */
    int32_t blocks_per_sm; /* its blocks per SM (4: _LAT form, 6: _OCC)      */
    int32_t max_support; /* largest support before peeling (set when stats
                            are requested or the form is chosen)           */
    int32_t compactions; /* row compactions the peel ran (sync = 1)          */
    int64_t walked;      /* shorter-row entries ProcessSubLevel walked: the
                            sum over sub-levels of the frontier's shorter-row
                            lengths as the rows stood then (dmin_sum without
                            compaction; sync = 1)                           */
    int64_t compacted_slots; /* row entries the compactions visited (sync)  */
    int64_t support_walked;  /* N+(v) entries the support kernels read (at
                            most wedges_up: a pair u < v whose v is a hub
                            with a bitmap and whose N+(v) is longer than
                            u's entries above v walks those entries instead,
                            probing v's bitmap; sync = 1)                   */
    int64_t support_hub_probes; /* those bitmap probes (sync = 1)          */
} truss_stats;

/*
 * truss_triangle_count -- the number of triangles T of the graph (§II; the
 * sum of all supports is 3T): the support kernels' walk (Algorithm 3, each
 * triangle found once at its lowest vertex) without edge ids or per-edge
 * atomics.  *h_count (host) receives T.  Synchronous on the stream.
 * Errors: TRUSS_EINVAL for null arguments.
 */
TRUSS_API int truss_triangle_count(truss_graph* g, int64_t* h_count, void* stream);

/*
 * truss_ktruss_components -- the k-trusses of the graph as subgraphs (§II:
 * a k-truss is a maximal connected subgraph whose every edge lies in at
 * least k-2 of its triangles): the connected components of the edges whose
 * trussness is >= k.
 *   d_truss : device int32[m], canonical order (as truss_decompose writes it).
 *   k       : any value; k <= 2 takes every edge.
 *   d_comp  : device int32[m], canonical order (written): the smallest input
 *             vertex label of the edge's k-truss, or -1 when the edge's
 *             trussness is below k.
 *   h_ncomp : host int64 (may be NULL): the number of k-trusses; when given
 *             the call waits for the result.
 * Errors: TRUSS_EINVAL for null arguments; TRUSS_EDEVICE if a union-find
 * loop hit its step bound (only on a corrupted state; reported when h_ncomp
 * is given).  Allocates and frees 8 bytes per vertex in the call.
 */
TRUSS_API int truss_ktruss_components(truss_graph* g, const int32_t* d_truss, int32_t k, int32_t* d_comp,
                                      int64_t* h_ncomp, void* stream);

/* Fill *opts with defaults: persistent loop, heuristic variants, no sync,
 * level jumps on, 10 s wait limit, no sub-level recording. */
TRUSS_API void truss_default_opts(truss_opts* opts);

/*
 * truss_decompose -- trussness of every edge (§II) by PKT: support
 * (Algorithm 3), then, level l = 0, 1, ...: Scan gathers the edges whose
 * support equals l (Algorithm 4); ProcessSubLevel (Algorithm 5) walks the
 * triangles of each such edge whose other two edges are unprocessed and
 * lowers the support of those other edges that are above l, by one per
 * triangle, never below l; edges that reach l form the next sub-level.  When
 * two edges of a triangle are in the same sub-level, the lower edge id
 * handles it (§III, Fig. 3).  Trussness = final support + 2.
 *   d_truss : device int32[m], canonical order (written).
 *   opts    : NULL for defaults (truss_default_opts).
 * Certificate: with opts->d_peel_step, ordering the edges by (peel step,
 * edge id) gives a removal order in which every edge, when removed, lies in
 * at most trussness-2 triangles of the edges not yet removed, and trussness
 * never decreases along it; together with "every edge of trussness k lies in
 * >= k-2 triangles of edges of trussness >= k" this proves the result exact.
 *   stats   : may be NULL; filled only when opts->sync is set.
 * Workspace: the first call on a graph allocates its peeling workspace and
 * keeps it until truss_free (roughly 100 to 150 bytes per edge with int32
 * offsets, plus neighbour bitmaps of its vertices of degree >= 1024 -- the
 * threshold doubles until the bitmaps fit 1024 bytes per edge and 3/4 of the
 * device memory free at that moment -- plus, for graphs that compact their
 * rows, about 60 bytes per edge more); TRUSS_ENOMEM when the device cannot
 * hold the rest.
 */
TRUSS_API int truss_decompose(truss_graph* g, int32_t* d_truss, const truss_opts* opts, truss_stats* stats, void* stream);

/*
 * truss_decompose_local -- the same trussness by the asynchronous local
 * iteration the paper contrasts with level-synchronous peeling (§II: the
 * MPM-style update rule and its nucleus/truss generalisation).  Starting
 * from S(e) + 2, every active edge repeatedly takes the value
 *   2 + min(its value - 2, h),  h = the largest k such that at least k of
 *   its triangles {e, e2, e3} have min(value(e2), value(e3)) - 2 >= k,
 * in place and without level or sub-level barriers, until a sweep changes
 * nothing; edges sharing a triangle with a changed edge are the next sweep's
 * active set.  The fixed point reached from these upper bounds is the
 * trussness, identical to truss_decompose.
 *   d_truss    : device int32[m], canonical order (written).
 *   max_sweeps : limit on sweeps (<= 0: none); TRUSS_ETIMEOUT when reached.
 *   h_sweeps, h_updates : may be NULL; receive the sweeps run and the value
 *                changes made.
 * Synchronises `stream` once per sweep.  Allocates 6 bytes per edge for the
 * call, and the graph's peeling workspace on first use.
 */
TRUSS_API int truss_decompose_local(truss_graph* g, int32_t* d_truss, int64_t max_sweeps, int64_t* h_sweeps,
                                    int64_t* h_updates, void* stream);

/*
 * truss_peel_sublevel -- one ProcessSubLevel (Algorithm 5) on a caller-set
 * state, for tests and tuning.  All arrays are device arrays in canonical
 * edge order:
 *   d_S     : int32[m] support, updated in place;
 *   d_flags : uint8[m], bit 0 = processed, bit 1 = in curr; on return curr
 *             edges are processed and not in curr, next edges are in curr;
 *   d_curr  : int32[ncurr] canonical edge ids, all with d_S == l (their
 *             in-curr bit is set by the call);
 *   d_next  : int32[m] receives the next frontier (any order);
 *   h_nnext : host int64, receives |next|.
 * Synchronises `stream`.  TRUSS_EINVAL when ncurr > m.  d_curr is checked
 * on the device before any other kernel reads it: TRUSS_EBADGRAPH when an id
 * lies outside [0, m) or appears twice (the state is then left untouched).
 */
TRUSS_API int truss_peel_sublevel(truss_graph* g, int32_t* d_S, uint8_t* d_flags, const int32_t* d_curr, int64_t ncurr,
                        int32_t l, int32_t* d_next, int64_t* h_nnext, int32_t variant, void* stream);

/*
 * truss_decompose_host -- the whole pipeline from host memory: copy the raw
 * edge list h_src/h_dst (int32[n_in], host; pinned memory is fastest) to the
 * device, build the graph (flags as truss_build_csr), decompose, and copy
 * the trussness back to h_truss (host int32, capacity m_cap >= m, canonical
 * order).  *m_out receives m.  Synchronous.  Device workspace is allocated
 * and freed inside the call.
 */
TRUSS_API int truss_decompose_host(const int32_t* h_src, const int32_t* h_dst, int64_t n_in, int32_t n, uint32_t flags,
                         int32_t* h_truss, int64_t m_cap, int64_t* m_out, const truss_opts* opts,
                         truss_stats* stats, void* stream);

/*
 * truss_decompose_batch -- trussness of every edge of G independent graphs
 * in one decomposition.  No triangle spans two graphs, so the graphs are
 * peeled together as one disjoint union (graph g's vertices relabelled to a
 * contiguous range): one support pass and one level loop (one persistent
 * launch) serve all of them, and a sub-level of the union is the union of
 * the graphs' sub-levels at the same level.
 *   d_src, d_dst : device int32 raw pairs of all graphs; graph g's pairs are
 *                  [h_eoff[g], h_eoff[g+1]), with vertex ids local to the
 *                  graph, in [0, h_nverts[g]).
 *   h_eoff       : host int64[G+1], h_eoff[0] = 0.
 *   h_nverts     : host int32[G]; their sum must be below 2^31.
 *   d_truss      : device int32[capacity] (capacity >= total edges; the total
 *                  number of pairs always suffices): graph after graph, each
 *                  in its own canonical edge order.
 *   h_moff       : host int64[G+1] out: graph g's trussness is
 *                  d_truss[h_moff[g] .. h_moff[g+1]).
 *   flags, opts, stats: as truss_build_csr / truss_decompose.
 * Synchronous.  Device workspace is allocated and freed inside the call.
 */
TRUSS_API int truss_decompose_batch(const int32_t* d_src, const int32_t* d_dst, const int64_t* h_eoff,
                                    const int32_t* h_nverts, int32_t G, uint32_t flags, int32_t* d_truss,
                                    int64_t capacity, int64_t* h_moff, const truss_opts* opts, truss_stats* stats,
                                    void* stream);

/* ---------------------------------------- learned scheduler, autotuner */

/* Features of each of n sub-level records (host): log2(1 + x) of the
 * frontier size, the sum and the maximum of its shorter-row lengths, the
 * level and the edges not yet peeled.  x: host float[n][5].  The persistent
 * kernel computes the same five values on the device. */
TRUSS_API void truss_sched_features(const truss_sublevel_trace* tr, int64_t n, float* x);

/* Random initial weights (He-style uniform, counter-based from seed) into
 * device float[TRUSS_SCHED_PARAMS].  Synchronises `stream`. */
TRUSS_API int truss_sched_init(float* d_params, uint64_t seed, void* stream);

/* Mean squared error L = sum over samples and variants of (o - y)^2 / (3n)
 * of the model on d_x (device float[n][5]) against d_y (device float[n][3],
 * log2 times), and its gradient with respect to every parameter (device
 * float[TRUSS_SCHED_PARAMS]; the normalisation entries receive their
 * gradient too but training keeps them fixed).  Synchronises `stream`. */
TRUSS_API int truss_sched_grad(const float* d_params, const float* d_x, const float* d_y, int64_t n, float* d_grad,
                               float* h_loss, void* stream);

/* Train on the device: set the normalisation from d_x, then `epochs` full-
 * batch Adam steps (learning rate lr, betas 0.9 / 0.999) on the loss of
 * truss_sched_grad.  *h_loss receives the final loss.  Synchronises. */
TRUSS_API int truss_sched_train(float* d_params, const float* d_x, const float* d_y, int64_t n, int32_t epochs,
                                float lr, float* h_loss, void* stream);

/* Predicted log2 times, d_out device float[n][3]. */
TRUSS_API int truss_sched_predict(const float* d_params, const float* d_x, int64_t n, float* d_out, void* stream);

/* Autotuner: decompose g once per light-edge variant (THREAD, GROUP, WARP),
 * `repeats` times each, timing every sub-level; for every class of
 * TRUSS_TUNE_CLASSES with data, h_table receives the variant with the least
 * total time (-1 for classes without data).  Synchronous. */
TRUSS_API int truss_autotune(truss_graph* g, int8_t* h_table, int32_t repeats, void* stream);

/* Wait for the graph's pending device work on `stream` and return any
 * latched device-side error (and clear it). */
TRUSS_API int truss_sync(truss_graph* g, void* stream);

/* truss_pool_keep -- how many bytes of freed device memory the stream-ordered
 * pool the library allocates from (this process's default pool on the
 * current device) keeps for reuse instead of returning it to the driver
 * (the library's default: 16 GiB, set by its first graph build).  Keeping
 * more saves mapping the memory again when graph after graph is built and
 * freed (R-MAT scale 24 through truss_decompose_host: 2.19 s a call with
 * 16 GiB kept, 1.99 s with 200 GB); the memory kept is not available to
 * other allocators in the process (cudaMalloc, frameworks' caching
 * allocators).  0 also returns what the pool holds now.  The paper has no
 * counterpart.  TRUSS_EINVAL for a negative size. */
TRUSS_API int truss_pool_keep(int64_t bytes);

/* ---------------------------------------------- allocation-free support */

/* Largest vertex count truss_support_noalloc accepts. */
#define TRUSS_NOALLOC_MAX_VERTICES (1 << 22)

/*
 * truss_support_noalloc -- per-edge triangle support S(e) (as truss_support)
 * for a graph the caller already holds on the device, without allocating
 * any device memory.  The paper has no counterpart: it exists for callers
 * that must not call cudaMalloc or cudaFree -- e.g. a process whose
 * framework allocator owns all device memory, or a latency-critical loop with
 * a fixed memory budget.  Every other entry point allocates workspace.
 *   d_rowptr : device int32[n+1], row offsets of the symmetric adjacency
 *              (Es of Fig. 2), d_rowptr[n] = 2m.
 *   d_col    : device int32[2m], neighbours, each row strictly ascending, no
 *              self-loops (N of Fig. 2).
 *   d_eid    : device int32[2m], the edge id in [0, m) of every slot; both
 *              slots of an edge carry the same id (Eid of Fig. 2).
 *   n, m     : vertices (0 <= n <= TRUSS_NOALLOC_MAX_VERTICES) and edges.
 *   d_support: device int32[m], indexed by edge id (written).
 * Scratch: a fixed array of (TRUSS_NOALLOC_MAX_VERTICES + 64) int32 (16 MiB)
 * in the library's device memory, held by every GPU that uses it until the
 * process exits.  CUDA loads the library's device code lazily, so the array
 * is reserved on a device by the first truss_support_noalloc call there
 * (which can fail with TRUSS_ENOMEM or TRUSS_ECUDA if device memory is
 * already exhausted); that call also looks up the array's address
 * (cudaGetSymbolAddress, with the device current) and caches it.  A caller
 * whose allocator will take all device memory should therefore make one call
 * first -- a call with n = 0 and m = 0 does only this set-up -- and make it
 * before any stream capture.  All calls share the array, so calls whose
 * device work overlaps (on two streams, or from two host threads) race and
 * must be serialised by the caller.
 * Checks: d_rowptr is validated on the device before any other array is read
 * through it (d_rowptr[0] = 0, d_rowptr[n] = 2m, no row ends before it
 * starts); neighbours and edge ids are range-checked where they are used.
 * Synchronises `stream`.  Returns TRUSS_ETOOBIG when n exceeds the maximum,
 * TRUSS_EOVERFLOW when 2m exceeds INT32_MAX, TRUSS_EBADGRAPH for bad row
 * offsets (nothing else is read) or a neighbour or edge id out of range
 * (those entries are skipped, never written through), TRUSS_EINVAL for null
 * pointers or negative sizes.  Rows that are not sorted are not detected;
 * they give wrong counts but every access stays within the arrays.
 */
TRUSS_API int truss_support_noalloc(const int32_t* d_rowptr, const int32_t* d_col, const int32_t* d_eid, int32_t n,
                                    int64_t m, int32_t* d_support, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TRUSS_H */
