/*
 * CPU ORACLE for truss decomposition -- test infrastructure only.
 *
 * Plain, serial, obviously-correct C.  Only the tests, the package's smoke
 * check and the bench's CPU-baseline leg may load this file's library; the
 * product path never does.  It shares no code with the CUDA path: it does
 * its own canonicalisation, adjacency build, support count and peeling.
 *
 * Definitions (paper §II): the support S(e) of an edge is the number of
 * triangles containing it; a k-truss is a subgraph in which every edge has
 * support >= k-2 within it; the trussness of e is the largest k such that e
 * lies in a k-truss.  Edges in no triangle have trussness 2.
 *
 * What is here:
 *   or_canonical      undirect, drop self-loops and repeated pairs, order
 *                     edges lexicographically by (min, max) endpoint (§IV-A).
 *                     The position in that order is the edge id everywhere.
 *   or_support        S(e) = |N(u) ∩ N(v)| for every edge (§II).
 *   or_truss_wc       the serial bottom-up peel of Algorithm 1 (Wang-Cheng):
 *                     edges kept in bins by support (the Batagelj-Zaversnik
 *                     bin structure the paper points to), the lowest-support
 *                     edge removed each step, the other two edges of each of
 *                     its live triangles decremented if above its support.
 *                     A sorted-adjacency binary search replaces the hash
 *                     table of Algorithm 1; a removed[] flag replaces
 *                     deletion from it.  Trussness = S + 2.
 *   or_pkt_serial     the level-synchronous loop of Algorithms 4 and 5 run
 *                     one edge at a time: Scan at level l, then sub-levels
 *                     of ProcessSubLevel until the frontier is empty.  It
 *                     reports the frontier size of every sub-level, which
 *                     the parallel method must reproduce exactly.
 *   or_sublevel       one ProcessSubLevel (Algorithm 5) on a caller-given
 *                     state (S, processed/inCurr flags, curr, l).
 *   or_truss_batch    or_truss_wc over many independent graphs, spread over
 *                     host threads (one graph per task).
 *   or_certify        checks a claimed trussness against the definition at
 *                     any size, given a claimed peeling order (the sub-level
 *                     each edge was peeled in).  Lower bound: every edge of
 *                     claimed trussness k lies in >= k-2 triangles whose
 *                     other edges have claimed trussness >= k, so each set
 *                     {claimed >= k} is a k-truss subgraph (§II) and the true
 *                     trussness is at least the claim.  Upper bound: ordering
 *                     edges by (step, id), the claim never decreases along
 *                     the order and every edge lies in <= claim-2 triangles
 *                     of edges after it; if e were in a k-truss H with
 *                     k > claim(e), the first edge of H in the order would
 *                     lie in >= k-2 triangles of later edges while its own
 *                     claim is <= claim(e) < k -- a contradiction.  Edges
 *                     are checked in parallel on host threads.
 *   or_certify_sample the same per-edge conditions for a sample of edges
 *                     (rows built only for the sampled edges' endpoints),
 *                     with the order check over all edges: the check used
 *                     where the whole certificate costs too long.
 *
 * Readings of the paper taken here (each is stated where it is used):
 *   - the level variable l of Algorithms 4 and 5 is a support value, so
 *     edges of trussness k are peeled at level l = k-2 (Algorithm 4 compares
 *     S[e] = l; the text speaks of support k-2);
 *   - the peel loop counts down the m edges (Algorithm 4 initialises the
 *     counter with n, but subtracts frontier sizes, which count edges);
 *   - Algorithm 5 prints only the decrement of e2; the rule is applied to
 *     e3 symmetrically: e2 is decremented when S[e2] > l and (e3 not in
 *     curr or e1 < e3), e3 when S[e3] > l and (e2 not in curr or e1 < e2).
 *     Two curr edges of one triangle thus let the lower id handle it (§III,
 *     "Concurrent triangle processing", Fig. 3).
 *
 * Error returns: -1 bad argument (vertex id outside [0, n), negative size,
 * more than 2^31-1 edges), -2 out of memory.
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ helpers */

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

typedef struct { int32_t w; int32_t e; } slot_t; /* neighbour and edge id */

static int cmp_slot(const void* a, const void* b) {
    int32_t x = ((const slot_t*)a)->w, y = ((const slot_t*)b)->w;
    return (x > y) - (x < y);
}

typedef struct {
    int32_t n;
    int64_t m;
    int64_t* off;  /* [n+1] */
    slot_t* adj;   /* [2m], each row ascending by neighbour */
} graph_t;

static void graph_free(graph_t* g) {
    free(g->off);
    free(g->adj);
    g->off = NULL;
    g->adj = NULL;
}

/* Adjacency lists from a canonical edge list (u < v, ids 0..m-1). */
static int graph_build(graph_t* g, int32_t n, int64_t m, const int32_t* eu, const int32_t* ev) {
    g->n = n;
    g->m = m;
    g->off = calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = malloc(sizeof(slot_t) * (size_t)(2 * m + 1));
    int64_t* cur = malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!g->off || !g->adj || !cur) { free(cur); graph_free(g); return -2; }
    for (int64_t e = 0; e < m; e++) {
        if (eu[e] < 0 || eu[e] >= n || ev[e] < 0 || ev[e] >= n || eu[e] == ev[e]) {
            free(cur); graph_free(g); return -1;
        }
        g->off[eu[e] + 1]++;
        g->off[ev[e] + 1]++;
    }
    for (int32_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
    memcpy(cur, g->off, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; e++) {
        g->adj[cur[eu[e]]].w = ev[e]; g->adj[cur[eu[e]]].e = (int32_t)e; cur[eu[e]]++;
        g->adj[cur[ev[e]]].w = eu[e]; g->adj[cur[ev[e]]].e = (int32_t)e; cur[ev[e]]++;
    }
    for (int32_t v = 0; v < n; v++)
        qsort(g->adj + g->off[v], (size_t)(g->off[v + 1] - g->off[v]), sizeof(slot_t), cmp_slot);
    free(cur);
    return 0;
}

static inline int64_t deg(const graph_t* g, int32_t v) { return g->off[v + 1] - g->off[v]; }

/* Edge id of {x, w}, or -1 when x and w are not adjacent (binary search). */
static int32_t find_edge(const graph_t* g, int32_t x, int32_t w) {
    int64_t lo = g->off[x], hi = g->off[x + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t y = g->adj[mid].w;
        if (y == w) return g->adj[mid].e;
        if (y < w) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------ canonical list */

int64_t or_canonical(const int32_t* src, const int32_t* dst, int64_t n_in, int32_t n,
                     int32_t* eu, int32_t* ev) {
    if (n_in < 0 || n < 0) return -1;
    uint64_t* key = malloc(sizeof(uint64_t) * (size_t)(n_in + 1));
    if (!key) return -2;
    int64_t k = 0;
    for (int64_t i = 0; i < n_in; i++) {
        int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n) { free(key); return -1; }
        if (a == b) continue; /* self-loop */
        int32_t lo = a < b ? a : b, hi = a < b ? b : a;
        key[k++] = ((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi;
    }
    qsort(key, (size_t)k, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (int64_t i = 0; i < k; i++) {
        if (i > 0 && key[i] == key[i - 1]) continue; /* repeated pair */
        if (m > INT32_MAX - 1) { free(key); return -1; }
        eu[m] = (int32_t)(key[i] >> 32);
        ev[m] = (int32_t)(key[i] & 0xffffffffu);
        m++;
    }
    free(key);
    return m;
}

/* ------------------------------------------------------------- support */

/* |N(u) ∩ N(v)|: walk the shorter list, binary search each entry in the
 * longer one. */
static int32_t common_count(const graph_t* g, int32_t u, int32_t v) {
    int32_t a = u, b = v;
    if (deg(g, a) > deg(g, b)) { a = v; b = u; }
    int32_t c = 0;
    for (int64_t j = g->off[a]; j < g->off[a + 1]; j++)
        if (find_edge(g, b, g->adj[j].w) >= 0) c++;
    return c;
}

static void support_all(const graph_t* g, const int32_t* eu, const int32_t* ev, int32_t* S) {
    for (int64_t e = 0; e < g->m; e++) S[e] = common_count(g, eu[e], ev[e]);
}

int or_support(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, int32_t* S) {
    graph_t g;
    int rc = graph_build(&g, n, m, eu, ev);
    if (rc) return rc;
    support_all(&g, eu, ev, S);
    graph_free(&g);
    return 0;
}

/* ------------------------------------------------ Algorithm 1 (WC peel) */

typedef struct {
    int32_t* S;
    int64_t* bin_start; /* first position of each support value */
    int32_t* vert;      /* edges in ascending support order */
    int64_t* pos;       /* position of each edge in vert */
} bins_t;

/* S[f] -= 1 if S[f] > k, keeping vert sorted: f swaps with the first edge of
 * its bin, and that bin's start moves one place right. */
static void dec_above(bins_t* b, int32_t f, int32_t k) {
    int32_t s = b->S[f];
    if (s <= k) return;
    int64_t pf = b->pos[f], pb = b->bin_start[s];
    int32_t g = b->vert[pb];
    if (g != f) {
        b->vert[pf] = g; b->pos[g] = pf;
        b->vert[pb] = f; b->pos[f] = pb;
    }
    b->bin_start[s]++;
    b->S[f] = s - 1;
}

static int truss_wc(const graph_t* g, const int32_t* eu, const int32_t* ev, int32_t* tau, int32_t* S0) {
    int64_t m = g->m;
    int32_t* S = malloc(sizeof(int32_t) * (size_t)(m + 1));
    uint8_t* removed = calloc((size_t)m + 1, 1);
    int32_t* vert = malloc(sizeof(int32_t) * (size_t)(m + 1));
    int64_t* pos = malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!S || !removed || !vert || !pos) { free(S); free(removed); free(vert); free(pos); return -2; }
    support_all(g, eu, ev, S);
    if (S0) memcpy(S0, S, sizeof(int32_t) * (size_t)m);
    int32_t smax = 0;
    for (int64_t e = 0; e < m; e++) if (S[e] > smax) smax = S[e];
    int64_t* bin_start = calloc((size_t)smax + 2, sizeof(int64_t));
    if (!bin_start) { free(S); free(removed); free(vert); free(pos); return -2; }
    /* counting sort of edges by support */
    for (int64_t e = 0; e < m; e++) bin_start[S[e] + 1]++;
    for (int32_t s = 0; s <= smax; s++) bin_start[s + 1] += bin_start[s];
    {
        int64_t* fill = malloc(sizeof(int64_t) * ((size_t)smax + 1));
        if (!fill) { free(bin_start); free(S); free(removed); free(vert); free(pos); return -2; }
        memcpy(fill, bin_start, sizeof(int64_t) * ((size_t)smax + 1));
        for (int64_t e = 0; e < m; e++) { pos[e] = fill[S[e]]++; vert[pos[e]] = (int32_t)e; }
        free(fill);
    }
    bins_t b = {S, bin_start, vert, pos};
    for (int64_t i = 0; i < m; i++) {
        int32_t e = vert[i];
        int32_t k = S[e];
        int32_t u = eu[e], v = ev[e];
        int32_t x = deg(g, u) <= deg(g, v) ? u : v; /* canonical: d(x) <= d(y) */
        int32_t y = x == u ? v : u;
        for (int64_t j = g->off[x]; j < g->off[x + 1]; j++) {
            int32_t w = g->adj[j].w, f1 = g->adj[j].e;
            if (w == y || removed[f1]) continue;
            int32_t f2 = find_edge(g, y, w);
            if (f2 < 0 || removed[f2]) continue;
            /* live triangle {x, y, w}: lower both other edges if above k */
            dec_above(&b, f1, k);
            dec_above(&b, f2, k);
        }
        removed[e] = 1;
    }
    for (int64_t e = 0; e < m; e++) tau[e] = S[e] + 2;
    free(bin_start); free(S); free(removed); free(vert); free(pos);
    return 0;
}

int or_truss_wc(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, int32_t* tau, int32_t* S0) {
    if (m < 0 || m > INT32_MAX - 1) return -1;
    graph_t g;
    int rc = graph_build(&g, n, m, eu, ev);
    if (rc) return rc;
    rc = truss_wc(&g, eu, ev, tau, S0);
    graph_free(&g);
    return rc;
}

/* ------------------------------------- Algorithms 4 and 5, one at a time */

enum { F_PROCESSED = 1, F_INCURR = 2 };

/* One ProcessSubLevel: every triangle through each e1 in curr whose other
 * two edges are unprocessed lowers those of them that are not in curr (or
 * whose curr partner has a higher id) by one, never below l.  Edges that
 * reach l are returned in next (ascending).  At the end, curr is processed
 * and next becomes the in-curr set of the following sub-level. */
static int64_t sublevel(const graph_t* g, const int32_t* eu, const int32_t* ev, int32_t* S, uint8_t* flag,
                        const int32_t* curr, int64_t ncurr, int32_t l, int32_t* next) {
    int64_t nnext = 0;
    for (int64_t c = 0; c < ncurr; c++) {
        int32_t e1 = curr[c];
        int32_t u = eu[e1], v = ev[e1];
        int32_t a = deg(g, u) <= deg(g, v) ? u : v;
        int32_t b = a == u ? v : u;
        for (int64_t j = g->off[a]; j < g->off[a + 1]; j++) {
            int32_t w = g->adj[j].w;
            if (w == b) continue;
            int32_t f_aw = g->adj[j].e;
            int32_t f_bw = find_edge(g, b, w);
            if (f_bw < 0) continue;
            /* name the other two edges as in Algorithm 5: e2 = {v, w}, e3 = {u, w} */
            int32_t e2 = (a == v) ? f_aw : f_bw;
            int32_t e3 = (a == u) ? f_aw : f_bw;
            if ((flag[e2] & F_PROCESSED) || (flag[e3] & F_PROCESSED)) continue;
            if (S[e2] > l && (!(flag[e3] & F_INCURR) || e1 < e3)) {
                S[e2] -= 1;
                if (S[e2] == l) next[nnext++] = e2;
            }
            if (S[e3] > l && (!(flag[e2] & F_INCURR) || e1 < e2)) {
                S[e3] -= 1;
                if (S[e3] == l) next[nnext++] = e3;
            }
        }
    }
    for (int64_t c = 0; c < ncurr; c++) flag[curr[c]] = (uint8_t)((flag[curr[c]] | F_PROCESSED) & ~F_INCURR);
    for (int64_t c = 0; c < nnext; c++) flag[next[c]] |= F_INCURR;
    /* ascending order, so the result does not depend on visit order */
    qsort(next, (size_t)nnext, sizeof(int32_t), cmp_i32);
    return nnext;
}

int64_t or_sublevel(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, int32_t* S, uint8_t* flag,
                    const int32_t* curr, int64_t ncurr, int32_t l, int32_t* next) {
    if (m < 0 || ncurr < 0 || m > INT32_MAX - 1) return -1;
    for (int64_t c = 0; c < ncurr; c++) {
        if (curr[c] < 0 || curr[c] >= m) return -1;
        flag[curr[c]] |= F_INCURR;
    }
    graph_t g;
    int rc = graph_build(&g, n, m, eu, ev);
    if (rc) return rc;
    int64_t r = sublevel(&g, eu, ev, S, flag, curr, ncurr, l, next);
    graph_free(&g);
    return r;
}

/* Algorithm 4 run serially.  tau: trussness per edge.  sub_level/sub_size:
 * level and frontier size of each non-empty sub-level, written up to
 * max_sub entries; the return value is the total number of sub-levels.
 * step (may be NULL): number of the sub-level each edge was peeled in. */
int64_t or_pkt_serial(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, int32_t* tau,
                      int32_t* sub_level, int64_t* sub_size, int64_t max_sub, int32_t* step) {
    if (m < 0 || m > INT32_MAX - 1) return -1;
    graph_t g;
    int rc = graph_build(&g, n, m, eu, ev);
    if (rc) return rc;
    int32_t* S = malloc(sizeof(int32_t) * (size_t)(m + 1));
    uint8_t* flag = calloc((size_t)m + 1, 1);
    int32_t* curr = malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t* next = malloc(sizeof(int32_t) * (size_t)(m + 1));
    if (!S || !flag || !curr || !next) {
        free(S); free(flag); free(curr); free(next); graph_free(&g); return -2;
    }
    support_all(&g, eu, ev, S);
    int64_t todo = m, nsub = 0;
    int32_t l = 0;
    while (todo > 0) {
        /* Scan: curr = {e : S[e] = l}; an edge with S[e] = l is unprocessed,
         * since processed edges keep the lower level they were peeled at */
        int64_t ncurr = 0;
        for (int64_t e = 0; e < m; e++)
            if (S[e] == l && !(flag[e] & F_PROCESSED)) { curr[ncurr++] = (int32_t)e; flag[e] |= F_INCURR; }
        while (ncurr > 0) {
            if (nsub < max_sub) { sub_level[nsub] = l; sub_size[nsub] = ncurr; }
            if (step)
                for (int64_t c = 0; c < ncurr; c++) step[curr[c]] = (int32_t)nsub;
            nsub++;
            todo -= ncurr;
            int64_t nn = sublevel(&g, eu, ev, S, flag, curr, ncurr, l, next);
            int32_t* t = curr; curr = next; next = t;
            ncurr = nn;
        }
        l++;
    }
    for (int64_t e = 0; e < m; e++) tau[e] = S[e] + 2;
    free(S); free(flag); free(curr); free(next);
    graph_free(&g);
    return nsub;
}

/* ------------------------------------------------ many graphs, threads */

typedef struct {
    int64_t G;
    const int32_t* nverts;
    const int64_t* eoff;
    const int32_t *src, *dst;
    int64_t* m_out;
    int32_t* tau;
    atomic_llong next_graph;
    atomic_int err;
} batch_ctx;

static void* batch_worker(void* p) {
    batch_ctx* c = (batch_ctx*)p;
    for (;;) {
        int64_t gi = atomic_fetch_add(&c->next_graph, 1);
        if (gi >= c->G) break;
        int64_t lo = c->eoff[gi], cnt = c->eoff[gi + 1] - lo;
        int32_t* eu = malloc(sizeof(int32_t) * (size_t)(cnt + 1));
        int32_t* ev = malloc(sizeof(int32_t) * (size_t)(cnt + 1));
        if (!eu || !ev) { free(eu); free(ev); atomic_store(&c->err, -2); continue; }
        int64_t m = or_canonical(c->src + lo, c->dst + lo, cnt, c->nverts[gi], eu, ev);
        int rc = m < 0 ? (int)m : or_truss_wc(c->nverts[gi], m, eu, ev, c->tau + lo, NULL);
        if (rc) atomic_store(&c->err, rc);
        c->m_out[gi] = m;
        free(eu); free(ev);
    }
    return NULL;
}

/* Graph gi has nverts[gi] vertices and raw edges [eoff[gi], eoff[gi+1]) of
 * src/dst.  Its trussness (canonical order, m_out[gi] entries) is written at
 * tau + eoff[gi].  Independent graphs run on up to nthreads host threads. */
int or_truss_batch(int64_t G, const int32_t* nverts, const int64_t* eoff, const int32_t* src,
                   const int32_t* dst, int64_t* m_out, int32_t* tau, int nthreads) {
    if (G < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    batch_ctx c;
    c.G = G; c.nverts = nverts; c.eoff = eoff; c.src = src; c.dst = dst; c.m_out = m_out; c.tau = tau;
    atomic_init(&c.next_graph, 0);
    atomic_init(&c.err, 0);
    pthread_t th[256];
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, batch_worker, &c);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    return atomic_load(&c.err);
}

/* ------------------------------------------------------ result certificate */

typedef struct {
    const graph_t* g;
    const int32_t *eu, *ev, *tau, *step;
    int64_t m;
    atomic_llong next_chunk;
    atomic_llong violations;
    int64_t first_bad;  /* smallest violating edge id found (or -1) */
    pthread_mutex_t lock;
} cert_ctx;

/* key order (step, id) */
static inline int later(const cert_ctx* c, int32_t f, int32_t e) {
    return c->step[f] > c->step[e] || (c->step[f] == c->step[e] && f > e);
}

static void* cert_worker(void* p) {
    cert_ctx* c = (cert_ctx*)p;
    const graph_t* g = c->g;
    const int64_t CH = 4096;
    for (;;) {
        int64_t lo = atomic_fetch_add(&c->next_chunk, CH);
        if (lo >= c->m) break;
        int64_t hi = lo + CH < c->m ? lo + CH : c->m;
        for (int64_t e = lo; e < hi; e++) {
            int32_t u = c->eu[e], v = c->ev[e];
            int32_t a = deg(g, u) <= deg(g, v) ? u : v, b = a == u ? v : u;
            int32_t k = c->tau[e];
            int64_t ge = 0, lat = 0;
            for (int64_t j = g->off[a]; j < g->off[a + 1]; j++) {
                int32_t w = g->adj[j].w;
                if (w == b) continue;
                int32_t f = g->adj[j].e, h = find_edge(g, b, w);
                if (h < 0) continue;
                if (c->tau[f] >= k && c->tau[h] >= k) ge++;
                if (later(c, f, (int32_t)e) && later(c, h, (int32_t)e)) lat++;
            }
            if (k < 2 || ge < k - 2 || lat > k - 2) {
                atomic_fetch_add(&c->violations, 1);
                pthread_mutex_lock(&c->lock);
                if (c->first_bad < 0 || e < c->first_bad) c->first_bad = e;
                pthread_mutex_unlock(&c->lock);
            }
        }
    }
    return NULL;
}

/* Returns the number of violating edges (0: the claim is exactly the
 * trussness), or -1 / -2 on bad arguments / allocation failure.  *first_bad
 * receives the smallest violating edge id, or -1. */
int64_t or_certify(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, const int32_t* tau,
                   const int32_t* step, int nthreads, int64_t* first_bad) {
    if (m < 0 || m > INT32_MAX - 1) return -1;
    *first_bad = -1;
    graph_t g;
    int rc = graph_build(&g, n, m, eu, ev);
    if (rc) return rc;
    int64_t bad = 0;
    /* the claim must not decrease along the (step, id) order: per step,
     * claims are compared across consecutive steps in step order */
    int32_t smax = -1;
    for (int64_t e = 0; e < m; e++) {
        if (step[e] < 0) { graph_free(&g); return -1; }
        if (step[e] > smax) smax = step[e];
    }
    int32_t* lo_t = malloc(sizeof(int32_t) * ((size_t)smax + 2));
    int32_t* hi_t = malloc(sizeof(int32_t) * ((size_t)smax + 2));
    if (!lo_t || !hi_t) { free(lo_t); free(hi_t); graph_free(&g); return -2; }
    for (int32_t s = 0; s <= smax; s++) { lo_t[s] = INT32_MAX; hi_t[s] = INT32_MIN; }
    for (int64_t e = 0; e < m; e++) {
        if (tau[e] < lo_t[step[e]]) lo_t[step[e]] = tau[e];
        if (tau[e] > hi_t[step[e]]) hi_t[step[e]] = tau[e];
    }
    int32_t run = INT32_MIN;
    for (int32_t s = 0; s <= smax; s++) {
        if (lo_t[s] == INT32_MAX) continue;
        if (lo_t[s] != hi_t[s] || lo_t[s] < run) bad++;
        run = hi_t[s];
    }
    free(lo_t);
    free(hi_t);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    cert_ctx c;
    c.g = &g; c.eu = eu; c.ev = ev; c.tau = tau; c.step = step; c.m = m; c.first_bad = -1;
    atomic_init(&c.next_chunk, 0);
    atomic_init(&c.violations, 0);
    pthread_mutex_init(&c.lock, NULL);
    pthread_t th[256];
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, cert_worker, &c);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&c.lock);
    graph_free(&g);
    *first_bad = c.first_bad;
    return bad + (int64_t)atomic_load(&c.violations);
}

/* ------------------------------------------- sampled result certificate */

/* The per-edge conditions of or_certify for the edges listed in `sample`
 * only, plus the whole-order monotonicity check and trussness <= support+2
 * for the sampled edges.  Only the adjacency rows of the sampled edges'
 * endpoints are built (one pass over all edges), so the cost is O(m) plus
 * the sampled rows.  Returns the number of violations (0 for an exact
 * answer; a wrong answer is caught when a sampled edge is wrong or the
 * order is not monotone), -1 / -2 on bad arguments / allocation failure. */
int64_t or_certify_sample(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, const int32_t* tau,
                          const int32_t* step, const int64_t* sample, int64_t ns, int64_t* first_bad) {
    if (m < 0 || n < 0 || ns < 0 || m > INT32_MAX - 1) return -1;
    *first_bad = -1;
    int64_t bad = 0;
    /* monotone claims along the step order, over all edges */
    int32_t smax = -1;
    for (int64_t e = 0; e < m; e++) {
        if (step[e] < 0 || tau[e] < 2) return -1;
        if (step[e] > smax) smax = step[e];
    }
    int32_t* lo_t = malloc(sizeof(int32_t) * ((size_t)smax + 2));
    int32_t* hi_t = malloc(sizeof(int32_t) * ((size_t)smax + 2));
    uint8_t* mark = calloc((size_t)n + 1, 1);
    int64_t* off = calloc((size_t)n + 2, sizeof(int64_t));
    if (!lo_t || !hi_t || !mark || !off) { free(lo_t); free(hi_t); free(mark); free(off); return -2; }
    for (int32_t s = 0; s <= smax; s++) { lo_t[s] = INT32_MAX; hi_t[s] = INT32_MIN; }
    for (int64_t e = 0; e < m; e++) {
        if (tau[e] < lo_t[step[e]]) lo_t[step[e]] = tau[e];
        if (tau[e] > hi_t[step[e]]) hi_t[step[e]] = tau[e];
    }
    int32_t run = INT32_MIN;
    for (int32_t s = 0; s <= smax; s++) {
        if (lo_t[s] == INT32_MAX) continue;
        if (lo_t[s] != hi_t[s] || lo_t[s] < run) bad++;
        run = hi_t[s];
    }
    free(lo_t);
    free(hi_t);
    /* rows of the sampled endpoints */
    for (int64_t i = 0; i < ns; i++) {
        if (sample[i] < 0 || sample[i] >= m) { free(mark); free(off); return -1; }
        mark[eu[sample[i]]] = 1;
        mark[ev[sample[i]]] = 1;
    }
    for (int64_t e = 0; e < m; e++) {
        if (mark[eu[e]]) off[eu[e] + 1]++;
        if (mark[ev[e]]) off[ev[e] + 1]++;
    }
    for (int32_t v = 0; v < n; v++) off[v + 1] += off[v];
    slot_t* adj = malloc(sizeof(slot_t) * (size_t)(off[n] + 1));
    int64_t* cur = malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!adj || !cur) { free(adj); free(cur); free(mark); free(off); return -2; }
    memcpy(cur, off, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; e++) {
        if (mark[eu[e]]) { adj[cur[eu[e]]].w = ev[e]; adj[cur[eu[e]]].e = (int32_t)e; cur[eu[e]]++; }
        if (mark[ev[e]]) { adj[cur[ev[e]]].w = eu[e]; adj[cur[ev[e]]].e = (int32_t)e; cur[ev[e]]++; }
    }
    for (int32_t v = 0; v < n; v++)
        if (mark[v]) qsort(adj + off[v], (size_t)(off[v + 1] - off[v]), sizeof(slot_t), cmp_slot);
    /* per sampled edge: merge the two rows */
    for (int64_t i = 0; i < ns; i++) {
        const int32_t e = (int32_t)sample[i], u = eu[e], v = ev[e], k = tau[e];
        int64_t p = off[u], q = off[v], ge = 0, lat = 0, sup = 0;
        while (p < off[u + 1] && q < off[v + 1]) {
            if (adj[p].w < adj[q].w) { p++; continue; }
            if (adj[p].w > adj[q].w) { q++; continue; }
            const int32_t f = adj[p].e, h = adj[q].e;
            sup++;
            if (tau[f] >= k && tau[h] >= k) ge++;
            if ((step[f] > step[e] || (step[f] == step[e] && f > e)) &&
                (step[h] > step[e] || (step[h] == step[e] && h > e)))
                lat++;
            p++;
            q++;
        }
        if (ge < k - 2 || lat > k - 2 || k > sup + 2) {
            bad++;
            if (*first_bad < 0 || e < *first_bad) *first_bad = e;
        }
    }
    free(adj); free(cur); free(mark); free(off);
    return bad;
}

/* ---- k-trusses as subgraphs (§II: a k-truss is a maximal connected
 * subgraph whose every edge lies in >= k-2 of its triangles).  The k-trusses
 * of a graph are the connected components of the edges of trussness >= k;
 * comp[e] = the smallest vertex label of e's component, -1 when tau[e] < k.
 * Plain union-find over those edges (union by smaller label, path halving).
 * Returns the number of components. */
static int32_t uf_root(int32_t* p, int32_t x) {
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

int64_t or_ktruss_components(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, const int32_t* tau,
                             int32_t k, int32_t* comp) {
    if (n < 0 || m < 0) return -1;
    int32_t* p = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!p) return -2;
    for (int32_t v = 0; v < n; v++) p[v] = v;
    for (int64_t e = 0; e < m; e++) {
        if (tau[e] < k) continue;
        const int32_t a = uf_root(p, eu[e]), b = uf_root(p, ev[e]);
        if (a < b) p[b] = a;
        else if (b < a) p[a] = b;
    }
    /* the root of a tree is its smallest label: a root is only ever hooked
     * under a smaller one */
    int64_t ncomp = 0;
    for (int64_t e = 0; e < m; e++) {
        if (tau[e] < k) {
            comp[e] = -1;
            continue;
        }
        comp[e] = uf_root(p, eu[e]);
    }
    for (int32_t v = 0; v < n; v++) p[v] = (p[v] == v) ? -1 : 0; /* reuse: mark roots */
    for (int64_t e = 0; e < m; e++)
        if (comp[e] >= 0 && p[comp[e]] == -1) {
            p[comp[e]] = 1;
            ncomp++;
        }
    free(p);
    return ncomp;
}
