/*
 * Seeded synthetic graph generators (R-MAT, Chung-Lu, 2-D random geometric).
 *
 * These produce raw undirected edge lists (int32 pairs) that may contain
 * self-loops and duplicate pairs; both the device graph build and the CPU
 * oracle canonicalise them on their own.  Nothing in this file computes any
 * part of the truss decomposition: it only draws inputs.
 *
 * Randomness is counter based, so a sample's value depends only on
 * (seed, stream, index) and never on the thread count: every draw is the
 * SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) applied to a key built from
 * those three numbers.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Counter-based 64-bit draw number `i` of stream `stream` under `seed`. */
uint64_t gg_rand64(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t k = mix64(seed ^ mix64(stream + 0x632BE59BD9B4E019ULL));
    return mix64(k + i * 0xD1B54A32D192ED03ULL);
}

static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

static int num_threads(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)c;
}

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } range_job;
static void* range_thunk(void* p) { range_job* j = (range_job*)p; j->fn(j->ctx, j->lo, j->hi); return NULL; }

/* Runs fn over [0, n) split into contiguous chunks, one per thread. */
static void parallel_for(int64_t n, range_fn fn, void* ctx) {
    int t = num_threads();
    if (n < 65536 || t == 1) { fn(ctx, 0, n); return; }
    pthread_t th[64];
    range_job jobs[64];
    for (int i = 0; i < t; i++) {
        jobs[i].fn = fn; jobs[i].ctx = ctx;
        jobs[i].lo = n * i / t; jobs[i].hi = n * (i + 1) / t;
        pthread_create(&th[i], NULL, range_thunk, &jobs[i]);
    }
    for (int i = 0; i < t; i++) pthread_join(th[i], NULL);
}

/* ---------------------------------------------------------------- R-MAT */
typedef struct { int scale; double a, ab, abc; uint64_t seed; int32_t *src, *dst; } rmat_ctx;

static void rmat_range(void* p, int64_t lo, int64_t hi) {
    rmat_ctx* c = (rmat_ctx*)p;
    for (int64_t i = lo; i < hi; i++) {
        uint32_t s = 0, d = 0;
        uint64_t r = 0;
        for (int k = 0; k < c->scale; k++) {
            if ((k & 1) == 0) r = gg_rand64(c->seed, 1, (uint64_t)i * 32 + (uint64_t)(k >> 1));
            double u = (double)((k & 1) ? (uint32_t)(r >> 32) : (uint32_t)r) * (1.0 / 4294967296.0);
            uint32_t sb, db;
            if (u < c->a) { sb = 0; db = 0; }
            else if (u < c->ab) { sb = 0; db = 1; }
            else if (u < c->abc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        c->src[i] = (int32_t)s;
        c->dst[i] = (int32_t)d;
    }
}

/* n_samples quadrant-recursive samples on 2^scale vertices; no noise, no
 * vertex permutation. */
int gg_rmat(int scale, int64_t n_samples, double a, double b, double c, uint64_t seed,
            int32_t* src, int32_t* dst) {
    if (scale < 1 || scale > 30 || n_samples < 0) return -1;
    rmat_ctx ctx = {scale, a, a + b, a + b + c, seed, src, dst};
    parallel_for(n_samples, rmat_range, &ctx);
    return 0;
}

/* ------------------------------------------------------------- Chung-Lu */
/* Expected-degree weights w_i = (i+1)^(-1/(gamma-1)), rescaled to mean
 * `mean_deg` and clipped at `max_deg`; the rescale-and-clip step is repeated
 * 64 times so the clipped sequence ends close to the requested mean. */
int gg_chung_lu_weights(int32_t n, double gamma, double mean_deg, double max_deg, double* w) {
    if (n < 1 || gamma <= 1.0) return -1;
    double e = -1.0 / (gamma - 1.0);
    for (int32_t i = 0; i < n; i++) w[i] = pow((double)i + 1.0, e);
    for (int it = 0; it < 64; it++) {
        double s = 0.0;
        for (int32_t i = 0; i < n; i++) s += w[i];
        double f = mean_deg * (double)n / s;
        for (int32_t i = 0; i < n; i++) {
            double x = w[i] * f;
            w[i] = x > max_deg ? max_deg : x;
        }
    }
    return 0;
}

typedef struct { int32_t n; const double* cum; double total; uint64_t seed; int32_t *src, *dst; } cl_ctx;

static inline int32_t cl_pick(const double* cum, int32_t n, double x) {
    /* first i with cum[i] > x, cum[i] = w_0 + ... + w_i */
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (cum[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static void cl_range(void* p, int64_t lo, int64_t hi) {
    cl_ctx* c = (cl_ctx*)p;
    for (int64_t i = lo; i < hi; i++) {
        double x = u01(gg_rand64(c->seed, 2, (uint64_t)i * 2)) * c->total;
        double y = u01(gg_rand64(c->seed, 2, (uint64_t)i * 2 + 1)) * c->total;
        c->src[i] = cl_pick(c->cum, c->n, x);
        c->dst[i] = cl_pick(c->cum, c->n, y);
    }
}

/* n_samples endpoint pairs, each endpoint drawn independently with
 * probability proportional to its weight. */
int gg_chung_lu(int32_t n, double gamma, double mean_deg, double max_deg, uint64_t seed,
                int64_t n_samples, int32_t* src, int32_t* dst) {
    if (n < 1 || n_samples < 0) return -1;
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    if (!w) return -2;
    gg_chung_lu_weights(n, gamma, mean_deg, max_deg, w);
    for (int32_t i = 1; i < n; i++) w[i] += w[i - 1];
    cl_ctx ctx = {n, w, w[n - 1], seed, src, dst};
    parallel_for(n_samples, cl_range, &ctx);
    free(w);
    return 0;
}

/* Per-graph parameters of the ragged batch: graph `seed` draws its vertex
 * count log-uniformly in [n_lo, n_hi] and its mean degree log-uniformly in
 * [d_lo, d_hi], clamped to n-1. */
void gg_batch_params(uint64_t seed, int32_t n_lo, int32_t n_hi, double d_lo, double d_hi,
                     int32_t* n_out, double* d_out) {
    double u = u01(gg_rand64(seed, 5, 0));
    double v = u01(gg_rand64(seed, 5, 1));
    int32_t n = (int32_t)floor(exp(log((double)n_lo) + u * (log((double)n_hi) - log((double)n_lo))));
    if (n < n_lo) n = n_lo;
    if (n > n_hi) n = n_hi;
    double d = exp(log(d_lo) + v * (log(d_hi) - log(d_lo)));
    if (d > (double)(n - 1)) d = (double)(n - 1);
    *n_out = n;
    *d_out = d;
}

/* ------------------------------------------------- 2-D random geometric */
typedef struct {
    int32_t n, C;
    double r2;
    const double *x, *y;
    const int32_t* cell_start; /* [C*C+1] */
    const int32_t* cell_pts;   /* point ids sorted by cell, ascending id within a cell */
    int64_t* row_count;        /* per cell row */
    const int64_t* row_off;
    int32_t *src, *dst;
    int fill;
} rgg_ctx;

static void rgg_rows(void* p, int64_t lo, int64_t hi) {
    rgg_ctx* c = (rgg_ctx*)p;
    const int C = c->C;
    static const int nbx[4] = {1, -1, 0, 1};
    static const int nby[4] = {0, 1, 1, 1};
    for (int64_t cy = lo; cy < hi; cy++) {
        int64_t cnt = 0;
        int64_t out = c->fill ? c->row_off[cy] : 0;
        for (int cx = 0; cx < C; cx++) {
            int cid = (int)cy * C + cx;
            for (int32_t a = c->cell_start[cid]; a < c->cell_start[cid + 1]; a++) {
                int32_t i = c->cell_pts[a];
                double xi = c->x[i], yi = c->y[i];
                for (int32_t b = a + 1; b < c->cell_start[cid + 1]; b++) {
                    int32_t j = c->cell_pts[b];
                    double dx = xi - c->x[j], dy = yi - c->y[j];
                    if (dx * dx + dy * dy <= c->r2) {
                        if (c->fill) { c->src[out] = i; c->dst[out] = j; out++; }
                        cnt++;
                    }
                }
                for (int q = 0; q < 4; q++) {
                    int nx = cx + nbx[q], ny = (int)cy + nby[q];
                    if (nx < 0 || nx >= C || ny >= C) continue;
                    int nid = ny * C + nx;
                    for (int32_t b = c->cell_start[nid]; b < c->cell_start[nid + 1]; b++) {
                        int32_t j = c->cell_pts[b];
                        double dx = xi - c->x[j], dy = yi - c->y[j];
                        if (dx * dx + dy * dy <= c->r2) {
                            if (c->fill) { c->src[out] = i; c->dst[out] = j; out++; }
                            cnt++;
                        }
                    }
                }
            }
        }
        if (!c->fill) c->row_count[cy] = cnt;
    }
}

typedef struct { uint64_t seed; double *x, *y; } pts_ctx;
static void rgg_points(void* p, int64_t lo, int64_t hi) {
    pts_ctx* c = (pts_ctx*)p;
    for (int64_t i = lo; i < hi; i++) {
        c->x[i] = u01(gg_rand64(c->seed, 3, (uint64_t)i * 2));
        c->y[i] = u01(gg_rand64(c->seed, 3, (uint64_t)i * 2 + 1));
    }
}

/* Random geometric graph: n uniform points in the unit square (no wrap),
 * an edge for every pair at distance <= r, r chosen so that the expected
 * degree of an interior point is mean_deg.  Two-call protocol: with src ==
 * NULL it returns the edge count; then call again with buffers of that size.
 * Returns -1 on bad arguments, -2 on allocation failure. */
int64_t gg_rgg2d(int32_t n, double mean_deg, uint64_t seed, int32_t* src, int32_t* dst) {
    if (n < 2 || mean_deg <= 0) return -1;
    double r = sqrt(mean_deg / (M_PI * (double)(n - 1)));
    int C = (int)floor(1.0 / r);
    if (C < 1) C = 1;
    if (C > 46000) C = 46000;
    double *x = malloc(sizeof(double) * (size_t)n), *y = malloc(sizeof(double) * (size_t)n);
    int32_t* cell_start = calloc((size_t)C * C + 1, sizeof(int32_t));
    int32_t* cell_pts = malloc(sizeof(int32_t) * (size_t)n);
    int32_t* cell_of = malloc(sizeof(int32_t) * (size_t)n);
    int64_t* row_count = calloc((size_t)C, sizeof(int64_t));
    int64_t* row_off = calloc((size_t)C + 1, sizeof(int64_t));
    int64_t ret = -2;
    if (!x || !y || !cell_start || !cell_pts || !cell_of || !row_count || !row_off) goto done;
    pts_ctx pc = {seed, x, y};
    parallel_for(n, rgg_points, &pc);
    for (int32_t i = 0; i < n; i++) {
        int cx = (int)(x[i] * C), cy = (int)(y[i] * C);
        if (cx >= C) cx = C - 1;
        if (cy >= C) cy = C - 1;
        cell_of[i] = cy * C + cx;
        cell_start[cell_of[i] + 1]++;
    }
    for (int64_t k = 0; k < (int64_t)C * C; k++) cell_start[k + 1] += cell_start[k];
    {
        int32_t* cur = malloc(sizeof(int32_t) * (size_t)C * C);
        if (!cur) goto done;
        memcpy(cur, cell_start, sizeof(int32_t) * (size_t)C * C);
        for (int32_t i = 0; i < n; i++) cell_pts[cur[cell_of[i]]++] = i;
        free(cur);
    }
    rgg_ctx ctx = {n, C, r * r, x, y, cell_start, cell_pts, row_count, row_off, src, dst, 0};
    int t = num_threads();
    if (C < 64) t = 1;
    /* count pass then fill pass; chunks are whole cell rows so the output
     * order is fixed by the cell layout, not by thread timing */
    {
        pthread_t th[64];
        range_job jobs[64];
        for (int pass = 0; pass < (src ? 2 : 1); pass++) {
            ctx.fill = pass;
            if (pass == 1) {
                for (int k = 0; k < C; k++) row_off[k + 1] = row_off[k] + row_count[k];
            }
            for (int i = 0; i < t; i++) {
                jobs[i].fn = rgg_rows; jobs[i].ctx = &ctx;
                jobs[i].lo = (int64_t)C * i / t; jobs[i].hi = (int64_t)C * (i + 1) / t;
                pthread_create(&th[i], NULL, range_thunk, &jobs[i]);
            }
            for (int i = 0; i < t; i++) pthread_join(th[i], NULL);
        }
    }
    ret = 0;
    for (int k = 0; k < C; k++) ret += row_count[k];
done:
    free(x); free(y); free(cell_start); free(cell_pts); free(cell_of); free(row_count); free(row_off);
    return ret;
}
