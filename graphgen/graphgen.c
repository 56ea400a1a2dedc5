/*
 * graphgen.c -- seeded synthetic edge-list generators.
 *
 * This module produces the INPUTS that both the CUDA path and the CPU oracle
 * consume: plain int32 (src, dst) edge lists and seeded source vertices.  It
 * holds none of the BFS arithmetic (no symmetrising, deduplication, CSR
 * construction or traversal); those are done independently by each side.
 *
 * Every random draw comes from Philox-4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11), a counter-based
 * generator, so each edge is a pure function of (seed, stream, edge index)
 * and the output does not depend on the number of threads.
 *
 * Generators (parameters follow the synthetic stand-ins for the paper's
 * dataset groups, Section 7.1: Kronecker/RMAT = high degree variance,
 * Barabasi-Albert = mid, Erdos-Renyi and grids = low / road-like):
 *   - RMAT (Chakrabarti, Zhan, Faloutsos 2004): `scale` independent quadrant
 *     draws per edge with probabilities a, b, c, d = 1-a-b-c, no noise and no
 *     vertex permutation.
 *   - Erdos-Renyi G(n, M): M ordered pairs, endpoints uniform in [0, n).
 *   - W x H 4-neighbour grid, each undirected edge deleted independently with
 *     probability p, then a seeded Fisher-Yates relabelling of the vertices.
 *   - Barabasi-Albert via the linear-time method of Batagelj and Brandes
 *     (Phys. Rev. E 71, 2005), started from an (m+1)-clique.
 *   - Source sampling: distinct vertices that have at least one non-self-loop
 *     edge, drawn uniformly by rejection.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GG_STREAM_RMAT 0x524d4154u
#define GG_STREAM_ER 0x45520000u
#define GG_STREAM_GRID 0x47524944u
#define GG_STREAM_PERM 0x5045524du
#define GG_STREAM_BA 0x42410000u
#define GG_STREAM_SRC 0x53524300u

/* Philox-4x32 round constants and key schedule (Salmon et al. 2011, Sec. 5). */
static inline void philox4x32_10(const uint32_t ctr_in[4], uint64_t seed, uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static inline void draw4(uint64_t seed, uint64_t index, uint32_t stream, uint32_t sub, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), stream, sub};
    philox4x32_10(ctr, seed, out);
}

/* Uniform integer in [0, bound) by the multiply-shift map of a 32-bit draw
 * (Lemire 2019); bound <= 2^32. */
static inline uint64_t scale32(uint32_t r, uint64_t bound) { return ((uint64_t)r * bound) >> 32; }

uint32_t gg_philox_word(uint64_t seed, uint64_t index, uint32_t stream, uint32_t sub, int which) {
    uint32_t o[4];
    draw4(seed, index, stream, sub, o);
    return o[which & 3];
}

/* ---------------------------------------------------------------- threads */
typedef struct {
    void (*fn)(void*, int64_t, int64_t);
    void* arg;
    int64_t lo, hi;
} gg_job;

static void* gg_thread_main(void* p) {
    gg_job* j = (gg_job*)p;
    j->fn(j->arg, j->lo, j->hi);
    return NULL;
}

static void gg_parallel_for(int64_t n, int nthreads, void (*fn)(void*, int64_t, int64_t), void* arg) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 65536 || nthreads == 1) {
        fn(arg, 0, n);
        return;
    }
    pthread_t th[256];
    gg_job jobs[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn;
        jobs[t].arg = arg;
        jobs[t].lo = n * t / nthreads;
        jobs[t].hi = n * (t + 1) / nthreads;
        if (pthread_create(&th[t], NULL, gg_thread_main, &jobs[t]) == 0) {
            started = t + 1;
        } else {
            /* could not spawn: run the rest on this thread */
            for (int u = t; u < nthreads; ++u) fn(arg, n * u / nthreads, n * (u + 1) / nthreads);
            break;
        }
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------ RMAT */
typedef struct {
    int scale;
    uint32_t tA, tAB, tABC;
    uint64_t seed;
    int32_t *src, *dst;
} rmat_arg;

static void rmat_range(void* p, int64_t lo, int64_t hi) {
    rmat_arg* a = (rmat_arg*)p;
    for (int64_t e = lo; e < hi; ++e) {
        uint32_t u = 0, v = 0, w[4] = {0, 0, 0, 0};
        for (int l = 0; l < a->scale; ++l) {
            if ((l & 3) == 0) draw4(a->seed, (uint64_t)e, GG_STREAM_RMAT, (uint32_t)(l >> 2), w);
            uint32_t r = w[l & 3];
            uint32_t bu, bv;
            if (r < a->tA) { bu = 0; bv = 0; }
            else if (r < a->tAB) { bu = 0; bv = 1; }
            else if (r < a->tABC) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        a->src[e] = (int32_t)u;
        a->dst[e] = (int32_t)v;
    }
}

static uint32_t prob_to_u32(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return 0xFFFFFFFFu;
    return (uint32_t)(p * 4294967296.0);
}

int gg_rmat(int scale, int64_t n_edges, double a, double b, double c, uint64_t seed,
            int32_t* src, int32_t* dst, int nthreads) {
    if (scale < 1 || scale > 30 || n_edges < 0 || !src || !dst) return 1;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0 + 1e-12) return 1;
    rmat_arg arg;
    arg.scale = scale;
    arg.tA = prob_to_u32(a);
    arg.tAB = prob_to_u32(a + b);
    arg.tABC = prob_to_u32(a + b + c);
    arg.seed = seed;
    arg.src = src;
    arg.dst = dst;
    gg_parallel_for(n_edges, nthreads, rmat_range, &arg);
    return 0;
}

/* ----------------------------------------------------------- Erdos-Renyi */
typedef struct {
    uint64_t n, seed;
    int32_t *src, *dst;
} er_arg;

static void er_range(void* p, int64_t lo, int64_t hi) {
    er_arg* a = (er_arg*)p;
    for (int64_t e = lo; e < hi; ++e) {
        uint32_t w[4];
        draw4(a->seed, (uint64_t)e, GG_STREAM_ER, 0, w);
        a->src[e] = (int32_t)scale32(w[0], a->n);
        a->dst[e] = (int32_t)scale32(w[1], a->n);
    }
}

int gg_erdos_renyi(int64_t n, int64_t m_pairs, uint64_t seed, int32_t* src, int32_t* dst, int nthreads) {
    if (n < 1 || n > 0x7FFFFFFF || m_pairs < 0 || !src || !dst) return 1;
    er_arg arg = {(uint64_t)n, seed, src, dst};
    gg_parallel_for(m_pairs, nthreads, er_range, &arg);
    return 0;
}

/* ------------------------------------------------------------------ grid */
/* Undirected grid edges are numbered: horizontal (r,c)-(r,c+1) as
 * r*(W-1)+c, then vertical (r,c)-(r+1,c) as H*(W-1) + r*W + c. */
static inline void grid_edge(int64_t id, int64_t W, int64_t H, int64_t* a, int64_t* b) {
    int64_t nh = H * (W - 1);
    if (id < nh) {
        int64_t r = id / (W - 1), c = id % (W - 1);
        *a = r * W + c;
        *b = r * W + c + 1;
    } else {
        int64_t k = id - nh;
        int64_t r = k / W, c = k % W;
        *a = r * W + c;
        *b = (r + 1) * W + c;
    }
}

int64_t gg_grid_num_edges(int64_t W, int64_t H) { return H * (W - 1) + (H - 1) * W; }

typedef struct {
    int64_t W, H;
    uint32_t keep_thr; /* keep an edge if its draw >= keep_thr */
    uint64_t seed;
    int64_t* counts; /* per chunk */
    int64_t chunk;
    int32_t *src, *dst;
    const int32_t* label;
    int pass;
} grid_arg;

static void grid_range(void* p, int64_t clo, int64_t chi) {
    grid_arg* a = (grid_arg*)p;
    int64_t total = gg_grid_num_edges(a->W, a->H);
    for (int64_t ch = clo; ch < chi; ++ch) {
        int64_t lo = ch * a->chunk, hi = lo + a->chunk;
        if (hi > total) hi = total;
        int64_t out = (a->pass == 0) ? 0 : a->counts[ch];
        int64_t cnt = 0;
        for (int64_t id = lo; id < hi; ++id) {
            uint32_t w[4];
            draw4(a->seed, (uint64_t)id, GG_STREAM_GRID, 0, w);
            if (w[0] < a->keep_thr) continue;
            if (a->pass == 1) {
                int64_t x, y;
                grid_edge(id, a->W, a->H, &x, &y);
                a->src[out + cnt] = a->label ? a->label[x] : (int32_t)x;
                a->dst[out + cnt] = a->label ? a->label[y] : (int32_t)y;
            }
            ++cnt;
        }
        if (a->pass == 0) a->counts[ch] = cnt;
    }
}

/* Fisher-Yates shuffle of the identity, position i swapped with a uniform
 * j in [0, i], the draw for i taken from counter i. */
int gg_permutation(int64_t n, uint64_t seed, int32_t* perm) {
    if (n < 1 || n > 0x7FFFFFFF || !perm) return 1;
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i >= 1; --i) {
        uint32_t w[4];
        draw4(seed, (uint64_t)i, GG_STREAM_PERM, 0, w);
        int64_t j = (int64_t)scale32(w[0], (uint64_t)(i + 1));
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    return 0;
}

/* Returns the number of kept edges written to src/dst (capacity must be at
 * least gg_grid_num_edges(W, H)), or -1 on bad arguments. */
int64_t gg_grid(int64_t W, int64_t H, double p_del, uint64_t seed, int relabel,
                int32_t* src, int32_t* dst, int nthreads) {
    if (W < 1 || H < 1 || W * H > 0x7FFFFFFF || !src || !dst || p_del < 0 || p_del > 1) return -1;
    int64_t total = gg_grid_num_edges(W, H);
    int32_t* label = NULL;
    if (relabel) {
        label = (int32_t*)malloc(sizeof(int32_t) * (size_t)(W * H));
        if (!label) return -1;
        gg_permutation(W * H, seed, label);
    }
    grid_arg arg;
    arg.W = W;
    arg.H = H;
    arg.keep_thr = prob_to_u32(p_del);
    arg.seed = seed;
    arg.chunk = 1 << 16;
    int64_t nch = (total + arg.chunk - 1) / arg.chunk;
    arg.counts = (int64_t*)calloc((size_t)(nch + 1), sizeof(int64_t));
    arg.src = src;
    arg.dst = dst;
    arg.label = label;
    if (!arg.counts) {
        free(label);
        return -1;
    }
    arg.pass = 0;
    gg_parallel_for(nch, nthreads, grid_range, &arg);
    int64_t run = 0;
    for (int64_t ch = 0; ch < nch; ++ch) {
        int64_t c = arg.counts[ch];
        arg.counts[ch] = run;
        run += c;
    }
    arg.pass = 1;
    gg_parallel_for(nch, nthreads, grid_range, &arg);
    free(arg.counts);
    free(label);
    return run;
}

/* ------------------------------------------------------- Barabasi-Albert */
/* Returns the number of edges written (capacity: m*(m+1)/2 + (n-m-1)*m). */
int64_t gg_barabasi_albert(int64_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst) {
    if (m < 1 || n < m + 2 || n > 0x7FFFFFFF || !src || !dst) return -1;
    int64_t cap = m * (m + 1) / 2 + (n - m - 1) * m;
    int32_t* ends = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * cap));
    if (!ends) return -1;
    int64_t e = 0;
    for (int64_t i = 0; i <= m; ++i)
        for (int64_t j = i + 1; j <= m; ++j) {
            src[e] = (int32_t)i;
            dst[e] = (int32_t)j;
            ends[2 * e] = (int32_t)i;
            ends[2 * e + 1] = (int32_t)j;
            ++e;
        }
    for (int64_t v = m + 1; v < n; ++v) {
        for (int64_t t = 0; t < m; ++t) {
            uint32_t w[4];
            draw4(seed, (uint64_t)e, GG_STREAM_BA, 0, w);
            /* endpoint of a uniformly chosen earlier edge end: degree-proportional */
            int64_t r = (int64_t)scale32(w[0], (uint64_t)(2 * e));
            int32_t tgt = ends[r];
            src[e] = (int32_t)v;
            dst[e] = tgt;
            ends[2 * e] = (int32_t)v;
            ends[2 * e + 1] = tgt;
            ++e;
        }
    }
    free(ends);
    return e;
}

/* -------------------------------------------------------------- sources */
/* k distinct vertices, each an endpoint of at least one edge with src != dst.
 * Returns 0, or 2 when fewer than k such vertices exist, 1 on bad arguments. */
int gg_sample_sources(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t k,
                      uint64_t seed, int32_t* out) {
    if (n < 1 || m < 0 || k < 0 || (k > 0 && !out)) return 1;
    uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
    if (!mark) return 1;
    int64_t eligible = 0;
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        if (u == v || u < 0 || v < 0 || u >= n || v >= n) continue;
        if (!mark[u]) { mark[u] = 1; ++eligible; }
        if (!mark[v]) { mark[v] = 1; ++eligible; }
    }
    if (eligible < k) {
        free(mark);
        return 2;
    }
    int32_t got = 0;
    for (uint64_t t = 0; got < k; ++t) {
        uint32_t w[4];
        draw4(seed, t, GG_STREAM_SRC, 0, w);
        int64_t v = (int64_t)scale32(w[0], (uint64_t)n);
        if (mark[v] == 1) {
            mark[v] = 2; /* taken */
            out[got++] = (int32_t)v;
        }
    }
    free(mark);
    return 0;
}
