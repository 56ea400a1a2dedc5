/*
 * oracle.c -- plain, slow, obviously correct CPU reference for the BFS hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it follows (paper: "The Einsum-Enabled Design Space for Graph
 * Algorithms: A BFS Case Study"):
 *   - Section 3, Cascade 1: BFS as a cascade over the iteration rank i.  The
 *     graph tensor G (Eq. G) is a 0/1 S x D matrix; the frontier F_i holds the
 *     vertices of depth i (Eq. F, empty = infinity); P_i is the visited set
 *     (Eq. P).  Initialisation puts the source in F_0 with depth 0 and in P_0.
 *     The advance Einsum (Eq. advance) gathers the neighbours d of every s in
 *     F_i, selects ANY one source per d, and keeps only d not in P_i; the
 *     update Einsum (Eq. update) sets P_{i+1} = P_i OR F_{i+1}; the loop stops
 *     when ||F_{i+1}|| = 0.  Depth is therefore the minimum hop count
 *     (Section 3, definition of depth), which is what a FIFO queue BFS
 *     computes; ANY is read as "first discoverer in FIFO order" for the
 *     oracle's own parent array.
 *   - Section 5 (push-to-pull derivation): the pull form visits every
 *     unvisited d and scans its in-neighbours s until one lies in F_i; the
 *     per-level statistics below count those scanned entries.
 *   - Section 4.C: graph in CSR (s-major); an undirected edge is the two
 *     directed edges (s,d) and (d,s) (Section 3).
 *
 * The brute-force all-pairs distance routine uses Boolean matrix powers and
 * the component routine uses union-find: both are independent of the queue
 * BFS so that they can pin it.
 *
 * The RCM routine numbers vertices by the Cuthill-McKee rule with fixed tie
 * breaks (see or_rcm); the tests pin it with hand-derived orders and an
 * independent check of the rules a Cuthill-McKee sequence must satisfy.
 *
 * The MLP routines are the FP64 reference for the learned direction policy:
 * 10 -> 32 -> 32 -> 3 with ReLU, softmax cross-entropy averaged over rows, and
 * the Adam update of Kingma & Ba (ICLR 2015, Algorithm 1).  The paper has no
 * learned policy; these follow the stated architecture only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------ adjacency */

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Adjacency (CSR) from an edge list: the S x D tensor G of Cascade 1 (Eq. G)
 * stored s-major (Section 4.C).  With `symmetrize`, an edge (s,d) contributes
 * both (s,d) and (d,s) (Section 3).  With `drop_self`, s == d is dropped; with
 * `dedup`, repeated (s,d) are kept once (G is 0/1).  Rows are sorted ascending.
 * row_ptr has n+1 entries; col must hold 2*m entries.  Returns the number of
 * directed entries, or -1 on bad input.
 */
int64_t or_build_adjacency(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                           int symmetrize, int drop_self, int dedup, int64_t* row_ptr, int32_t* col) {
    if (n < 1 || m < 0) return -1;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t e = 0; e < m; ++e) {
        int32_t s = src[e], d = dst[e];
        if (s < 0 || d < 0 || s >= n || d >= n) { free(cnt); return -1; }
        if (drop_self && s == d) continue;
        cnt[s]++;
        if (symmetrize) cnt[d]++;
    }
    /* bucket by row */
    row_ptr[0] = 0;
    for (int64_t v = 0; v < n; ++v) row_ptr[v + 1] = row_ptr[v] + cnt[v];
    for (int64_t v = 0; v < n; ++v) cnt[v] = row_ptr[v];
    for (int64_t e = 0; e < m; ++e) {
        int32_t s = src[e], d = dst[e];
        if (drop_self && s == d) continue;
        col[cnt[s]++] = d;
        if (symmetrize) col[cnt[d]++] = s;
    }
    /* sort each row, then drop repeats, compacting in place */
    int64_t out = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t b = row_ptr[v], e = row_ptr[v + 1];
        qsort(col + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
        row_ptr[v] = out;
        for (int64_t j = b; j < e; ++j) {
            if (dedup && j > b && col[j] == col[j - 1]) continue;
            col[out++] = col[j];
        }
    }
    row_ptr[n] = out;
    free(cnt);
    return out;
}

/* ------------------------------------------------------------------ BFS */

/*
 * Cascade 1 evaluated with a FIFO queue: F_0 = {s} at depth 0 (initialisation),
 * each dequeued vertex advances over its row of G in ascending order, and a
 * neighbour not yet in P receives depth+1 and joins P (Eqs. advance, update).
 * The queue empties exactly when ||F_{i+1}|| = 0.
 * depth[v] = -1 and parent[v] = -1 for unreached v; parent[s] = s.
 * Returns the number of levels with a non-empty frontier (max depth + 1).
 */
int32_t or_bfs(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t s, int32_t* depth,
               int32_t* parent) {
    if (s < 0 || s >= n) return -1;
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!queue) return -1;
    for (int64_t v = 0; v < n; ++v) {
        depth[v] = -1;
        if (parent) parent[v] = -1;
    }
    int64_t head = 0, tail = 0;
    depth[s] = 0;
    if (parent) parent[s] = s;
    queue[tail++] = s;
    int32_t maxd = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            int32_t v = col[j];
            if (depth[v] == -1) {
                depth[v] = depth[u] + 1;
                if (parent) parent[v] = u;
                if (depth[v] > maxd) maxd = depth[v];
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return maxd + 1;
}

/* ------------------------------------------------- min-label components */

/*
 * Connected components with the min operator of the paper's operator table
 * in place of ANY: starting from L_0[v] = v, the cascade
 *   L_{i+1}[d] = min(L_i[d], min over s adjacent to d of L_i[s])
 * reaches a fixed point in which every vertex holds the smallest id of its
 * component.  That fixed point is written out directly here: vertices are
 * visited in ascending id order, and each one not yet labelled labels its
 * whole component, found by a FIFO search, with its own id.  This is the
 * smallest id there, because every smaller id was reached earlier from a
 * smaller start.
 * The adjacency must be symmetric.  Returns 0, or -1 on allocation failure.
 */
int or_min_label(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t* label) {
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!queue) return -1;
    for (int64_t v = 0; v < n; ++v) label[v] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (label[s] >= 0) continue;
        int64_t head = 0, tail = 0;
        label[s] = (int32_t)s;
        queue[tail++] = (int32_t)s;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
                int32_t v = col[j];
                if (label[v] < 0) {
                    label[v] = (int32_t)s;
                    queue[tail++] = v;
                }
            }
        }
    }
    free(queue);
    return 0;
}

/* ------------------------------------------------------------------ RCM */

static const int64_t* rank_deg;  /* degrees seen by cmp_rank (single-threaded use) */

/* rank order: degree ascending, then vertex id ascending */
static int cmp_rank(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    int64_t dx = rank_deg[x], dy = rank_deg[y];
    if (dx != dy) return (dx > dy) - (dx < dy);
    return (x > y) - (x < y);
}

/*
 * Reverse Cuthill-McKee ordering.  Section 7.1 reorders every input graph
 * with RCM (Cuthill & McKee 1969; George & Liu).  The choices the method
 * leaves open are fixed here so that the order is unique:
 *   - vertices are ranked by (degree, id) ascending, degree = row length;
 *   - each connected component starts at its lowest-ranked vertex, and the
 *     components follow each other in the rank order of those starts;
 *   - a vertex taken from the FIFO queue numbers its not-yet-numbered
 *     neighbours next, in rank order (the Cuthill-McKee step);
 *   - the whole sequence is reversed.
 * newid[v] = n - 1 - (position of v in the Cuthill-McKee sequence).
 * Returns 0, or -1 on allocation failure.
 */
int or_rcm(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t* newid) {
    int64_t* deg = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int32_t* byrank = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!deg || !byrank || !order || !pos) {
        free(deg); free(byrank); free(order); free(pos);
        return -1;
    }
    for (int64_t v = 0; v < n; ++v) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        byrank[v] = (int32_t)v;
        pos[v] = -1;
    }
    rank_deg = deg;
    qsort(byrank, (size_t)n, sizeof(int32_t), cmp_rank);
    int64_t next = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t s = byrank[i];
        if (pos[s] >= 0) continue;  /* already numbered in an earlier component */
        pos[s] = next;
        order[next++] = s;
        int64_t head = pos[s];
        while (head < next) {
            int32_t u = order[head++];
            int64_t first = next;
            for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
                int32_t v = col[j];
                if (pos[v] < 0) {
                    pos[v] = next;
                    order[next++] = v;
                }
            }
            qsort(order + first, (size_t)(next - first), sizeof(int32_t), cmp_rank);
            for (int64_t k = first; k < next; ++k) pos[order[k]] = k;
        }
    }
    for (int64_t v = 0; v < n; ++v) newid[v] = (int32_t)(n - 1 - pos[v]);
    free(deg); free(byrank); free(order); free(pos);
    return 0;
}

/*
 * Per-level work statistics of Cascade 1 for a given depth array, six int64
 * per level i = 0 .. levels-1:
 *   [0] f     = |F_i|                         (vertices of depth i)
 *   [1] e_f   = sum of out-degrees over F_i   (edges a push level reads)
 *   [2] u     = |{v : deg v > 0, v not in P_{i+1} before the level}|, i.e.
 *               non-isolated vertices with depth > i or unreached
 *   [3] s_u   = CSR entries a pull level reads: for each such v its row is
 *               scanned in ascending order up to and including the first
 *               neighbour of depth i, or completely (Section 5, pull form)
 *   [4] d_new = |F_{i+1}|
 *   [5] e_u   = sum of degrees over the u vertices of [2]
 * Returns the number of levels written (<= max_levels), or -1.
 */
int32_t or_level_stats(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* depth,
                       int32_t max_levels, int64_t* stats) {
    int32_t maxd = -1;
    for (int64_t v = 0; v < n; ++v)
        if (depth[v] > maxd) maxd = depth[v];
    int32_t levels = maxd + 1;
    if (levels > max_levels) return -1;
    memset(stats, 0, sizeof(int64_t) * 6 * (size_t)(levels > 0 ? levels : 0));
    for (int32_t i = 0; i < levels; ++i) {
        int64_t* st = stats + 6 * (int64_t)i;
        for (int64_t v = 0; v < n; ++v) {
            int64_t deg = row_ptr[v + 1] - row_ptr[v];
            if (depth[v] == i) {
                st[0] += 1;
                st[1] += deg;
            }
            if (depth[v] == i + 1) st[4] += 1;
            if (deg > 0 && (depth[v] == -1 || depth[v] > i)) {
                st[2] += 1;
                st[5] += deg;
                int64_t scanned = 0;
                for (int64_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
                    ++scanned;
                    if (depth[col[j]] == i) break;
                }
                st[3] += scanned;
            }
        }
    }
    return levels;
}

/* ------------------------------------------------------ independent pins */

/*
 * All-pairs hop distances for n <= 64 by Boolean matrix powers: R_0 = I and
 * R_k = R_{k-1} OR (R_{k-1} x A); dist(s,v) is the least k with R_k[s][v]
 * set, -1 if none.  adj[s] is the bit-row of s (bit v set iff (s,v) in E).
 * This shares nothing with the queue BFS.
 */
int or_apsp_boolean(int32_t n, const uint64_t* adj, int32_t* dist) {
    if (n < 1 || n > 64) return 1;
    uint64_t R[64], nxt[64];
    for (int s = 0; s < n; ++s) {
        R[s] = 1ull << s;
        for (int v = 0; v < n; ++v) dist[s * n + v] = (v == s) ? 0 : -1;
    }
    for (int k = 1; k < n; ++k) {
        int changed = 0;
        for (int s = 0; s < n; ++s) {
            uint64_t row = R[s];
            for (int w = 0; w < n; ++w)
                if (R[s] >> w & 1) row |= adj[w];
            nxt[s] = row;
        }
        for (int s = 0; s < n; ++s) {
            uint64_t fresh = nxt[s] & ~R[s];
            for (int v = 0; v < n; ++v)
                if (fresh >> v & 1) dist[s * n + v] = k;
            if (fresh) changed = 1;
            R[s] = nxt[s];
        }
        if (!changed) break;
    }
    return 0;
}

static int64_t uf_find(int64_t* p, int64_t x) {
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

/* Connected components of the undirected graph given by the raw edge list
 * (union-find with path halving); comp[v] = smallest vertex of v's component. */
int or_components(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t* comp) {
    int64_t* p = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!p) return 1;
    for (int64_t v = 0; v < n; ++v) p[v] = v;
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = uf_find(p, src[e]), b = uf_find(p, dst[e]);
        if (a == b) continue;
        if (a < b) p[b] = a; else p[a] = b;
    }
    for (int64_t v = 0; v < n; ++v) comp[v] = (int32_t)uf_find(p, v);
    free(p);
    return 0;
}

static int has_edge(const int64_t* row_ptr, const int32_t* col, int32_t a, int32_t b) {
    int64_t lo = row_ptr[a], hi = row_ptr[a + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < b) lo = mid + 1;
        else hi = mid;
    }
    return lo < row_ptr[a + 1] && col[lo] == b;
}

/*
 * Validation of a BFS result against the graph alone (Graph500-style checks):
 *   1 depth[s] != 0 or parent[s] != s
 *   2 depth and parent disagree on reachability (exactly one is -1)
 *   3 some edge (u,v) has both ends reached and |depth u - depth v| > 1
 *   4 some edge joins a reached and an unreached vertex
 *   5 a reached v != s whose parent is out of range or unreached
 *   6 (parent[v], v) is not an edge of G
 *   7 depth[parent[v]] != depth[v] - 1
 *   8 a vertex other than s has depth 0 or depth < -1
 * Pass parent = NULL to check only the depth conditions.  Returns 0 if valid.
 * Rows must be sorted (for the edge lookup).
 * With `directed`, conditions 3 and 4 follow the edge direction only (a
 * directed edge is the tuple (s,d) of Section 3): for an edge (u,v) with u
 * reached, v is reached (4) and depth v <= depth u + 1 (3).
 */
int or_validate(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t s, const int32_t* depth,
                const int32_t* parent, int directed) {
    if (depth[s] != 0) return 1;
    if (parent && parent[s] != s) return 1;
    for (int64_t v = 0; v < n; ++v) {
        if (depth[v] < -1 || (v != s && depth[v] == 0)) return 8;
        if (parent && ((depth[v] == -1) != (parent[v] == -1))) return 2;
    }
    for (int64_t u = 0; u < n; ++u)
        for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            int32_t v = col[j];
            int ru = depth[u] >= 0, rv = depth[v] >= 0;
            if (directed) {
                if (ru && !rv) return 4;
                if (ru && depth[v] > depth[u] + 1) return 3;
                continue;
            }
            if (ru != rv) return 4;
            if (ru && rv && abs(depth[u] - depth[v]) > 1) return 3;
        }
    if (!parent) return 0;
    for (int64_t v = 0; v < n; ++v) {
        if (v == s || depth[v] < 0) continue;
        int32_t p = parent[v];
        if (p < 0 || p >= n || depth[p] < 0) return 5;
        if (!has_edge(row_ptr, col, p, (int32_t)v)) return 6;
        if (depth[p] != depth[v] - 1) return 7;
    }
    return 0;
}

/* ------------------------------------------------------------- MLP (FP64) */
/*
 * Parameter vector layout (float64 here, float32 on the device), row-major:
 *   W1[32][10], b1[32], W2[32][32], b2[32], W3[3][32], b3[3]   (1507 values)
 * Forward: h1 = relu(W1 x + b1); h2 = relu(W2 h1 + b2); z = W3 h2 + b3.
 */
enum { OR_IN = 10, OR_H = 32, OR_OUT = 3 };
#define OR_NPARAM (OR_H * OR_IN + OR_H + OR_H * OR_H + OR_H + OR_OUT * OR_H + OR_OUT)

int32_t or_mlp_num_params(void) { return OR_NPARAM; }

static void mlp_forward_row(const double* P, const double* x, double* h1, double* h2, double* z) {
    const double *W1 = P, *b1 = W1 + OR_H * OR_IN, *W2 = b1 + OR_H, *b2 = W2 + OR_H * OR_H;
    const double *W3 = b2 + OR_H, *b3 = W3 + OR_OUT * OR_H;
    for (int j = 0; j < OR_H; ++j) {
        double a = b1[j];
        for (int k = 0; k < OR_IN; ++k) a += W1[j * OR_IN + k] * x[k];
        h1[j] = a > 0 ? a : 0;
    }
    for (int j = 0; j < OR_H; ++j) {
        double a = b2[j];
        for (int k = 0; k < OR_H; ++k) a += W2[j * OR_H + k] * h1[k];
        h2[j] = a > 0 ? a : 0;
    }
    for (int j = 0; j < OR_OUT; ++j) {
        double a = b3[j];
        for (int k = 0; k < OR_H; ++k) a += W3[j * OR_H + k] * h2[k];
        z[j] = a;
    }
}

/* logits[rows][3] for inputs X[rows][10]. */
int or_mlp_forward(const double* P, const double* X, int64_t rows, double* logits) {
    double h1[OR_H], h2[OR_H];
    for (int64_t r = 0; r < rows; ++r) mlp_forward_row(P, X + r * OR_IN, h1, h2, logits + r * OR_OUT);
    return 0;
}

/*
 * Add one row's contribution to dL/dP given dL/dz for that row: the chain rule
 * written out layer by layer (ReLU derivative taken as 0 at 0).
 */
static void mlp_backprop_row(const double* P, const double* x, const double* h1, const double* h2, const double* dz,
                             double* grad) {
    const double *W2 = P + OR_H * OR_IN + OR_H, *W3 = W2 + OR_H * OR_H + OR_H;
    double *gW1 = grad, *gb1 = gW1 + OR_H * OR_IN, *gW2 = gb1 + OR_H, *gb2 = gW2 + OR_H * OR_H;
    double *gW3 = gb2 + OR_H, *gb3 = gW3 + OR_OUT * OR_H;
    double dh2[OR_H];
    for (int k = 0; k < OR_H; ++k) dh2[k] = 0;
    for (int j = 0; j < OR_OUT; ++j) {
        gb3[j] += dz[j];
        for (int k = 0; k < OR_H; ++k) {
            gW3[j * OR_H + k] += dz[j] * h2[k];
            dh2[k] += W3[j * OR_H + k] * dz[j];
        }
    }
    double dh1[OR_H];
    for (int k = 0; k < OR_H; ++k) dh1[k] = 0;
    for (int j = 0; j < OR_H; ++j) {
        double da = h2[j] > 0 ? dh2[j] : 0;
        gb2[j] += da;
        for (int k = 0; k < OR_H; ++k) {
            gW2[j * OR_H + k] += da * h1[k];
            dh1[k] += W2[j * OR_H + k] * da;
        }
    }
    for (int j = 0; j < OR_H; ++j) {
        double da = h1[j] > 0 ? dh1[j] : 0;
        gb1[j] += da;
        for (int k = 0; k < OR_IN; ++k) gW1[j * OR_IN + k] += da * x[k];
    }
}

/* log(sum_j exp(z_j)) of one row of logits, shifted by the largest logit. */
static double logsumexp_row(const double* z) {
    double zmax = z[0];
    for (int j = 1; j < OR_OUT; ++j) zmax = z[j] > zmax ? z[j] : zmax;
    double se = 0;
    for (int j = 0; j < OR_OUT; ++j) se += exp(z[j] - zmax);
    return zmax + log(se);
}

/*
 * Mean softmax cross-entropy over rows, L = (1/R) sum_r [logsumexp(z_r) - z_r[y_r]],
 * and its gradient dL/dP.  grad has OR_NPARAM entries.
 */
int or_mlp_loss_grad(const double* P, const double* X, const int32_t* y, int64_t rows, double* loss,
                     double* grad) {
    memset(grad, 0, sizeof(double) * OR_NPARAM);
    double total = 0;
    for (int64_t r = 0; r < rows; ++r) {
        const double* x = X + r * OR_IN;
        double h1[OR_H], h2[OR_H], z[OR_OUT];
        mlp_forward_row(P, x, h1, h2, z);
        const double lse = logsumexp_row(z);
        total += lse - z[y[r]];
        double dz[OR_OUT];
        for (int j = 0; j < OR_OUT; ++j) dz[j] = (exp(z[j] - lse) - (j == y[r] ? 1.0 : 0.0)) / (double)rows;
        mlp_backprop_row(P, x, h1, h2, dz, grad);
    }
    *loss = total / (double)rows;
    return 0;
}

/*
 * Least-squares regression of the outputs on per-row targets,
 * L = (1/R) sum_r sum_j (z_rj - t_rj)^2 / 2, and dL/dP; dL/dz_rj = (z_rj - t_rj) / R.
 * grad has OR_NPARAM entries.
 */
int or_mlp_regress_loss_grad(const double* P, const double* X, const double* t, int64_t rows, double* loss,
                             double* grad) {
    memset(grad, 0, sizeof(double) * OR_NPARAM);
    double total = 0;
    for (int64_t r = 0; r < rows; ++r) {
        const double* x = X + r * OR_IN;
        const double* tr = t + r * OR_OUT;
        double h1[OR_H], h2[OR_H], z[OR_OUT], dz[OR_OUT];
        mlp_forward_row(P, x, h1, h2, z);
        for (int j = 0; j < OR_OUT; ++j) {
            total += 0.5 * (z[j] - tr[j]) * (z[j] - tr[j]);
            dz[j] = (z[j] - tr[j]) / (double)rows;
        }
        mlp_backprop_row(P, x, h1, h2, dz, grad);
    }
    *loss = total / (double)rows;
    return 0;
}

/* One Adam step (Kingma & Ba 2015, Algorithm 1) at step t >= 1, in place. */
int or_adam_step(double* P, double* m1, double* m2, const double* g, int64_t np, int64_t t, double lr,
                 double beta1, double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < np; ++i) {
        m1[i] = beta1 * m1[i] + (1 - beta1) * g[i];
        m2[i] = beta2 * m2[i] + (1 - beta2) * g[i] * g[i];
        double mh = m1[i] / c1, vh = m2[i] / c2;
        P[i] -= lr * mh / (sqrt(vh) + eps);
    }
    return 0;
}
