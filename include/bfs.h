/*
 * bfs.h -- C ABI of the GB300-native breadth-first-search library (libbfsgb).
 *
 * The operation is level-synchronous BFS as written in the paper's Cascade 1
 * ("The Einsum-Enabled Design Space for Graph Algorithms: A BFS Case Study",
 * Section 3): every level is a masked Boolean sparse-matrix sparse-vector
 * product F_{i+1} = (G x F_i) masked by NOT P_i (Eq. advance) followed by the
 * visited-set update P_{i+1} = P_i OR F_{i+1} (Eq. update), stopping when the
 * new frontier is empty.  A level runs either in push form (loop order s -> d,
 * CSR expand of the frontier) or in pull form (loop order d -> s, Section 5:
 * unvisited vertices scan their in-neighbours with early exit).
 *
 * Conventions for every call:
 *   - The caller owns all input and output buffers.  A pointer may be host or
 *     device memory; the library detects which (cudaPointerGetAttributes) and
 *     copies through device staging buffers when needed.
 *   - Work is ordered on `cuda_stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Calls whose outputs are device memory return after enqueueing;
 *     calls with host outputs synchronise the stream before returning.
 *   - No exception crosses the ABI.  Every call returns a bfs_status; the
 *     message of the last failure on the calling thread is bfs_last_error().
 *   - A bfs_graph owns device memory and a per-graph workspace.  Runs on the
 *     same graph must not overlap in time (use one stream per graph, or
 *     synchronise between streams).
 */
#ifndef BFSGB_BFS_H
#define BFSGB_BFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BFS_OK = 0,
    BFS_EINVAL = 1,    /* bad argument: null pointer, n <= 0, vertex id out of range, k <= 0 ... */
    BFS_ENOMEM = 2,    /* device or host allocation failed */
    BFS_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    BFS_ETIMEOUT = 4,  /* a device-side wait (grid barrier) exceeded its limit; outputs undefined */
    BFS_ERANGE = 5,    /* a limit was passed: more than 2^31-1 directed CSR entries, a search's
                          max_levels, or the rows a statistics call may write */
    BFS_EVALIDATE = 6  /* internal consistency check failed (e.g. device error flag set) */
} bfs_status;

typedef struct bfs_graph bfs_graph;   /* opaque, library-owned */
typedef struct bfs_policy bfs_policy; /* opaque, library-owned learned direction policy */

/* Build flags for bfs_build_graph. */
enum {
    BFS_SYMMETRIZE = 1, /* add (d,s) for every (s,d): an undirected edge is two directed edges (Sec. 3) */
    BFS_DEDUP = 2,      /* G is a 0/1 tensor (Eq. G): keep each (s,d) once */
    BFS_DROP_SELF = 4,  /* drop s == d */
    BFS_BUILD_CSC = 8,  /* build the d-major copy used by pull levels; aliases CSR when symmetric */
    BFS_DEFAULT_FLAGS = 15,
    BFS_REORDER_RCM = 16, /* renumber the vertices in Reverse Cuthill-McKee order (Section 7.1); needs
                             BFS_SYMMETRIZE.  The graph then lives in the new ids: sources, depths and
                             parents of bfs_run are new ids; bfs_graph_permutation maps them */
    BFS_PULL_HUBS_FIRST = 32 /* order each d-major row by the degree of its entries, highest first (ties by
                                id), instead of by id; pull scans then meet likely frontier vertices first
                                whatever the numbering.  Symmetric graphs get a second column array */
};

/*
 * Build the graph tensor G (Cascade 1, Eq. G) in CSR form (Section 4.C) from an
 * int32 edge list of m entries (src[e], dst[e]) over vertices [0, n).
 * Rows are sorted ascending and, with BFS_DEDUP, free of repeats.  With
 * BFS_BUILD_CSC the transpose (the rank swizzle of Section 4.B, B.4) is built
 * for pull levels; when BFS_SYMMETRIZE is set it is the CSR itself.
 * src/dst: host or device, not modified.  *out receives a new graph, freed
 * with bfs_free_graph.  Errors: EINVAL (null pointer, n <= 0, m < 0, id
 * outside [0, n)), ERANGE (more than 2^31-1 directed entries before or after
 * deduplication), ENOMEM, ECUDA.  Synchronises `cuda_stream`.
 *
 * BFS_REORDER_RCM: the paper reorders every input with Reverse Cuthill-McKee
 * (Section 7.1).  Vertices are ranked by (degree, id) in the symmetric, built
 * CSR.  Each connected component starts at its lowest-ranked vertex, and the
 * components follow in the rank order of their starts.  Inside a component the
 * Cuthill-McKee sequence is built level by level on the device: a level's
 * vertices are ordered by (lowest position of a neighbour in the previous
 * level, rank), which is the order in which a FIFO queue that numbers each
 * dequeued vertex's neighbours in rank order would number them.  The sequence
 * is then reversed, and the CSR is rebuilt in the new ids.  The EINVAL case
 * without BFS_SYMMETRIZE is added to the errors above.
 *
 * BFS_PULL_HUBS_FIRST: a pull scan (Section 5) may stop at any in-neighbour in
 * F_i, since the ANY of Eq. advance picks one.  A high-degree in-neighbour is
 * the most likely to be in F_i, so rows of the d-major copy are ordered by the
 * entry's out-degree, descending, ties by id.  Depths are unchanged; the
 * parent chosen is the first frontier entry in this order.  The CSR keeps
 * ascending rows, and the level statistics are taken on it.
 */
bfs_status bfs_build_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, uint32_t flags,
                           void* cuda_stream, bfs_graph** out);

/* Graph summary.  deg_* are out-degree statistics of the built CSR. */
typedef struct {
    int32_t n;
    int64_t m;            /* directed CSR entries */
    int32_t symmetric;    /* 1 when the CSC aliases the CSR */
    int32_t n_isolated;   /* vertices of degree 0 */
    int32_t deg_max;
    double deg_mean;
    double deg_var;       /* population variance of the out-degree */
} bfs_graph_stats;

bfs_status bfs_graph_info(const bfs_graph* g, bfs_graph_stats* out);

/*
 * Copy the CSR out: row_ptr[n+1] (int32) and col[m] (int32), host or device.
 * With csc != 0 the d-major copy is copied instead.  Synchronises the stream
 * when a destination is host memory.
 */
bfs_status bfs_graph_csr(const bfs_graph* g, int32_t csc, int32_t* row_ptr, int32_t* col, void* cuda_stream);

/*
 * newid[v] (int32 [n], host or device) = the id in this graph of vertex v of
 * the edge list it was built from: the Reverse Cuthill-McKee number with
 * BFS_REORDER_RCM, v itself otherwise.  Synchronises the stream when newid is
 * host memory.  Errors: EINVAL (null argument), ECUDA.
 */
bfs_status bfs_graph_permutation(const bfs_graph* g, int32_t* newid, void* cuda_stream);

void bfs_free_graph(bfs_graph* g);

/* Traversal form of one level (the third class of the 3-way policy). */
enum {
    BFS_DIR_PUSH_QUEUE = 0,  /* push, sparse int32 queue frontier (GraphIt SparsePush) */
    BFS_DIR_PUSH_BITMAP = 1, /* push, frontier read from the dense bitmap in vertex order (DensePush) */
    BFS_DIR_PULL = 2         /* pull over unvisited vertices with early exit (DensePull, Section 5) */
};

/* How the level loop is driven. */
enum {
    BFS_MODE_PERSISTENT = 0, /* one cooperative kernel, levels separated by a grid barrier (default) */
    BFS_MODE_HOST_LOOP = 1,  /* one launch sequence per level, 4-byte readback per level */
    BFS_MODE_GRAPH = 2       /* CUDA graph with a conditional WHILE node: no host work per level */
};

/* How a push level's advance and its visited update are arranged (Section 7.2:
 * the conflict/predicate and visited-mask variants).  Single-source persistent
 * and host-loop drives; MS-BFS batches always claim during the advance. */
enum {
    BFS_PUSH_FUSED = 0,             /* each neighbour is claimed in P during the advance (default) */
    BFS_PUSH_FILTER = 1,            /* Variants 13/14: the advance appends every (neighbour, source) pair
                                       to an edge frontier without a predicate; after a grid barrier a
                                       filter pass claims them in P and records depth, parent and F_{i+1} */
    BFS_PUSH_FILTER_PREDICATED = 2  /* Variants 20/23: the advance appends only neighbours not yet set in P;
                                       the visited update happens in the filter pass */
};

/* Frontier order of push-queue levels (Section 7.2, Variants 6 and 7: the
 * swizzle of F on its ranks, i.e. sorting the frontier).  Single-source
 * persistent and host-loop drives; MS-BFS batches ignore it. */
enum {
    BFS_SORT_NONE = 0,   /* entries in the order they were claimed (default) */
    BFS_SORT_DEVICE = 1, /* Variant 6: device-wide ascending vertex order before each push-queue level,
                            built by a round trip through the frontier bitmap (F_i's vertices are distinct,
                            so the bitmap is a counting sort of the queue) and an order-preserving compaction */
    BFS_SORT_TILE = 2    /* Variant 7: each CTA sorts the frontier entries of its tile (bitonic sort in shared
                            memory) before expanding them */
};

/* Small levels of a single-source search (persistent drive).  While a push
 * level's frontier is small, one thread-block cluster (16 CTAs where the GPU
 * can co-schedule them, else 8) runs the levels with the cluster's hardware
 * barrier instead of the grid-wide barrier; the first level that would pull
 * or that has more frontier edges than the cluster's threads, and every level
 * after it, runs in the full persistent kernel (a second launch on the same
 * stream, no host round trip).  Sources run one launch pair each. */
enum {
    BFS_SMALL_AUTO = -1, /* on for graphs whose maximum degree is at most 16 (grids, road-like graphs) */
    BFS_SMALL_OFF = 0,
    BFS_SMALL_CLUSTER = 1
};

/* Per-level direction policy. */
enum {
    BFS_POLICY_HEURISTIC = 0, /* Beamer: push->pull if e_f > m_u/alpha, pull->push if f < n/beta */
    BFS_POLICY_PUSH = 1,      /* push every level (queue or bitmap by the gamma threshold) */
    BFS_POLICY_PULL = 2,      /* pull every level */
    BFS_POLICY_SCHEDULE = 3,  /* level i uses schedule[i % schedule_len] */
    BFS_POLICY_MLP = 4        /* learned policy `mlp` where the HEURISTIC's test is close (1/8 < e_f*alpha/m_u < 8),
                                 the HEURISTIC elsewhere and when `mlp` is NULL */
};

/* One record per executed level, written when bfs_options.level_log != NULL.
 * The single-source persistent and host-loop drives add, capacity allowing,
 * a closing record after the last level (dir = -1, f = 0) whose t_ns marks
 * the end of that level. */
typedef struct {
    int32_t level;
    int32_t dir;          /* BFS_DIR_* used for this level */
    int64_t f;            /* |F_i| */
    int64_t e_f;          /* sum of degrees over F_i */
    int64_t m_u;          /* sum of degrees over vertices unvisited before the level */
    int64_t t_ns;         /* device %globaltimer at the start of the level */
} bfs_level_record;

typedef struct {
    uint32_t struct_size;    /* sizeof(bfs_options); set by bfs_options_init */
    int32_t mode;            /* BFS_MODE_* */
    int32_t policy;          /* BFS_POLICY_* */
    float alpha;             /* Beamer alpha of single-source searches (14) */
    float beta;              /* Beamer beta of single-source searches (48) */
    float gamma;             /* push levels read the bitmap when f > n / gamma (16) */
    int32_t chunk;           /* push: vertices with degree >= chunk are split into chunk-edge units (1024) */
    int32_t medium;          /* push: degree >= medium is expanded by a whole warp (32) */
    int32_t pull_serial;     /* pull: row entries a lane tests before its row is finished by the whole warp (16; MS-BFS: twice this many) */
    int32_t block_threads;   /* threads per CTA of the persistent single-source kernel: 256, 512 or 1024 (1024) */
    int32_t blocks_per_sm;   /* CTAs per SM, 0 = as many as fit (persistent/cooperative launch) */
    int32_t claim_aggregate; /* push: warp-aggregate the visited-bitmap OR by word (0) */
    int64_t barrier_timeout_ns; /* limit of one device-side wait before BFS_ETIMEOUT (2e9) */
    const int8_t* schedule;  /* host array for BFS_POLICY_SCHEDULE */
    int32_t schedule_len;
    int32_t max_levels;      /* stop with BFS_ERANGE after this many levels, 0 = n + 1 */
    const bfs_policy* mlp;   /* for BFS_POLICY_MLP */
    bfs_level_record* level_log; /* optional host array, one record per level (k > 1: first 64-lane unit) */
    int32_t level_log_cap;
    int32_t* levels_out;     /* optional host int32: number of levels executed (k = 1: last run) */
    int32_t batch;           /* k > 1: 1 = 64-lane MS-BFS batches (default), 0 = one source at a time */
    int32_t push_filter;     /* BFS_PUSH_* (BFS_PUSH_FUSED).  A filter form holds an edge frontier of up to
                                m (target, source) pairs, 8 B each, allocated on first use; the CUDA-graph
                                drive rejects it with EINVAL */
    int32_t frontier_sort;   /* BFS_SORT_* (BFS_SORT_NONE); the CUDA-graph drive rejects a sort with EINVAL */
    float batch_alpha;       /* alpha of the 64-lane batched direction test (4) */
    float batch_beta;        /* beta of the 64-lane batched direction test (48) */
    int32_t small_levels;    /* BFS_SMALL_* (BFS_SMALL_AUTO); single-source persistent drive with fused claiming
                                and no frontier sort, else ignored */
} bfs_options;

/* Fill `opt` with the defaults listed above. */
void bfs_options_init(bfs_options* opt);

/*
 * Breadth-first search from k sources (Cascade 1).  For every source j:
 *   depth[j*n + v]  = hop distance from sources[j] to v, -1 if unreachable
 *                     (the paper's empty value infinity, Eq. F)
 *   parent[j*n + v] = a vertex u with (u, v) in G and depth u = depth v - 1
 *                     (the ANY reduction of Eq. advance picks one; not unique),
 *                     sources[j] for v = sources[j], -1 if unreachable.
 * parent may be NULL.  Depths do not depend on the options; parents may.
 * sources[k]: host or device.  depth/parent: [k][n] int32, host or device.
 * k == 1 runs the single-source path; k > 1 runs 64-lane MS-BFS batches (or
 * single sources when opt->batch == 0: one search after another, all in one
 * persistent launch when the outputs are device memory, the drive is
 * persistent and no level log or level count is requested).
 * Errors: EINVAL (null g/sources/depth, k <= 0, source outside [0, n)),
 * ENOMEM, ECUDA, ETIMEOUT (outputs undefined), ERANGE (max_levels exceeded).
 */
bfs_status bfs_run(const bfs_graph* g, const int32_t* sources, int32_t k, int32_t* depth, int32_t* parent,
                   const bfs_options* opt, void* cuda_stream);

/*
 * Wait for `cuda_stream` and report the first device-side failure (barrier
 * timeout, work-list overflow, level limit) raised by any asynchronous run on
 * `g` since the previous check; the failure is cleared once reported.
 */
bfs_status bfs_sync(const bfs_graph* g, void* cuda_stream);

/*
 * Many queries over several graphs in ONE persistent launch: query q searches
 * graphs[graph_of_query[q]] from sources[q]; its outputs go to depth[q] and
 * parent[q] (each an int32 array of that graph's n; device memory).
 * graph_of_query/sources are host arrays of length nq; graphs has n_graphs
 * entries; depth/parent are host arrays of nq device pointers (parent or its
 * entries may be NULL).  Queries are grouped per graph into 64-lane units and
 * the units are handed out to CTA teams by a device work counter.
 * Errors as bfs_run.
 */
bfs_status bfs_run_mixed(const bfs_graph* const* graphs, int32_t n_graphs, const int32_t* graph_of_query,
                         const int32_t* sources, int32_t nq, int32_t* const* depth, int32_t* const* parent,
                         const bfs_options* opt, void* cuda_stream);

/*
 * Per-level work statistics of a finished search, for the roofline model:
 * for levels i = 0 .. L-1 six int64 values [f, e_f, u, s_u, d_new, e_u]:
 * |F_i|, degree sum over F_i, non-isolated vertices unvisited before level i,
 * CSR entries a pull level reads (each unvisited row scanned in ascending
 * order up to its first neighbour of depth i, or fully; Section 5), |F_{i+1}|
 * and the degree sum over the unvisited vertices.  s_u is computed in closed
 * form: a row is read fully at every level before the one that finds its
 * vertex, and up to the first neighbour one level up at that level.  This is
 * exact for symmetric graphs, where no neighbour lies more than one level
 * away.  For a directed graph it is an upper bound, and a pull level there
 * scans in-rows instead.  depth[n]: host or device
 * output of bfs_run for one source.  stats: host array of 6*max_levels int64.
 * *levels receives L.  Errors: EINVAL (null argument, max_levels <= 0, graph
 * or depth on another device than the current one, a depth value outside
 * [-1, n)), ERANGE (L > max_levels).  Synchronises.
 */
bfs_status bfs_level_stats(const bfs_graph* g, const int32_t* depth, int32_t max_levels, int64_t* stats,
                           int32_t* levels, void* cuda_stream);

/*
 * bfs_level_stats without any allocation.  The paper has no counterpart; this
 * exists for callers that must not allocate memory while they run: a serving
 * process whose device memory is reserved up front by its own allocator, code
 * that may not take the driver's allocation lock, or a program that audits
 * that no allocation happens after start-up.  All scratch lives in one
 * file-scope device array of fixed size (about 360 KB, held by every GPU that
 * loads the library until the process exits), so at most 4096 levels are
 * supported: a larger max_levels, or a search with more levels, returns
 * BFS_ERANGE.  depth[n] must be device memory; stats (6*max_levels int64, the
 * same table as bfs_level_stats) may be host or device; *levels (host)
 * receives L.  The first call on a device looks up the scratch array's device
 * address, so make that first call before any stream capture.  Every call
 * shares the one array: calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  The table is
 * computed as by bfs_level_stats, with the same caveat for directed graphs
 * (s_u is then an upper bound).  Synchronises `cuda_stream`.  Errors: EINVAL
 * (as bfs_level_stats, and depth in host memory), ERANGE, ECUDA.
 */
bfs_status bfs_level_stats_noalloc(const bfs_graph* g, const int32_t* depth, int32_t max_levels, int64_t* stats,
                                   int32_t* levels, void* cuda_stream);

/*
 * Connected components by min-label propagation.  This is the cascade of
 * Cascade 1 over the same graph tensor with the min operator of the paper's
 * operator table (Section 2) in place of ANY: L_0[v] = v, F_0 = the vertices
 * with an edge, L_{i+1}[d] = min(L_i[d], min over s in F_i adjacent to d of
 * L_i[s]), F_{i+1} = the vertices whose label dropped, stop when F_{i+1} is
 * empty.  label[v] (int32 [n], host or device) receives the smallest vertex id
 * of v's connected component.  *iterations (host, may be NULL) receives the
 * number of iterations run.  One cooperative launch, no host work per
 * iteration.  The graph must be symmetric (built with BFS_SYMMETRIZE).
 * Synchronises `cuda_stream`.  Errors: EINVAL (null argument, directed graph,
 * wrong device), ENOMEM, ECUDA, ETIMEOUT.
 */
bfs_status bfs_components(const bfs_graph* g, int32_t* label, int32_t* iterations, void* cuda_stream);

/* ----------------------------------------------------- learned policy (MLP) */
/*
 * Direction policy: an FP32 MLP 10 -> 32 -> 32 -> 3 (ReLU) whose argmax picks
 * BFS_DIR_*.  The paper has no learned policy; it replaces the Beamer switch
 * it cites (Section 5) where that switch's own test is close -- e_f * alpha /
 * m_u within (1/8, 8) -- and only when it predicts its choice a to beat the
 * heuristic's form h clearly (outputs z_a - z_h > 1.0, about 2.7x in time);
 * the heuristic decides everywhere else (and costs no network evaluation on
 * the clear-cut levels).  Parameter layout (1507 floats, row-major):
 *   W1[32][10] b1[32] W2[32][32] b2[32] W3[3][32] b3[3]
 * followed by 20 floats of input normalisation: mean[10], inv_std[10].
 */
#define BFS_MLP_IN 10
#define BFS_MLP_HIDDEN 32
#define BFS_MLP_OUT 3
#define BFS_MLP_NPARAM 1507
#define BFS_MLP_NNORM 20

/*
 * Features of one level (host or device float[10]) from its counters: f =
 * |F_i|, e_f = degree sum over F_i, m_u = degree sum over unvisited vertices,
 * f_prev = |F_{i-1}|, prev_dir = form of level i-1.  Scale-free:
 * log2 of e_f/m_u, f/n, m_u/m, mean frontier degree over mean degree,
 * (f+1)/(f_prev+1); prev_dir one-hot (pull, push-bitmap); min(log2(n), 22)/32
 * (graph size, clamped to the largest training scale); log2(deg_max / mean
 * degree) capped at 12; log2(mean degree)/4.  `level` is accepted for the
 * interface and not used.
 */
bfs_status bfs_policy_features(const bfs_graph* g, int32_t level, int64_t f, int64_t e_f, int64_t m_u,
                               int64_t f_prev, int32_t prev_dir, float* out10);

/*
 * Training signal of the policy: run the plain method (opt->policy, heuristic
 * by default) from `source` one level at a time; before each level i, save
 * the level state and time every form BFS_DIR_* from that same state
 * (median of `repeats` launches, format conversions included), then continue
 * with the plain method's own choice.  Host outputs, L = *levels rows each:
 * features[L][10] (bfs_policy_features of the level), times_us[L][3],
 * taken[L] (form the plain method used; may be NULL).  Synchronous.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT.
 */
bfs_status bfs_profile_levels(const bfs_graph* g, int32_t source, const bfs_options* opt, int32_t repeats,
                              int32_t max_levels, float* features, float* times_us, int32_t* taken, int32_t* levels,
                              void* cuda_stream);

/* weights: host float[nw], nw = BFS_MLP_NPARAM + BFS_MLP_NNORM. */
bfs_status bfs_policy_load(const float* weights, int32_t nw, bfs_policy** out);
bfs_status bfs_policy_weights(const bfs_policy* p, float* out, int32_t nw); /* host copy */
void bfs_policy_free(bfs_policy* p);

/* logits[rows][3] for raw (unnormalised) features X[rows][10]; device pointers. */
bfs_status bfs_policy_forward(const bfs_policy* p, const float* X, int64_t rows, float* logits,
                              void* cuda_stream);

/*
 * One optimiser step of mean softmax cross-entropy on (X[rows][10], y[rows])
 * with Adam (Kingma & Ba 2015): forward, backward and update run in the
 * library's FP32 kernels on the device.  X/y: device.  loss_out: host float or
 * NULL.  grad_out: optional device float[BFS_MLP_NPARAM] receiving the
 * gradient before the update.  step is 1-based.
 */
bfs_status bfs_policy_train_step(bfs_policy* p, const float* X, const int32_t* y, int64_t rows, float lr,
                                 int32_t step, float* loss_out, float* grad_out, void* cuda_stream);

/*
 * The same step on a least-squares objective: L = (1/R) sum_r sum_c
 * (z_rc - target_rc)^2 / 2 over the raw outputs z (no softmax), target device
 * float [rows][3] row-major; dL/dz = (z - target) / R.  Trained on
 * -log(T_c / T_min) of profiled levels, the outputs estimate how much slower
 * each traversal form is, and their argmax -- the form the search takes -- is
 * the one predicted fastest.  Other arguments and errors as
 * bfs_policy_train_step.
 */
bfs_status bfs_policy_train_step_regress(bfs_policy* p, const float* X, const float* target, int64_t rows, float lr,
                                         int32_t step, float* loss_out, float* grad_out, void* cuda_stream);

/* Replace the normalisation (mean[10], inv_std[10], host) used by forward/train. */
bfs_status bfs_policy_set_norm(bfs_policy* p, const float* mean_inv_std);

/* ------------------------------------------------------------------ errors */
const char* bfs_status_string(bfs_status s);
const char* bfs_last_error(void); /* thread-local message of the last failure */
const char* bfs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BFSGB_BFS_H */
