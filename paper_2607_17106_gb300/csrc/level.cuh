// level.cuh -- device code of one BFS level (Cascade 1), shared by the
// persistent kernel (bfs_single.cu) and the CUDA-graph level kernels
// (bfs_graph.cu).  See bfs_single.cu for the design notes.
#pragma once

#include "common.cuh"
#include "policy_dev.cuh"

namespace bfsgb {

struct Counters {
    unsigned long long q_len;  // vertices appended to the next queue (= |F_{i+1}|)
    unsigned long long u_len;  // chunk units appended for the next level
    unsigned long long e_f;    // sum of out-degrees of the appended vertices
    unsigned long long conv;   // cursor of a bitmap -> queue conversion of this frontier
    unsigned long long e_len;  // push_filter: (target, source) pairs in the edge frontier of the level
};

struct Ctl1 {
    GridBarrier bar;
    // level i of search si of a launch counts in slot[3 * (si & 1) + i % 3]:
    // consecutive searches use different sets, so one search's first CTA
    // can reset its set while another CTA still reads the previous search's
    // last counters
    Counters slot[6];
    // loop state carried between launches
    int32_t next_level;
    int32_t prev_dir;
    int32_t bm_valid;   // level whose frontier bitmap is current, -1 if none
    int32_t q_valid;    // level whose frontier queue (and chunk units) is current
    int32_t done;
    long long m_u;
    long long f_prev;
    unsigned bar_base;  // barrier arrivals of earlier launches (host-loop mode)
    // graph mode: the level being run, its form and the run's outputs
    int32_t cur_level;
    int32_t cur_dir;
    int32_t units_valid;
    int32_t src;
    int32_t* depth;
    int32_t* parent;
};

struct Workspace1 {
    int32_t n = 0;
    int64_t W = 0;
    int32_t chunk = 0;
    int64_t ucap = 0;
    uint32_t* P = nullptr;
    uint32_t* F[2] = {nullptr, nullptr};
    int4* Q[2] = {nullptr, nullptr};
    int2* U[2] = {nullptr, nullptr};
    int2* E = nullptr;  // push_filter: edge frontier, capacity ecap pairs (allocated on first use)
    unsigned* cta_cnt = nullptr;  // frontier_sort: one count per CTA of the persistent launch
    int64_t ecap = 0;
    Ctl1* ctl = nullptr;
    int* d_sticky = nullptr;
    int32_t* stage_depth = nullptr;
    int32_t* stage_parent = nullptr;
    int32_t* d_srcs = nullptr;  // sources of a multi-search launch
    int32_t src_cap = 0;
    bfs_level_record* d_log = nullptr;
    int32_t log_cap = 0;
    int8_t* d_sched = nullptr;
    int32_t sched_cap = 0;
    Ctl1* h_ctl = nullptr;  // pinned host mirror for host-loop readbacks
    // CUDA-graph mode: the instantiated level loop and what it was built for
    cudaGraphExec_t gexec = nullptr;
    unsigned char gkey[512] = {0};
    int gkey_len = 0;
};

void free_ws1(Workspace1* w);  // bfs_single.cu

struct Params1 {
    int32_t n;
    int64_t W;
    int64_t m;
    int32_t symmetric;
    const int32_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col;
    const int32_t* __restrict__ csc_ptr;
    const int32_t* __restrict__ csc_col;
    const uint32_t* __restrict__ isolated;
    uint32_t* P;
    uint32_t* F0;
    uint32_t* F1;
    int4* Q0;  // frontier queues: {vertex, row begin, row end, 0}
    int4* Q1;
    int2* U0;
    int2* U1;
    int64_t ucap;
    int2* E;       // push_filter: edge frontier of the level, {target, source}
    int64_t ecap;
    Ctl1* ctl;
    int32_t src_value;
    const int32_t* srcs;  // nsrc sources searched one after another in one launch (device), or null
    int32_t nsrc;
    int* sticky;          // first device error of any run, cleared by the host
    int32_t* depth;
    int32_t* parent;
    // policy
    int32_t policy;
    int32_t force_dir;  // >= 0: every level uses this form (level profiling)
    float alpha, beta, gamma;
    const int8_t* schedule;
    int32_t schedule_len;
    const float* mlp;
    int32_t deg_max;
    // tuning
    int32_t chunk, medium, pull_serial, aggregate;
    int32_t push_filter;  // BFS_PUSH_FUSED / _FILTER / _FILTER_PREDICATED
    int32_t frontier_sort;  // BFS_SORT_*
    unsigned* cta_cnt;    // BFS_SORT_DEVICE: frontier vertices of each CTA's word range
    int64_t timeout_ns;
    int32_t max_levels;
    bfs_level_record* log;
    int32_t log_cap;
    // launch control
    int32_t do_init;
    int32_t level_count;  // levels to run in this launch (host loop: 1)
    int64_t small_ef_max; // cluster launch: leave before a level with more frontier edges (or a pull)
    int32_t rows_filled;  // the -1 of the depth and parent rows was stored before the launch
};

// ------------------------------------------------------------- direction
// Direction tests use FP32: every thread of every CTA evaluates them at every
// level, and GB300's FP64 rate is a small fraction of its FP32 rate (a
// double division per thread per level measurably lengthened each level).
__device__ __forceinline__ int push_kind(const Params1& p, long long f) {
    return ((float)f * p.gamma > (float)p.n) ? BFS_DIR_PUSH_BITMAP : BFS_DIR_PUSH_QUEUE;
}

// Beamer et al. 2012 (cited in Section 5): top-down while the frontier's
// edges are few relative to the unexplored edges; bottom-up while the
// frontier is growing or large.
__device__ __forceinline__ int heuristic_dir(const Params1& p, long long f, long long e_f, long long m_u,
                                             long long f_prev, int prev_dir) {
    if (prev_dir == BFS_DIR_PULL) {
        bool stay = (f >= f_prev) || ((float)f * p.beta > (float)p.n);
        return stay ? BFS_DIR_PULL : push_kind(p, f);
    }
    if ((float)e_f * p.alpha > (float)m_u && f > f_prev) return BFS_DIR_PULL;
    return push_kind(p, f);
}

// Same inputs on every CTA -> same decision (all arithmetic is deterministic).
// mlp_w: the policy weights to evaluate (a shared-memory copy when the
// caller staged one), else p.mlp.  Block-uniform.
__device__ inline int decide_dir(const Params1& p, int level, long long f, long long e_f, long long m_u, long long f_prev,
                          int prev_dir, float* s_feat, float* s_mlp_out, const float* mlp_w = nullptr) {
    if (p.force_dir >= 0) return p.force_dir;
    switch (p.policy) {
        case BFS_POLICY_PUSH:
            return push_kind(p, f);
        case BFS_POLICY_PULL:
            return BFS_DIR_PULL;
        case BFS_POLICY_SCHEDULE: {
            int d = p.schedule[level % p.schedule_len];
            return (d < 0 || d > 2) ? BFS_DIR_PUSH_QUEUE : d;
        }
        case BFS_POLICY_MLP: {
            const int h = heuristic_dir(p, f, e_f, m_u, f_prev, prev_dir);
            if (p.mlp && policy_in_band(e_f, m_u, p.alpha)) {
                // thread 0 forms the features; the whole CTA evaluates
                __shared__ float s_h2[MLP_H];
                __shared__ int s_choice;
                if (threadIdx.x == 0) policy_features(s_feat, f, e_f, m_u, f_prev, level, prev_dir, p.n, p.m, p.deg_max);
                __syncthreads();
                return policy_choice_block(mlp_w ? mlp_w : p.mlp, s_feat, h, MLP_MARGIN, s_h2, &s_choice);
            }
            return h;
        }
        default:
            return heuristic_dir(p, f, e_f, m_u, f_prev, prev_dir);
    }
}

// Loads of P and of the frontier bitmaps are ordinary (L1-cacheable) loads:
// the writes of the previous level are ordered before them by the grid
// barrier's acquire (or by the kernel boundary in graph mode), and within a
// level P only gains bits, so a stale word can only cost an extra OR.  Hub
// rows make a few frontier words very hot, which the L1 then serves.

// ------------------------------------------------------------ claiming
constexpr int QBUF = 64;  // per-warp shared-memory staging of next-queue entries

struct LevelCtx {
    int32_t level;          // i: discovered vertices get depth i+1
    int32_t* depth;         // outputs of this run
    int32_t* parent;
    int4* q_next;
    int2* u_next;
    Counters* next;         // counters of F_{i+1}
    unsigned long long ef;  // this thread's share of e_f(F_{i+1})
    unsigned long long cnt; // this thread's share of |F_{i+1}| (pull levels)
    int32_t* qv;            // this warp's staging of next-queue entries (QBUF
    int32_t* qb;            // each): vertex, row begin, row end
    int32_t* qe;
    int qn;                 // entries staged (warp-uniform)
    long long qcap;         // capacity of q_next (n entries)
    int* err;               // device error word of the run
    bool precheck;          // push: read P before the OR (most targets already visited)
};

#ifndef BFS_PRECHECK_MIN_EF
#define BFS_PRECHECK_MIN_EF 65536
#endif
// A push target is visited with probability about 1 - m_u / m (the explored
// share of the edges); reading P before the OR pays once most are and the
// level has enough candidates for the ORs' throughput to matter (on a small
// level the extra read only lengthens the chain).
__device__ __forceinline__ bool push_precheck(long long m_u, long long m, long long e_f) {
    return 2 * m_u < m && e_f >= BFS_PRECHECK_MIN_EF;
}


// Move the warp's staged queue entries to the next queue: one atomic per
// flush instead of one per claiming round.  An entry carries its vertex's
// row bounds (loaded when the vertex was claimed), so expanding it next
// level needs no row-offset load.  Warp-uniform.
__device__ __forceinline__ void flush_qbuf(LevelCtx& L) {
    if (L.qn == 0) return;
    const unsigned lane = lane_id();
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&L.next->q_len, (unsigned long long)L.qn);
    base = __shfl_sync(0xffffffffu, base, 0);
    // a vertex is claimed once, so the queue never outgrows n; were that ever
    // broken, record the overflow instead of writing past the buffer
    if (base + (unsigned long long)L.qn <= (unsigned long long)L.qcap) {
        for (int i = (int)lane; i < L.qn; i += 32) {
            L.q_next[base + i] = make_int4(L.qv[i], L.qb[i], L.qe[i], 0);
        }
    } else if (lane == 0) {
        atomicCAS(L.err, 0, (int)DEV_OVERFLOW);
    }
    __syncwarp();
    L.qn = 0;
}

__device__ __forceinline__ void emit_units(const Params1& p, int2* u_out, Counters* c, int v, int deg) {
    append_units(u_out, &c->u_len, p.ucap, &p.ctl->bar.err, v, deg, p.chunk);
}

// Chunk units of the big rows among a warp's claims: one atomic per warp.
// Warp-uniform call.
__device__ __forceinline__ void emit_units_warp(const Params1& p, int2* u_out, Counters* c, bool big, int v, int deg) {
    append_units_warp(u_out, &c->u_len, p.ucap, &p.ctl->bar.err, big, v, deg, p.chunk);
}

// Record vertices claimed in a push level: depth/parent, staged next-queue
// slot (with the row bounds rb..re of v), degree sum, chunk units for big
// rows.  Warp-uniform call.
__device__ __forceinline__ void emit(const Params1& p, LevelCtx& L, bool claimed, int v, int u, int rb, int re) {
    unsigned cm = __ballot_sync(0xffffffffu, claimed);
    if (!cm) return;
    int c = __popc(cm);
    if (L.qn + c > QBUF) flush_qbuf(L);
    const int deg = re - rb;
    if (claimed) {
        const int slot = L.qn + __popc(cm & lanemask_lt());
        L.qv[slot] = v;
        L.qb[slot] = rb;
        L.qe[slot] = re;
        L.depth[v] = L.level + 1;
        if (L.parent) L.parent[v] = u;
        L.ef += (unsigned long long)deg;
    }
    L.qn += c;
    emit_units_warp(p, L.u_next, L.next, claimed && deg >= p.chunk, v, deg);
}

// Claim v for parent u in P if not yet visited, and record the claim.
// Warp-uniform.
__device__ __forceinline__ void claim_candidate(const Params1& p, LevelCtx& L, bool has, int v, int u) {
    bool want = false;
    unsigned w = 0, bit = 0;
    if (has) {
        w = (unsigned)v >> 5;
        bit = 1u << (v & 31);
        want = !L.precheck || !(p.P[w] & bit);  // may be stale (bits only grow): the OR decides
    }
    // the row bounds of a likely claim are fetched before the OR so that both
    // round trips overlap
    int rb = 0, re = 0;
    if (want) {
        rb = __ldg(p.row_ptr + v);
        re = __ldg(p.row_ptr + v + 1);
    }
    bool claimed = false;
    if (p.aggregate) {
        unsigned act = __ballot_sync(0xffffffffu, want);
        if (act && want) {
            unsigned lane = lane_id();
            unsigned peers = __match_any_sync(act, w);
            unsigned same = __match_any_sync(act, (unsigned)v);
            bool first = (unsigned)(__ffs(same) - 1) == lane;
            unsigned orb = __reduce_or_sync(peers, first ? bit : 0u);
            int leader = __ffs(peers) - 1;
            unsigned old = 0;
            if ((int)lane == leader) old = atomicOr(p.P + w, orb);
            old = __shfl_sync(peers, old, leader);
            claimed = first && !(old & bit);
        }
    } else if (want) {
        claimed = !(atomicOr(p.P + w, bit) & bit);
    }
    emit(p, L, claimed, v, u, rb, re);
}

// push_filter: move the warp's staged (target, source) pairs to the level's
// edge frontier, one atomic per flush.  Warp-uniform.
__device__ __forceinline__ void flush_pairs(const Params1& p, LevelCtx& L) {
    if (L.qn == 0) return;
    const unsigned lane = lane_id();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&L.next->e_len, (unsigned long long)L.qn);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    if (base + (unsigned long long)L.qn <= (unsigned long long)p.ecap) {
        for (int i = (int)lane; i < L.qn; i += 32) p.E[base + i] = make_int2(L.qv[i], L.qb[i]);
    } else if (lane == 0) {
        atomicCAS(&p.ctl->bar.err, 0, (int)DEV_OVERFLOW);
    }
    __syncwarp();
    L.qn = 0;
}

// End of a push level's expansion: staged queue entries, or staged pairs when
// the claims are left to a filter pass.  Warp-uniform.
__device__ __forceinline__ void flush_push(const Params1& p, LevelCtx& L) {
    if (p.push_filter != BFS_PUSH_FUSED) flush_pairs(p, L);
    else flush_qbuf(L);
}

// Push candidate (u -> v).  Fused (the default): claim v at once.  With a
// filter pass, the advance only appends (v, u) to the level's edge frontier:
// every pair (BFS_PUSH_FILTER, Variants 13/14: advance without the predicate),
// or those whose v is not yet set in P (BFS_PUSH_FILTER_PREDICATED, Variants
// 20/23: the visited test in the advance, the visited update in the filter).
// The warp's queue staging holds the pairs (target in qv, source in qb).
// Warp-uniform.
__device__ __forceinline__ void push_candidate(const Params1& p, LevelCtx& L, bool has, int v, int u) {
    if (p.push_filter == BFS_PUSH_FUSED) {
        claim_candidate(p, L, has, v, u);
        return;
    }
    bool want = has;
    if (has && p.push_filter == BFS_PUSH_FILTER_PREDICATED) want = !(p.P[(unsigned)v >> 5] & (1u << (v & 31)));
    const unsigned cm = __ballot_sync(0xffffffffu, want);
    if (!cm) return;
    const int c = __popc(cm);
    if (L.qn + c > QBUF) flush_pairs(p, L);
    if (want) {
        const int slot = L.qn + __popc(cm & lanemask_lt());
        L.qv[slot] = v;
        L.qb[slot] = u;
    }
    L.qn += c;
}

// push_filter: claim the pairs of the level's edge frontier E[0, len) (after
// a grid barrier that ends the advance), strided over all warps in order.
template <int T>
__device__ void filter_level(const Params1& p, LevelCtx& L, long long len) {
    const long long wstride = (long long)gridDim.x * T;
    for (long long b = (long long)blockIdx.x * T + (threadIdx.x & ~31u); b < len; b += wstride) {  // warp-uniform
        const long long i = b + lane_id();
        const bool has = i < len;
        const int2 e = has ? __ldcg(p.E + i) : make_int2(0, 0);
        claim_candidate(p, L, has, e.x, e.y);
    }
    flush_qbuf(L);
}

// ------------------------------------------------------------ shared memory
// A warp's scratch in the word-based pull (pull_level, graph mode).
struct PullWarpSmem {
    unsigned nb[32];                   // new bits of the block's words (slot = the word's lane)
    int lv[32], lj[32], le[32], lb[32], ls[32];  // deferred rows: vertex, next entry, end, row start, slot
    int nl;
};

// A round of the list-driven pull (pull_level_list): the new bits found for
// the P words the CTA's warps own in the round (slot = warp * 32 + lane); the
// round's unvisited vertices are listed in dynamic shared memory as 16-bit
// (slot, bit) entries.
template <int T>
struct PullListSmem {
    int n;           // unvisited vertices listed in the round
    int next;        // cursor of the warps draining the list
    unsigned nb[T];  // bits of F_{i+1} found in each slot's word
};

// The warps' staging of next-queue entries in push levels (QBUF each).
template <int T>
struct QueueStage {
    int32_t qv[(T / 32) * QBUF];
    int32_t qb[(T / 32) * QBUF];
    int32_t qe[(T / 32) * QBUF];
};

// Shared memory of a CTA running level kernels.  Push levels use the tile
// scratch (their next-queue staging is a QueueStage of its own: in the
// persistent kernel it shares the pull list's dynamic shared memory); pull
// levels use the round's new-bit words; no level uses both, so they share
// storage.
template <int T>
struct TileSmem {
    union {
        struct {
            int off[T + 1];
            int beg[T];
            int lim[T];
            int src[T];
        } t;
        PullListSmem<T> list;
    };
    int scan_tmp[33];
    unsigned long long red[T / 32];
    unsigned long long red2[T / 32];
    unsigned long long base;
};

// One CTA expands up to T frontier vertices (one per thread, u < 0 = none)
// whose rows are beg..end.  Rows of degree >= chunk are skipped when chunk
// units cover them.
template <int T>
__device__ __forceinline__ void push_tile(const Params1& p, LevelCtx& L, TileSmem<T>& sm, int u, int beg, int end,
                                          bool skip_big) {
    unsigned lane = lane_id();
    if (u < 0) beg = end = 0;
    if (skip_big && end - beg >= p.chunk) end = beg;
    // medium rows: cut into 32-edge segments that the CTA's warps take in
    // turn (a warp walking only its own lanes' rows would serialise them while
    // the other warps idle)
    const bool med = (end - beg) >= p.medium;
    int nseg_total;
    const int soff = block_exclusive_scan(med ? (end - beg + 31) >> 5 : 0, sm.scan_tmp, &nseg_total);
    if (nseg_total > 0) {
        sm.t.off[threadIdx.x] = soff;
        sm.t.beg[threadIdx.x] = beg;
        sm.t.lim[threadIdx.x] = end;
        sm.t.src[threadIdx.x] = u;
        __syncthreads();
        for (int s = (int)(threadIdx.x >> 5); s < nseg_total; s += T / 32) {
            // the row holding segment s: largest t with off[t] <= s
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (sm.t.off[mid] <= s) lo = mid; else hi = mid - 1;
            }
            const int j = sm.t.beg[lo] + ((s - sm.t.off[lo]) << 5) + (int)lane;
            const bool has = j < sm.t.lim[lo];
            const int v = has ? __ldg(p.col + j) : 0;
            push_candidate(p, L, has, v, sm.t.src[lo]);
        }
        // the scan below passes a barrier before anything overwrites off/beg/src
    }
    if (med) end = beg;
    // small rows: flatten (u, j) pairs over the CTA
    int deg = end - beg, total;
    int off = block_exclusive_scan(deg, sm.scan_tmp, &total);
    sm.t.off[threadIdx.x] = off;
    sm.t.beg[threadIdx.x] = beg;
    sm.t.src[threadIdx.x] = u;
    if (threadIdx.x == T - 1) sm.t.off[T] = total;
    __syncthreads();
    for (int k0 = 0; k0 < total; k0 += T) {
        int k = k0 + threadIdx.x;
        bool has = k < total;
        int v = 0, su = 0;
        if (has) {
            // largest t with off[t] <= k
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (sm.t.off[mid] <= k) lo = mid; else hi = mid - 1;
            }
            su = sm.t.src[lo];
            v = __ldg(p.col + sm.t.beg[lo] + (k - sm.t.off[lo]));
        }
        push_candidate(p, L, has, v, su);
    }
    __syncthreads();
}

// One CTA expands one chunk unit (vertex u, edges [c*chunk, (c+1)*chunk)).
template <int T>
__device__ __forceinline__ void push_unit(const Params1& p, LevelCtx& L, int2 unit) {
    int u = unit.x;
    int b = __ldg(p.row_ptr + u), e = __ldg(p.row_ptr + u + 1);
    int lo = b + unit.y * p.chunk, hi = min(e, lo + p.chunk);
    for (int base = lo; base < hi; base += T) {
        int j = base + threadIdx.x;
        bool has = j < hi;
        int v = has ? __ldg(p.col + j) : 0;
        push_candidate(p, L, has, v, u);
    }
}

// Variant 7 (BFS_SORT_TILE): the CTA's tile of frontier entries -- entries of
// threads 0 .. cnt-1 are valid -- sorted by vertex in shared memory with a
// bitonic network over the next power of two >= cnt.  Block-uniform.
template <int T>
__device__ __forceinline__ void tile_sort(TileSmem<T>& sm, int4& e, int cnt) {
    int p2 = 1;
    while (p2 < cnt) p2 <<= 1;
    const int t = (int)threadIdx.x;
    __syncthreads();  // a previous tile's readers of sm.t are done
    if (t < p2) {
        sm.t.src[t] = t < cnt ? e.x : INT32_MAX;
        sm.t.beg[t] = e.y;
        sm.t.lim[t] = e.z;
    }
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int o = t ^ j;
            if (t < p2 && o > t) {
                const bool up = (t & k) == 0;
                const int a = sm.t.src[t], b = sm.t.src[o];
                if ((a > b) == up) {
                    sm.t.src[t] = b;
                    sm.t.src[o] = a;
                    const int by = sm.t.beg[t], bz = sm.t.lim[t];
                    sm.t.beg[t] = sm.t.beg[o];
                    sm.t.lim[t] = sm.t.lim[o];
                    sm.t.beg[o] = by;
                    sm.t.lim[o] = bz;
                }
            }
            __syncthreads();
        }
    }
    if (t < cnt) e = make_int4(sm.t.src[t], sm.t.beg[t], sm.t.lim[t], 0);
    __syncthreads();  // push_tile reuses sm.t
}

// Push level.  Queue levels deal the frontier in passes of gridDim * T
// entries: thread t of CTA b takes entry pass * gridDim * T + b + gridDim * t,
// so a small frontier spreads over one thread of many CTAs.  Each entry carries
// its row bounds.  Bitmap levels deal tiles of T/32 words of F_i round-robin.
// Then the chunk units of F_i's big rows, round robin (their rows are skipped
// in the tiles).
template <int T, bool SORT = false>
__device__ void push_level(const Params1& p, LevelCtx& L, TileSmem<T>& sm, int dir, const int4* q_cur,
                           const int2* u_cur, const uint32_t* f_cur, long long f, long long nunits, bool units_valid) {
    const long long G = gridDim.x;
    if (dir == BFS_DIR_PUSH_QUEUE) {
        for (long long base = 0; base + blockIdx.x < f; base += G * T) {  // CTA-uniform
            const long long q = base + blockIdx.x + G * threadIdx.x;
            int4 e = q < f ? __ldcg(q_cur + q) : make_int4(-1, 0, 0, 0);
            if (SORT && p.frontier_sort == BFS_SORT_TILE) {
                const long long cnt = (f - base - blockIdx.x + G - 1) / G;  // entries of this tile
                tile_sort<T>(sm, e, (int)min(cnt, (long long)T));
            }
            push_tile<T>(p, L, sm, e.x, e.y, e.z, units_valid);
        }
    } else {
        const long long ntiles = (p.W + (T / 32) - 1) / (T / 32);
        for (long long t = blockIdx.x; t < ntiles; t += G) {
            const long long w = t * (T / 32) + (threadIdx.x >> 5);
            int u = -1, rb = 0, re = 0;
            if (w < p.W) {
                const unsigned fw = f_cur[w];
                if ((fw >> (threadIdx.x & 31)) & 1u) {
                    u = (int)(w * 32 + (threadIdx.x & 31));
                    rb = __ldg(p.row_ptr + u);
                    re = __ldg(p.row_ptr + u + 1);
                }
            }
            push_tile<T>(p, L, sm, u, rb, re, units_valid);
        }
    }
    if (!units_valid || nunits == 0) {
        flush_push(p, L);
        return;
    }
    if (p.chunk <= T && T % p.chunk == 0 && p.chunk % 32 == 0) {
        // T / chunk units at a time, one per group of chunk threads (whole
        // warps), one edge per thread: a CTA is not left three-quarters idle
        // on 256-edge units
        const int per = T / p.chunk;
        const int grp = (int)threadIdx.x / p.chunk, lt = (int)threadIdx.x % p.chunk;
        for (long long it = (long long)blockIdx.x * per; it < nunits; it += G * per) {  // CTA-uniform
            const long long ui = it + grp;
            int u = 0, j = 0, hi = 0;
            if (ui < nunits) {
                const int2 un = __ldcg(u_cur + ui);
                u = un.x;
                const int b = __ldg(p.row_ptr + u), e = __ldg(p.row_ptr + u + 1);
                j = b + un.y * p.chunk + lt;
                hi = min(e, b + (un.y + 1) * p.chunk);
            }
            const bool has = j < hi;
            push_candidate(p, L, has, has ? __ldg(p.col + j) : 0, u);
        }
    } else {
        for (long long it = blockIdx.x; it < nunits; it += G) push_unit<T>(p, L, __ldcg(u_cur + it));
    }
    flush_push(p, L);
}

// ------------------------------------------------------------ pull level
constexpr int PULL_SERIAL_MAX = 32;  // row entries one lane scans before its warp takes over
#ifndef BFS_PULL_R
#define BFS_PULL_R 1
#endif
// in-neighbours a lane loads and tests per serial step: the loads of one step
// are independent, so a step costs about one memory round trip whatever R is
constexpr int PULL_R = BFS_PULL_R;
// 32-entry groups a warp loads per step when it finishes a deferred long row
// (4 groups measured no faster than 1)
constexpr int PULL_LONG_U = 1;

template <bool NC>
__device__ __forceinline__ unsigned ld_word(const uint32_t* a, long long i) {
    return NC ? __ldg(a + i) : a[i];
}


// Words a warp finishes at a time in the dense pull (3 or 4 measured within
// +-3 % of 2 on RMAT, ER, BA and the grid).
constexpr int PULL_WPI = 2;

// Dense words of a pull level, PULL_WPI at a time, lane = vertex: wv[k] is a
// word index of P (-1 for none) and pw[k] its P word.  An unvisited lane
// scans its in-neighbours in ascending order and stops at the first one in
// F_i (ANY = the lowest-index frontier neighbour); rows longer than
// `pull_serial` entries are finished by the whole warp, 4 x 32 entries a step.
// The warp writes the words of P and of F_{i+1} with plain stores (it owns
// them).  Warp-uniform.
// Row bounds of the lanes' vertices of words wv (the first memory step of
// pull_words, separate so that a caller can issue it ahead).
__device__ __forceinline__ void pull_word_bounds(const Params1& p, const long long (&wv)[PULL_WPI],
                                                 const unsigned (&pw)[PULL_WPI], int (&beg)[PULL_WPI],
                                                 int (&end)[PULL_WPI]) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int k = 0; k < PULL_WPI; ++k) {
        const bool unvis = !((pw[k] >> lane) & 1u);
        const long long v = wv[k] * 32 + lane;
        beg[k] = unvis ? __ldg(p.csc_ptr + v) : 0;
        end[k] = unvis ? __ldg(p.csc_ptr + v + 1) : 0;
    }
}

template <bool NC>
__device__ __forceinline__ void pull_words_scan(const Params1& p, LevelCtx& L, const uint32_t* f_cur,
                                                uint32_t* f_next, const long long (&wv)[PULL_WPI],
                                                const unsigned (&pw)[PULL_WPI], const int (&beg)[PULL_WPI],
                                                const int (&end)[PULL_WPI]) {
    const unsigned lane = lane_id();
    const int dnext = L.level + 1;
    const int serial = min(p.pull_serial, PULL_SERIAL_MAX);
    bool unvis[PULL_WPI], found[PULL_WPI];
    int j[PULL_WPI], par[PULL_WPI];
#pragma unroll
    for (int k = 0; k < PULL_WPI; ++k) {
        unvis[k] = !((pw[k] >> lane) & 1u);
        j[k] = beg[k];
        found[k] = false;
        par[k] = -1;
    }
    // ascending scans of the rows advance together, PULL_R entries a step;
    // the first frontier entry in row order is the parent
    for (int step = 0; step < serial; step += PULL_R) {
        int u[PULL_WPI][PULL_R];
        unsigned fw[PULL_WPI][PULL_R];
        bool live = false;
#pragma unroll
        for (int k = 0; k < PULL_WPI; ++k) {
            const bool lk = !found[k] && j[k] < end[k];
#pragma unroll
            for (int r = 0; r < PULL_R; ++r)
                u[k][r] = (lk && j[k] + r < end[k]) ? __ldg(p.csc_col + j[k] + r) : -1;
            live |= lk;
        }
        if (!live) break;
#pragma unroll
        for (int k = 0; k < PULL_WPI; ++k)
#pragma unroll
            for (int r = 0; r < PULL_R; ++r) fw[k][r] = u[k][r] >= 0 ? ld_word<NC>(f_cur, u[k][r] >> 5) : 0u;
#pragma unroll
        for (int k = 0; k < PULL_WPI; ++k) {
            if (u[k][0] < 0) continue;
            int adv = PULL_R;
#pragma unroll
            for (int r = PULL_R - 1; r >= 0; --r)
                if (u[k][r] >= 0 && ((fw[k][r] >> (u[k][r] & 31)) & 1u)) adv = r;
            if (adv < PULL_R) {
                found[k] = true;
                par[k] = u[k][adv];
                j[k] += adv;
            } else {
                j[k] += PULL_R;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PULL_WPI; ++k) {
        if (wv[k] < 0) break;  // warp-uniform
        unsigned rm = __ballot_sync(0xffffffffu, unvis[k] && !found[k] && j[k] < end[k]);
        while (rm) {
            const int l = __ffs(rm) - 1;
            const int bl = __shfl_sync(0xffffffffu, j[k], l);
            const int el = __shfl_sync(0xffffffffu, end[k], l);
            // 4 x 32 entries a step, all column loads issued before the
            // frontier tests; the first hit in row order is the parent
            int hit = -1;
            for (int base = bl; base < el && hit < 0; base += 128) {
                int uu[4];
                unsigned fw[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int idx = base + q * 32 + (int)lane;
                    uu[q] = idx < el ? __ldg(p.csc_col + idx) : -1;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) fw[q] = uu[q] >= 0 ? ld_word<NC>(f_cur, uu[q] >> 5) : 0u;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const unsigned hb = __ballot_sync(0xffffffffu, uu[q] >= 0 && ((fw[q] >> (uu[q] & 31)) & 1u));
                    if (hb && hit < 0) hit = __shfl_sync(0xffffffffu, uu[q], __ffs(hb) - 1);
                }
            }
            if ((int)lane == l && hit >= 0) {
                found[k] = true;
                par[k] = hit;
            }
            rm &= rm - 1;
        }
        const long long w = wv[k];
        const unsigned nb = __ballot_sync(0xffffffffu, found[k]);
        if (lane == 0) {
            f_next[w] = nb;
            if (nb) p.P[w] = pw[k] | nb;
        }
        if (found[k]) {
            const long long v = w * 32 + lane;
            L.depth[v] = dnext;
            if (L.parent) L.parent[v] = par[k];
            L.ef += (unsigned long long)(p.symmetric ? (end[k] - beg[k])
                                                     : (__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v)));
            L.cnt += 1;
        }
    }
}

template <bool NC>
__device__ __forceinline__ void pull_words(const Params1& p, LevelCtx& L, const uint32_t* f_cur, uint32_t* f_next,
                                           const long long (&wv)[PULL_WPI], const unsigned (&pw)[PULL_WPI]) {
    int beg[PULL_WPI], end[PULL_WPI];
    pull_word_bounds(p, wv, pw, beg, end);
    pull_words_scan<NC>(p, L, f_cur, f_next, wv, pw, beg, end);
}

// Dense block of a pull level (32 words, the block's word l in lane l): the
// warp finishes its words PULL_WPI at a time.  Warp-uniform.
template <bool NC>
__device__ __forceinline__ void pull_block_pairs(const Params1& p, LevelCtx& L, const uint32_t* f_cur,
                                                 uint32_t* f_next, long long bi, long long S, unsigned pwl) {
    const unsigned lane = lane_id();
    const long long wl = bi + lane * S;
    if (wl < p.W && pwl == 0xffffffffu) f_next[wl] = 0;
    unsigned todo = __ballot_sync(0xffffffffu, pwl != 0xffffffffu);
    while (todo) {
        long long wv[PULL_WPI];
        unsigned pw[PULL_WPI];
#pragma unroll
        for (int k = 0; k < PULL_WPI; ++k) {
            const int wi = todo ? __ffs(todo) - 1 : -1;
            if (todo) todo &= todo - 1;
            pw[k] = __shfl_sync(0xffffffffu, pwl, wi < 0 ? 0 : wi);
            if (wi < 0) pw[k] = 0xffffffffu;
            wv[k] = wi < 0 ? -1 : bi + wi * S;
        }
        pull_words<NC>(p, L, f_cur, f_next, wv, pw);
    }
}

// Sparse block of a pull level (same ANY reading as pull_block_pairs): the
// lanes take the unvisited vertices of the block in ascending order and each
// lane runs its scans as a pipeline of one memory step per iteration:
//   bounds  csc_ptr[v], csc_ptr[v+1]
//   first   csc_col[j]
//   test    the F_i word of the current in-neighbour, and csc_col[j+1]
// so a lane whose scan ends (hit, row exhausted) takes the next vertex at
// once instead of idling until the slowest lane of its word finishes.  After
// `pull_serial` tested entries a row is deferred to the block's long-row list,
// scanned by the whole warp 32 entries at a time.  New bits of the block's
// words collect in shared memory; the warp then writes its words of F_{i+1}
// and P with plain stores (it owns them).


// Position of the r-th (0-based) set bit of m; m must have more than r bits set.
__device__ __forceinline__ int nth_set_bit(unsigned m, int r) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const unsigned lo = m & ((1u << s) - 1u);
        const int c = __popc(lo);
        if (r >= c) {
            r -= c;
            m >>= s;
            pos += s;
        } else {
            m = lo;
        }
    }
    return pos;
}

// Record a vertex found by a pull scan (parent u).  Any lane, any time.
__device__ __forceinline__ void pull_found(const Params1& p, LevelCtx& L, unsigned* nb, int slot, int v, int u,
                                           int b0, int e) {
    atomicOr(nb + slot, 1u << (v & 31));
    L.depth[v] = L.level + 1;
    if (L.parent) L.parent[v] = u;
    L.ef += (unsigned long long)(p.symmetric ? (e - b0) : (__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v)));
    L.cnt += 1;
}

// The deferred rows of the block, each scanned by the whole warp.  Warp-uniform.
template <bool NC>
__device__ __forceinline__ void pull_long_rows(const Params1& p, LevelCtx& L, PullWarpSmem& ws, unsigned* nb,
                                               const uint32_t* f_cur) {
    __syncwarp();
    const int nl = min(ws.nl, 32);
    const unsigned lane = lane_id();
    for (int r = 0; r < nl; ++r) {
        const int v = ws.lv[r], jl = ws.lj[r], el = ws.le[r], bl = ws.lb[r];
        // PULL_LONG_U x 32 entries a step: every column load, then every
        // frontier test, then the first hit in row order
        int hit = -1;
        for (int base = jl; base < el && hit < 0; base += 32 * PULL_LONG_U) {
            int uu[PULL_LONG_U];
            unsigned fw[PULL_LONG_U];
#pragma unroll
            for (int q = 0; q < PULL_LONG_U; ++q) {
                const int idx = base + q * 32 + (int)lane;
                uu[q] = idx < el ? __ldg(p.csc_col + idx) : -1;
            }
#pragma unroll
            for (int q = 0; q < PULL_LONG_U; ++q) fw[q] = uu[q] >= 0 ? ld_word<NC>(f_cur, uu[q] >> 5) : 0u;
#pragma unroll
            for (int q = 0; q < PULL_LONG_U; ++q) {
                const unsigned hb = __ballot_sync(0xffffffffu, uu[q] >= 0 && ((fw[q] >> (uu[q] & 31)) & 1u));
                if (hb && hit < 0) hit = __shfl_sync(0xffffffffu, uu[q], __ffs(hb) - 1);
            }
        }
        if (hit >= 0 && lane == 0) pull_found(p, L, nb, ws.ls[r], v, hit, bl, el);
    }
    __syncwarp();
    if (lane == 0) ws.nl = 0;
    __syncwarp();
}

constexpr int PULL_SLOTS = 2;         // vertices a lane scans at once in a sparse block (3 or 4: slower)
constexpr int PULL_SPARSE_MAX = 128;  // unvisited vertices (of 1024) up to which a block is sparse

// Pull level (Section 5, loop order d -> s).  Warps take blocks of 32 words
// of P (1024 vertices) round-robin; block b holds the words b + l * S
// (l = 0..31, S = the number of blocks), so each block samples the whole
// vertex range and a cluster of costly vertices (consecutive ids in a
// bandwidth-reducing order such as Reverse Cuthill-McKee) is spread over many
// warps instead of landing on a few.  A block with many unvisited vertices,
// where most scans end at their first entries, is finished two words at a
// time (pull_block_pairs: few instructions per vertex); a block with few
// runs the lane pipeline below, which keeps every lane busy on the long
// scans that dominate late levels.  |F_{i+1}| and e_f are counted in
// registers.  NC selects non-coherent loads of P and F_i, valid when no other
// CTA writes them during the kernel (the graph-mode kernel); the persistent
// kernel uses ordinary loads ordered by its grid barrier.
// The unvisited vertices of the block whose word l (P word pwl) is in lane
// l: per lane um = ~pwl, excl = unvisited vertices in the words before its
// own; returns U, their number in the block.  Warp-uniform.
__device__ __forceinline__ int pull_block_census(unsigned pwl, unsigned& um, int& excl) {
    um = ~pwl;
    const int c = __popc(um);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane_id() >= o) incl += y;
    }
    excl = incl - c;
    return __shfl_sync(0xffffffffu, incl, 31);
}

// Sparse block: the lane pipeline described above.  Warp-uniform.
template <bool NC>
__device__ __forceinline__ void pull_block_sparse(const Params1& p, LevelCtx& L, const uint32_t* f_cur,
                                                  uint32_t* f_next, PullWarpSmem& ws, long long bi, long long S,
                                                  long long wl, unsigned pwl, unsigned um, int excl, int U) {
    constexpr unsigned FULL = 0xffffffffu;
    enum { IDLE = 0, BOUNDS = 1, FIRST = 2, TEST = 3 };
    const unsigned lane = lane_id();
    const int serial = max(1, min(p.pull_serial, PULL_SERIAL_MAX));
    {
        ws.nb[lane] = 0;
        if (lane == 0) ws.nl = 0;
        __syncwarp();
        int next = 0;  // unvisited vertices of the block handed out (warp-uniform)
        int st[PULL_SLOTS], v[PULL_SLOTS], j[PULL_SLOTS], e[PULL_SLOTS], b0[PULL_SLOTS], u[PULL_SLOTS],
            tried[PULL_SLOTS], sl[PULL_SLOTS];
#pragma unroll
        for (int q = 0; q < PULL_SLOTS; ++q) {
            st[q] = IDLE;
            v[q] = j[q] = e[q] = b0[q] = u[q] = tried[q] = sl[q] = 0;
        }
        // every iteration advances each busy slot by one step; a vertex takes
        // at most serial + 2 steps of its slot before it ends or is deferred
        const long long guard = (long long)U * (serial + 3) + 2;
        for (long long it = 0;; ++it) {
            // idle slots take the next unvisited vertices (ascending)
#pragma unroll
            for (int q = 0; q < PULL_SLOTS; ++q) {
                const unsigned idle = __ballot_sync(FULL, st[q] == IDLE);
                if (idle != 0 && next < U) {
                    const int k = next + __popc(idle & lanemask_lt());
                    int lo = 0;  // word of the k-th unvisited vertex: largest i with excl_i <= k
#pragma unroll
                    for (int s2 = 16; s2 > 0; s2 >>= 1) {
                        const int ex = __shfl_sync(FULL, excl, (lo + s2) & 31);
                        if (lo + s2 < 32 && ex <= k) lo += s2;
                    }
                    const unsigned umw = __shfl_sync(FULL, um, lo);
                    const int exw = __shfl_sync(FULL, excl, lo);
                    if (st[q] == IDLE && k < U) {
                        v[q] = (int)((bi + lo * S) * 32 + nth_set_bit(umw, k - exw));
                        sl[q] = lo;
                        st[q] = BOUNDS;
                        tried[q] = 0;
                    }
                    next = min(U, next + __popc(idle));
                }
            }
            bool busy = false;
#pragma unroll
            for (int q = 0; q < PULL_SLOTS; ++q) busy |= st[q] != IDLE;
            if (!__any_sync(FULL, busy)) break;
            if (it > guard) {  // cannot happen; stop rather than spin
                if (lane == 0) atomicCAS(&p.ctl->bar.err, 0, (int)DEV_OVERFLOW);
                break;
            }
            // one memory step per busy slot, all issued before any is used
            unsigned x1[PULL_SLOTS], x2[PULL_SLOTS];
#pragma unroll
            for (int q = 0; q < PULL_SLOTS; ++q) {
                x1[q] = 0;
                x2[q] = 0;
                if (st[q] == BOUNDS) {
                    x1[q] = (unsigned)__ldg(p.csc_ptr + v[q]);
                    x2[q] = (unsigned)__ldg(p.csc_ptr + v[q] + 1);
                } else if (st[q] == FIRST) {
                    x1[q] = (unsigned)__ldg(p.csc_col + j[q]);
                } else if (st[q] == TEST) {
                    x1[q] = ld_word<NC>(f_cur, u[q] >> 5);
                    if (j[q] + 1 < e[q]) x2[q] = (unsigned)__ldg(p.csc_col + j[q] + 1);
                }
            }
            bool defer[PULL_SLOTS];
#pragma unroll
            for (int q = 0; q < PULL_SLOTS; ++q) {
                defer[q] = false;
                if (st[q] == BOUNDS) {
                    b0[q] = (int)x1[q];
                    j[q] = b0[q];
                    e[q] = (int)x2[q];
                    st[q] = (j[q] < e[q]) ? FIRST : IDLE;
                } else if (st[q] == FIRST) {
                    u[q] = (int)x1[q];
                    st[q] = TEST;
                } else if (st[q] == TEST) {
                    if ((x1[q] >> (u[q] & 31)) & 1u) {
                        pull_found(p, L, ws.nb, sl[q], v[q], u[q], b0[q], e[q]);
                        st[q] = IDLE;
                    } else if (++j[q] >= e[q]) {
                        st[q] = IDLE;
                    } else {
                        u[q] = (int)x2[q];
                        defer[q] = ++tried[q] >= serial;
                    }
                }
            }
            // long rows go to the block's list; a full list is drained first
#pragma unroll
            for (int q = 0; q < PULL_SLOTS; ++q) {
                const unsigned dm = __ballot_sync(FULL, defer[q]);
                if (dm) {
                    if (ws.nl + __popc(dm) > 32) pull_long_rows<NC>(p, L, ws, ws.nb, f_cur);
                    if (defer[q]) {
                        const int slot = ws.nl + __popc(dm & lanemask_lt());
                        ws.lv[slot] = v[q];
                        ws.lj[slot] = j[q];
                        ws.le[slot] = e[q];
                        ws.lb[slot] = b0[q];
                        ws.ls[slot] = sl[q];
                        st[q] = IDLE;
                    }
                    __syncwarp();
                    if (lane == 0) ws.nl += __popc(dm);
                    __syncwarp();
                }
            }
        }
        pull_long_rows<NC>(p, L, ws, ws.nb, f_cur);
        if (wl < p.W) {
            const unsigned nb = ws.nb[lane];
            f_next[wl] = nb;
            if (nb) p.P[wl] = pwl | nb;
        }
        __syncwarp();
    }
}

template <bool NC>
__device__ __forceinline__ void pull_level(const Params1& p, LevelCtx& L, const uint32_t* f_cur, uint32_t* f_next,
                                           PullWarpSmem& ws) {
    const unsigned lane = lane_id();
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long S = (p.W + 31) >> 5;
    for (long long bi = gwarp; bi < S; bi += nwarps) {
        const long long wl = bi + lane * S;
        const unsigned pwl = wl < p.W ? ld_word<NC>(p.P, wl) : 0xffffffffu;
        unsigned um;
        int excl;
        const int U = pull_block_census(pwl, um, excl);
        if (U == 0) {  // warp-uniform: every vertex of the block is visited
            if (wl < p.W) f_next[wl] = 0;
        } else if (U > PULL_SPARSE_MAX) {
            pull_block_pairs<NC>(p, L, f_cur, f_next, bi, S, pwl);
        } else {
            pull_block_sparse<NC>(p, L, f_cur, f_next, ws, bi, S, wl, pwl, um, excl, U);
        }
    }
}

// Listed vertices a lane scans at once in the list-driven pull (1 and 4
// measured slower on RMAT, ER and BA).
constexpr int PULL_LPI = 2;

// Scans of up to PULL_LPI listed vertices per lane (v < 0: none), as in
// pull_words_scan: ascending in-neighbours, the first one in F_i is the
// parent; rows still open after `serial` entries are finished by the whole
// warp, 4 x 32 entries a step.  Found vertices set their bit in the slot's
// shared-memory word nb[sl].  Warp-uniform.
template <bool NC>
__device__ __forceinline__ void pull_list_scan(const Params1& p, LevelCtx& L, unsigned* nb, const uint32_t* f_cur,
                                               const int (&v)[PULL_LPI], const int (&sl)[PULL_LPI], int serial) {
    const unsigned lane = lane_id();
    int beg[PULL_LPI], end[PULL_LPI], j[PULL_LPI], par[PULL_LPI];
    bool found[PULL_LPI];
#pragma unroll
    for (int q = 0; q < PULL_LPI; ++q) {
        beg[q] = v[q] >= 0 ? __ldg(p.csc_ptr + v[q]) : 0;
        end[q] = v[q] >= 0 ? __ldg(p.csc_ptr + v[q] + 1) : 0;
        j[q] = beg[q];
        par[q] = -1;
        found[q] = false;
    }
    // software-pipelined scan: each step tests the current entry's F_i word
    // and loads the next entry, so a step costs one memory round trip (two
    // or four entries a step measured no faster)
    int u[PULL_LPI];
#pragma unroll
    for (int q = 0; q < PULL_LPI; ++q) u[q] = j[q] < end[q] ? __ldg(p.csc_col + j[q]) : -1;
    for (int step = 0; step < serial; ++step) {
        unsigned fw[PULL_LPI];
        int un[PULL_LPI];
        bool live = false;
#pragma unroll
        for (int q = 0; q < PULL_LPI; ++q) {
            live |= u[q] >= 0;
            fw[q] = u[q] >= 0 ? ld_word<NC>(f_cur, u[q] >> 5) : 0u;
            un[q] = (u[q] >= 0 && j[q] + 1 < end[q] && step + 1 < serial) ? __ldg(p.csc_col + j[q] + 1) : -1;
        }
        if (!live) break;
#pragma unroll
        for (int q = 0; q < PULL_LPI; ++q) {
            if (u[q] < 0) continue;
            if ((fw[q] >> (u[q] & 31)) & 1u) {
                found[q] = true;
                par[q] = u[q];
                u[q] = -1;
            } else {
                ++j[q];
                u[q] = un[q];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PULL_LPI; ++q) {
        unsigned rm = __ballot_sync(0xffffffffu, v[q] >= 0 && !found[q] && j[q] < end[q]);
        while (rm) {
            const int l = __ffs(rm) - 1;
            const int bl = __shfl_sync(0xffffffffu, j[q], l);
            const int el = __shfl_sync(0xffffffffu, end[q], l);
            int hit = -1;
            for (int base = bl; base < el && hit < 0; base += 128) {
                int uu[4];
                unsigned fw[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int idx = base + t * 32 + (int)lane;
                    uu[t] = idx < el ? __ldg(p.csc_col + idx) : -1;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) fw[t] = uu[t] >= 0 ? ld_word<NC>(f_cur, uu[t] >> 5) : 0u;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const unsigned hb = __ballot_sync(0xffffffffu, uu[t] >= 0 && ((fw[t] >> (uu[t] & 31)) & 1u));
                    if (hb && hit < 0) hit = __shfl_sync(0xffffffffu, uu[t], __ffs(hb) - 1);
                }
            }
            if ((int)lane == l && hit >= 0) {
                found[q] = true;
                par[q] = hit;
            }
            rm &= rm - 1;
        }
        if (found[q]) {
            atomicOr(nb + sl[q], 1u << (v[q] & 31));
            L.depth[v[q]] = L.level + 1;
            if (L.parent) L.parent[v[q]] = par[q];
            L.ef += (unsigned long long)(p.symmetric ? (end[q] - beg[q])
                                                     : (__ldg(p.row_ptr + v[q] + 1) - __ldg(p.row_ptr + v[q])));
            L.cnt += 1;
        }
    }
}

// Vertex of round-list entry e (slot = warp * 32 + lane of the word's owner,
// bit) in round r.
__device__ __forceinline__ int pull_list_vertex(int e, long long r, long long G, long long S) {
    const int s2 = e >> 5;
    const long long w = r + (long long)(s2 >> 5) * G + (long long)(s2 & 31) * S;
    return (int)(w * 32 + (e & 31));
}

// Pull level of the persistent kernel, driven by a list of the unvisited
// vertices (Section 5, loop order d -> s).  Blocks of 32 words of P are
// strided over the vertex range as in pull_level (block b = words b + l * S,
// so a cluster of costly vertices is spread over many CTAs); CTA c owns the
// blocks c, c + G, c + 2G, ... (G CTAs), one per warp per round.  In each
// round every warp reads its block's 32 words and appends their unvisited
// vertices to the CTA's list in shared memory; the warps then drain the list
// 32 * PULL_LPI entries at a time, so every lane scans a vertex that is
// still open, however sparse the words are, and the cost of a dense block is
// spread over all the CTA's warps.  New bits collect in shared memory per
// word and are stored with plain stores by the word's owner after the round.
// `lst` holds T * 32 entries.  Block-uniform.
template <bool NC, int T>
__device__ void pull_level_list(const Params1& p, LevelCtx& L, const uint32_t* f_cur, uint32_t* f_next,
                                PullListSmem<T>& ls, uint16_t* lst) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NW = T / 32;
    static_assert(T * 32 <= 65536, "16-bit list entries");
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const long long S = (p.W + 31) >> 5;
    const long long G = gridDim.x;
    const int serial = max(1, min(p.pull_serial, PULL_SERIAL_MAX));
    for (long long r = blockIdx.x; r < S; r += G * NW) {  // CTA-uniform
        if (threadIdx.x == 0) {
            ls.n = 0;
            ls.next = 0;
        }
        __syncthreads();
        const long long bi = r + (long long)warp * G;
        const long long wl = bi + (long long)lane * S;
        const bool own = bi < S && wl < p.W;
        const unsigned pwl = own ? ld_word<NC>(p.P, wl) : FULL;
        const int slot = (int)(warp * 32 + lane);
        ls.nb[slot] = 0;
        unsigned um = ~pwl;
        const int c = __popc(um);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const int tot = __shfl_sync(FULL, incl, 31);
        int base = 0;
        if (lane == 0 && tot) base = atomicAdd(&ls.n, tot);
        int k = __shfl_sync(FULL, base, 0) + incl - c;
        while (um) {
            const int b = __ffs(um) - 1;
            um &= um - 1;
            lst[k++] = (uint16_t)(slot * 32 + b);
        }
        __syncthreads();
        const int n = ls.n;
        for (;;) {  // warp-uniform
            int k0 = 0;
            if (lane == 0) k0 = atomicAdd(&ls.next, 32 * PULL_LPI);
            k0 = __shfl_sync(FULL, k0, 0);
            if (k0 >= n) break;
            int v[PULL_LPI], sl[PULL_LPI];
#pragma unroll
            for (int q = 0; q < PULL_LPI; ++q) {
                const int idx = k0 + q * 32 + (int)lane;
                v[q] = -1;
                sl[q] = 0;
                if (idx < n) {
                    const int e = lst[idx];
                    v[q] = pull_list_vertex(e, r, G, S);
                    sl[q] = e >> 5;
                }
            }
            pull_list_scan<NC>(p, L, ls.nb, f_cur, v, sl, serial);
        }
        __syncthreads();
        if (own) {
            const unsigned nb = ls.nb[slot];
            f_next[wl] = nb;
            if (nb) p.P[wl] = pwl | nb;
        }
    }
}

// ------------------------------------------------------------ conversions
// Variant 6 (BFS_SORT_DEVICE): F_i's bitmap -> queue in ascending vertex
// order over the whole device.  CTA b owns words [b W / G, (b+1) W / G).
// Phase 1 counts the frontier vertices of each CTA's range into cta_cnt[b];
// after a grid barrier, phase 2 places each range at the sum of the counts
// before it and writes its vertices in order (no atomics: the ranges are
// disjoint).  With units set, chunk units of big rows are appended as in
// bitmap_to_queue.
__device__ __forceinline__ void sort_range(const Params1& p, long long& lo, long long& hi) {
    lo = (long long)blockIdx.x * p.W / gridDim.x;
    hi = (long long)(blockIdx.x + 1) * p.W / gridDim.x;
}

template <int T>
__device__ void sort_count(const Params1& p, TileSmem<T>& sm, const uint32_t* f_cur) {
    long long lo, hi;
    sort_range(p, lo, hi);
    int c = 0;
    for (long long w = lo + threadIdx.x; w < hi; w += T) c += __popc(__ldcg(f_cur + w));
    int total;
    block_exclusive_scan(c, sm.scan_tmp, &total);
    if (threadIdx.x == 0) p.cta_cnt[blockIdx.x] = (unsigned)total;
}

template <int T>
__device__ void sort_emit(const Params1& p, TileSmem<T>& sm, const uint32_t* f_cur, int4* q_cur, int2* u_cur,
                          Counters* cur, bool units) {
    long long lo, hi;
    sort_range(p, lo, hi);
    unsigned long long before = 0;
    for (unsigned b = threadIdx.x; b < blockIdx.x; b += T) before += __ldcg(p.cta_cnt + b);
    before = warp_sum(before);
    if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = before;
    __syncthreads();
    unsigned long long base = 0;
    for (int i = 0; i < T / 32; ++i) base += sm.red[i];
    for (long long wb = lo; wb < hi; wb += T) {  // CTA-uniform
        const long long w = wb + threadIdx.x;
        unsigned fw = w < hi ? __ldcg(f_cur + w) : 0u;
        int total;
        const int off = block_exclusive_scan(__popc(fw), sm.scan_tmp, &total);
        int r = 0;
        while (fw) {
            const int b = __ffs(fw) - 1;
            fw &= fw - 1;
            const int v = (int)(w * 32 + b);
            const int rb = __ldg(p.row_ptr + v), re = __ldg(p.row_ptr + v + 1);
            q_cur[base + off + r++] = make_int4(v, rb, re, 0);
            if (units && re - rb >= p.chunk) emit_units(p, u_cur, cur, v, re - rb);
        }
        base += (unsigned long long)total;
    }
}

// F_i bitmap -> queue Q_i (ascending vertex order inside each CTA chunk) and
// chunk units for its big rows.  Cursor: cur->conv.
template <int T>
__device__ void bitmap_to_queue(const Params1& p, TileSmem<T>& sm, const uint32_t* f_cur, int4* q_cur, int2* u_cur,
                                Counters* cur) {
    for (long long wb = (long long)blockIdx.x * T; wb < p.W; wb += (long long)gridDim.x * T) {
        long long w = wb + threadIdx.x;
        unsigned fw = w < p.W ? __ldcg(f_cur + w) : 0u;
        int c = __popc(fw), total;
        int off = block_exclusive_scan(c, sm.scan_tmp, &total);
        if (threadIdx.x == 0 && total) sm.base = atomicAdd(&cur->conv, (unsigned long long)total);
        __syncthreads();
        unsigned long long base = sm.base;
        int r = 0;
        while (fw) {
            int b = __ffs(fw) - 1;
            fw &= fw - 1;
            const int v = (int)(w * 32 + b);
            const int rb = __ldg(p.row_ptr + v), re = __ldg(p.row_ptr + v + 1);
            q_cur[base + off + r++] = make_int4(v, rb, re, 0);
            if (re - rb >= p.chunk) emit_units(p, u_cur, cur, v, re - rb);
        }
        __syncthreads();
    }
}

}  // namespace bfsgb
