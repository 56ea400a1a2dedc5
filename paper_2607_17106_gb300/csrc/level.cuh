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
};

struct Ctl1 {
    GridBarrier bar;
    Counters slot[3];
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
    int32_t* Q[2] = {nullptr, nullptr};
    int2* U[2] = {nullptr, nullptr};
    Ctl1* ctl = nullptr;
    int* d_sticky = nullptr;
    int32_t* stage_depth = nullptr;
    int32_t* stage_parent = nullptr;
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
    int32_t* Q0;
    int32_t* Q1;
    int2* U0;
    int2* U1;
    int64_t ucap;
    Ctl1* ctl;
    int32_t src_value;
    int* sticky;          // first device error of any run, cleared by the host
    int32_t* depth;
    int32_t* parent;
    // policy
    int32_t policy;
    float alpha, beta, gamma;
    const int8_t* schedule;
    int32_t schedule_len;
    const float* mlp;
    float log_n, log_m, log_degmax;
    // tuning
    int32_t chunk, medium, pull_serial, aggregate;
    int64_t timeout_ns;
    int32_t max_levels;
    bfs_level_record* log;
    int32_t log_cap;
    // launch control
    int32_t do_init;
    int32_t level_count;  // levels to run in this launch (host loop: 1)
};

// ------------------------------------------------------------- direction
__device__ __forceinline__ int push_kind(const Params1& p, long long f) {
    return ((double)f * p.gamma > (double)p.n) ? BFS_DIR_PUSH_BITMAP : BFS_DIR_PUSH_QUEUE;
}

// Same inputs on every CTA -> same decision (all arithmetic is deterministic).
__device__ inline int decide_dir(const Params1& p, int level, long long f, long long e_f, long long m_u, long long f_prev,
                          int prev_dir, float* s_feat, float* s_mlp_out) {
    switch (p.policy) {
        case BFS_POLICY_PUSH:
            return push_kind(p, f);
        case BFS_POLICY_PULL:
            return BFS_DIR_PULL;
        case BFS_POLICY_SCHEDULE: {
            int d = p.schedule[level % p.schedule_len];
            return (d < 0 || d > 2) ? BFS_DIR_PUSH_QUEUE : d;
        }
        case BFS_POLICY_MLP:
            if (p.mlp) {
                // warp 0 evaluates; result broadcast through shared memory
                if (threadIdx.x < 32) {
                    if (threadIdx.x == 0)
                        policy_features(s_feat, f, e_f, m_u, level, prev_dir, p.n, p.log_n, p.log_m, p.log_degmax);
                    __syncwarp();
                    int a = policy_argmax_warp(p.mlp, s_feat);
                    if (threadIdx.x == 0) *s_mlp_out = (float)a;
                }
                __syncthreads();
                int a = (int)*s_mlp_out;
                __syncthreads();
                return a;
            }
            // fall through to the heuristic
        default: {
            // Beamer et al. 2012 (cited in Section 5): top-down while the
            // frontier's edges are few relative to the unexplored edges;
            // bottom-up while the frontier is growing or large.
            if (prev_dir == BFS_DIR_PULL) {
                bool stay = (f >= f_prev) || ((double)f * p.beta > (double)p.n);
                return stay ? BFS_DIR_PULL : push_kind(p, f);
            }
            if ((double)e_f * p.alpha > (double)m_u && f > f_prev) return BFS_DIR_PULL;
            return push_kind(p, f);
        }
    }
}

// ------------------------------------------------------------ claiming
constexpr int QBUF = 64;  // per-warp shared-memory staging of next-queue entries

struct LevelCtx {
    int32_t level;          // i: discovered vertices get depth i+1
    int32_t* depth;         // outputs of this run
    int32_t* parent;
    int32_t* q_next;
    int2* u_next;
    Counters* next;         // counters of F_{i+1}
    unsigned long long ef;  // this thread's share of e_f(F_{i+1})
    unsigned long long cnt; // this thread's share of |F_{i+1}| (pull levels)
    int32_t* qbuf;          // this warp's staging buffer (QBUF entries)
    int qn;                 // entries staged (warp-uniform)
};

// Move the warp's staged queue entries to the next queue: one atomic per
// flush instead of one per claiming round.  Warp-uniform.
__device__ __forceinline__ void flush_qbuf(LevelCtx& L) {
    if (L.qn == 0) return;
    unsigned lane = lane_id();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&L.next->q_len, (unsigned long long)L.qn);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    for (int i = (int)lane; i < L.qn; i += 32) L.q_next[base + i] = L.qbuf[i];
    __syncwarp();
    L.qn = 0;
}

__device__ __forceinline__ void emit_units(const Params1& p, int2* u_out, Counters* c, int v, int deg) {
    int nch = (deg + p.chunk - 1) / p.chunk;
    unsigned long long ub = atomicAdd(&c->u_len, (unsigned long long)nch);
    if (ub + nch <= (unsigned long long)p.ucap) {
        for (int k = 0; k < nch; ++k) u_out[ub + k] = make_int2(v, k);
    } else {
        atomicCAS(&p.ctl->bar.err, 0, (int)DEV_OVERFLOW);
    }
}

// Record vertices claimed in a push level: depth/parent, staged next-queue
// slot, degree sum, chunk units for big rows.  Warp-uniform call.
__device__ __forceinline__ void emit(const Params1& p, LevelCtx& L, bool claimed, int v, int u, int deg) {
    unsigned cm = __ballot_sync(0xffffffffu, claimed);
    if (!cm) return;
    int c = __popc(cm);
    if (L.qn + c > QBUF) flush_qbuf(L);
    if (claimed) {
        L.qbuf[L.qn + __popc(cm & lanemask_lt())] = v;
        L.depth[v] = L.level + 1;
        if (L.parent) L.parent[v] = u;
        L.ef += (unsigned long long)deg;
        if (deg >= p.chunk) emit_units(p, L.u_next, L.next, v, deg);
    }
    L.qn += c;
}

// Push candidate (u -> v): claim v in P if not yet visited.  Warp-uniform.
__device__ __forceinline__ void push_candidate(const Params1& p, LevelCtx& L, bool has, int v, int u) {
    bool want = false;
    unsigned w = 0, bit = 0;
    if (has) {
        w = (unsigned)v >> 5;
        bit = 1u << (v & 31);
        want = !(__ldcg(p.P + w) & bit);
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
    int deg = 0;
    if (claimed) deg = __ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v);
    emit(p, L, claimed, v, u, deg);
}

// ------------------------------------------------------------ push tiles
template <int T>
struct TileSmem {
    int off[T + 1];
    int beg[T];
    int src[T];
    int scan_tmp[33];
    int32_t qbuf[(T / 32) * QBUF];
    unsigned long long red[T / 32];
    unsigned long long base;
};

// One CTA expands up to T frontier vertices (one per thread, u < 0 = none).
// Rows of degree >= chunk are skipped when chunk units cover them.
template <int T>
__device__ __forceinline__ void push_tile(const Params1& p, LevelCtx& L, TileSmem<T>& sm, int u, bool skip_big) {
    unsigned lane = lane_id();
    int beg = 0, end = 0;
    if (u >= 0) {
        beg = __ldg(p.row_ptr + u);
        end = __ldg(p.row_ptr + u + 1);
        if (skip_big && end - beg >= p.chunk) end = beg;
    }
    // medium rows: one warp each
    bool med = (end - beg) >= p.medium;
    unsigned mm = __ballot_sync(0xffffffffu, med);
    while (mm) {
        int l = __ffs(mm) - 1;
        int ub = __shfl_sync(0xffffffffu, u, l);
        int bb = __shfl_sync(0xffffffffu, beg, l);
        int ee = __shfl_sync(0xffffffffu, end, l);
        for (int base = bb; base < ee; base += 32) {
            int j = base + (int)lane;
            bool has = j < ee;
            int v = has ? __ldg(p.col + j) : 0;
            push_candidate(p, L, has, v, ub);
        }
        mm &= mm - 1;
    }
    if (med) end = beg;
    // small rows: flatten (u, j) pairs over the CTA
    int deg = end - beg, total;
    int off = block_exclusive_scan(deg, sm.scan_tmp, &total);
    sm.off[threadIdx.x] = off;
    sm.beg[threadIdx.x] = beg;
    sm.src[threadIdx.x] = u;
    if (threadIdx.x == T - 1) sm.off[T] = total;
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
                if (sm.off[mid] <= k) lo = mid; else hi = mid - 1;
            }
            su = sm.src[lo];
            v = __ldg(p.col + sm.beg[lo] + (k - sm.off[lo]));
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

// Push level: items are [chunk units of F_i] then [tiles of the frontier],
// dealt to CTAs round-robin (units are equal-sized; tiles hold rows below
// the chunk size).
template <int T>
__device__ void push_level(const Params1& p, LevelCtx& L, TileSmem<T>& sm, int dir, const int32_t* q_cur,
                           const int2* u_cur, const uint32_t* f_cur, long long f, long long nunits, bool units_valid) {
    long long ntiles;
    if (dir == BFS_DIR_PUSH_QUEUE) ntiles = (f + T - 1) / T;
    else ntiles = (p.W + (T / 32) - 1) / (T / 32);
    if (!units_valid) nunits = 0;
    long long nitems = nunits + ntiles;
    for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
        if (it < nunits) {
            push_unit<T>(p, L, __ldcg(u_cur + it));
        } else {
            long long t = it - nunits;
            int u = -1;
            if (dir == BFS_DIR_PUSH_QUEUE) {
                long long q = t * T + threadIdx.x;
                if (q < f) u = __ldcg(q_cur + q);
            } else {
                long long w = t * (T / 32) + (threadIdx.x >> 5);
                if (w < p.W) {
                    unsigned fw = __ldcg(f_cur + w);
                    if ((fw >> (threadIdx.x & 31)) & 1u) u = (int)(w * 32 + (threadIdx.x & 31));
                }
            }
            push_tile<T>(p, L, sm, u, units_valid);
        }
    }
    flush_qbuf(L);
}

// ------------------------------------------------------------ pull level
constexpr int PULL_ILP = 8;     // words a warp handles per step
constexpr int PULL_BLOCK = 16;  // words of P a warp reads per block
constexpr int PULL_LIST = 32 * PULL_ILP;  // leftover rows of one step (at most every row)

// Per-warp shared memory of the pull level.
struct PullSmem {
    int v[PULL_LIST];     // leftover row: vertex
    int j[PULL_LIST];     //   next position to test
    int end[PULL_LIST];   //   row end
    int off[PULL_LIST + 1];
    unsigned hit[PULL_LIST];  // lowest hit position of this round, ~0u if none
    unsigned word_nb[PULL_ILP];  // found bits per word of the step
};

// One pull step over up to PULL_ILP 32-vertex words (lane = vertex of each
// word).  Phase 1: every unvisited row tests its first in-neighbour, all
// rows' loads in flight together.  Phase 2: rows not yet resolved go to a
// shared-memory list that the warp scans flattened: each round every live row
// contributes up to `pull_serial` entries, a prefix over the list lays the
// entries out over the lanes, and the lowest hit position of a row (a min in
// shared memory) gives its parent.  Phase 3 writes the words of P and F_{i+1}.
__device__ __forceinline__ void pull_step(const Params1& p, LevelCtx& L, const uint32_t* f_cur, uint32_t* f_next,
                                          long long wb, const int (&wi)[PULL_ILP], const unsigned (&pwi)[PULL_ILP],
                                          PullSmem& ps) {
    const unsigned lane = lane_id();
    const int dnext = L.level + 1;
    int beg[PULL_ILP], end[PULL_ILP], u0[PULL_ILP];
#pragma unroll
    for (int k = 0; k < PULL_ILP; ++k) {
        bool unvis = !((pwi[k] >> lane) & 1u);
        long long v = (wb + wi[k]) * 32 + lane;
        beg[k] = unvis ? __ldg(p.csc_ptr + v) : 0;
        end[k] = unvis ? __ldg(p.csc_ptr + v + 1) : 0;
    }
#pragma unroll
    for (int k = 0; k < PULL_ILP; ++k) u0[k] = (beg[k] < end[k]) ? __ldg(p.csc_col + beg[k]) : -1;
    int nlist = 0;
#pragma unroll
    for (int k = 0; k < PULL_ILP; ++k) {
        bool found = u0[k] >= 0 && ((__ldcg(f_cur + (u0[k] >> 5)) >> (u0[k] & 31)) & 1u);
        long long v = (wb + wi[k]) * 32 + lane;
        if (found) {
            L.depth[v] = dnext;
            if (L.parent) L.parent[v] = u0[k];
            int dg = p.symmetric ? end[k] - beg[k] : (__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v));
            L.ef += (unsigned long long)dg;
            L.cnt += 1;
        }
        unsigned nb = __ballot_sync(0xffffffffu, found);
        if (lane == 0) ps.word_nb[k] = nb;
        bool left = u0[k] >= 0 && !found && beg[k] + 1 < end[k];
        unsigned lm = __ballot_sync(0xffffffffu, left);
        if (left) {
            int r = nlist + __popc(lm & lanemask_lt());
            ps.v[r] = (int)v;
            ps.j[r] = beg[k] + 1;
            ps.end[r] = end[k];
        }
        nlist += __popc(lm);
    }
    __syncwarp();
    const int cap = p.pull_serial;
    while (nlist > 0) {
        // contributions and their prefix (rows lane, lane+32, ...)
        int loc = 0;
        for (int r = (int)lane; r < nlist; r += 32) loc += min(ps.end[r] - ps.j[r], cap);
        int incl = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        // per-lane rows are strided, so lay offsets out row by row
        // (prefix in row order = sum over earlier rows): recompute serially
        // per lane group of 32 rows
        int run = 0;
        for (int r0 = 0; r0 < nlist; r0 += 32) {
            int r = r0 + (int)lane;
            int c = r < nlist ? min(ps.end[r] - ps.j[r], cap) : 0;
            int ci = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, ci, o);
                if ((int)lane >= o) ci += y;
            }
            if (r < nlist) {
                ps.off[r] = run + ci - c;
                ps.hit[r] = ~0u;
            }
            run += __shfl_sync(0xffffffffu, ci, 31);
        }
        if (lane == 0) ps.off[nlist] = total;
        __syncwarp();
        for (int e0 = 0; e0 < total; e0 += 32) {
            int x = e0 + (int)lane;
            if (x < total) {
                int lo = 0, hi = nlist - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (ps.off[mid] <= x) lo = mid; else hi = mid - 1;
                }
                int pos = ps.j[lo] + (x - ps.off[lo]);
                int u = __ldg(p.csc_col + pos);
                if ((__ldcg(f_cur + (u >> 5)) >> (u & 31)) & 1u) atomicMin(&ps.hit[lo], (unsigned)pos);
            }
        }
        __syncwarp();
        // resolve rows; keep the live ones (compacted) for the next round
        int keep = 0;
        for (int r0 = 0; r0 < nlist; r0 += 32) {
            int r = r0 + (int)lane;
            bool live = false;
            int rv = 0, rj = 0, re = 0;
            if (r < nlist) {
                rv = ps.v[r];
                rj = ps.j[r];
                re = ps.end[r];
                unsigned h = ps.hit[r];
                if (h != ~0u) {
                    int par = __ldg(p.csc_col + h);
                    L.depth[rv] = dnext;
                    if (L.parent) L.parent[rv] = par;
                    int dg = p.symmetric ? (__ldg(p.csc_ptr + rv + 1) - __ldg(p.csc_ptr + rv))
                                         : (__ldg(p.row_ptr + rv + 1) - __ldg(p.row_ptr + rv));
                    L.ef += (unsigned long long)dg;
                    L.cnt += 1;
                    long long w = rv >> 5;
                    // the word's index within the step
#pragma unroll
                    for (int k = 0; k < PULL_ILP; ++k)
                        if (wi[k] >= 0 && wb + wi[k] == w) atomicOr(&ps.word_nb[k], 1u << (rv & 31));
                } else {
                    rj += min(re - rj, cap);
                    live = rj < re;
                }
            }
            unsigned lm = __ballot_sync(0xffffffffu, live);
            __syncwarp();
            if (live) {
                int q = keep + __popc(lm & lanemask_lt());
                ps.v[q] = rv;
                ps.j[q] = rj;
                ps.end[q] = re;
            }
            keep += __popc(lm);
            __syncwarp();
        }
        nlist = keep;
    }
    __syncwarp();
    if ((int)lane < PULL_ILP && wi[lane] >= 0) {
        long long w = wb + wi[lane];
        unsigned nb = ps.word_nb[lane];
        f_next[w] = nb;
        if (nb) p.P[w] = pwi[lane] | nb;
    }
    __syncwarp();
}

// Pull level: each warp reads PULL_BLOCK words of P with one coalesced load,
// writes F_{i+1} = 0 for the fully visited ones, and handles the others
// PULL_ILP at a time.
__device__ inline void pull_level(const Params1& p, LevelCtx& L, const uint32_t* f_cur, uint32_t* f_next, PullSmem& ps) {
    unsigned lane = lane_id();
    long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long wb = gwarp * PULL_BLOCK; wb < p.W; wb += nwarps * PULL_BLOCK) {
        long long wl = wb + lane;
        bool mine = lane < PULL_BLOCK && wl < p.W;
        unsigned pw = mine ? __ldcg(p.P + wl) : 0xffffffffu;
        if (mine && pw == 0xffffffffu) f_next[wl] = 0;
        unsigned todo = __ballot_sync(0xffffffffu, pw != 0xffffffffu);
        while (todo) {
            int wi[PULL_ILP];
            unsigned pwi[PULL_ILP];
#pragma unroll
            for (int k = 0; k < PULL_ILP; ++k) {
                if (todo) {
                    wi[k] = __ffs(todo) - 1;
                    todo &= todo - 1;
                    pwi[k] = __shfl_sync(0xffffffffu, pw, wi[k]);
                } else {
                    wi[k] = -1;
                    pwi[k] = 0xffffffffu;
                }
            }
            pull_step(p, L, f_cur, f_next, wb, wi, pwi, ps);
        }
    }
}

// ------------------------------------------------------------ conversions
// F_i bitmap -> queue Q_i (ascending vertex order inside each CTA chunk) and
// chunk units for its big rows.  Cursor: cur->conv.
template <int T>
__device__ void bitmap_to_queue(const Params1& p, TileSmem<T>& sm, const uint32_t* f_cur, int32_t* q_cur, int2* u_cur,
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
            int v = (int)(w * 32 + b);
            q_cur[base + off + r++] = v;
            int deg = __ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v);
            if (deg >= p.chunk) emit_units(p, u_cur, cur, v, deg);
        }
        __syncthreads();
    }
}

}  // namespace bfsgb
