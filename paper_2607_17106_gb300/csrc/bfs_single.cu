// bfs_single.cu -- single-source level-synchronous BFS (Cascade 1) on one GPU.
//
// One level computes F_{i+1} = (G x F_i) masked by NOT P_i (Eq. advance) and
// P_{i+1} = P_i OR F_{i+1} (Eq. update).  Three traversal forms are built:
//
//   push-queue  : loop order s -> d over a sparse int32 queue frontier
//   push-bitmap : the same, frontier read from the dense bitmap in vertex order
//   pull        : loop order d -> s (Section 5): every unvisited d scans its
//                 in-neighbours in ascending order and stops at the first one
//                 in F_i (the ANY reduction of Eq. advance)
//
// Claiming (push): the visited bitmap P is both the mask NOT P_i and the
// update target.  A candidate d first reads its P word; if the bit is clear it
// ORs the bit in (one atomicOr per distinct word per warp when
// claim_aggregate is on: lanes are grouped by word with match-any and the
// group's bits are OR-reduced).  The OR's return value names exactly one
// claimer, which alone writes depth/parent (no atomics on depth, cf. the
// paper's ping-pong Depths variants 11/12: P_i is only read, P_{i+1} only
// grows) and appends d to the next queue.
//
// Pull levels own whole 32-vertex words: a warp handles one word of P, so the
// new bits of P and of F_{i+1} are written with plain stores.
//
// Load balance (push): vertices with degree >= `chunk` are split at claim time
// into chunk-edge units that whole CTAs take round-robin; the rest of
// the frontier is cut into CTA tiles; inside a tile, degree >= `medium` goes
// to a whole warp and smaller rows are flattened over the CTA by a block scan
// of degrees (the flatten/partition mappings of Section 7.2.1).
//
// The whole loop runs in ONE cooperative kernel: levels are separated by a
// grid barrier with a %globaltimer limit, and every CTA evaluates the same
// direction decision from the same device counters, so there is no host
// round trip per level.  The host-loop mode launches the same kernel once per
// level and carries the loop state in device memory.
#include "common.cuh"
#include "policy_dev.cuh"

#include <algorithm>
#include <vector>

namespace bfsgb {

int msbfs_sticky_error(bfs_graph* g);  // msbfs.cu

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
};

void free_ws1(Workspace1* w) {
    if (!w) return;
    cudaFree(w->P);
    for (int i = 0; i < 2; ++i) {
        cudaFree(w->F[i]);
        cudaFree(w->Q[i]);
        cudaFree(w->U[i]);
    }
    cudaFree(w->ctl);
    cudaFree(w->d_sticky);
    cudaFree(w->stage_depth);
    cudaFree(w->stage_parent);
    cudaFree(w->d_log);
    cudaFree(w->d_sched);
    cudaFreeHost(w->h_ctl);
    delete w;
}

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
__device__ int decide_dir(const Params1& p, int level, long long f, long long e_f, long long m_u, long long f_prev,
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
        p.depth[v] = L.level + 1;
        if (p.parent) p.parent[v] = u;
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
            p.depth[v] = dnext;
            if (p.parent) p.parent[v] = u0[k];
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
                    p.depth[rv] = dnext;
                    if (p.parent) p.parent[rv] = par;
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
__device__ void pull_level(const Params1& p, LevelCtx& L, const uint32_t* f_cur, uint32_t* f_next, PullSmem& ps) {
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

// ------------------------------------------------------------ the kernel
template <int T>
__device__ __forceinline__ void bfs1_body(const Params1& p) {
    __shared__ TileSmem<T> sm;
    __shared__ PullSmem s_pull[T / 32];
    __shared__ float s_feat[BFS_MLP_IN];
    __shared__ float s_mlp_out;
    Ctl1* ctl = p.ctl;
    const unsigned nblocks = gridDim.x;
    const long long gtid = (long long)blockIdx.x * T + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * T;

    if (p.do_init) {
        int s = p.src_value;
        for (long long w = gtid; w < p.W; w += gthreads) {
            unsigned bits = __ldg(p.isolated + w);
            if (w == (s >> 5)) bits |= 1u << (s & 31);
            if (w == p.W - 1 && (p.n & 31)) bits |= ~((1u << (p.n & 31)) - 1u);  // phantom vertices
            p.P[w] = bits;
        }
        for (long long v = gtid; v < p.n; v += gthreads) {
            p.depth[v] = (v == s) ? 0 : -1;
            if (p.parent) p.parent[v] = (v == s) ? s : -1;
        }
        if (gtid == 0) {
            int deg = __ldg(p.row_ptr + s + 1) - __ldg(p.row_ptr + s);
            p.Q0[0] = s;
            int nch = deg >= p.chunk ? (deg + p.chunk - 1) / p.chunk : 0;
            for (int c = 0; c < nch; ++c) p.U0[c] = make_int2(s, c);
            ctl->slot[0].q_len = 1;
            ctl->slot[0].u_len = nch;
            ctl->slot[0].e_f = deg;
            ctl->next_level = 0;
            ctl->prev_dir = BFS_DIR_PUSH_QUEUE;
            ctl->bm_valid = -1;
            ctl->q_valid = 0;
            ctl->done = 0;
            ctl->m_u = p.m - deg;
            ctl->f_prev = 0;
        }
        if (!grid_sync(&ctl->bar, nblocks, p.timeout_ns)) return;
    }

    int level = __ldcg(&ctl->next_level);
    int prev_dir = __ldcg(&ctl->prev_dir);
    int bm_valid = __ldcg(&ctl->bm_valid);
    int q_valid = __ldcg(&ctl->q_valid);
    long long m_u = __ldcg(&ctl->m_u);
    long long f_prev = __ldcg(&ctl->f_prev);
    bool done = __ldcg(&ctl->done) != 0;
    int level_end = level + p.level_count;
    const unsigned warp = threadIdx.x >> 5;

    while (!done && level < level_end) {
        Counters* cur = &ctl->slot[level % 3];
        Counters* nxt = &ctl->slot[(level + 1) % 3];
        long long f = (long long)__ldcg(&cur->q_len);
        long long nunits = (long long)__ldcg(&cur->u_len);
        long long e_f = (long long)__ldcg(&cur->e_f);
        if (f == 0) {
            done = true;
            break;
        }
        if (level >= p.max_levels) {
            if (gtid == 0) atomicCAS(&ctl->bar.err, 0, (int)DEV_LEVELS);
            done = true;
            break;
        }
        if (level > 0) m_u -= e_f;
        int dir = decide_dir(p, level, f, e_f, m_u, f_prev, prev_dir, s_feat, &s_mlp_out);
        if (gtid == 0 && p.log && level < p.log_cap) {
            bfs_level_record r;
            r.level = level;
            r.dir = dir;
            r.f = f;
            r.e_f = e_f;
            r.m_u = m_u;
            r.t_ns = (int64_t)globaltimer_ns();
            p.log[level] = r;
        }
        int32_t* q_cur = (level & 1) ? p.Q1 : p.Q0;
        int2* u_cur = (level & 1) ? p.U1 : p.U0;
        uint32_t* f_cur = (level & 1) ? p.F1 : p.F0;
        uint32_t* f_nxt = (level & 1) ? p.F0 : p.F1;
        if (dir != BFS_DIR_PUSH_QUEUE && bm_valid != level) {
            // queue -> bitmap conversion of F_i
            for (long long w = gtid; w < p.W; w += gthreads) f_cur[w] = 0;
            if (!grid_sync(&ctl->bar, nblocks, p.timeout_ns)) return;
            for (long long q = gtid; q < f; q += gthreads) {
                int v = __ldcg(q_cur + q);
                atomicOr(f_cur + (v >> 5), 1u << (v & 31));
            }
            if (!grid_sync(&ctl->bar, nblocks, p.timeout_ns)) return;
            bm_valid = level;
        }
        if (dir == BFS_DIR_PUSH_QUEUE && q_valid != level) {
            // bitmap -> queue conversion of F_i (after pull levels)
            bitmap_to_queue<T>(p, sm, f_cur, q_cur, u_cur, cur);
            if (!grid_sync(&ctl->bar, nblocks, p.timeout_ns)) return;
            nunits = (long long)__ldcg(&cur->u_len);
            q_valid = level;
        }
        if (gtid == 0) {
            Counters* z = &ctl->slot[(level + 2) % 3];
            z->q_len = 0;
            z->u_len = 0;
            z->e_f = 0;
            z->conv = 0;
        }
        LevelCtx L;
        L.level = level;
        L.q_next = (level & 1) ? p.Q0 : p.Q1;
        L.u_next = (level & 1) ? p.U0 : p.U1;
        L.next = nxt;
        L.ef = 0;
        L.cnt = 0;
        L.qbuf = sm.qbuf + warp * QBUF;
        L.qn = 0;
        if (dir == BFS_DIR_PULL) {
            pull_level(p, L, f_cur, f_nxt, s_pull[warp]);
        } else {
            push_level<T>(p, L, sm, dir, q_cur, u_cur, f_cur, f, nunits, q_valid == level);
        }
        // e_f (and |F_{i+1}| for pull) of the next frontier: one atomic per CTA
        unsigned long long ef = warp_sum(L.ef);
        unsigned long long cn = warp_sum(L.cnt);
        if ((threadIdx.x & 31) == 0) sm.red[warp] = ef;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int i = 0; i < T / 32; ++i) t += sm.red[i];
            if (t) atomicAdd(&nxt->e_f, t);
        }
        __syncthreads();
        if (dir == BFS_DIR_PULL) {
            if ((threadIdx.x & 31) == 0) sm.red[warp] = cn;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned long long t = 0;
                for (int i = 0; i < T / 32; ++i) t += sm.red[i];
                if (t) atomicAdd(&nxt->q_len, t);
            }
            bm_valid = level + 1;
        } else {
            q_valid = level + 1;
        }
        prev_dir = dir;
        f_prev = f;
        ++level;
        if (!grid_sync(&ctl->bar, nblocks, p.timeout_ns)) return;
    }
    if (gtid == 0) {
        ctl->next_level = level;
        ctl->prev_dir = prev_dir;
        ctl->bm_valid = bm_valid;
        ctl->q_valid = q_valid;
        ctl->m_u = m_u;
        ctl->f_prev = f_prev;
        ctl->done = done ? 1 : 0;
    }
}

// 64 registers a thread so that 1024 threads fit on an SM with the pull
// level's shared memory (32 warps of memory-level parallelism).
template <int T>
__global__ void __launch_bounds__(T, (1024 / T) > 0 ? (1024 / T) : 1) bfs1_kernel(Params1 p) {
    bfs1_body<T>(p);
    if (threadIdx.x == 0) {
        int e = ld_volatile_i32(&p.ctl->bar.err);
        if (e) atomicCAS(p.sticky, 0, e);
    }
}

// ------------------------------------------------------------- host side
struct LaunchCfg {
    int threads;
    int blocks;
};

template <int T>
cudaError_t launch_bfs1(const Params1& p, int blocks, cudaStream_t st) {
    void* args[] = {(void*)&p};
    return cudaLaunchCooperativeKernel((const void*)bfs1_kernel<T>, dim3(blocks), dim3(T), args, 0, st);
}

template <int T>
int max_coop_blocks(int blocks_per_sm) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs1_kernel<T>, T, 0);
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
    return per_sm * num_sms();
}

__global__ void count_units_kernel(const int32_t* row_ptr, int32_t n, int32_t chunk, unsigned long long* out) {
    unsigned long long s = 0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        int d = row_ptr[v + 1] - row_ptr[v];
        if (d >= chunk) s += (unsigned long long)((d + chunk - 1) / chunk);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

static bfs_status ensure_ws1(bfs_graph* g, int32_t chunk, cudaStream_t st, Workspace1** out) {
    Workspace1* w = g->ws1;
    if (w && w->chunk == chunk) {
        *out = w;
        return BFS_OK;
    }
    if (w) {
        BFS_CUDA(cudaStreamSynchronize(st));
        free_ws1(w);
        g->ws1 = nullptr;
    }
    w = new (std::nothrow) Workspace1();
    if (!w) return fail(BFS_ENOMEM, "host allocation");
    w->n = g->n;
    w->W = div_up(g->n, 32);
    w->chunk = chunk;
    unsigned long long* d_cnt = nullptr;
    unsigned long long units = 0;
    bool ok = cudaMalloc(&d_cnt, 8) == cudaSuccess;
    if (ok) {
        cudaMemsetAsync(d_cnt, 0, 8, st);
        count_units_kernel<<<num_sms() * 8, 256, 0, st>>>(g->row_ptr, g->n, chunk, d_cnt);
        cudaMemcpyAsync(&units, d_cnt, 8, cudaMemcpyDeviceToHost, st);
        ok = cudaStreamSynchronize(st) == cudaSuccess;
        cudaFree(d_cnt);
    }
    w->ucap = (int64_t)units + 1;
    ok = ok && cudaMalloc(&w->P, w->W * 4) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i) {
        ok = cudaMalloc(&w->F[i], w->W * 4) == cudaSuccess && cudaMalloc(&w->Q[i], (int64_t)g->n * 4) == cudaSuccess &&
             cudaMalloc(&w->U[i], w->ucap * sizeof(int2)) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&w->ctl, sizeof(Ctl1)) == cudaSuccess;
    ok = ok && cudaMalloc(&w->d_sticky, 4) == cudaSuccess && cudaMemset(w->d_sticky, 0, 4) == cudaSuccess;
    ok = ok && cudaMallocHost(&w->h_ctl, sizeof(Ctl1)) == cudaSuccess;
    if (!ok) {
        free_ws1(w);
        cudaGetLastError();
        return fail(BFS_ENOMEM, "single-source workspace for n=%d", g->n);
    }
    g->ws1 = w;
    *out = w;
    return BFS_OK;
}

bfs_status device_error(int err, int64_t timeout_ns) {
    if (err == DEV_TIMEOUT) return fail(BFS_ETIMEOUT, "grid barrier wait exceeded %lld ns", (long long)timeout_ns);
    if (err == DEV_OVERFLOW) return fail(BFS_EVALIDATE, "device work list overflow");
    if (err == DEV_LEVELS) return fail(BFS_ERANGE, "level limit exceeded");
    return fail(BFS_EVALIDATE, "device error %d", err);
}

// Waits for the stream and reports (then clears) the first device-side error
// raised by any run on this graph since the last check.
bfs_status sync_graph(bfs_graph* g, cudaStream_t st) {
    BFS_CUDA(cudaStreamSynchronize(st));
    int err = 0;
    if (g->ws1) {
        BFS_CUDA(cudaMemcpy(&err, g->ws1->d_sticky, 4, cudaMemcpyDeviceToHost));
        if (err) BFS_CUDA(cudaMemset(g->ws1->d_sticky, 0, 4));
    }
    if (!err) err = msbfs_sticky_error(g);
    if (err) return device_error(err, 0);
    return BFS_OK;
}

static float flog2(double x) { return (float)std::log2(x); }

// Runs one source (already validated).  Returns after enqueueing unless a
// host readback is needed (host loop, level log, level count); device-side
// failures of asynchronous runs are reported by sync_graph / bfs_sync.
bfs_status run_single(bfs_graph* g, int32_t src_value, int32_t* depth, int32_t* parent, const bfs_options& o,
                      const float* mlp_dev, cudaStream_t st) {
    Workspace1* w;
    bfs_status s = ensure_ws1(g, o.chunk, st, &w);
    if (s != BFS_OK) return s;
    Params1 p{};
    p.n = g->n;
    p.W = w->W;
    p.m = g->m;
    p.symmetric = g->symmetric;
    p.row_ptr = g->row_ptr;
    p.col = g->col;
    p.csc_ptr = g->csc_ptr;
    p.csc_col = g->csc_col;
    p.isolated = g->isolated;
    p.P = w->P;
    p.F0 = w->F[0];
    p.F1 = w->F[1];
    p.Q0 = w->Q[0];
    p.Q1 = w->Q[1];
    p.U0 = w->U[0];
    p.U1 = w->U[1];
    p.ucap = w->ucap;
    p.ctl = w->ctl;
    p.src_value = src_value;
    p.sticky = w->d_sticky;
    p.depth = depth;
    p.parent = parent;
    p.policy = o.policy;
    p.alpha = o.alpha;
    p.beta = o.beta;
    p.gamma = o.gamma;
    p.mlp = mlp_dev;
    p.log_n = flog2((double)g->n);
    p.log_m = flog2(1.0 + (double)g->m);
    p.log_degmax = flog2(1.0 + (double)g->deg_max);
    p.chunk = o.chunk;
    p.medium = o.medium;
    p.pull_serial = o.pull_serial;
    p.aggregate = o.claim_aggregate;
    p.timeout_ns = o.barrier_timeout_ns;
    p.max_levels = o.max_levels > 0 ? o.max_levels : g->n + 1;
    if (o.policy == BFS_POLICY_SCHEDULE) {
        if (!o.schedule || o.schedule_len <= 0) return fail(BFS_EINVAL, "schedule policy needs a schedule");
        if (w->sched_cap < o.schedule_len) {
            cudaFree(w->d_sched);
            w->d_sched = nullptr;
            if (cudaMalloc(&w->d_sched, o.schedule_len) != cudaSuccess) return fail(BFS_ENOMEM, "schedule");
            w->sched_cap = o.schedule_len;
        }
        BFS_CUDA(cudaMemcpyAsync(w->d_sched, o.schedule, o.schedule_len, cudaMemcpyHostToDevice, st));
        p.schedule = w->d_sched;
        p.schedule_len = o.schedule_len;
    }
    if (o.level_log && o.level_log_cap > 0) {
        if (w->log_cap < o.level_log_cap) {
            cudaFree(w->d_log);
            w->d_log = nullptr;
            if (cudaMalloc(&w->d_log, sizeof(bfs_level_record) * o.level_log_cap) != cudaSuccess)
                return fail(BFS_ENOMEM, "level log");
            w->log_cap = o.level_log_cap;
        }
        p.log = w->d_log;
        p.log_cap = o.level_log_cap;
    }
    BFS_CUDA(cudaMemsetAsync(w->ctl, 0, sizeof(Ctl1), st));
    int T = o.block_threads;
    int blocks = 0;
    switch (T) {
        case 256: blocks = max_coop_blocks<256>(o.blocks_per_sm); break;
        case 1024: blocks = max_coop_blocks<1024>(o.blocks_per_sm); break;
        default: T = 512; blocks = max_coop_blocks<512>(o.blocks_per_sm); break;
    }
    auto launch = [&](const Params1& pp) -> cudaError_t {
        switch (T) {
            case 256: return launch_bfs1<256>(pp, blocks, st);
            case 1024: return launch_bfs1<1024>(pp, blocks, st);
            default: return launch_bfs1<512>(pp, blocks, st);
        }
    };
    if (o.mode == BFS_MODE_HOST_LOOP) {
        p.do_init = 1;
        p.level_count = 0;
        BFS_CUDA(launch(p));
        p.do_init = 0;
        p.level_count = 1;
        for (int it = 0;; ++it) {
            BFS_CUDA(launch(p));
            BFS_CUDA(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl1), cudaMemcpyDeviceToHost, st));
            BFS_CUDA(cudaStreamSynchronize(st));
            if (w->h_ctl->done || w->h_ctl->bar.err) break;
        }
    } else {
        p.do_init = 1;
        p.level_count = INT32_MAX / 2;
        BFS_CUDA(launch(p));
    }
    bool need_sync = o.level_log || o.levels_out || o.mode == BFS_MODE_HOST_LOOP;
    if (!need_sync) return BFS_OK;
    BFS_CUDA(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl1), cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    Ctl1& h = *w->h_ctl;
    if (h.bar.err) {
        cudaMemsetAsync(w->d_sticky, 0, 4, st);
        return device_error(h.bar.err, o.barrier_timeout_ns);
    }
    if (o.levels_out) *o.levels_out = h.next_level;
    if (o.level_log && o.level_log_cap > 0) {
        int nl = std::min(h.next_level, o.level_log_cap);
        if (nl > 0) BFS_CUDA(cudaMemcpy(o.level_log, w->d_log, sizeof(bfs_level_record) * nl, cudaMemcpyDeviceToHost));
    }
    return BFS_OK;
}

}  // namespace bfsgb
