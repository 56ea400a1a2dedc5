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
    int32_t force_dir;  // >= 0: every level uses this form (level profiling)
    float alpha, beta, gamma;
    const int8_t* schedule;
    int32_t schedule_len;
    const float* mlp;
    int32_t deg_max;
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
        case BFS_POLICY_MLP:
            if (p.mlp) {
                // warp 0 evaluates; result broadcast through shared memory
                if (threadIdx.x < 32) {
                    if (threadIdx.x == 0)
                        policy_features(s_feat, f, e_f, m_u, f_prev, level, prev_dir, p.n, p.m, p.deg_max);
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

// Chunk units of the big rows among a warp's claims: one atomic per warp.
// Warp-uniform call.
__device__ __forceinline__ void emit_units_warp(const Params1& p, int2* u_out, Counters* c, bool big, int v, int deg) {
    const unsigned bm = __ballot_sync(0xffffffffu, big);
    if (!bm) return;
    const unsigned lane = lane_id();
    int nch = big ? (deg + p.chunk - 1) / p.chunk : 0;
    int incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&c->u_len, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + total > (unsigned long long)p.ucap) {
        if (lane == 0) atomicCAS(&p.ctl->bar.err, 0, (int)DEV_OVERFLOW);
        return;
    }
    const unsigned long long off = base + (incl - nch);
    for (int k = 0; k < nch; ++k) u_out[off + k] = make_int2(v, k);
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
    }
    L.qn += c;
    emit_units_warp(p, L.u_next, L.next, claimed && deg >= p.chunk, v, deg);
}

// Push candidate (u -> v): claim v in P if not yet visited.  Warp-uniform.
__device__ __forceinline__ void push_candidate(const Params1& p, LevelCtx& L, bool has, int v, int u) {
    bool want = false;
    unsigned w = 0, bit = 0;
    if (has) {
        w = (unsigned)v >> 5;
        bit = 1u << (v & 31);
        want = !(p.P[w] & bit);  // may be stale (bits only grow): the OR decides
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
    emit(p, L, claimed, v, u, claimed ? re - rb : 0);
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
    // queue tiles hold about f / gridDim vertices (at most T), so that a small
    // frontier is spread over every CTA instead of a few full tiles
    long long per_tile = (f + gridDim.x - 1) / gridDim.x;
    per_tile = per_tile < 1 ? 1 : (per_tile > T ? T : per_tile);
    long long ntiles;
    if (dir == BFS_DIR_PUSH_QUEUE) ntiles = (f + per_tile - 1) / per_tile;
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
                long long q = t * per_tile + threadIdx.x;
                if (threadIdx.x < per_tile && q < f) u = __ldcg(q_cur + q);
            } else {
                long long w = t * (T / 32) + (threadIdx.x >> 5);
                if (w < p.W) {
                    unsigned fw = f_cur[w];
                    if ((fw >> (threadIdx.x & 31)) & 1u) u = (int)(w * 32 + (threadIdx.x & 31));
                }
            }
            push_tile<T>(p, L, sm, u, units_valid);
        }
    }
    flush_qbuf(L);
}

// ------------------------------------------------------------ pull level
constexpr int PULL_SERIAL_MAX = 32;  // row entries one lane scans before its warp takes over

template <bool NC>
__device__ __forceinline__ unsigned ld_word(const uint32_t* a, long long i) {
    return NC ? __ldg(a + i) : a[i];
}

// Pull level (Section 5, loop order d -> s): one warp per 32-vertex word of P
// (lane = vertex); warps take blocks of 32 words round-robin.  An
// unvisited lane scans its in-neighbours in ascending order and stops at the
// first one in F_i (ANY = the lowest-index frontier neighbour); rows longer
// than `pull_serial` entries are finished by the whole warp 32 entries at a
// time.  The warp writes the word of P and of F_{i+1} with plain stores (it
// owns the word) and counts |F_{i+1}| and e_f in registers.  NC selects
// non-coherent loads of P and F_i, valid when no other CTA writes them during
// the kernel (the graph-mode kernel); the persistent kernel uses ordinary
// loads ordered by its grid barrier.
template <bool NC>
__device__ __forceinline__ void pull_level_words(const Params1& p, LevelCtx& L, const uint32_t* f_cur,
                                                 uint32_t* f_next) {
    const unsigned lane = lane_id();
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int dnext = L.level + 1;
    const int serial = min(p.pull_serial, PULL_SERIAL_MAX);
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // each warp reads 32 words of P at once; fully visited words get an empty
    // F_{i+1} word, the others are finished two at a time
    for (long long wb = gwarp * 32; wb < p.W; wb += nwarps * 32) {
        const long long wl = wb + lane;
        const unsigned pwl = wl < p.W ? ld_word<NC>(p.P, wl) : 0xffffffffu;
        if (wl < p.W && pwl == 0xffffffffu) f_next[wl] = 0;
        unsigned todo = __ballot_sync(0xffffffffu, pwl != 0xffffffffu);
        while (todo) {
            int wi[2];
            unsigned pw[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                wi[k] = todo ? __ffs(todo) - 1 : -1;
                if (todo) todo &= todo - 1;
                pw[k] = __shfl_sync(0xffffffffu, pwl, wi[k] < 0 ? 0 : wi[k]);
                if (wi[k] < 0) pw[k] = 0xffffffffu;
            }
            bool unvis[2], found[2];
            int beg[2], end[2], j[2], par[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                unvis[k] = !((pw[k] >> lane) & 1u);
                const long long v = (wb + wi[k]) * 32 + lane;
                beg[k] = unvis[k] ? __ldg(p.csc_ptr + v) : 0;
                end[k] = unvis[k] ? __ldg(p.csc_ptr + v + 1) : 0;
                j[k] = beg[k];
                found[k] = false;
                par[k] = -1;
            }
            // ascending scans of both rows advance together
            for (int step = 0; step < serial; ++step) {
                int u[2];
                bool live = false;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const bool lk = !found[k] && j[k] < end[k];
                    u[k] = lk ? __ldg(p.csc_col + j[k]) : -1;
                    live |= lk;
                }
                if (!live) break;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (u[k] >= 0) {
                        if ((ld_word<NC>(f_cur, u[k] >> 5) >> (u[k] & 31)) & 1u) {
                            found[k] = true;
                            par[k] = u[k];
                        } else {
                            ++j[k];
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (wi[k] < 0) break;  // warp-uniform
                unsigned rm = __ballot_sync(0xffffffffu, unvis[k] && !found[k] && j[k] < end[k]);
                while (rm) {
                    const int l = __ffs(rm) - 1;
                    const int bl = __shfl_sync(0xffffffffu, j[k], l);
                    const int el = __shfl_sync(0xffffffffu, end[k], l);
                    int hit = -1;
                    for (int base = bl; base < el; base += 32) {
                        const int idx = base + (int)lane;
                        int uu = 0;
                        bool h = false;
                        if (idx < el) {
                            uu = __ldg(p.csc_col + idx);
                            h = (ld_word<NC>(f_cur, uu >> 5) >> (uu & 31)) & 1u;
                        }
                        const unsigned hb = __ballot_sync(0xffffffffu, h);
                        if (hb) {
                            hit = __shfl_sync(0xffffffffu, uu, __ffs(hb) - 1);
                            break;
                        }
                    }
                    if ((int)lane == l && hit >= 0) {
                        found[k] = true;
                        par[k] = hit;
                    }
                    rm &= rm - 1;
                }
                const long long w = wb + wi[k];
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
