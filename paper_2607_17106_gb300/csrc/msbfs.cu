// msbfs.cu -- batched multi-source BFS: up to 64 sources per unit, each
// vertex carrying 64-bit frontier / seen masks (one bit per source lane).
//
// Per lane j this is exactly Cascade 1 for source j; the 64 lanes share every
// read of G.  With seen_i the lanes that reached v before level i and front_i
// the lanes whose frontier holds v:
//   push: for u with front_i[u] != 0, for v in N(u):
//           new = front_i[u] & ~seen[v]; atomicOr(next[v], new)
//   pull: for v with missing = ~seen[v] != 0, OR front_i[u] over in-neighbours
//           u in ascending order, stopping once every missing lane is found
//   then front_{i+1} = next and seen |= next: the three-array identity
//   F_{i+1} = P_{i+1} AND NOT P_i of the paper's variant 26.
// The ANY reduction picks, per lane, the first u (push: the one whose OR set
// the bit; pull: the lowest-index in-neighbour), which is written as parent.
//
// One cooperative kernel runs all levels of all units of a launch: units are
// independent searches (possibly over different graphs: bfs_run_mixed), and
// levels are separated by a grid barrier with a %globaltimer limit.
#include "common.cuh"
#include "policy_dev.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

namespace bfsgb {

struct MsUnit {
    const int32_t* row_ptr;
    const int32_t* col;
    const int32_t* csc_ptr;
    const int32_t* csc_col;
    const uint32_t* isolated;
    int64_t m;
    int32_t n;
    int32_t k;
    int32_t symmetric;
    int32_t deg_max;
    int32_t src[64];
    int32_t* depth[64];
    int32_t* parent[64];
};

struct CountersMS {
    unsigned long long a_len;  // active vertices appended (front != 0)
    unsigned long long u_len;  // chunk units appended
    unsigned long long e_f;    // degree sum of the appended vertices
    unsigned long long conv;   // cursor of a masks -> active-list conversion
    unsigned long long lanes;  // OR of the frontier masks: lanes that can still find vertices
    unsigned long long done_e; // degree sum of the vertices that the level left seen by every live lane
    unsigned long long pull_next;  // pull level: cursor of the warps over the words of the vertex range
};

struct CtlMS {
    GridBarrier bar;
    CountersMS slot[3];
    int32_t levels;
    unsigned long long long_len;  // deferred long rows of the current pull level
};

struct WorkspaceMS {
    int32_t ncap = 0;
    int64_t ucap = 0;
    int32_t chunk = 0;
    uint64_t* seen = nullptr;
    uint64_t* front[2] = {nullptr, nullptr};
    int32_t* act[2] = {nullptr, nullptr};
    int2* U[2] = {nullptr, nullptr};
    CtlMS* ctl = nullptr;
    int* d_sticky = nullptr;
    MsUnit* d_units = nullptr;
    int32_t units_cap = 0;
    CtlMS* h_ctl = nullptr;
    int32_t* longv = nullptr;            // pull: deferred long rows of the level
    unsigned long long* acc_long = nullptr;  // their lanes found so far
    uint64_t* hist = nullptr;            // frontier masks of levels 0 .. MS_HIST-1, [MS_HIST][ncap]
    int* hist_dirty = nullptr;           // device flag, see ParamsMS
};

void free_wsms(WorkspaceMS* w) {
    if (!w) return;
    cudaFree(w->seen);
    for (int i = 0; i < 2; ++i) {
        cudaFree(w->front[i]);
        cudaFree(w->act[i]);
        cudaFree(w->U[i]);
    }
    cudaFree(w->ctl);
    cudaFree(w->d_sticky);
    cudaFree(w->d_units);
    cudaFree(w->longv);
    cudaFree(w->acc_long);
    cudaFree(w->hist);
    cudaFree(w->hist_dirty);
    cudaFreeHost(w->h_ctl);
    delete w;
}

int msbfs_sticky_error(bfs_graph* g) {
    if (!g || !g->wsms) return 0;
    int err = 0;
    if (cudaMemcpy(&err, g->wsms->d_sticky, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return DEV_OK;
    if (err) cudaMemset(g->wsms->d_sticky, 0, 4);
    return err;
}

bfs_status device_error(int err, int64_t timeout_ns);
const float* policy_device_weights(const bfs_policy* p);

struct ParamsMS {
    const MsUnit* units;
    int32_t n_units;
    uint64_t* seen;
    uint64_t* F0;
    uint64_t* F1;
    int32_t* A0;
    int32_t* A1;
    int2* U0;
    int2* U1;
    int64_t ucap;
    CtlMS* ctl;
    int* sticky;
    int32_t policy;
    float alpha, beta;
    const int8_t* schedule;
    int32_t schedule_len;
    const float* mlp;
    int32_t chunk, medium, pull_serial;
    int64_t timeout_ns;
    int32_t max_levels;
    bfs_level_record* log;  // per-level records of the first unit
    int32_t log_cap;
    int32_t* longv;
    unsigned long long* acc_long;
    uint64_t* hist;  // frontier masks of the first MS_HIST levels (zero between units)
    int64_t ncap;    // vertices per history level
    int* hist_dirty; // set while a launch runs; still set at the next launch if it ended early
};

// Unit fields kept in registers / shared memory while a unit runs.
struct UnitView {
    const int32_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col;
    const int32_t* __restrict__ csc_ptr;
    const int32_t* __restrict__ csc_col;
    const uint32_t* __restrict__ isolated;
    int64_t m;
    int32_t n;
    int32_t k;
    int32_t symmetric;
    uint64_t lanes;
};

constexpr int MS_T = 512;
// Depths of the first MS_HIST levels are not written as lanes find vertices:
// the frontier masks of those levels are kept, and one pass after the last
// level writes every depth row whole (the level of the first mask holding
// the lane, -1 for an unreached vertex).  Written as found, a lane's depth
// entries are scattered 4-byte stores into partly written sectors, which the
// memory system fills from DRAM, and every row would first be set to -1.
constexpr int MS_HIST = 16;
constexpr int MS_QBUF = 64;       // per-warp staging of active-list appends
constexpr int MS_LONG_ROW = 1024; // pull rows longer than this are scanned grid-wide
static_assert(MS_LONG_ROW < 65536, "pull parent positions are staged as 16-bit row offsets");
constexpr int MS_LONG_ITEMS = 4;  // entries a thread tests per long-row chunk

#ifndef BFS_MS_PULL_R
#define BFS_MS_PULL_R 4
#endif
constexpr int MS_PULL_R = BFS_MS_PULL_R;  // in-neighbours loaded per serial pull step
constexpr int MS_COOP_U = 4;  // 32-entry groups a warp loads per step when it finishes a long row
// Words a warp takes at a time in a pull level: one while many vertices
// still miss live lanes (costly words: finest balance), eight once few do
// (the takes of one word each then queue on the cursor's atomics).
constexpr int MS_PULL_CHUNK_DENSE = 1, MS_PULL_CHUNK_SPARSE = 8;

struct MsSmem {
    int32_t* depth[64];
    int32_t* parent[64];
    int off[MS_T + 1];
    int beg[MS_T];
    int lim[MS_T];
    int src[MS_T];
    unsigned long long fmask[MS_T];
    int scan_tmp[33];
    int32_t qbuf[(MS_T / 32) * MS_QBUF];
    float feat[BFS_MLP_IN];
    float mlp_out;
    unsigned long long red[MS_T / 32];
    unsigned long long base;
};

struct MsLevel {
    int32_t level;
    uint64_t* f_next;
    int32_t* a_next;
    int2* u_next;
    CountersMS* next;
    unsigned long long ef;   // degree sum of F_{i+1} vertices (this thread's share)
    unsigned long long cnt;  // |{v : F_{i+1}[v] != 0}| (pull levels, this thread's share)
    uint64_t lanes;          // OR of the F_{i+1} masks this thread wrote
    uint64_t live;           // lanes with a non-empty frontier F_i
    unsigned long long done_e;  // degree sum of vertices now seen by every live lane (this thread's share)
    int32_t* qbuf;
    int qn;                  // staged appends (warp-uniform)
    unsigned long long* cursor;  // pull: next word to take (zero when the level starts)
    int pull_chunk;              // pull: words a warp takes at a time
    bool write_depth;        // depths of F_{i+1} are written now (levels past the history)
};

__device__ __forceinline__ void write_lanes(MsSmem& sm, uint64_t bits, int v, int par, int d, bool write_depth) {
    while (bits) {
        int j = __ffsll((long long)bits) - 1;
        if (write_depth) sm.depth[j][v] = d;
        if (sm.parent[j]) sm.parent[j][v] = par;
        bits &= bits - 1;
    }
}

__device__ __forceinline__ void ms_units(const ParamsMS& p, int2* u_out, CountersMS* c, int v, int deg) {
    append_units(u_out, &c->u_len, p.ucap, &p.ctl->bar.err, v, deg, p.chunk);
}

__device__ __forceinline__ void ms_flush(MsLevel& L) {
    if (L.qn == 0) return;
    unsigned lane = lane_id();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&L.next->a_len, (unsigned long long)L.qn);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    for (int i = (int)lane; i < L.qn; i += 32) L.a_next[base + i] = L.qbuf[i];
    __syncwarp();
    L.qn = 0;
}

// v entered F_{i+1} (first OR into its mask this level): stage it for the
// active list, add its degree, split big rows into chunk units.  Warp-uniform.
__device__ __forceinline__ void ms_emit(const ParamsMS& p, MsLevel& L, bool first, int v, int deg) {
    unsigned cm = __ballot_sync(0xffffffffu, first);
    if (!cm) return;
    int c = __popc(cm);
    if (L.qn + c > MS_QBUF) ms_flush(L);
    if (first) {
        L.qbuf[L.qn + __popc(cm & lanemask_lt())] = v;
        L.ef += (unsigned long long)deg;
        if (deg >= p.chunk) ms_units(p, L.u_next, L.next, v, deg);
    }
    L.qn += c;
}

// Push candidate u -> v with frontier lanes fu: the lanes of fu that v has
// not seen are ORed into next[v]; the OR's old value names exactly one
// claimer per (v, lane), which writes that lane's depth and parent.
__device__ __forceinline__ void ms_candidate(const ParamsMS& p, const UnitView& g, MsLevel& L, MsSmem& sm, bool has,
                                             int v, int u, uint64_t fu) {
    uint64_t bits = 0;
    if (has) bits = fu & ~((const unsigned long long*)p.seen)[v];
    bool first = false;
    int deg = 0;
    if (bits) {
        uint64_t old = atomicOr((unsigned long long*)L.f_next + v, (unsigned long long)bits);
        uint64_t nb = bits & ~old;
        first = (old == 0);
        L.lanes |= nb;
        if (nb) write_lanes(sm, nb, v, u, L.level + 1, L.write_depth);
        if (first) deg = __ldg(g.row_ptr + v + 1) - __ldg(g.row_ptr + v);
    }
    ms_emit(p, L, first, v, deg);
}

template <int T>
__device__ void ms_push_tile(const ParamsMS& p, const UnitView& g, MsLevel& L, MsSmem& sm, int u,
                             const uint64_t* f_cur) {
    static_assert(T <= MS_T, "tile arrays are sized for MS_T threads");
    unsigned lane = lane_id();
    int beg = 0, end = 0;
    uint64_t fu = 0;
    if (u >= 0) {
        beg = __ldg(g.row_ptr + u);
        end = __ldg(g.row_ptr + u + 1);
        fu = ((const unsigned long long*)f_cur)[u];
        if (end - beg >= p.chunk) end = beg;  // chunk units cover it
    }
    // medium rows: 32-edge segments taken in turn by every warp of the CTA
    const bool med = (end - beg) >= p.medium;
    int nseg_total;
    const int soff = block_exclusive_scan(med ? (end - beg + 31) >> 5 : 0, sm.scan_tmp, &nseg_total);
    if (nseg_total > 0) {
        sm.off[threadIdx.x] = soff;
        sm.beg[threadIdx.x] = beg;
        sm.lim[threadIdx.x] = end;
        sm.src[threadIdx.x] = u;
        sm.fmask[threadIdx.x] = fu;
        __syncthreads();
        for (int s = (int)(threadIdx.x >> 5); s < nseg_total; s += T / 32) {
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (sm.off[mid] <= s) lo = mid; else hi = mid - 1;
            }
            const int j = sm.beg[lo] + ((s - sm.off[lo]) << 5) + (int)lane;
            const bool has = j < sm.lim[lo];
            const int v = has ? __ldg(g.col + j) : 0;
            ms_candidate(p, g, L, sm, has, v, sm.src[lo], sm.fmask[lo]);
        }
    }
    if (med) end = beg;
    int deg = end - beg, total;
    int off = block_exclusive_scan(deg, sm.scan_tmp, &total);
    sm.off[threadIdx.x] = off;
    sm.beg[threadIdx.x] = beg;
    sm.src[threadIdx.x] = u;
    sm.fmask[threadIdx.x] = fu;
    if (threadIdx.x == T - 1) sm.off[T] = total;
    __syncthreads();
    for (int k0 = 0; k0 < total; k0 += T) {
        int k = k0 + threadIdx.x;
        bool has = k < total;
        int v = 0, su = 0;
        uint64_t sf = 0;
        if (has) {
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (sm.off[mid] <= k) lo = mid; else hi = mid - 1;
            }
            su = sm.src[lo];
            sf = sm.fmask[lo];
            v = __ldg(g.col + sm.beg[lo] + (k - sm.off[lo]));
        }
        ms_candidate(p, g, L, sm, has, v, su, sf);
    }
    __syncthreads();
}

// Push level: items = chunk units of big rows, then CTA tiles of the active
// list, dealt round-robin over the CTAs.
template <int T>
__device__ void ms_push_level(const ParamsMS& p, const UnitView& g, MsLevel& L, MsSmem& sm, const int32_t* a_cur,
                              const int2* u_cur, const uint64_t* f_cur, long long a, long long nunits) {
    long long per_tile = (a + gridDim.x - 1) / gridDim.x;
    per_tile = per_tile < 1 ? 1 : (per_tile > T ? T : per_tile);
    long long nitems = nunits + (a + per_tile - 1) / per_tile;
    for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
        if (it < nunits) {
            int2 un = u_cur[it];
            int u = un.x;
            uint64_t fu = ((const unsigned long long*)f_cur)[u];
            int b = __ldg(g.row_ptr + u), e = __ldg(g.row_ptr + u + 1);
            int lo = b + un.y * p.chunk, hi = min(e, lo + p.chunk);
            for (int base = lo; base < hi; base += T) {
                int j = base + threadIdx.x;
                bool has = j < hi;
                int v = has ? __ldg(g.col + j) : 0;
                ms_candidate(p, g, L, sm, has, v, u, fu);
            }
        } else {
            long long q = (it - nunits) * per_tile + threadIdx.x;
            int u = (threadIdx.x < per_tile && q < a) ? a_cur[q] : -1;
            ms_push_tile<T>(p, g, L, sm, u, f_cur);
        }
    }
    ms_flush(L);
}

__device__ __forceinline__ uint64_t warp_or64(uint64_t x) {
    unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)x);
    unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(x >> 32));
    return ((uint64_t)hi << 32) | lo;
}

// Pull level, one warp per 32 consecutive vertices (lane = vertex): a vertex
// missing some live lanes (lanes whose frontier F_i is not empty: only those
// can reach it at this level) ORs the frontier masks of its in-neighbours in
// ascending order and stops once every such lane is found; the first
// neighbour that supplies a lane is that lane's parent.  Rows longer than
// `pull_serial` entries are finished by the whole warp.  Depths are written
// lane-major in a warp-uniform loop over the union of the new lanes, so the
// 32 vertices' entries of one lane's depth row go out together.
// Dynamic shared memory of the MS-BFS kernel: per warp, the row offset of
// the parent found for each (lane l, vertex of the warp's word) in a pull
// level, [l][vertex], so that parents are written lane-major like depths.
constexpr size_t MS_PIDX_BYTES = (size_t)(MS_T / 32) * 64 * 32 * sizeof(unsigned short);
extern __shared__ __align__(16) unsigned short ms_pidx_smem[];

__device__ void ms_pull_level(const ParamsMS& p, const UnitView& g, MsLevel& L, MsSmem& sm, const uint64_t* f_cur) {
    const unsigned lane = lane_id();
    unsigned short* pidx = ms_pidx_smem + (threadIdx.x >> 5) * (64 * 32);
    const int dnext = L.level + 1;
    const long long W = (g.n + 31) >> 5;
    const unsigned long long* F = (const unsigned long long*)f_cur;
    // warps take L.pull_chunk words at a time from a level-wide cursor: the
    // cost of a word varies by orders of magnitude (hubs, early exits), and a
    // fixed deal left most warps waiting at the level barrier.  The next take
    // is requested when a chunk starts, so its round trip overlaps the work.
    const unsigned long long chunk = (unsigned long long)L.pull_chunk;
    unsigned long long take = 0;
    if (lane == 0) take = atomicAdd(L.cursor, chunk);
    for (;;) {  // warp-uniform
        const long long w0 = (long long)__shfl_sync(0xffffffffu, take, 0);
        if (w0 >= W) break;
        if (lane == 0) take = atomicAdd(L.cursor, chunk);
        const long long w1 = min(w0 + (long long)chunk, W);
        for (long long w = w0; w < w1; ++w) {
        const long long v = w * 32 + lane;
        uint64_t miss = 0;
        if (v < g.n) {
            bool iso = (__ldg(g.isolated + w) >> lane) & 1u;
            if (!iso) miss = L.live & ~((const unsigned long long*)p.seen)[v];
        }
        if (!__ballot_sync(0xffffffffu, miss != 0)) continue;
        int beg = 0, end = 0;
        if (miss) {
            beg = __ldg(g.csc_ptr + v);
            end = __ldg(g.csc_ptr + v + 1);
        }
        // rows longer than MS_LONG_ROW are scanned by the whole grid after
        // this pass (ms_long_rows); defer them
        const bool longrow = miss != 0 && end - beg > MS_LONG_ROW;
        const unsigned lm = __ballot_sync(0xffffffffu, longrow);
        if (lm) {
            unsigned long long base = 0;
            const int leader = __ffs(lm) - 1;
            if ((int)lane == leader) base = atomicAdd(&p.ctl->long_len, (unsigned long long)__popc(lm));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (longrow) {
                const unsigned long long r = base + __popc(lm & lanemask_lt());
                p.longv[r] = (int)v;
                p.acc_long[r] = 0;
                miss = 0;
                end = beg;
            }
        }
        uint64_t acc = 0;
        int j = beg;
        const int lim = min(end, beg + p.pull_serial);
        // MS_PULL_R entries per step (independent loads), tested in row order
        while (j < lim && acc != miss) {
            int uu[MS_PULL_R];
            uint64_t fm[MS_PULL_R];
#pragma unroll
            for (int r = 0; r < MS_PULL_R; ++r) uu[r] = j + r < lim ? __ldg(g.csc_col + j + r) : -1;
#pragma unroll
            for (int r = 0; r < MS_PULL_R; ++r) fm[r] = uu[r] >= 0 ? F[uu[r]] : 0ull;
#pragma unroll
            for (int r = 0; r < MS_PULL_R; ++r) {
                if (uu[r] < 0 || acc == miss) break;
                const uint64_t got = fm[r] & miss & ~acc;
                if (got) {
                    acc |= got;
                    uint64_t b = got;
                    while (b) {
                        int lj = __ffsll((long long)b) - 1;
                        pidx[lj * 32 + lane] = (unsigned short)(j - beg);
                        b &= b - 1;
                    }
                }
                ++j;
            }
        }
        unsigned rm = __ballot_sync(0xffffffffu, miss != 0 && acc != miss && j < end);
        while (rm) {
            const int l = __ffs(rm) - 1;
            const int jl = __shfl_sync(0xffffffffu, j, l);
            const int el = __shfl_sync(0xffffffffu, end, l);
            const int bl = __shfl_sync(0xffffffffu, beg, l);
            const uint64_t ml = __shfl_sync(0xffffffffu, (unsigned long long)miss, l);
            uint64_t al = __shfl_sync(0xffffffffu, (unsigned long long)acc, l);
            // MS_COOP_U * 32 entries a step: all column loads, then all mask loads
            for (int b2 = jl; b2 < el && al != ml; b2 += 32 * MS_COOP_U) {
                int uu[MS_COOP_U];
                uint64_t fu[MS_COOP_U];
#pragma unroll
                for (int q = 0; q < MS_COOP_U; ++q) {
                    const int idx = b2 + q * 32 + (int)lane;
                    uu[q] = idx < el ? __ldg(g.csc_col + idx) : -1;
                }
                uint64_t mine = 0;
#pragma unroll
                for (int q = 0; q < MS_COOP_U; ++q) {
                    fu[q] = uu[q] >= 0 ? (F[uu[q]] & ml & ~al) : 0ull;
                    mine |= fu[q];
                }
                const uint64_t got = warp_or64(mine);
                uint64_t gb = got;
                while (gb) {  // warp-uniform: the first (lowest index) provider of each lane
                    const int bj = __ffsll((long long)gb) - 1;
#pragma unroll
                    for (int q = 0; q < MS_COOP_U; ++q) {
                        const unsigned who = __ballot_sync(0xffffffffu, (fu[q] >> bj) & 1ull);
                        if (who) {
                            if (lane == 0) pidx[bj * 32 + l] = (unsigned short)(b2 + q * 32 + __ffs(who) - 1 - bl);
                            break;
                        }
                    }
                    gb &= gb - 1;
                }
                al |= got;
            }
            if ((int)lane == l) acc = al;
            rm &= rm - 1;
        }
        // depths and parents of the word, lane-major: for each lane found
        // anywhere in the word, its row entries of the 32 vertices go out together
        uint64_t all = warp_or64(acc);
        __syncwarp();
        while (all) {  // warp-uniform
            const int bj = __ffsll((long long)all) - 1;
            if ((acc >> bj) & 1ull) {
                if (L.write_depth) sm.depth[bj][v] = dnext;
                int32_t* pp = sm.parent[bj];
                if (pp) pp[v] = __ldg(g.csc_col + beg + pidx[bj * 32 + lane]);
            }
            all &= all - 1;
        }
        __syncwarp();
        if (acc) {
            ((unsigned long long*)L.f_next)[v] = acc;
            ((unsigned long long*)p.seen)[v] |= acc;
            L.lanes |= acc;
            L.cnt += 1;
            const unsigned long long dv =
                (unsigned long long)(g.symmetric ? (end - beg) : (__ldg(g.row_ptr + v + 1) - __ldg(g.row_ptr + v)));
            L.ef += dv;
            if (acc == miss) L.done_e += dv;  // no live lane misses v any more
        }
        }
    }
}

// Long rows of a pull level: each is scanned by a whole CTA (rows dealt
// round-robin), MS_LONG_ITEMS*T entries per step, stopping once every live
// missing lane is found.  The CTA ORs the supplied lanes in shared memory and
// keeps the first supplier of each lane as its parent; it owns the row, so
// the accumulator and the parents are written with plain stores.
template <int T>
__device__ void ms_long_rows(const ParamsMS& p, const UnitView& g, MsSmem& sm, const uint64_t* f_cur, uint64_t live,
                             long long nl) {
    __shared__ unsigned long long s_or;
    __shared__ int s_prov[64];
    const unsigned long long* F = (const unsigned long long*)f_cur;
    const int per = MS_LONG_ITEMS * T;
    for (long long r = blockIdx.x; r < nl; r += gridDim.x) {
        const int v = p.longv[r];
        const int beg = __ldg(g.csc_ptr + v), end = __ldg(g.csc_ptr + v + 1);
        const uint64_t miss = live & ~((const unsigned long long*)p.seen)[v];
        if (threadIdx.x == 0) s_or = 0;
        __syncthreads();
        for (int lo = beg; lo < end; lo += per) {
            if ((s_or & miss) == miss) break;  // CTA-uniform: read after the barrier below
            const int hi = min(end, lo + per);
#pragma unroll
            for (int k = 0; k < MS_LONG_ITEMS; ++k) {
                const int e = lo + k * T + (int)threadIdx.x;
                if (e < hi) {
                    const int u = __ldg(g.csc_col + e);
                    const uint64_t got = F[u] & miss;
                    if (got) {
                        const uint64_t old = atomicOr(&s_or, (unsigned long long)got);
                        uint64_t nb = got & ~old;
                        while (nb) {
                            const int b = __ffsll((long long)nb) - 1;
                            s_prov[b] = u;
                            nb &= nb - 1;
                        }
                    }
                }
            }
            __syncthreads();
        }
        const uint64_t acc = s_or;
        if (threadIdx.x == 0) p.acc_long[r] = acc;
        if (threadIdx.x < 64 && ((acc >> threadIdx.x) & 1ull) && sm.parent[threadIdx.x])
            sm.parent[threadIdx.x][v] = s_prov[threadIdx.x];
        __syncthreads();
    }
}

// The deferred long rows found their lanes: depth, F_{i+1}, seen and the
// level counters (after ms_long_rows, before the next level).
__device__ void ms_long_finalize(const ParamsMS& p, const UnitView& g, MsSmem& sm, uint64_t* f_next, long long nl,
                                 int dnext, CountersMS* nxt, uint64_t live, bool write_depth) {
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    unsigned long long cnt = 0, ef = 0, done = 0;
    uint64_t ln = 0;
    for (long long r = gtid; r < nl; r += gthreads) {
        const uint64_t acc = __ldcg(p.acc_long + r);
        if (!acc) continue;
        const int v = p.longv[r];
        ((unsigned long long*)f_next)[v] = acc;
        const uint64_t old = ((const unsigned long long*)p.seen)[v];
        ((unsigned long long*)p.seen)[v] = old | acc;
        uint64_t b = write_depth ? acc : 0ull;
        while (b) {
            const int j = __ffsll((long long)b) - 1;
            sm.depth[j][v] = dnext;
            b &= b - 1;
        }
        cnt += 1;
        const unsigned long long dv = (unsigned long long)(__ldg(g.row_ptr + v + 1) - __ldg(g.row_ptr + v));
        ef += dv;
        if (((old | acc) & live) == live) done += dv;
        ln |= acc;
    }
    cnt = warp_sum(cnt);
    ef = warp_sum(ef);
    done = warp_sum(done);
    ln = warp_or64(ln);
    if ((threadIdx.x & 31) == 0) {
        if (cnt) atomicAdd(&nxt->a_len, cnt);
        if (ef) atomicAdd(&nxt->e_f, ef);
        if (done) atomicAdd(&nxt->done_e, done);
        if (ln) atomicOr((unsigned long long*)&nxt->lanes, (unsigned long long)ln);
    }
}

// Active list of F_i from its masks (after a pull level), with chunk units.
template <int T>
__device__ void ms_masks_to_list(const ParamsMS& p, const UnitView& g, MsSmem& sm, const uint64_t* f_cur,
                                 int32_t* a_cur, int2* u_cur, CountersMS* cur) {
    for (long long vb = (long long)blockIdx.x * T; vb < g.n; vb += (long long)gridDim.x * T) {
        long long v = vb + threadIdx.x;
        int flag = (v < g.n && ((const unsigned long long*)f_cur)[v] != 0) ? 1 : 0;
        int total;
        int off = block_exclusive_scan(flag, sm.scan_tmp, &total);
        if (threadIdx.x == 0 && total) sm.base = atomicAdd(&cur->conv, (unsigned long long)total);
        __syncthreads();
        if (flag) {
            a_cur[sm.base + off] = (int)v;
            int deg = __ldg(g.row_ptr + v + 1) - __ldg(g.row_ptr + v);
            if (deg >= p.chunk) ms_units(p, u_cur, cur, (int)v, deg);
        }
        __syncthreads();
    }
}

// The MS-BFS heuristic: Beamer's test on the lanes' summed counters.
__device__ __forceinline__ int ms_heuristic(const ParamsMS& p, const UnitView& g, long long a, long long e_f,
                                            long long m_u, long long a_prev, int prev_dir) {
    if (prev_dir == BFS_DIR_PULL) {
        bool stay = (a >= a_prev) || ((float)a * p.beta > (float)g.n);
        return stay ? BFS_DIR_PULL : BFS_DIR_PUSH_QUEUE;
    }
    if ((float)e_f * p.alpha > (float)m_u && a > a_prev) return BFS_DIR_PULL;
    return BFS_DIR_PUSH_QUEUE;
}

__device__ int ms_decide(const ParamsMS& p, const UnitView& g, MsSmem& sm, int level, long long a, long long e_f,
                         long long m_u, long long a_prev, int prev_dir, int deg_max) {
    int d;
    switch (p.policy) {
        case BFS_POLICY_PUSH: return BFS_DIR_PUSH_QUEUE;
        case BFS_POLICY_PULL: return BFS_DIR_PULL;
        case BFS_POLICY_SCHEDULE:
            d = p.schedule[level % p.schedule_len];
            return d == BFS_DIR_PULL ? BFS_DIR_PULL : BFS_DIR_PUSH_QUEUE;
        case BFS_POLICY_MLP: {
            const int h = ms_heuristic(p, g, a, e_f, m_u, a_prev, prev_dir);
            if (p.mlp && policy_in_band(e_f, m_u, p.alpha)) {
                if (threadIdx.x < 32) {
                    if (threadIdx.x == 0)
                        policy_features(sm.feat, a, e_f, m_u, a_prev, level, prev_dir, g.n, g.m, deg_max);
                    __syncwarp();
                    int c = policy_choice_warp(p.mlp, sm.feat, h, MLP_MARGIN);
                    if (threadIdx.x == 0) sm.mlp_out = (float)c;
                }
                __syncthreads();
                d = (int)sm.mlp_out;
                __syncthreads();
                return d == BFS_DIR_PULL ? BFS_DIR_PULL : BFS_DIR_PUSH_QUEUE;
            }
            return h;  // no weights, or a clear-cut level: the heuristic decides
        }
        default:
            return ms_heuristic(p, g, a, e_f, m_u, a_prev, prev_dir);
    }
}

// The frontier mask of level i: kept in the history for the first MS_HIST
// levels, two alternating buffers after that.
__device__ __forceinline__ uint64_t* ms_front(const ParamsMS& p, int i) {
    return i < MS_HIST ? p.hist + (int64_t)i * p.ncap : ((i & 1) ? p.F1 : p.F0);
}

// After the last level L of a unit: every depth row written whole.  A warp
// takes 32 consecutive vertices (lane = vertex) and records, in its
// shared-memory table [lane j][vertex], the first history level whose mask
// holds lane j; a lane found only after the history (written as found) is
// left alone, an unreached one gets -1.  Each lane's 32 entries then go out
// as one coalesced row segment.  The history masks used are cleared for the
// next unit.
__device__ void ms_depth_pass(const ParamsMS& p, const UnitView& g, MsSmem& sm, int levels) {
    const unsigned lane = lane_id();
    signed char* tab = (signed char*)(ms_pidx_smem + (threadIdx.x >> 5) * (64 * 32));  // [64][32] int8
    const int lh = min(levels, MS_HIST);
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long ntiles = ((long long)g.n + 31) >> 5;
    for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nwarps) {
        const long long v = t * 32 + lane;
        const bool valid = v < g.n;
#pragma unroll 4
        for (int j = 0; j < 64; ++j) tab[j * 32 + lane] = -1;
        uint64_t found = 0;
        for (int i = 0; i < lh; ++i) {
            uint64_t* hp = p.hist + (int64_t)i * p.ncap + v;
            const uint64_t b = valid ? *hp : 0ull;
            uint64_t nb = b & ~found;
            found |= b;
            while (nb) {
                const int j = __ffsll((long long)nb) - 1;
                tab[j * 32 + lane] = (signed char)i;
                nb &= nb - 1;
            }
            if (b) *hp = 0ull;
        }
        const uint64_t later = valid ? (((const unsigned long long*)p.seen)[v] & ~found) : 0ull;
        __syncwarp();
        for (int j = 0; j < g.k; ++j) {
            if (valid && !((later >> j) & 1ull)) sm.depth[j][v] = (int)tab[j * 32 + lane];
        }
        __syncwarp();
    }
}

template <int T>
__device__ void msbfs_body(const ParamsMS& p) {
    __shared__ MsSmem sm;
    CtlMS* ctl = p.ctl;
    const unsigned nblocks = gridDim.x;
    const long long gtid = (long long)blockIdx.x * T + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * T;
    const unsigned warp = threadIdx.x >> 5;
    unsigned bar_target = 0;
    int total_levels = 0;
    // a launch that ended early (error, time limit) left history masks set:
    // clear the whole history before use
    if (ld_volatile_i32(p.hist_dirty)) {
        for (long long i = gtid; i < (long long)MS_HIST * p.ncap; i += gthreads) p.hist[i] = 0;
    }
    if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
    if (gtid == 0) *p.hist_dirty = 1;
    for (int ui = 0; ui < p.n_units; ++ui) {
        const MsUnit* U = p.units + ui;
        UnitView g;
        g.row_ptr = U->row_ptr;
        g.col = U->col;
        g.csc_ptr = U->csc_ptr;
        g.csc_col = U->csc_col;
        g.isolated = U->isolated;
        g.m = U->m;
        g.n = U->n;
        g.k = U->k;
        g.symmetric = U->symmetric;
        g.lanes = (g.k >= 64) ? ~0ull : ((1ull << g.k) - 1);
        int deg_max = U->deg_max;
        if (threadIdx.x < 64) {
            sm.depth[threadIdx.x] = threadIdx.x < g.k ? U->depth[threadIdx.x] : nullptr;
            sm.parent[threadIdx.x] = threadIdx.x < g.k ? U->parent[threadIdx.x] : nullptr;
        }
        __syncthreads();
        // init: masks, outputs (-1), counters
        for (long long v = gtid; v < g.n; v += gthreads) {
            p.seen[v] = 0;
            p.F0[v] = 0;
            p.F1[v] = 0;
        }
        // depths are written whole by ms_depth_pass; parents start at -1
        for (int j = 0; j < g.k; ++j) {
            int32_t* pp = sm.parent[j];
            if (!pp) continue;
            for (long long v = gtid; v < g.n; v += gthreads) pp[v] = -1;
        }
        if (gtid == 0) {
            for (int s = 0; s < 3; ++s) {
                ctl->slot[s].a_len = 0;
                ctl->slot[s].u_len = 0;
                ctl->slot[s].e_f = 0;
                ctl->slot[s].conv = 0;
                ctl->slot[s].lanes = 0;
                ctl->slot[s].done_e = 0;
                ctl->slot[s].pull_next = 0;
            }
            ctl->slot[0].lanes = g.lanes;
        }
        if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
        if (blockIdx.x == 0 && threadIdx.x < (unsigned)g.k) {
            int j = threadIdx.x;
            int s = U->src[j];
            atomicOr((unsigned long long*)p.seen + s, 1ull << j);
            unsigned long long old = atomicOr((unsigned long long*)ms_front(p, 0) + s, 1ull << j);
            if (sm.parent[j]) sm.parent[j][s] = s;
            if (old == 0) {
                int deg = g.row_ptr[s + 1] - g.row_ptr[s];
                unsigned long long idx = atomicAdd(&ctl->slot[0].a_len, 1ull);
                p.A0[idx] = s;
                atomicAdd(&ctl->slot[0].e_f, (unsigned long long)deg);
                if (deg >= p.chunk) ms_units(p, p.U0, &ctl->slot[0], s, deg);
            }
        }
        if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
        long long m_u = g.m, a_prev = 0;
        int prev_dir = BFS_DIR_PUSH_QUEUE;
        int unit_levels = 0;
        int list_valid = 0;  // level whose active list (and chunk units) exists
        for (int level = 0;; ++level) {
            CountersMS* cur = &ctl->slot[level % 3];
            CountersMS* nxt = &ctl->slot[(level + 1) % 3];
            const unsigned long long* const csrc[5] = {&cur->a_len, &cur->e_f, &cur->lanes, &cur->u_len,
                                                       &cur->done_e};
            unsigned long long cv[5];
            cta_load_u64<5>(csrc, cv);
            long long a = (long long)cv[0];
            long long e_f = (long long)cv[1];
            const uint64_t live = (uint64_t)cv[2];
            if (a == 0) break;
            if (level >= p.max_levels) {
                if (gtid == 0) atomicCAS(&ctl->bar.err, 0, (int)DEV_LEVELS);
                return;
            }
            // m_u: degree sum of the vertices some live lane has not seen,
            // the rows a pull level would scan (the batched reading of
            // Beamer's unexplored edges; summing every lane's frontier edges
            // instead drove it to zero within a few levels of a long search)
            m_u = max(m_u - (long long)cv[4], 1ll);
            int dir = ms_decide(p, g, sm, level, a, e_f, m_u, a_prev, prev_dir, deg_max);
            if (ui == 0 && gtid == 0 && p.log && level < p.log_cap) {
                bfs_level_record r;
                r.level = level;
                r.dir = dir;
                r.f = a;
                r.e_f = e_f;
                r.m_u = m_u;
                r.t_ns = (int64_t)globaltimer_ns();
                p.log[level] = r;
            }
            int32_t* a_cur = (level & 1) ? p.A1 : p.A0;
            int2* u_cur = (level & 1) ? p.U1 : p.U0;
            uint64_t* f_cur = ms_front(p, level);
            long long nunits = (long long)cv[3];
            if (dir != BFS_DIR_PULL && list_valid != level) {
                // active list of a pull-made frontier (it appends the chunk units)
                ms_masks_to_list<T>(p, g, sm, f_cur, a_cur, u_cur, cur);
                if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
                list_valid = level;
                const unsigned long long* const usrc[1] = {&cur->u_len};
                unsigned long long uv[1];
                cta_load_u64<1>(usrc, uv);
                nunits = (long long)uv[0];
            }
            if (gtid == 0) {
                CountersMS* z = &ctl->slot[(level + 2) % 3];
                z->a_len = 0;
                z->u_len = 0;
                z->e_f = 0;
                z->conv = 0;
                z->lanes = 0;
                z->done_e = 0;
                z->pull_next = 0;
            }
            MsLevel L;
            L.level = level;
            L.f_next = ms_front(p, level + 1);
            L.write_depth = level + 1 >= MS_HIST;
            L.a_next = (level & 1) ? p.A0 : p.A1;
            L.u_next = (level & 1) ? p.U0 : p.U1;
            L.next = nxt;
            L.ef = 0;
            L.cnt = 0;
            L.lanes = 0;
            L.live = live;
            L.done_e = 0;
            L.qbuf = sm.qbuf + warp * MS_QBUF;
            L.qn = 0;
            L.cursor = &cur->pull_next;
            // m_u: degree sum of the vertices some live lane has not seen
            L.pull_chunk = 8 * m_u >= g.m ? MS_PULL_CHUNK_DENSE : MS_PULL_CHUNK_SPARSE;
            if (dir == BFS_DIR_PULL) ms_pull_level(p, g, L, sm, f_cur);
            else ms_push_level<T>(p, g, L, sm, a_cur, u_cur, f_cur, a, nunits);
            const uint64_t ln = warp_or64(L.lanes);
            if ((threadIdx.x & 31) == 0 && ln) atomicOr((unsigned long long*)&nxt->lanes, (unsigned long long)ln);
            const unsigned long long dn = warp_sum(L.done_e);
            if ((threadIdx.x & 31) == 0 && dn) atomicAdd(&nxt->done_e, dn);
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
                    if (t) atomicAdd(&nxt->a_len, t);
                }
            } else {
                list_valid = level + 1;
            }
            if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            long long nl = 0;
            if (dir == BFS_DIR_PULL) {
                const unsigned long long* const lsrc[1] = {&ctl->long_len};
                unsigned long long lv[1];
                cta_load_u64<1>(lsrc, lv);
                nl = (long long)lv[0];
                if (nl > 0) {
                    ms_long_rows<T>(p, g, sm, f_cur, live, nl);
                    if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
                    ms_long_finalize(p, g, sm, L.f_next, nl, level + 1, nxt, live, L.write_depth);
                }
            }
            if (gtid == 0) ctl->long_len = 0;
            // F_i is consumed: past the history its buffer is F_{i+2}'s, so
            // clear its masks (history levels are kept for the depth pass);
            // after a push level fold F_{i+1} into seen (a pull level already did)
            if (level >= MS_HIST) {
                if (list_valid >= level) {
                    for (long long q = gtid; q < a; q += gthreads) f_cur[a_cur[q]] = 0;
                } else {
                    for (long long v = gtid; v < g.n; v += gthreads) f_cur[v] = 0;
                }
            }
            if (dir != BFS_DIR_PULL) {
                const unsigned long long* const asrc[1] = {&nxt->a_len};
                unsigned long long av[1];
                cta_load_u64<1>(asrc, av);
                long long an = (long long)av[0];
                unsigned long long done = 0;
                for (long long q = gtid; q < an; q += gthreads) {
                    const int v = L.a_next[q];
                    const uint64_t old = p.seen[v];
                    const uint64_t nw = old | ((const unsigned long long*)L.f_next)[v];
                    p.seen[v] = nw;
                    if ((nw & live) == live && (old & live) != live)
                        done += (unsigned long long)(__ldg(g.row_ptr + v + 1) - __ldg(g.row_ptr + v));
                }
                done = warp_sum(done);
                if ((threadIdx.x & 31) == 0 && done) atomicAdd(&nxt->done_e, done);
            }
            if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            a_prev = a;
            prev_dir = dir;
            ++total_levels;
            ++unit_levels;
        }
        // the unit's depth rows; a barrier before the next unit reuses seen
        ms_depth_pass(p, g, sm, unit_levels);
        if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
    }
    if (gtid == 0) {
        ctl->levels = total_levels;
        *p.hist_dirty = 0;  // every history level used was cleared by its depth pass
    }
}

template <int T>
__global__ void __launch_bounds__(T, 2) msbfs_kernel(ParamsMS p) {
    msbfs_body<T>(p);
    if (threadIdx.x == 0) {
        int e = ld_volatile_i32(&p.ctl->bar.err);
        if (e) atomicCAS(p.sticky, 0, e);
    }
}


__global__ void ms_count_units_kernel(const int32_t* row_ptr, int32_t n, int32_t chunk, unsigned long long* out) {
    unsigned long long s = 0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        int d = row_ptr[v + 1] - row_ptr[v];
        if (d >= chunk) s += (unsigned long long)((d + chunk - 1) / chunk);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

static int64_t count_units(const bfs_graph* g, int32_t chunk, cudaStream_t st) {
    unsigned long long* d = nullptr;
    unsigned long long h = 0;
    if (cudaMallocAsync(&d, 8, st) != cudaSuccess) return -1;
    cudaMemsetAsync(d, 0, 8, st);
    ms_count_units_kernel<<<num_sms() * 8, 256, 0, st>>>(g->row_ptr, g->n, chunk, d);
    cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    return (int64_t)h;
}

static bfs_status alloc_wsms(int32_t ncap, int64_t ucap, int32_t chunk, int32_t units_cap, WorkspaceMS** out) {
    WorkspaceMS* w = new (std::nothrow) WorkspaceMS();
    if (!w) return fail(BFS_ENOMEM, "host allocation");
    w->ncap = ncap;
    w->ucap = ucap;
    w->chunk = chunk;
    w->units_cap = units_cap;
    bool ok = cudaMalloc(&w->seen, (size_t)ncap * 8) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i)
        ok = cudaMalloc(&w->front[i], (size_t)ncap * 8) == cudaSuccess &&
             cudaMalloc(&w->act[i], (size_t)ncap * 4) == cudaSuccess &&
             cudaMalloc(&w->U[i], (size_t)ucap * sizeof(int2)) == cudaSuccess;
    ok = ok && cudaMalloc(&w->ctl, sizeof(CtlMS)) == cudaSuccess;
    ok = ok && cudaMalloc(&w->d_sticky, 4) == cudaSuccess && cudaMemset(w->d_sticky, 0, 4) == cudaSuccess;
    ok = ok && cudaMalloc(&w->d_units, sizeof(MsUnit) * (size_t)units_cap) == cudaSuccess;
    ok = ok && cudaMalloc(&w->longv, (size_t)ncap * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&w->acc_long, (size_t)ncap * 8) == cudaSuccess;
    ok = ok && cudaMalloc(&w->hist, (size_t)MS_HIST * ncap * 8) == cudaSuccess &&
         cudaMemset(w->hist, 0, (size_t)MS_HIST * ncap * 8) == cudaSuccess;
    ok = ok && cudaMalloc(&w->hist_dirty, 4) == cudaSuccess && cudaMemset(w->hist_dirty, 0, 4) == cudaSuccess;
    ok = ok && cudaMallocHost(&w->h_ctl, sizeof(CtlMS)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_wsms(w);
        return fail(BFS_ENOMEM, "MS-BFS workspace for n=%d", ncap);
    }
    *out = w;
    return BFS_OK;
}

static int coop_blocks_ms(int blocks_per_sm) {
    int per_sm = 0;
    cudaFuncSetAttribute(msbfs_kernel<MS_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MS_PIDX_BYTES);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, msbfs_kernel<MS_T>, MS_T, MS_PIDX_BYTES);
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
    return per_sm * num_sms();
}

static MsUnit make_unit(const bfs_graph* g) {
    MsUnit u;
    memset(&u, 0, sizeof(u));
    u.row_ptr = g->row_ptr;
    u.col = g->col;
    u.csc_ptr = g->csc_ptr;
    u.csc_col = g->csc_col;
    u.isolated = g->isolated;
    u.m = g->m;
    u.n = g->n;
    u.symmetric = g->symmetric;
    u.deg_max = g->deg_max;
    return u;
}

static bfs_status launch_ms(WorkspaceMS* w, const std::vector<MsUnit>& units, const bfs_options& o, const float* mlp,
                            const int8_t* d_sched, cudaStream_t st, bfs_level_record* d_log = nullptr) {
    if ((int32_t)units.size() > w->units_cap) return fail(BFS_EINVAL, "too many units");
    BFS_CUDA(cudaMemcpyAsync(w->d_units, units.data(), sizeof(MsUnit) * units.size(), cudaMemcpyHostToDevice, st));
    BFS_CUDA(cudaMemsetAsync(w->ctl, 0, sizeof(CtlMS), st));
    ParamsMS p{};
    p.units = w->d_units;
    p.n_units = (int32_t)units.size();
    p.seen = w->seen;
    p.F0 = w->front[0];
    p.F1 = w->front[1];
    p.A0 = w->act[0];
    p.A1 = w->act[1];
    p.U0 = w->U[0];
    p.U1 = w->U[1];
    p.ucap = w->ucap;
    p.ctl = w->ctl;
    p.sticky = w->d_sticky;
    p.policy = o.policy;
    p.alpha = o.batch_alpha;
    p.beta = o.batch_beta;
    p.schedule = d_sched;
    p.schedule_len = o.schedule_len;
    p.mlp = mlp;
    p.chunk = o.chunk;
    p.medium = o.medium;
    p.pull_serial = std::max(o.pull_serial, 1) * 2;  // all missing lanes are rarely found early: longer serial scans
    p.timeout_ns = o.barrier_timeout_ns;
    p.max_levels = o.max_levels > 0 ? o.max_levels : INT32_MAX / 2;
    p.log = d_log;
    p.log_cap = d_log ? o.level_log_cap : 0;
    p.longv = w->longv;
    p.acc_long = w->acc_long;
    p.hist = w->hist;
    p.ncap = w->ncap;
    p.hist_dirty = w->hist_dirty;
    int blocks = coop_blocks_ms(o.blocks_per_sm);
    void* args[] = {(void*)&p};
    BFS_CUDA(cudaLaunchCooperativeKernel((const void*)msbfs_kernel<MS_T>, dim3(blocks), dim3(MS_T), args, MS_PIDX_BYTES,
                                         st));
    return BFS_OK;
}

// k sources over one graph, in units of 64 lanes; depth/parent: [k][n].
bfs_status run_msbfs(bfs_graph* g, const int32_t* sources, int32_t k, int32_t* depth, int32_t* parent,
                     const bfs_options& o, const float* mlp_dev, cudaStream_t st) {
    int32_t nunits = (int32_t)div_up(k, 64);
    WorkspaceMS* w = g->wsms;
    if (!w || w->chunk != o.chunk || w->units_cap < nunits) {
        if (w) {
            BFS_CUDA(cudaStreamSynchronize(st));
            free_wsms(w);
            g->wsms = nullptr;
        }
        int64_t uc = count_units(g, o.chunk, st);
        if (uc < 0) return fail(BFS_ECUDA, "unit count");
        bfs_status s = alloc_wsms(g->n, uc + 64, o.chunk, std::max(nunits, 4), &w);
        if (s != BFS_OK) return s;
        g->wsms = w;
    }
    const int64_t n = g->n;
    bool dev_out = is_device_ptr(depth) && (!parent || is_device_ptr(parent));
    int32_t *dd = depth, *dp = parent;
    if (!dev_out) {
        if (cudaMallocAsync(&dd, (size_t)k * n * 4, st) != cudaSuccess ||
            (parent && cudaMallocAsync(&dp, (size_t)k * n * 4, st) != cudaSuccess)) {
            cudaGetLastError();
            return fail(BFS_ENOMEM, "staging outputs for %d sources", k);
        }
    }
    int8_t* d_sched = nullptr;
    if (o.policy == BFS_POLICY_SCHEDULE) {
        if (!o.schedule || o.schedule_len <= 0) return fail(BFS_EINVAL, "schedule policy needs a schedule");
        BFS_CUDA(cudaMallocAsync(&d_sched, o.schedule_len, st));
        BFS_CUDA(cudaMemcpyAsync(d_sched, o.schedule, o.schedule_len, cudaMemcpyHostToDevice, st));
    }
    std::vector<MsUnit> units;
    for (int32_t u0 = 0; u0 < k; u0 += 64) {
        MsUnit u = make_unit(g);
        u.k = std::min(64, k - u0);
        for (int j = 0; j < u.k; ++j) {
            u.src[j] = sources[u0 + j];
            u.depth[j] = dd + (int64_t)(u0 + j) * n;
            u.parent[j] = dp ? dp + (int64_t)(u0 + j) * n : nullptr;
        }
        units.push_back(u);
    }
    bfs_level_record* d_log = nullptr;
    if (o.level_log && o.level_log_cap > 0)
        BFS_CUDA(cudaMallocAsync(&d_log, sizeof(bfs_level_record) * o.level_log_cap, st));
    bfs_status s = launch_ms(w, units, o, mlp_dev, d_sched, st, d_log);
    if (d_sched) cudaFreeAsync(d_sched, st);
    if (d_log) {
        if (s == BFS_OK) {
            BFS_CUDA(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(CtlMS), cudaMemcpyDeviceToHost, st));
            BFS_CUDA(cudaStreamSynchronize(st));
            int nl = std::min(w->h_ctl->levels, o.level_log_cap);
            if (nl > 0) BFS_CUDA(cudaMemcpy(o.level_log, d_log, sizeof(bfs_level_record) * nl, cudaMemcpyDeviceToHost));
        }
        cudaFreeAsync(d_log, st);
    }
    if (s == BFS_OK && o.levels_out) {
        BFS_CUDA(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(CtlMS), cudaMemcpyDeviceToHost, st));
        BFS_CUDA(cudaStreamSynchronize(st));
        *o.levels_out = w->h_ctl->levels;
    }
    if (!dev_out) {
        cudaError_t e = cudaSuccess;
        if (s == BFS_OK) e = cudaMemcpyAsync(depth, dd, (size_t)k * n * 4, cudaMemcpyDeviceToHost, st);
        if (s == BFS_OK && e == cudaSuccess && parent) e = cudaMemcpyAsync(parent, dp, (size_t)k * n * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFreeAsync(dd, st);
        if (dp) cudaFreeAsync(dp, st);
        if (s == BFS_OK && e != cudaSuccess) s = cuda_fail(e, "copy outputs to host");
        if (s == BFS_OK) {
            int err = msbfs_sticky_error(g);
            if (err) s = device_error(err, o.barrier_timeout_ns);
        }
    }
    return s;
}

// Queries over several graphs in one launch: grouped per graph, 64 lanes a unit.
bfs_status run_mixed(const bfs_graph* const* graphs, int32_t n_graphs, const int32_t* graph_of_query,
                     const int32_t* sources, int32_t nq, int32_t* const* depth, int32_t* const* parent,
                     const bfs_options& o, cudaStream_t st) {
    (void)n_graphs;  // bfs_run_mixed has checked every graph_of_query[q] against it
    std::map<int, std::vector<int>> by_graph;
    for (int q = 0; q < nq; ++q) by_graph[graph_of_query[q]].push_back(q);
    std::vector<MsUnit> units;
    int32_t ncap = 1;
    int64_t ucap = 1;
    for (auto& kv : by_graph) {
        const bfs_graph* g = graphs[kv.first];
        ncap = std::max(ncap, g->n);
        int64_t uc = count_units(g, o.chunk, st);
        if (uc < 0) return fail(BFS_ECUDA, "unit count");
        ucap = std::max(ucap, uc + 64);
        const std::vector<int>& qs = kv.second;
        for (size_t i = 0; i < qs.size(); i += 64) {
            MsUnit u = make_unit(g);
            u.k = (int32_t)std::min<size_t>(64, qs.size() - i);
            for (int j = 0; j < u.k; ++j) {
                int q = qs[i + j];
                u.src[j] = sources[q];
                u.depth[j] = depth[q];
                u.parent[j] = parent ? parent[q] : nullptr;
            }
            units.push_back(u);
        }
    }
    WorkspaceMS* w = nullptr;
    bfs_status s = alloc_wsms(ncap, ucap, o.chunk, (int32_t)units.size(), &w);
    if (s != BFS_OK) return s;
    int8_t* d_sched = nullptr;
    if (o.policy == BFS_POLICY_SCHEDULE && o.schedule && o.schedule_len > 0) {
        if (cudaMalloc(&d_sched, o.schedule_len) == cudaSuccess)
            cudaMemcpy(d_sched, o.schedule, o.schedule_len, cudaMemcpyHostToDevice);
    }
    bfs_options oo = o;
    if (oo.policy == BFS_POLICY_SCHEDULE && !d_sched) oo.policy = BFS_POLICY_HEURISTIC;
    const float* mlp = nullptr;
    if (oo.policy == BFS_POLICY_MLP && oo.mlp) mlp = policy_device_weights(oo.mlp);
    s = launch_ms(w, units, oo, mlp, d_sched, st);
    if (s == BFS_OK) {
        cudaError_t e = cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(CtlMS), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "mixed batch");
        else if (w->h_ctl->bar.err) s = device_error(w->h_ctl->bar.err, o.barrier_timeout_ns);
        if (s == BFS_OK && o.levels_out) *o.levels_out = w->h_ctl->levels;
    } else {
        cudaStreamSynchronize(st);
    }
    cudaFree(d_sched);
    free_wsms(w);
    return s;
}

}  // namespace bfsgb
