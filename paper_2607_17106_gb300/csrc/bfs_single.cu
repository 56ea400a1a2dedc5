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
// Pull levels own whole 32-vertex words: each CTA lists the unvisited
// vertices of its words in shared memory, its warps scan them, and the new
// bits of P and of F_{i+1} go out with plain stores by the words' owners.
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
// level and carries the loop state in device memory.  On bounded-degree
// graphs a launch of one thread-block cluster runs the small levels first
// and the grid-wide launch continues from its saved state.
#include "level.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace bfsgb {

int msbfs_sticky_error(bfs_graph* g);  // msbfs.cu
bfs_status run_graph_mode(bfs_graph* g, Workspace1* w, Params1& p, int32_t src, int32_t* depth, int32_t* parent,
                          const bfs_options& o, cudaStream_t st);  // bfs_graph.cu

void free_ws1(Workspace1* w) {
    if (!w) return;
    cudaFree(w->P);
    for (int i = 0; i < 2; ++i) {
        cudaFree(w->F[i]);
        cudaFree(w->Q[i]);
        cudaFree(w->U[i]);
    }
    cudaFree(w->E);
    cudaFree(w->cta_cnt);
    cudaFree(w->ctl);
    cudaFree(w->d_sticky);
    cudaFree(w->stage_depth);
    cudaFree(w->stage_parent);
    cudaFree(w->d_srcs);
    cudaFree(w->d_log);
    cudaFree(w->d_sched);
    cudaFreeHost(w->h_ctl);
    if (w->gexec) cudaGraphExecDestroy(w->gexec);
    delete w;
}


// ------------------------------------------------------------ the kernel
// Dynamic shared memory of the persistent kernel: the round list of the
// list-driven pull (T * 32 16-bit entries; push levels use the same bytes
// for the warps' next-queue staging, QueueStage<T>), then a copy of the
// policy weights, evaluated by every CTA at every level when the policy is
// the MLP.
template <int T>
constexpr size_t bfs1_list_bytes() {
    static_assert(sizeof(QueueStage<T>) <= (size_t)T * 32 * sizeof(uint16_t), "staging fits the list bytes");
    return (size_t)T * 32 * sizeof(uint16_t);
}

template <int T>
constexpr size_t bfs1_dyn_smem() {
    return bfs1_list_bytes<T>() + (size_t)NWEIGHTS * sizeof(float);
}
extern __shared__ __align__(16) unsigned char bfs1_dyn[];

// a[0, len) = -1 by the whole grid: 16-byte stores from the first 16-byte
// boundary, 4-byte stores for the head and the tail.  a is 4-byte aligned.
__device__ __forceinline__ void fill_minus1(int32_t* a, long long len, long long gtid, long long gthreads) {
    long long head = (long long)((16u - ((unsigned)(uintptr_t)a & 15u)) & 15u) >> 2;
    if (head > len) head = len;
    if (gtid < head) a[gtid] = -1;
    const long long nv = (len - head) >> 2;
    int4* const a4 = reinterpret_cast<int4*>(a + head);
    for (long long i = gtid; i < nv; i += gthreads) a4[i] = make_int4(-1, -1, -1, -1);
    const long long t0 = head + nv * 4;
    if (gtid < len - t0) a[t0 + gtid] = -1;
}

// Address of `p` (this CTA's shared memory) in the cluster's CTA 0.
template <typename X>
__device__ __forceinline__ X* cluster_map_rank0(X* p) {
    uint64_t r;
    asm volatile("mapa.u64 %0, %1, 0;" : "=l"(r) : "l"((uint64_t)p));
    return reinterpret_cast<X*>(r);
}

// A level counter read right after the level barrier: from L2 in a
// grid-wide launch, through distributed shared memory in a cluster launch.
template <bool CL>
__device__ __forceinline__ unsigned long long ld_counter(const unsigned long long* a) {
    if constexpr (CL) return *reinterpret_cast<const volatile unsigned long long*>(a);
    else return ld_cg_u64(a);
}

// The barrier between phases of a level.  A grid-wide launch uses the
// %globaltimer-limited grid barrier; a launch of one thread-block cluster
// (CL) uses the cluster's hardware barrier, whose arrive/wait orders every
// thread's memory operations at cluster scope.  before_arrival and
// after_open run on thread 0 as in grid_sync.
template <bool CL, typename F = NoArrivalWork, typename A = NoArrivalWork>
__device__ __forceinline__ bool level_sync(GridBarrier* b, unsigned nblocks, unsigned& target, int64_t timeout_ns,
                                           F before_arrival = F(), A after_open = A()) {
    if constexpr (CL) {
        __syncthreads();
        if (threadIdx.x == 0) before_arrival();
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        if (threadIdx.x == 0) after_open();
        __syncthreads();
        return true;
    } else {
        return grid_sync(b, nblocks, target, timeout_ns, before_arrival, after_open);
    }
}

// SORT: the frontier-sort variants are compiled in (a separate instantiation,
// so that the default kernel carries none of their registers).
// CL: one thread-block cluster runs the small levels of one search (see
// bfs_options.small_levels) and leaves the first level that is not a small
// push-queue level to the grid-wide launch that follows it.
template <int T, bool SORT, bool CL>
__device__ __forceinline__ void bfs1_body(const Params1& p) {
    __shared__ TileSmem<T> sm;
    __shared__ float s_feat[BFS_MLP_IN];
    __shared__ float s_mlp_out;
    const float* mlp_w = nullptr;
    if (p.policy == BFS_POLICY_MLP && p.mlp) {
        float* w = reinterpret_cast<float*>(bfs1_dyn + bfs1_list_bytes<T>());
        for (int i = threadIdx.x; i < NWEIGHTS; i += T) w[i] = __ldg(p.mlp + i);
        __syncthreads();
        mlp_w = w;
    }
    Ctl1* ctl = p.ctl;
    const unsigned nblocks = gridDim.x;
    const long long gtid = (long long)blockIdx.x * T + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * T;
    unsigned bar_target = p.do_init ? 0u : __ldcg(&ctl->bar_base);

    // One launch runs nsrc searches one after another (do_init), or continues
    // the search whose state the control block holds (host-loop drive).
    const int nsearch = p.do_init ? max(p.nsrc, 1) : 1;
    int level = 0, prev_dir = BFS_DIR_PUSH_QUEUE, bm_valid = -1, q_valid = 0;
    long long m_u = 0, f_prev = 0;
    bool done = false;
    // counters of the level about to start (|F_i|, chunk units, e_f): set by
    // the init, or read by thread 0 right after the level barrier opens
    // (s_cnt_ok), else read at the top of the level
    __shared__ unsigned long long s_cnt[3];
    // A cluster launch keeps the level counters in CTA 0's shared memory
    // (reached by every CTA of the cluster through distributed shared
    // memory) and copies them to the control block when it leaves.
    __shared__ Counters s_ctr[3];
    const unsigned warp = threadIdx.x >> 5;
    QueueStage<T>* const qs = reinterpret_cast<QueueStage<T>*>(bfs1_dyn);
    for (int si = 0; si < nsearch; ++si) {
    int32_t* const depth = p.depth + (int64_t)si * p.n;
    int32_t* const parent = p.parent ? p.parent + (int64_t)si * p.n : nullptr;
    Counters* const cs = CL ? cluster_map_rank0(s_ctr) : ctl->slot + 3 * (si & 1);
    bool s_cnt_ok = false;
    if (p.do_init) {
        const int s = p.srcs ? __ldg(p.srcs + si) : p.src_value;
        for (long long w = gtid; w < p.W; w += gthreads) {
            unsigned bits = __ldg(p.isolated + w);
            if (w == (s >> 5)) bits |= 1u << (s & 31);
            if (w == p.W - 1 && (p.n & 31)) bits |= ~((1u << (p.n & 31)) - 1u);  // phantom vertices
            p.P[w] = bits;
        }
        if (!p.rows_filled) {
            fill_minus1(depth, p.n, gtid, gthreads);
            if (parent) fill_minus1(parent, p.n, gtid, gthreads);
        }
        __syncthreads();  // the CTA's warps have read s_cnt of the previous search's last level
        if (threadIdx.x == 0) {
            // every CTA knows level 0's counters without reading them back
            const int rb = __ldg(p.row_ptr + s), re = __ldg(p.row_ptr + s + 1);
            const int deg = re - rb;
            const int nch = deg >= p.chunk ? (deg + p.chunk - 1) / p.chunk : 0;
            s_cnt[0] = 1;
            s_cnt[1] = (unsigned long long)nch;
            s_cnt[2] = (unsigned long long)deg;
            if (blockIdx.x == 0) {
                p.Q0[0] = make_int4(s, rb, re, 0);
                for (int c = 0; c < nch; ++c) p.U0[c] = make_int2(s, c);
                for (int k = 1; k < 3; ++k) {  // the search before the previous one used them
                    cs[k].q_len = 0;
                    cs[k].u_len = 0;
                    cs[k].e_f = 0;
                    cs[k].conv = 0;
                    cs[k].e_len = 0;
                }
                cs[0].q_len = 1;
                cs[0].u_len = nch;
                cs[0].e_f = deg;
                cs[0].conv = 0;
                cs[0].e_len = 0;
                ctl->next_level = 0;
                ctl->prev_dir = BFS_DIR_PUSH_QUEUE;
                ctl->bm_valid = -1;
                ctl->q_valid = 0;
                ctl->done = 0;
                ctl->m_u = p.m - deg;
                ctl->f_prev = 0;
            }
        }
        if (!level_sync<CL>(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
        // after the barrier: ordered after every -1 store of the rows
        if (gtid == 0) {
            depth[s] = 0;
            if (parent) parent[s] = s;
        }
        level = 0;
        prev_dir = BFS_DIR_PUSH_QUEUE;
        bm_valid = -1;
        q_valid = 0;
        m_u = p.m - (long long)s_cnt[2];
        f_prev = 0;
        done = false;
        s_cnt_ok = true;
    } else {
        level = __ldcg(&ctl->next_level);
        prev_dir = __ldcg(&ctl->prev_dir);
        bm_valid = __ldcg(&ctl->bm_valid);
        q_valid = __ldcg(&ctl->q_valid);
        m_u = __ldcg(&ctl->m_u);
        f_prev = __ldcg(&ctl->f_prev);
        done = __ldcg(&ctl->done) != 0;
    }
    const int level_end = level + p.level_count;

    while (!done && level < level_end) {
        Counters* cur = &cs[level % 3];
        Counters* nxt = &cs[(level + 1) % 3];
        int4* q_cur = (level & 1) ? p.Q1 : p.Q0;
        unsigned long long cv[3];
        if (s_cnt_ok) {
#pragma unroll
            for (int i = 0; i < 3; ++i) cv[i] = s_cnt[i];
        } else {
            const unsigned long long* const csrc[3] = {&cur->q_len, &cur->u_len, &cur->e_f};
            cta_load_u64<3>(csrc, cv);
        }
        long long f = (long long)cv[0];
        long long nunits = (long long)cv[1];
        long long e_f = (long long)cv[2];
        if (f == 0) {
            // closing record: marks the end time of the last level
            if (gtid == 0 && p.log && level < p.log_cap) {
                bfs_level_record r;
                r.level = level;
                r.dir = -1;
                r.f = 0;
                r.e_f = 0;
                r.m_u = m_u;
                r.t_ns = (int64_t)globaltimer_ns();
                p.log[level] = r;
            }
            done = true;
            break;
        }
        if (level >= p.max_levels) {
            if (gtid == 0) atomicCAS(&ctl->bar.err, 0, (int)DEV_LEVELS);
            done = true;
            break;
        }
        if (level > 0) m_u -= e_f;
        int dir = decide_dir(p, level, f, e_f, m_u, f_prev, prev_dir, s_feat, &s_mlp_out, mlp_w);
        // a cluster launch leaves every level but a small push-queue level to
        // the grid-wide launch (the state, m_u as it was before the level, is
        // saved as the loop exits)
        if (CL && (dir != BFS_DIR_PUSH_QUEUE || e_f > p.small_ef_max || q_valid != level)) {
            if (level > 0) m_u += e_f;
            break;
        }
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
        int2* u_cur = (level & 1) ? p.U1 : p.U0;
        uint32_t* f_cur = (level & 1) ? p.F1 : p.F0;
        uint32_t* f_nxt = (level & 1) ? p.F0 : p.F1;
        // Variant 6: a push-queue level expands F_i in ascending vertex order
        const bool sort_dev = SORT && p.frontier_sort == BFS_SORT_DEVICE && dir == BFS_DIR_PUSH_QUEUE;
        if ((dir != BFS_DIR_PUSH_QUEUE || sort_dev) && bm_valid != level) {
            // queue -> bitmap conversion of F_i
            for (long long w = gtid; w < p.W; w += gthreads) f_cur[w] = 0;
            if (!level_sync<CL>(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            for (long long q = gtid; q < f; q += gthreads) {
                const int v = __ldcg(q_cur + q).x;
                atomicOr(f_cur + (v >> 5), 1u << (v & 31));
            }
            if (!level_sync<CL>(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            bm_valid = level;
        }
        if (sort_dev) {
            // ordered bitmap -> queue of F_i; chunk units only when no push
            // level has made them (after pull levels)
            sort_count<T>(p, sm, f_cur);
            if (!level_sync<CL>(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            sort_emit<T>(p, sm, f_cur, q_cur, u_cur, cur, q_valid != level);
            if (!level_sync<CL>(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            const unsigned long long* const usrc[1] = {&cur->u_len};
            unsigned long long uv[1];
            cta_load_u64<1>(usrc, uv);
            nunits = (long long)uv[0];
            q_valid = level;
        } else if (dir == BFS_DIR_PUSH_QUEUE && q_valid != level) {
            // bitmap -> queue conversion of F_i (after pull levels)
            bitmap_to_queue<T>(p, sm, f_cur, q_cur, u_cur, cur);
            if (!level_sync<CL>(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            const unsigned long long* const usrc[1] = {&cur->u_len};
            unsigned long long uv[1];
            cta_load_u64<1>(usrc, uv);
            nunits = (long long)uv[0];
            q_valid = level;
        }
        if (gtid == 0) {
            Counters* z = &cs[(level + 2) % 3];
            z->q_len = 0;
            z->u_len = 0;
            z->e_f = 0;
            z->conv = 0;
            z->e_len = 0;
        }
        LevelCtx L;
        L.level = level;
        L.depth = depth;
        L.parent = parent;
        L.q_next = (level & 1) ? p.Q0 : p.Q1;
        L.u_next = (level & 1) ? p.U0 : p.U1;
        L.next = nxt;
        L.ef = 0;
        L.cnt = 0;
        L.qv = qs->qv + warp * QBUF;
        L.qb = qs->qb + warp * QBUF;
        L.qe = qs->qe + warp * QBUF;
        L.qn = 0;
        L.qcap = p.n;
        L.err = &p.ctl->bar.err;
        L.precheck = push_precheck(m_u, p.m, e_f);
        if (dir == BFS_DIR_PULL) {
            pull_level_list<false, T>(p, L, f_cur, f_nxt, sm.list, reinterpret_cast<uint16_t*>(bfs1_dyn));
        } else {
            push_level<T, SORT>(p, L, sm, dir, q_cur, u_cur, f_cur, f, nunits, q_valid == level);
            if (p.push_filter != BFS_PUSH_FUSED) {
                // the advance is complete everywhere before any pair is claimed
                if (!level_sync<CL>(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
                const unsigned long long* const esrc[1] = {&nxt->e_len};
                unsigned long long ev[1];
                cta_load_u64<1>(esrc, ev);
                filter_level<T>(p, L, (long long)min(ev[0], (unsigned long long)p.ecap));
            }
        }
        // e_f (and |F_{i+1}| for pull) of the next frontier: one atomic per
        // CTA, issued by thread 0 after the barrier's own __syncthreads and
        // before its arrival
        const unsigned long long ef = warp_sum(L.ef);
        const unsigned long long cn = warp_sum(L.cnt);
        if ((threadIdx.x & 31) == 0) {
            sm.red[warp] = ef;
            sm.red2[warp] = cn;
        }
        const bool pull_dir = dir == BFS_DIR_PULL;
        if (pull_dir) bm_valid = level + 1;
        else q_valid = level + 1;
        prev_dir = dir;
        f_prev = f;
        const int done_level = level;
        ++level;
        const bool ok = level_sync<CL>(&ctl->bar, nblocks, bar_target, p.timeout_ns, [&]() {
            unsigned long long te = 0, tc = 0;
            for (int i = 0; i < T / 32; ++i) {
                te += sm.red[i];
                tc += sm.red2[i];
            }
            if (te) atomicAdd(&nxt->e_f, te);
            if (pull_dir && tc) atomicAdd(&nxt->q_len, tc);
#if BFS_LEVEL_PHASES
            if (p.log && done_level < p.log_cap / 2)
                atomicMax((unsigned long long*)&p.log[p.log_cap / 2 + done_level].t_ns, (unsigned long long)globaltimer_ns());
#endif
        }, [&]() {
            s_cnt[0] = ld_counter<CL>(&nxt->q_len);
            s_cnt[1] = ld_counter<CL>(&nxt->u_len);
            s_cnt[2] = ld_counter<CL>(&nxt->e_f);
        });
        if (!ok) return;
        // the next iteration reads them before any CTA can change them: the
        // slot is zeroed two levels later
        s_cnt_ok = true;
#if BFS_LEVEL_PHASES
        if (gtid == 0 && p.log && done_level < p.log_cap / 2) p.log[p.log_cap / 2 + done_level].m_u = (int64_t)globaltimer_ns();
#else
        (void)done_level;
#endif
    }
    // No barrier before the next search: after the last level's barrier a CTA
    // reads only its own shared memory (s_cnt) before it leaves the loop, so
    // the next search's init may overwrite P, the queues and the other
    // counter set while slower CTAs are still leaving.
    }  // searches
    if (CL && gtid == 0) {
        // the grid-wide launch that continues the search reads them there
        for (int k = 0; k < 3; ++k) ctl->slot[k] = s_ctr[k];
    }
    if (gtid == 0) {
        ctl->next_level = level;
        ctl->prev_dir = prev_dir;
        ctl->bm_valid = bm_valid;
        ctl->q_valid = q_valid;
        ctl->m_u = m_u;
        ctl->f_prev = f_prev;
        ctl->done = done ? 1 : 0;
        ctl->bar_base = bar_target;
    }
    if constexpr (CL) {
        // CTA 0's shared memory holds the counters the other CTAs read
        // through distributed shared memory: no CTA leaves before all are done
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
}

// At most 40 registers a thread for T <= 512, so that 1536 threads (48 warps
// of memory-level parallelism for the latency-bound gathers) fit on an SM.
template <int T, bool SORT, bool CL = false>
__global__ void __launch_bounds__(T, (1536 / T) > 0 ? (1536 / T) : 1) bfs1_kernel(Params1 p) {
    bfs1_body<T, SORT, CL>(p);
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
    const void* k = p.frontier_sort != BFS_SORT_NONE ? (const void*)bfs1_kernel<T, true> : (const void*)bfs1_kernel<T, false>;
    return cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(T), args, bfs1_dyn_smem<T>(), st);
}

template <int T>
int max_coop_blocks(int blocks_per_sm) {
    int per_sm = 0;
    int per_sm_sorted = 0;
    const size_t dyn = bfs1_dyn_smem<T>();
    cudaFuncSetAttribute(bfs1_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    cudaFuncSetAttribute(bfs1_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs1_kernel<T, false>, T, dyn);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_sorted, bfs1_kernel<T, true>, T, dyn);
    per_sm = std::min(per_sm, per_sm_sorted);  // one grid size whichever instantiation runs
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
    return per_sm * num_sms();
}

// Small levels (bfs_options.small_levels): one cluster of 1024-thread CTAs,
// 16 where the GPU can co-schedule such a cluster, else 8 (0: none).
constexpr int SMALL_T = 1024;
static int small_cluster_size() {
    static int cached[64] = {};
    const int d = device_id();
    if (d < 0 || d >= 64) return 0;
    if (cached[d]) return cached[d] > 0 ? cached[d] : 0;
    int found = -1;
    const size_t dyn = bfs1_dyn_smem<SMALL_T>();
    auto k = bfs1_kernel<SMALL_T, false, true>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) == cudaSuccess) {
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        for (int cl : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cl);
            cfg.blockDim = dim3(SMALL_T);
            cfg.dynamicSmemBytes = dyn;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cl;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, k, &cfg) == cudaSuccess && nc >= 1) {
                found = cl;
                break;
            }
        }
    }
    cudaGetLastError();  // an unsupported size leaves a non-sticky error
    cached[d] = found;
    return found > 0 ? found : 0;
}

static cudaError_t launch_small(const Params1& p, int cl, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(SMALL_T);
    cfg.dynamicSmemBytes = bfs1_dyn_smem<SMALL_T>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bfs1_kernel<SMALL_T, false, true>, p);
}

// The cluster size to run a search's small levels with, 0 for none.  The
// automatic choice takes graphs of bounded degree (grid- and road-like),
// whose frontiers stay small for many levels; on ER-22 (maximum degree
// about 40) the cluster's first levels and the second launch cost more
// than the cheaper barrier saves.
static int small_levels_for(const bfs_graph* g, const bfs_options& o) {
    if (o.mode != BFS_MODE_PERSISTENT || o.frontier_sort != BFS_SORT_NONE || o.push_filter != BFS_PUSH_FUSED) return 0;
    if (o.small_levels == BFS_SMALL_OFF) return 0;
    if (o.small_levels == BFS_SMALL_AUTO && g->deg_max > 16) return 0;
    return small_cluster_size();
}

// The small-level launch pair of one search: the -1 rows stored by the copy
// engines' memset (the cluster's few SMs would take long to store them),
// the cluster launch, then the grid-wide launch that finishes the search.
template <typename L>
static cudaError_t run_small_pair(Params1 q, int cl, const L& launcher, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(q.depth, 0xff, (size_t)q.n * sizeof(int32_t), st);
    if (!e && q.parent) e = cudaMemsetAsync(q.parent, 0xff, (size_t)q.n * sizeof(int32_t), st);
    q.do_init = 1;
    q.level_count = INT32_MAX / 2;
    q.small_ef_max = (int64_t)cl * SMALL_T;  // about one frontier edge a thread
    q.rows_filled = 1;
    if (!e) e = launch_small(q, cl, st);
    q.do_init = 0;
    q.small_ef_max = 0;
    q.rows_filled = 0;
    if (!e) e = launcher(q, st);
    return e;
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
        ok = cudaMalloc(&w->F[i], w->W * 4) == cudaSuccess && cudaMalloc(&w->Q[i], (int64_t)g->n * sizeof(int4)) == cudaSuccess &&
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


// Kernel parameters of one single-source run (workspace, graph, options).
static bfs_status make_params(bfs_graph* g, Workspace1* w, const bfs_options& o, const float* mlp_dev, int32_t src_value,
                              int32_t* depth, int32_t* parent, cudaStream_t st, Params1& p) {
    p = Params1{};
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
    p.srcs = nullptr;
    p.nsrc = 1;
    p.sticky = w->d_sticky;
    p.depth = depth;
    p.parent = parent;
    p.policy = o.policy;
    p.force_dir = -1;
    p.alpha = o.alpha;
    p.beta = o.beta;
    p.gamma = o.gamma;
    p.mlp = mlp_dev;
    p.deg_max = g->deg_max;
    p.chunk = o.chunk;
    p.medium = o.medium;
    p.pull_serial = o.pull_serial;
    p.aggregate = o.claim_aggregate;
    p.push_filter = o.push_filter;
    p.frontier_sort = o.frontier_sort;
    if (o.frontier_sort == BFS_SORT_DEVICE) {
        if (!w->cta_cnt && cudaMalloc(&w->cta_cnt, 4096 * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            return fail(BFS_ENOMEM, "frontier sort counts");
        }
        p.cta_cnt = w->cta_cnt;
    }
    if (o.push_filter != BFS_PUSH_FUSED) {
        // edge frontier: one level's advance appends at most m pairs
        if (w->ecap < g->m) {
            cudaFree(w->E);
            w->E = nullptr;
            w->ecap = 0;
            if (cudaMalloc(&w->E, (size_t)g->m * sizeof(int2)) != cudaSuccess) {
                cudaGetLastError();
                return fail(BFS_ENOMEM, "edge frontier of %lld pairs", (long long)g->m);
            }
            w->ecap = g->m;
        }
        p.E = w->E;
        p.ecap = w->ecap;
    }
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
#if BFS_LEVEL_PHASES
        BFS_CUDA(cudaMemsetAsync(w->d_log, 0, sizeof(bfs_level_record) * o.level_log_cap, st));
#endif
        p.log = w->d_log;
        p.log_cap = o.level_log_cap;
    }
    return BFS_OK;
}

struct CoopLauncher {
    int T = 512, blocks = 0;
    explicit CoopLauncher(const bfs_options& o) {
        T = o.block_threads;
        switch (T) {
            case 256: blocks = max_coop_blocks<256>(o.blocks_per_sm); break;
            case 1024: blocks = max_coop_blocks<1024>(o.blocks_per_sm); break;
            default: T = 512; blocks = max_coop_blocks<512>(o.blocks_per_sm); break;
        }
    }
    cudaError_t operator()(const Params1& pp, cudaStream_t st) const {
        switch (T) {
            case 256: return launch_bfs1<256>(pp, blocks, st);
            case 1024: return launch_bfs1<1024>(pp, blocks, st);
            default: return launch_bfs1<512>(pp, blocks, st);
        }
    }
};

// Runs one source (already validated).  Returns after enqueueing unless a
// host readback is needed (host loop, level log, level count); device-side
// failures of asynchronous runs are reported by sync_graph / bfs_sync.
bfs_status run_single(bfs_graph* g, int32_t src_value, int32_t* depth, int32_t* parent, const bfs_options& o,
                      const float* mlp_dev, cudaStream_t st) {
    Workspace1* w;
    bfs_status s = ensure_ws1(g, o.chunk, st, &w);
    if (s != BFS_OK) return s;
    Params1 p;
    s = make_params(g, w, o, mlp_dev, src_value, depth, parent, st, p);
    if (s != BFS_OK) return s;
    if (o.mode == BFS_MODE_GRAPH) return run_graph_mode(g, w, p, src_value, depth, parent, o, st);
    BFS_CUDA(cudaMemsetAsync(w->ctl, 0, sizeof(Ctl1), st));
    CoopLauncher launcher(o);
    if (o.frontier_sort == BFS_SORT_DEVICE && launcher.blocks > 4096)
        return fail(BFS_EINVAL, "frontier_sort supports at most 4096 CTAs (launch has %d)", launcher.blocks);
    auto launch = [&](const Params1& pp) -> cudaError_t { return launcher(pp, st); };
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
        if (const int cl = small_levels_for(g, o)) {
            // the small levels in one cluster, the rest grid-wide (a launch
            // that finds the search done returns at once)
            BFS_CUDA(run_small_pair(p, cl, launcher, st));
        } else {
            BFS_CUDA(launch(p));
        }
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
#if BFS_LEVEL_PHASES
        int nl = o.level_log_cap;  // the second half holds the phase times
#else
        int nl = std::min(h.next_level + (h.done ? 1 : 0), o.level_log_cap);
#endif
        if (nl > 0) BFS_CUDA(cudaMemcpy(o.level_log, w->d_log, sizeof(bfs_level_record) * nl, cudaMemcpyDeviceToHost));
    }
    return BFS_OK;
}

// k sources, one search after another, all in ONE persistent launch (device
// outputs [k][n], persistent drive, no level log): the per-search launch and
// control-block reset are paid once.  A barrier separates the searches.
bfs_status run_single_many(bfs_graph* g, const int32_t* src_host, int32_t k, int32_t* depth, int32_t* parent,
                           const bfs_options& o, const float* mlp_dev, cudaStream_t st) {
    Workspace1* w;
    bfs_status s = ensure_ws1(g, o.chunk, st, &w);
    if (s != BFS_OK) return s;
    Params1 p;
    s = make_params(g, w, o, mlp_dev, src_host[0], depth, parent, st, p);
    if (s != BFS_OK) return s;
    if (w->src_cap < k) {
        cudaFree(w->d_srcs);
        w->d_srcs = nullptr;
        w->src_cap = 0;
        if (cudaMalloc(&w->d_srcs, (size_t)k * 4) != cudaSuccess) {
            cudaGetLastError();
            return fail(BFS_ENOMEM, "sources of %d searches", k);
        }
        w->src_cap = k;
    }
    BFS_CUDA(cudaMemcpyAsync(w->d_srcs, src_host, (size_t)k * 4, cudaMemcpyHostToDevice, st));
    p.srcs = w->d_srcs;
    p.nsrc = k;
    CoopLauncher launcher(o);
    if (o.frontier_sort == BFS_SORT_DEVICE && launcher.blocks > 4096)
        return fail(BFS_EINVAL, "frontier_sort supports at most 4096 CTAs (launch has %d)", launcher.blocks);
    if (const int cl = small_levels_for(g, o)) {
        // a pair of launches per source: the small levels in one cluster,
        // the rest grid-wide
        for (int32_t si = 0; si < k; ++si) {
            Params1 q = p;
            q.srcs = nullptr;
            q.nsrc = 1;
            q.src_value = src_host[si];
            q.depth = depth + (int64_t)si * g->n;
            q.parent = parent ? parent + (int64_t)si * g->n : nullptr;
            BFS_CUDA(cudaMemsetAsync(w->ctl, 0, sizeof(Ctl1), st));
            BFS_CUDA(run_small_pair(q, cl, launcher, st));
        }
        return BFS_OK;
    }
    BFS_CUDA(cudaMemsetAsync(w->ctl, 0, sizeof(Ctl1), st));
    p.do_init = 1;
    p.level_count = INT32_MAX / 2;
    BFS_CUDA(launcher(p, st));
    return BFS_OK;
}

}  // namespace bfsgb

// ------------------------------------------------------------ level profiling
using namespace bfsgb;

// Per-level timings of the three traversal forms from identical states: the
// training signal of the learned direction policy.  See bfs.h.
extern "C" bfs_status bfs_profile_levels(const bfs_graph* gc, int32_t source, const bfs_options* opt, int32_t repeats,
                                         int32_t max_levels, float* features, float* times_us, int32_t* taken,
                                         int32_t* levels, void* cuda_stream) {
    bfs_graph* g = const_cast<bfs_graph*>(gc);
    if (!g || !features || !times_us || !levels) return fail(BFS_EINVAL, "null argument");
    if (source < 0 || source >= g->n) return fail(BFS_EINVAL, "source %d outside [0, %d)", source, g->n);
    if (repeats < 1 || max_levels < 1) return fail(BFS_EINVAL, "repeats and max_levels must be >= 1");
    bfs_options o;
    bfs_options_init(&o);
    if (opt) {
        if (opt->struct_size != sizeof(bfs_options)) return fail(BFS_EINVAL, "bfs_options.struct_size mismatch");
        o = *opt;
    }
    if (o.policy == BFS_POLICY_MLP || o.policy == BFS_POLICY_SCHEDULE) o.policy = BFS_POLICY_HEURISTIC;
    o.level_log = nullptr;
    o.levels_out = nullptr;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::lock_guard<std::mutex> lk(g->lock);
    Workspace1* w;
    bfs_status s = ensure_ws1(g, o.chunk, st, &w);
    if (s != BFS_OK) return s;
    if (!w->stage_depth) {
        if (cudaMalloc(&w->stage_depth, (size_t)g->n * 4) != cudaSuccess ||
            cudaMalloc(&w->stage_parent, (size_t)g->n * 4) != cudaSuccess) {
            cudaGetLastError();
            return fail(BFS_ENOMEM, "profiling outputs");
        }
    }
    Params1 p;
    s = make_params(g, w, o, nullptr, source, w->stage_depth, w->stage_parent, st, p);
    if (s != BFS_OK) return s;
    uint32_t *snapP = nullptr, *snapF = nullptr;
    Ctl1* snapC = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(snapP);
        cudaFree(snapF);
        cudaFree(snapC);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&snapP, w->W * 4) != cudaSuccess || cudaMalloc(&snapF, w->W * 4) != cudaSuccess ||
        cudaMalloc(&snapC, sizeof(Ctl1)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(BFS_ENOMEM, "profiling snapshot");
    }
    CoopLauncher launch(o);
    cudaError_t e = cudaMemsetAsync(w->ctl, 0, sizeof(Ctl1), st);
    p.do_init = 1;
    p.level_count = 0;
    if (!e) e = launch(p, st);
    p.do_init = 0;
    p.level_count = 1;
    int L = 0;
    std::vector<float> samples(repeats);
    while (!e && L < max_levels) {
        e = cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl1), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (e) break;
        Ctl1 h = *w->h_ctl;
        if (h.bar.err) {
            cleanup();
            return device_error(h.bar.err, o.barrier_timeout_ns);
        }
        const Counters& c = h.slot[L % 3];
        if (h.done || c.q_len == 0) break;
        long long m_u = L > 0 ? h.m_u - (long long)c.e_f : h.m_u;
        policy_features(features + (size_t)L * BFS_MLP_IN, (long long)c.q_len, (long long)c.e_f, m_u, h.f_prev, L,
                        h.prev_dir, g->n, g->m, g->deg_max);
        uint32_t* f_cur = (L & 1) ? w->F[1] : w->F[0];
        e = cudaMemcpyAsync(snapP, w->P, w->W * 4, cudaMemcpyDeviceToDevice, st);
        if (!e) e = cudaMemcpyAsync(snapF, f_cur, w->W * 4, cudaMemcpyDeviceToDevice, st);
        if (!e) e = cudaMemcpyAsync(snapC, w->ctl, sizeof(Ctl1), cudaMemcpyDeviceToDevice, st);
        for (int d = 0; d < 3 && !e; ++d) {
            Params1 q = p;
            q.force_dir = d;
            for (int r = 0; r < repeats && !e; ++r) {
                e = cudaMemcpyAsync(w->P, snapP, w->W * 4, cudaMemcpyDeviceToDevice, st);
                if (!e) e = cudaMemcpyAsync(f_cur, snapF, w->W * 4, cudaMemcpyDeviceToDevice, st);
                if (!e) e = cudaMemcpyAsync(w->ctl, snapC, sizeof(Ctl1), cudaMemcpyDeviceToDevice, st);
                if (!e) e = cudaEventRecord(e0, st);
                if (!e) e = launch(q, st);
                if (!e) e = cudaEventRecord(e1, st);
                if (!e) e = cudaEventSynchronize(e1);
                float ms = 0;
                if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
                samples[r] = ms * 1000.0f;
            }
            std::sort(samples.begin(), samples.end());
            times_us[(size_t)L * 3 + d] = samples[repeats / 2];
        }
        // continue with the plain method's own choice from the same state
        if (!e) e = cudaMemcpyAsync(w->P, snapP, w->W * 4, cudaMemcpyDeviceToDevice, st);
        if (!e) e = cudaMemcpyAsync(f_cur, snapF, w->W * 4, cudaMemcpyDeviceToDevice, st);
        if (!e) e = cudaMemcpyAsync(w->ctl, snapC, sizeof(Ctl1), cudaMemcpyDeviceToDevice, st);
        if (!e) e = launch(p, st);
        if (!e) e = cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl1), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (!e && taken) taken[L] = w->h_ctl->prev_dir;
        ++L;
    }
    cleanup();
    if (e) return cuda_fail(e, "level profiling");
    *levels = L;
    return BFS_OK;
}
