// bfs_graph.cu -- the level loop of Cascade 1 as a CUDA graph with a
// conditional WHILE node, so that no host work happens per level.
//
//   init kernel (ordinary launch: outputs, P, F_0 = {s}, counters)
//   WHILE (||F_i|| != 0):
//       decide      <<<1, 32>>>   direction of level i from the device counters;
//                                 sets the conditions of the nodes below
//       IF q2bm     { zero F_i bitmap -> scatter the queue into it }
//       IF bm2q     { bitmap -> queue (+ chunk units) after pull levels }
//       SWITCH dir  { 0: push-queue | 1: push-bitmap | 2: pull }
//
// Unlike the persistent kernel, each level's expansion is its own launch, so
// the pull kernel runs at full occupancy with few registers (one warp per
// 32-vertex word of P, lane = vertex), while the push kernel keeps the tile /
// chunk-unit load balance of level.cuh.  The graph is instantiated once per
// workspace and option set; a run's source and outputs reach it through the
// device control block written by the init kernel.
#include "level.cuh"

#include <cstring>

namespace bfsgb {

bfs_status device_error(int err, int64_t timeout_ns);

namespace {

constexpr int GT = 512;        // threads of the push / conversion kernels
constexpr int PULL_T = 256;    // threads of the pull kernel

__global__ void __launch_bounds__(256) g_init(Params1 p, int32_t s, int32_t* depth, int32_t* parent) {
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    for (long long w = gtid; w < p.W; w += gthreads) {
        unsigned bits = __ldg(p.isolated + w);
        if (w == (s >> 5)) bits |= 1u << (s & 31);
        if (w == p.W - 1 && (p.n & 31)) bits |= ~((1u << (p.n & 31)) - 1u);  // phantom vertices
        p.P[w] = bits;
    }
    for (long long v = gtid; v < p.n; v += gthreads) {
        depth[v] = (v == s) ? 0 : -1;
        if (parent) parent[v] = (v == s) ? s : -1;
    }
    if (gtid == 0) {
        Ctl1* ctl = p.ctl;
        const int rb = __ldg(p.row_ptr + s), re = __ldg(p.row_ptr + s + 1);
        const int deg = re - rb;
        p.Q0[0] = make_int4(s, rb, re, 0);
        int nch = deg >= p.chunk ? (deg + p.chunk - 1) / p.chunk : 0;
        for (int c = 0; c < nch; ++c) p.U0[c] = make_int2(s, c);
        for (int k = 0; k < 3; ++k) {
            ctl->slot[k].q_len = 0;
            ctl->slot[k].u_len = 0;
            ctl->slot[k].e_f = 0;
            ctl->slot[k].conv = 0;
        }
        ctl->slot[0].q_len = 1;
        ctl->slot[0].u_len = nch;
        ctl->slot[0].e_f = deg;
        ctl->bar.count = 0;
        ctl->bar.abort = 0;
        ctl->bar.err = 0;
        ctl->next_level = 0;
        ctl->prev_dir = BFS_DIR_PUSH_QUEUE;
        ctl->bm_valid = -1;
        ctl->q_valid = 0;
        ctl->done = 0;
        ctl->m_u = p.m - deg;
        ctl->f_prev = 0;
        ctl->cur_level = -1;
        ctl->cur_dir = BFS_DIR_PUSH_QUEUE;
        ctl->units_valid = 1;
        ctl->src = s;
        ctl->depth = depth;
        ctl->parent = parent;
    }
}

// Direction of the next level; every decision input lives in the control
// block.  One warp (the MLP is evaluated warp-cooperatively).
__global__ void g_decide(Params1 p, cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_q2bm,
                         cudaGraphConditionalHandle h_bm2q, cudaGraphConditionalHandle h_dir) {
    __shared__ float s_feat[BFS_MLP_IN];
    __shared__ float s_out;
    Ctl1* ctl = p.ctl;
    const int level = ctl->next_level;
    int prev_dir = ctl->prev_dir;
    int bm_valid = ctl->bm_valid, q_valid = ctl->q_valid;
    long long m_u = ctl->m_u, f_prev = ctl->f_prev;
    if (ctl->cur_level >= 0) {  // account for the level that just ran
        if (ctl->cur_dir == BFS_DIR_PULL) bm_valid = level;
        else q_valid = level;
        prev_dir = ctl->cur_dir;
    }
    Counters* cur = &ctl->slot[level % 3];
    const long long f = (long long)cur->q_len;
    const long long e_f = (long long)cur->e_f;
    const bool over = level >= p.max_levels;
    if (f == 0 || over || ctl->bar.err) {
        if (threadIdx.x == 0) {
            if (over && f != 0) atomicCAS(&ctl->bar.err, 0, (int)DEV_LEVELS);
            int e = ctl->bar.err;
            if (e) atomicCAS(p.sticky, 0, e);
            ctl->done = 1;
            cudaGraphSetConditional(h_while, 0);
            cudaGraphSetConditional(h_q2bm, 0);
            cudaGraphSetConditional(h_bm2q, 0);
            cudaGraphSetConditional(h_dir, 3);  // no branch
        }
        return;
    }
    if (level > 0) m_u -= e_f;
    int dir = decide_dir(p, level, f, e_f, m_u, f_prev, prev_dir, s_feat, &s_out);
    if (threadIdx.x == 0) {
        bool q2bm = dir != BFS_DIR_PUSH_QUEUE && bm_valid != level;
        bool bm2q = dir == BFS_DIR_PUSH_QUEUE && q_valid != level;
        ctl->units_valid = (q_valid == level || bm2q) ? 1 : 0;
        if (q2bm) bm_valid = level;
        if (bm2q) q_valid = level;
        Counters* z = &ctl->slot[(level + 2) % 3];
        z->q_len = 0;
        z->u_len = 0;
        z->e_f = 0;
        z->conv = 0;
        if (p.log && level < p.log_cap) {
            bfs_level_record r;
            r.level = level;
            r.dir = dir;
            r.f = f;
            r.e_f = e_f;
            r.m_u = m_u;
            r.t_ns = (int64_t)globaltimer_ns();
            p.log[level] = r;
        }
        ctl->cur_level = level;
        ctl->cur_dir = dir;
        ctl->next_level = level + 1;
        ctl->prev_dir = prev_dir;
        ctl->bm_valid = bm_valid;
        ctl->q_valid = q_valid;
        ctl->m_u = m_u;
        ctl->f_prev = f;
        cudaGraphSetConditional(h_while, 1);
        cudaGraphSetConditional(h_q2bm, q2bm ? 1 : 0);
        cudaGraphSetConditional(h_bm2q, bm2q ? 1 : 0);
        cudaGraphSetConditional(h_dir, (unsigned)dir);
    }
}

// What a level kernel needs from the control block, read by thread 0 and
// shared with the CTA: every thread of every CTA reading the same words put
// thousands of requests on one L2 sector (see cta_load_u64).
struct GHead {
    int level, units_valid;
    long long f, nunits, m_u, e_f;
    int32_t* depth;
    int32_t* parent;
};

__device__ __forceinline__ GHead cta_head(const Ctl1* ctl) {
    __shared__ GHead s;
    if (threadIdx.x == 0) {
        GHead h;
        h.level = ctl->cur_level;
        const Counters* c = &ctl->slot[h.level % 3];
        h.f = (long long)c->q_len;
        h.nunits = (long long)c->u_len;
        h.m_u = ctl->m_u;
        h.e_f = (long long)c->e_f;
        h.units_valid = ctl->units_valid;
        h.depth = ctl->depth;
        h.parent = ctl->parent;
        s = h;
    }
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(256) g_q2bm_zero(Params1 p) {
    const int level = cta_head(p.ctl).level;
    uint32_t* f_cur = (level & 1) ? p.F1 : p.F0;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < p.W; w += (long long)gridDim.x * blockDim.x)
        f_cur[w] = 0;
}

__global__ void __launch_bounds__(256) g_q2bm_scatter(Params1 p) {
    const GHead h = cta_head(p.ctl);
    const int level = h.level;
    uint32_t* f_cur = (level & 1) ? p.F1 : p.F0;
    const int4* q_cur = (level & 1) ? p.Q1 : p.Q0;
    const long long f = h.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < f; q += (long long)gridDim.x * blockDim.x) {
        const int v = q_cur[q].x;
        atomicOr(f_cur + (v >> 5), 1u << (v & 31));
    }
}

__global__ void __launch_bounds__(GT) g_bm2q(Params1 p) {
    __shared__ TileSmem<GT> sm;
    const int level = cta_head(p.ctl).level;
    uint32_t* f_cur = (level & 1) ? p.F1 : p.F0;
    int4* q_cur = (level & 1) ? p.Q1 : p.Q0;
    int2* u_cur = (level & 1) ? p.U1 : p.U0;
    bitmap_to_queue<GT>(p, sm, f_cur, q_cur, u_cur, &p.ctl->slot[level % 3]);
}

template <int DIR>
__global__ void __launch_bounds__(GT, 2) g_push(Params1 p) {
    __shared__ TileSmem<GT> sm;
    __shared__ QueueStage<GT> qs;
    Ctl1* ctl = p.ctl;
    const GHead h = cta_head(ctl);
    const int level = h.level;
    Counters* nxt = &ctl->slot[(level + 1) % 3];
    const long long f = h.f;
    const long long nunits = h.nunits;
    LevelCtx L;
    L.level = level;
    L.depth = h.depth;
    L.parent = h.parent;
    L.q_next = (level & 1) ? p.Q0 : p.Q1;
    L.u_next = (level & 1) ? p.U0 : p.U1;
    L.next = nxt;
    L.ef = 0;
    L.cnt = 0;
    L.qv = qs.qv + (threadIdx.x >> 5) * QBUF;
    L.qb = qs.qb + (threadIdx.x >> 5) * QBUF;
    L.qe = qs.qe + (threadIdx.x >> 5) * QBUF;
    L.qn = 0;
    L.qcap = p.n;
    L.err = &p.ctl->bar.err;
    L.precheck = push_precheck(h.m_u, p.m, h.e_f);
    const int4* q_cur = (level & 1) ? p.Q1 : p.Q0;
    const int2* u_cur = (level & 1) ? p.U1 : p.U0;
    const uint32_t* f_cur = (level & 1) ? p.F1 : p.F0;
    push_level<GT>(p, L, sm, DIR, q_cur, u_cur, f_cur, f, nunits, h.units_valid != 0);
    unsigned long long ef = warp_sum(L.ef);
    if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = ef;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < GT / 32; ++i) t += sm.red[i];
        if (t) atomicAdd(&nxt->e_f, t);
    }
}

// Pull level at full occupancy (few registers): pull_level with
// non-coherent loads of P and F_i, which no CTA writes during this kernel
// except the word owner after its last read.
__global__ void __launch_bounds__(PULL_T) g_pull(Params1 p) {
    __shared__ unsigned long long s_ef[PULL_T / 32], s_cn[PULL_T / 32];
    __shared__ PullWarpSmem s_pull[PULL_T / 32];
    Ctl1* ctl = p.ctl;
    const GHead h = cta_head(ctl);
    const int level = h.level;
    LevelCtx L;
    L.level = level;
    L.depth = h.depth;
    L.parent = h.parent;
    L.ef = 0;
    L.cnt = 0;
    const uint32_t* f_cur = (level & 1) ? p.F1 : p.F0;
    uint32_t* f_next = (level & 1) ? p.F0 : p.F1;
    pull_level<true>(p, L, f_cur, f_next, s_pull[threadIdx.x >> 5]);
    unsigned long long ef = warp_sum(L.ef);
    unsigned long long cn = warp_sum(L.cnt);
    if (lane_id() == 0) {
        s_ef[threadIdx.x >> 5] = ef;
        s_cn[threadIdx.x >> 5] = cn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long te = 0, tc = 0;
        for (int i = 0; i < PULL_T / 32; ++i) {
            te += s_ef[i];
            tc += s_cn[i];
        }
        Counters* nxt = &ctl->slot[(level + 1) % 3];
        if (te) atomicAdd(&nxt->e_f, te);
        if (tc) atomicAdd(&nxt->q_len, tc);
    }
}

template <typename K>
int occupancy_blocks(K kernel, int threads) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    return (per_sm < 1 ? 1 : per_sm) * num_sms();
}

struct KernelNode {
    void* func;
    int grid, block;
};

cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, size_t ndeps, void* func,
                       int grid, int block, void** args) {
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

cudaError_t add_conditional(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, size_t ndeps,
                            cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, unsigned size,
                            cudaGraph_t** bodies) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = size;
    cudaError_t e = cudaGraphAddNode(node, g, deps, nullptr, ndeps, &np);
    if (e == cudaSuccess) *bodies = np.conditional.phGraph_out;
    return e;
}

// Build and instantiate the level-loop graph for the static part of `p`.
cudaError_t build_graph(Workspace1* w, Params1 p, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e) return e;
    cudaGraphConditionalHandle h_while;
    cudaGraph_t* wb = nullptr;
    cudaGraphNode_t n_while;
    e = cudaGraphConditionalHandleCreate(&h_while, g, 1, cudaGraphCondAssignDefault);
    if (!e) e = add_conditional(g, &n_while, nullptr, 0, h_while, cudaGraphCondTypeWhile, 1, &wb);
    cudaGraph_t body = wb ? wb[0] : nullptr;
    cudaGraphConditionalHandle h_q2bm, h_bm2q, h_dir;
    if (!e) e = cudaGraphConditionalHandleCreate(&h_q2bm, body, 0, 0);
    if (!e) e = cudaGraphConditionalHandleCreate(&h_bm2q, body, 0, 0);
    if (!e) e = cudaGraphConditionalHandleCreate(&h_dir, body, 3, 0);
    const int nb_small = num_sms() * 4;
    const int nb_push = occupancy_blocks(g_push<BFS_DIR_PUSH_QUEUE>, GT);
    const int nb_bm = occupancy_blocks(g_bm2q, GT);
    const int nb_pull = occupancy_blocks(g_pull, PULL_T);
    void* a_decide[] = {&p, &h_while, &h_q2bm, &h_bm2q, &h_dir};
    void* a_p[] = {&p};
    cudaGraphNode_t n_dec, n_q2bm, n_bm2q, n_dir, tmp, tmp2;
    if (!e) e = add_kernel(body, &n_dec, nullptr, 0, (void*)g_decide, 1, 32, a_decide);
    cudaGraph_t* bq = nullptr;
    if (!e) e = add_conditional(body, &n_q2bm, &n_dec, 1, h_q2bm, cudaGraphCondTypeIf, 1, &bq);
    if (!e) e = add_kernel(bq[0], &tmp, nullptr, 0, (void*)g_q2bm_zero, nb_small, 256, a_p);
    if (!e) e = add_kernel(bq[0], &tmp2, &tmp, 1, (void*)g_q2bm_scatter, nb_small, 256, a_p);
    cudaGraph_t* bb = nullptr;
    if (!e) e = add_conditional(body, &n_bm2q, &n_q2bm, 1, h_bm2q, cudaGraphCondTypeIf, 1, &bb);
    if (!e) e = add_kernel(bb[0], &tmp, nullptr, 0, (void*)g_bm2q, nb_bm, GT, a_p);
    cudaGraph_t* bs = nullptr;
    if (!e) e = add_conditional(body, &n_dir, &n_bm2q, 1, h_dir, cudaGraphCondTypeSwitch, 3, &bs);
    if (!e) e = add_kernel(bs[0], &tmp, nullptr, 0, (void*)g_push<BFS_DIR_PUSH_QUEUE>, nb_push, GT, a_p);
    if (!e) e = add_kernel(bs[1], &tmp, nullptr, 0, (void*)g_push<BFS_DIR_PUSH_BITMAP>, nb_push, GT, a_p);
    if (!e) e = add_kernel(bs[2], &tmp, nullptr, 0, (void*)g_pull, nb_pull, PULL_T, a_p);
    if (!e) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    (void)w;
    return e;
}

}  // namespace

// Runs one source through the graph-mode level loop (p is fully set up by
// run_single; its per-run fields are passed through the init kernel).
bfs_status run_graph_mode(bfs_graph* g, Workspace1* w, Params1& p, int32_t src, int32_t* depth, int32_t* parent,
                          const bfs_options& o, cudaStream_t st) {
    Params1 key = p;
    key.src_value = 0;
    key.depth = nullptr;
    key.parent = nullptr;
    static_assert(sizeof(Params1) <= sizeof(w->gkey), "graph key buffer");
    if (!w->gexec || w->gkey_len != (int)sizeof(Params1) || memcmp(w->gkey, &key, sizeof(Params1)) != 0) {
        BFS_CUDA(cudaStreamSynchronize(st));
        if (w->gexec) {
            cudaGraphExecDestroy(w->gexec);
            w->gexec = nullptr;
        }
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = build_graph(w, key, &ex);
        if (e != cudaSuccess) return cuda_fail(e, "building the level-loop graph");
        w->gexec = ex;
        memcpy(w->gkey, &key, sizeof(Params1));
        w->gkey_len = (int)sizeof(Params1);
    }
    g_init<<<num_sms() * 4, 256, 0, st>>>(key, src, depth, parent);
    BFS_CUDA(cudaGetLastError());
    BFS_CUDA(cudaGraphLaunch(w->gexec, st));
    bool need_sync = o.level_log || o.levels_out;
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
        int nl = h.next_level < o.level_log_cap ? h.next_level : o.level_log_cap;
        if (nl > 0) BFS_CUDA(cudaMemcpy(o.level_log, w->d_log, sizeof(bfs_level_record) * nl, cudaMemcpyDeviceToHost));
    }
    (void)g;
    return BFS_OK;
}

}  // namespace bfsgb
