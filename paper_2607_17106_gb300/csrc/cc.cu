// cc.cu -- connected components by min-label propagation.
//
// The BFS cascade over the same graph tensor G with the min operator of the
// paper's operator table (Section 2) in place of ANY:
//   L_0[v] = v,  F_0 = the vertices with an edge,
//   L_{i+1}[d] = min(L_i[d], min over s in F_i adjacent to d of L_i[s]),
//   F_{i+1} = the vertices whose label dropped, stop when F_{i+1} is empty.
// The fixed point gives every vertex the smallest id of its component.
//
// One persistent cooperative kernel runs every iteration; iterations are
// separated by the grid barrier of common.cuh.  Like BFS, an iteration has a
// push and a pull form of the same Einsum:
//   push (sparse F_i): the words of F_i are dealt over warps, the rows of a
//     word's active vertices flattened over the warp (32 entries a step); a
//     relaxation reads the target's label and issues the atomicMin only when
//     it would lower it.  Rows of at least CC_CHUNK entries become chunk units
//     that whole CTAs expand one edge per thread in the next iteration (safe:
//     labels only drop, and a unit reads its vertex's label when it runs).
//   pull (dense F_i, and iteration 0): every vertex takes the minimum over
//     all its neighbours' labels with no atomics.  This equals the minimum
//     over its neighbours in F_i, because a neighbour outside F_i has already
//     pushed its current label.  Rows of at least CC_CHUNK entries are fixed
//     chunk units, listed once, whose CTA-wide minimum goes in with one
//     atomicMin.
// After each iteration the vertices of F_{i+1} shortcut their labels
// (cc_jump), which leaves the fixed point unchanged and shortens the chains
// a label travels along on long-diameter graphs.
#include "common.cuh"

#include <algorithm>
#include <numeric>

namespace bfsgb {

bfs_status device_error(int err, int64_t timeout_ns);  // bfs_single.cu

namespace {

constexpr int CC_T = 1024;
constexpr int CC_CHUNK = 1024;  // rows of at least this many entries are expanded as chunk units
constexpr int CC_PULL_DIV = 16;  // pull when |F_i| > n / CC_PULL_DIV

struct CountersCC {
    unsigned long long changed;  // vertices set in F_{i+1}
    unsigned long long u_len;    // chunk units appended for the next iteration
};

struct CtlCC {
    GridBarrier bar;
    CountersCC slot[3];  // iteration i: slot[i % 3]; slot[(i + 2) % 3] is cleared during i
    unsigned long long n_big;  // fixed chunk units of the big rows (pull iterations)
    int32_t iters;
};

struct ParamsCC {
    int32_t n;
    int64_t W;
    const int32_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col;
    const uint32_t* __restrict__ isolated;
    int32_t* label;
    uint32_t* F0;
    uint32_t* F1;
    int2* U0;
    int2* U1;
    int2* B;  // fixed chunk units of every row of at least CC_CHUNK entries
    int64_t ucap;
    uint64_t wmul;  // odd multiplier coprime to W: word i of the dealing order is (i * wmul) mod W
    CtlCC* ctl;
    int64_t timeout_ns;
    int32_t max_iters;
};

// s -> d with s's label ls: lower d's label, and on a drop put d in F_{i+1}
__device__ __forceinline__ void cc_relax(const ParamsCC& p, uint32_t* f_nxt, int ls, int d, unsigned long long& cnt) {
    if (ls < __ldcg(p.label + d)) {  // labels only drop, so a stale read costs an atomic at most
        const int old = atomicMin(p.label + d, ls);
        if (ls < old) {
            const unsigned bit = 1u << (d & 31);
            if (!(atomicOr(f_nxt + (d >> 5), bit) & bit)) cnt += 1;
        }
    }
}

// Word of position i in the dealing order.  Warp k takes the contiguous
// positions [k * per, (k + 1) * per).  The multiplicative scramble spreads
// costly words over the warps: RMAT ids that share bit patterns have similar
// degrees, and a stride of warps over plain word order (or over a scramble
// modulo a power of two, which keeps low bits) gave one warp 10x the mean work.
__device__ __forceinline__ long long cc_word(const ParamsCC& p, long long i) {
    return (long long)(((unsigned long long)i * p.wmul) % (unsigned long long)p.W);
}

// Shortcut step after an iteration's relaxations (the pointer jumping of
// Shiloach-Vishkin-style algorithms): every vertex of F_{i+1} takes the label
// of the vertex its label names, label[v] <- min(label[v], label[label[v]]).
// A label is always the id of a vertex of the same component and labels only
// drop, so the fixed point is unchanged (each vertex's smallest component
// id); the step lets a label travel through the vertex it names instead of
// one edge per iteration, which on long-diameter graphs cuts the iteration
// count.  A thread takes words of F_{i+1} in a grid stride.
__device__ __forceinline__ void cc_jump(const ParamsCC& p, const uint32_t* f_nxt) {
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    for (long long w = gtid; w < p.W; w += gthreads) {
        unsigned fw = __ldcg(f_nxt + w);
        while (fw) {
            const int v = (int)(w * 32 + __ffs(fw) - 1);
            fw &= fw - 1;
            const int l = __ldcg(p.label + v);
            const int ll = __ldcg(p.label + l);
            if (ll < l) atomicMin(p.label + v, ll);
        }
    }
}

// |F_{i+1}|: one atomic per CTA
__device__ __forceinline__ void cc_count(CountersCC* nxt, unsigned long long cnt, unsigned long long* s_red) {
    cnt = warp_sum(cnt);
    if (lane_id() == 0) s_red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < CC_T / 32; ++i) t += s_red[i];
        if (t) atomicAdd(&nxt->changed, t);
    }
    __syncthreads();
}

// d's label dropped (this thread's atomic lowered it): record d in F_{i+1}
__device__ __forceinline__ void cc_mark(uint32_t* f_nxt, int d, unsigned long long& cnt) {
    const unsigned bit = 1u << (d & 31);
    if (!(atomicOr(f_nxt + (d >> 5), bit) & bit)) cnt += 1;
}

// Pull iteration.  Units left by a push iteration are expanded in push form
// first (their rows were in F_{i-1}); then each fixed unit of a big row gives
// a warp-wide minimum, and warps take the words of all vertices, each word's
// rows below CC_CHUNK flattened over the warp.  F_i is consumed (cleared)
// because a pull reads every neighbour anyway.
template <int T>
__device__ void cc_pull(const ParamsCC& p, uint32_t* f_cur, uint32_t* f_nxt, const int2* u_cur,
                        long long nunits, long long n_big, unsigned long long& cnt) {
    const unsigned lane = lane_id();
    const long long gwarp = ((long long)blockIdx.x * T + threadIdx.x) >> 5, nwarps = ((long long)gridDim.x * T) >> 5;
    for (long long u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int2 un = __ldcg(u_cur + u);
        const int s = un.x;
        const int ls = __ldcg(p.label + s);
        const int b = __ldg(p.row_ptr + s) + un.y * CC_CHUNK;
        const int e = min(__ldg(p.row_ptr + s + 1), b + CC_CHUNK);
        const int j = b + (int)threadIdx.x;
        if (j < e) cc_relax(p, f_nxt, ls, __ldg(p.col + j), cnt);
    }
    for (long long u = gwarp; u < n_big; u += nwarps) {  // a warp per fixed unit, warp-uniform
        const int2 un = __ldcg(p.B + u);  // written by this kernel's init phase
        const int d = un.x;
        const int b = __ldg(p.row_ptr + d) + un.y * CC_CHUNK;
        const int e = min(__ldg(p.row_ptr + d + 1), b + CC_CHUNK);
        int m = INT32_MAX;
        for (int j = b + (int)lane; j < e; j += 32) m = min(m, __ldcg(p.label + __ldg(p.col + j)));
        m = __reduce_min_sync(0xffffffffu, m);
        if (lane == 0 && m < __ldcg(p.label + d)) {
            if (m < atomicMin(p.label + d, m)) cc_mark(f_nxt, d, cnt);
        }
    }
    const long long per = (p.W + nwarps - 1) / nwarps;
    const long long iend = min((gwarp + 1) * per, (long long)p.W);
    for (long long i0 = gwarp * per; i0 < iend; i0 += 32) {  // 32 words of the dealing order a step
        const long long il = i0 + (long long)lane;
        const long long wl = il < iend ? cc_word(p, il) : -1;
        if (wl >= 0 && __ldcg(f_cur + wl)) f_cur[wl] = 0u;  // the buffer holds F_{i+2} next
        for (unsigned todo = __ballot_sync(0xffffffffu, wl >= 0); todo; todo &= todo - 1) {  // warp-uniform
            const long long w = __shfl_sync(0xffffffffu, wl, __ffs(todo) - 1);
            const int d = (int)(w * 32 + lane);
            int beg = 0, deg = 0, ld = INT32_MAX;
            if (d < p.n) {
                beg = __ldg(p.row_ptr + d);
                deg = __ldg(p.row_ptr + d + 1) - beg;
                ld = __ldcg(p.label + d);
            }
            const int fdeg = deg < CC_CHUNK ? deg : 0;
            int incl = fdeg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (total == 0) continue;
            const int excl = incl - fdeg;
            int mine = INT32_MAX;  // minimum over this lane's row
            for (int base = 0; base < total; base += 32) {
                const int idx = base + (int)lane;
                int o = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int ex = __shfl_sync(0xffffffffu, excl, (o + st) & 31);
                    if (o + st < 32 && ex <= idx) o += st;
                }
                const int ob = __shfl_sync(0xffffffffu, beg, o);
                const int oex = __shfl_sync(0xffffffffu, excl, o);
                const int val = idx < total ? __ldcg(p.label + __ldg(p.col + ob + (idx - oex))) : INT32_MAX;
                // segmented minimum: owners are non-decreasing over the lanes, so
                // each lane keeps the minimum of its owner's entries in this step
                int segmin = val;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int y = __shfl_down_sync(0xffffffffu, segmin, off);
                    const int oy = __shfl_down_sync(0xffffffffu, o, off);
                    if ((int)lane + off < 32 && oy == o) segmin = min(segmin, y);
                }
                // the first lane of each owner's run holds its minimum; hand it to the owner
                const int op = __shfl_up_sync(0xffffffffu, o, 1);
                const bool head = idx < total && (lane == 0 || op != o);
                const unsigned hm = __ballot_sync(0xffffffffu, head);
                // owner lane L takes the value of the head lane whose o == L (at most one per step)
                for (unsigned h = hm; h; h &= h - 1) {
                    const int hl = __ffs(h) - 1;
                    const int ho = __shfl_sync(0xffffffffu, o, hl);
                    const int hv = __shfl_sync(0xffffffffu, segmin, hl);
                    if ((int)lane == ho) mine = min(mine, hv);
                }
            }
            if (mine < ld) {  // units may lower labels concurrently: the atomic decides
                const int old = atomicMin(p.label + d, mine);
                if (mine < old) cc_mark(f_nxt, d, cnt);
            }
        }
    }
}

__global__ void __launch_bounds__(CC_T, 1) cc_kernel(ParamsCC p) {
    __shared__ unsigned long long s_red[CC_T / 32];
    CtlCC* ctl = p.ctl;
    const unsigned nblocks = gridDim.x;
    const unsigned lane = lane_id();
    const long long gtid = (long long)blockIdx.x * CC_T + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * CC_T;
    const long long gwarp = gtid >> 5, nwarps = gthreads >> 5;
    unsigned bar_target = 0;

    // L_0 = identity, F_0 = vertices with an edge (phantom bits past n stay clear)
    for (long long v = gtid; v < p.n; v += gthreads) p.label[v] = (int32_t)v;
    for (long long w = gtid; w < p.W; w += gthreads) {
        unsigned bits = ~__ldg(p.isolated + w);
        if (w == p.W - 1 && (p.n & 31)) bits &= (1u << (p.n & 31)) - 1u;
        p.F0[w] = bits;
        p.F1[w] = 0u;
    }
    // the fixed unit list of the big rows, for pull iterations
    for (long long v0 = gwarp * 32; v0 < p.n; v0 += nwarps * 32) {  // warp-uniform
        const long long v = v0 + lane;
        const int deg = v < p.n ? __ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v) : 0;
        append_units_warp(p.B, &ctl->n_big, p.ucap, &ctl->bar.err, deg >= CC_CHUNK, (int)v, deg, CC_CHUNK);
    }
    if (gtid == 0) ctl->slot[0].changed = (unsigned long long)p.n;  // F_0: dense, so iteration 0 pulls
    if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
    const long long n_big = (long long)min(__ldcg(&ctl->n_big), (unsigned long long)p.ucap);

    int it = 0;
    for (;; ++it) {
        CountersCC* cur = &ctl->slot[it % 3];
        CountersCC* nxt = &ctl->slot[(it + 1) % 3];
        const unsigned long long* const csrc[2] = {&cur->changed, &cur->u_len};
        unsigned long long cv[2];
        cta_load_u64<2>(csrc, cv);
        if (cv[0] == 0 && cv[1] == 0) break;
        if (it >= p.max_iters) {
            if (gtid == 0) atomicCAS(&ctl->bar.err, 0, (int)DEV_LEVELS);
            break;
        }
        if (gtid == 0) {
            CountersCC* z = &ctl->slot[(it + 2) % 3];
            z->changed = 0;
            z->u_len = 0;
        }
        uint32_t* f_cur = (it & 1) ? p.F1 : p.F0;
        uint32_t* f_nxt = (it & 1) ? p.F0 : p.F1;
        const int2* u_cur = (it & 1) ? p.U1 : p.U0;
        int2* u_nxt = (it & 1) ? p.U0 : p.U1;
        unsigned long long cnt = 0;
        if (cv[0] * CC_PULL_DIV > (unsigned long long)p.n) {
            cc_pull<CC_T>(p, f_cur, f_nxt, u_cur, (long long)min(cv[1], (unsigned long long)p.ucap), n_big, cnt);
            cc_count(nxt, cnt, s_red);
            if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            cc_jump(p, f_nxt);
            if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
            continue;
        }

        // chunk units of the previous iteration's big rows: a CTA per unit, an edge per thread
        // (an overflow was recorded and its units dropped; never read past the list)
        const long long nunits = (long long)min(cv[1], (unsigned long long)p.ucap);
        for (long long u = blockIdx.x; u < nunits; u += gridDim.x) {
            const int2 un = __ldcg(u_cur + u);
            const int s = un.x;
            const int ls = __ldcg(p.label + s);
            const int b = __ldg(p.row_ptr + s) + un.y * CC_CHUNK;
            const int e = min(__ldg(p.row_ptr + s + 1), b + CC_CHUNK);
            const int j = b + (int)threadIdx.x;
            if (j < e) cc_relax(p, f_nxt, ls, __ldg(p.col + j), cnt);
        }

        // the words of F_i, 32 of the dealing order loaded a step (one per lane);
        // each non-empty word's rows flattened over the warp
        const long long per = (p.W + nwarps - 1) / nwarps;
        const long long iend = min((gwarp + 1) * per, (long long)p.W);
        for (long long i0 = gwarp * per; i0 < iend; i0 += 32) {
            const long long il = i0 + (long long)lane;
            const long long wl = il < iend ? cc_word(p, il) : -1;
            const unsigned fwl = wl >= 0 ? __ldcg(f_cur + wl) : 0u;
            if (fwl) f_cur[wl] = 0u;  // the buffer holds F_{i+2} next
            for (unsigned todo = __ballot_sync(0xffffffffu, fwl != 0); todo; todo &= todo - 1) {  // warp-uniform
                const int src = __ffs(todo) - 1;
                const long long w = __shfl_sync(0xffffffffu, wl, src);
                const unsigned fw = __shfl_sync(0xffffffffu, fwl, src);
                const bool act = (fw >> lane) & 1u;
                const int s = (int)(w * 32 + lane);
                int beg = 0, deg = 0, ls = 0;
                if (act) {
                    beg = __ldg(p.row_ptr + s);
                    deg = __ldg(p.row_ptr + s + 1) - beg;
                    ls = __ldcg(p.label + s);
                }
                const bool big = act && deg >= CC_CHUNK;
                append_units_warp(u_nxt, &nxt->u_len, p.ucap, &p.ctl->bar.err, big, s, deg, CC_CHUNK);
                const int fdeg = (act && !big) ? deg : 0;
                int incl = fdeg;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((int)lane >= o) incl += y;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                const int excl = incl - fdeg;
                for (int base = 0; base < total; base += 32) {
                    const int idx = base + (int)lane;
                    // owner: the last lane whose first entry is at or before idx
                    int o = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) {
                        const int ex = __shfl_sync(0xffffffffu, excl, (o + st) & 31);
                        if (o + st < 32 && ex <= idx) o += st;
                    }
                    const int ob = __shfl_sync(0xffffffffu, beg, o);
                    const int oex = __shfl_sync(0xffffffffu, excl, o);
                    const int ol = __shfl_sync(0xffffffffu, ls, o);
                    if (idx < total) cc_relax(p, f_nxt, ol, __ldg(p.col + ob + (idx - oex)), cnt);
                }
            }
        }

        cc_count(nxt, cnt, s_red);
        if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
        cc_jump(p, f_nxt);
        if (!grid_sync(&ctl->bar, nblocks, bar_target, p.timeout_ns)) return;
    }
    if (gtid == 0) ctl->iters = it;
}

__global__ void cc_count_units_kernel(const int32_t* row_ptr, int32_t n, unsigned long long* out) {
    unsigned long long s = 0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int d = row_ptr[v + 1] - row_ptr[v];
        if (d >= CC_CHUNK) s += (unsigned long long)((d + CC_CHUNK - 1) / CC_CHUNK);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

struct StreamAllocs {
    cudaStream_t st;
    void* ptrs[12] = {};
    int k = 0;
    explicit StreamAllocs(cudaStream_t s) : st(s) {}
    template <typename T>
    bool alloc(T** p, size_t count) {
        if (cudaMallocAsync((void**)p, std::max<size_t>(count, 1) * sizeof(T), st) != cudaSuccess) return false;
        ptrs[k++] = *p;
        return true;
    }
    ~StreamAllocs() {
        for (int i = 0; i < k; ++i) cudaFreeAsync(ptrs[i], st);
    }
};

}  // namespace

}  // namespace bfsgb

using namespace bfsgb;

extern "C" bfs_status bfs_components(const bfs_graph* gc, int32_t* label, int32_t* iterations, void* cuda_stream) {
    bfs_graph* g = const_cast<bfs_graph*>(gc);
    if (!g || !label) return fail(BFS_EINVAL, "null argument");
    if (!g->symmetric) return fail(BFS_EINVAL, "bfs_components needs a symmetric graph (BFS_SYMMETRIZE)");
    if (device_id() != g->device) return fail(BFS_EINVAL, "graph lives on device %d, current device is %d", g->device, device_id());
    std::lock_guard<std::mutex> guard(g->lock);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int32_t n = g->n;
    const int64_t W = div_up(n, 32);
    const bool host = !is_device_ptr(label);

    StreamAllocs sa(st);
    unsigned long long* d_units;
    if (!sa.alloc(&d_units, 1)) {
        cudaGetLastError();
        return fail(BFS_ENOMEM, "components scratch");
    }
    BFS_CUDA(cudaMemsetAsync(d_units, 0, 8, st));
    cc_count_units_kernel<<<num_sms() * 8, 256, 0, st>>>(g->row_ptr, n, d_units);
    unsigned long long units = 0;
    BFS_CUDA(cudaMemcpyAsync(&units, d_units, 8, cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));

    ParamsCC p{};
    p.n = n;
    p.W = W;
    p.row_ptr = g->row_ptr;
    p.col = g->col;
    p.isolated = g->isolated;
    p.ucap = (int64_t)units + 1;
    uint64_t K = 2654435761ull % (uint64_t)W;  // a multiplier coprime to W makes the dealing a permutation
    if (K == 0) K = 1;
    while (std::gcd(K, (uint64_t)W) != 1) ++K;
    p.wmul = K;
    p.timeout_ns = 2000000000ll;
    p.max_iters = n + 1;
    int32_t* d_label = label;
    if ((host && !sa.alloc(&d_label, (size_t)n)) || !sa.alloc(&p.F0, (size_t)W) || !sa.alloc(&p.F1, (size_t)W) ||
        !sa.alloc(&p.U0, (size_t)p.ucap) || !sa.alloc(&p.U1, (size_t)p.ucap) || !sa.alloc(&p.B, (size_t)p.ucap) ||
        !sa.alloc(&p.ctl, 1)) {
        cudaGetLastError();
        return fail(BFS_ENOMEM, "components workspace for n=%d", n);
    }
    p.label = d_label;
    BFS_CUDA(cudaMemsetAsync(p.ctl, 0, sizeof(CtlCC), st));
    int per_sm = 0;
    BFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cc_kernel, CC_T, 0));
    if (per_sm < 1) return fail(BFS_ECUDA, "components kernel does not fit on an SM");
    void* args[] = {(void*)&p};
    BFS_CUDA(cudaLaunchCooperativeKernel((const void*)cc_kernel, dim3(per_sm * num_sms()), dim3(CC_T), args, 0, st));
    CtlCC h{};
    BFS_CUDA(cudaMemcpyAsync(&h, p.ctl, sizeof(CtlCC), cudaMemcpyDeviceToHost, st));
    if (host) BFS_CUDA(cudaMemcpyAsync(label, d_label, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    if (h.bar.err) return device_error(h.bar.err, p.timeout_ns);
    if (iterations) *iterations = h.iters;
    return BFS_OK;
}
