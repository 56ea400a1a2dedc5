// stats.cu -- per-level work statistics of a finished search (measurement
// utility for the roofline model; not on the timed path).
//
// For a depth array of Cascade 1 the per-level quantities are
//   f_i   = |F_i|,   e_f_i = sum deg over F_i,   d_new_i = |F_{i+1}|,
//   u_i   = non-isolated v with depth > i or unreached, e_u_i their degree sum,
//   s_u_i = entries a pull level reads: each such row scanned in ascending
//           order up to the first neighbour of depth i, else completely.
// A reached vertex of depth d has all neighbours at depth d-1, d or d+1, so
// its row is scanned completely at every level i < d-1 and up to the first
// depth-(d-1) neighbour at level d-1; unreached rows are always scanned
// completely.  Hence s_u_i = e_u_i - sum_{v in F_{i+1}} (deg v - p_v), with
// p_v the 1-based position of v's first depth-(d-1) neighbour, which makes
// the whole table O(n + m) instead of O(levels * m).  The shortcut holds for
// symmetric graphs (the configuration every benchmark uses).
#include "common.cuh"

#include <vector>

namespace bfsgb {
namespace {

// Largest depth of the search; a value outside [-1, n) (an uninitialised or
// foreign buffer) makes the result INT32_MAX, which the host rejects.
__global__ void max_depth_kernel(const int32_t* depth, int32_t n, int* out) {
    int mx = -1;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int d = depth[v];
        mx = (d < -1 || d >= n) ? INT32_MAX : max(mx, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// arrays: [5][L] = f, e_f, diff_u, diff_eu, corr ; consts: [2] = unreached count, unreached degree sum
template <bool SMEM>
__global__ void level_accum_kernel(const int32_t* row_ptr, const int32_t* col, const int32_t* depth, int32_t n, int L,
                                   unsigned long long* arrays, unsigned long long* consts) {
    extern __shared__ unsigned long long sh[];
    unsigned long long* acc = SMEM ? sh : arrays;
    if (SMEM) {
        for (int i = threadIdx.x; i < 5 * L; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    unsigned long long un = 0, undeg = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int d = depth[v];
        int b = row_ptr[v], e = row_ptr[v + 1];
        unsigned long long deg = (unsigned long long)(e - b);
        if (d < 0) {
            if (deg > 0) {
                ++un;
                undeg += deg;
            }
            continue;
        }
        atomicAdd(&acc[0 * L + d], 1ull);
        atomicAdd(&acc[1 * L + d], deg);
        if (d >= 1 && deg > 0) {
            // unvisited at levels 0 .. d-1
            atomicAdd(&acc[2 * L + 0], 1ull);
            atomicAdd(&acc[3 * L + 0], deg);
            if (d < L) {
                atomicAdd(&acc[2 * L + d], (unsigned long long)-1ll);
                atomicAdd(&acc[3 * L + d], (unsigned long long)(-(long long)deg));
            }
            long long pv = 0;
            for (int j = b; j < e; ++j) {
                ++pv;
                if (depth[col[j]] == d - 1) break;
            }
            atomicAdd(&acc[4 * L + (d - 1)], deg - (unsigned long long)pv);
        }
    }
    un = warp_sum(un);
    undeg = warp_sum(undeg);
    if ((threadIdx.x & 31) == 0) {
        if (un) atomicAdd(&consts[0], un);
        if (undeg) atomicAdd(&consts[1], undeg);
    }
    if (SMEM) {
        __syncthreads();
        for (int i = threadIdx.x; i < 5 * L; i += blockDim.x)
            if (sh[i]) atomicAdd(&arrays[i], sh[i]);
    }
}

// Frees the call's stream-ordered scratch on every return path.
struct AsyncFrees {
    cudaStream_t st;
    void* p[4] = {nullptr, nullptr, nullptr, nullptr};
    ~AsyncFrees() {
        for (void* q : p)
            if (q) cudaFreeAsync(q, st);
    }
};

// Checks shared by both statistics calls.
bfs_status check_stats_args(const bfs_graph* g, const int32_t* depth, const int64_t* stats, int32_t max_levels) {
    if (!g || !depth || !stats) return fail(BFS_EINVAL, "null argument");
    if (max_levels <= 0) return fail(BFS_EINVAL, "max_levels must be positive");
    if (device_id() != g->device)
        return fail(BFS_EINVAL, "graph lives on device %d, current device is %d", g->device, device_id());
    return BFS_OK;
}

bfs_status depth_levels(int h_max, int32_t n, int32_t max_levels, int* L) {
    if (h_max >= n) return fail(BFS_EINVAL, "depth holds values outside [-1, %d)", n);
    *L = h_max + 1;
    if (*L > max_levels) return fail(BFS_ERANGE, "search has %d levels, max_levels = %d", *L, max_levels);
    return BFS_OK;
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" bfs_status bfs_level_stats(const bfs_graph* g, const int32_t* depth, int32_t max_levels, int64_t* stats,
                                      int32_t* levels, void* cuda_stream) {
    bfs_status rc = check_stats_args(g, depth, stats, max_levels);
    if (rc != BFS_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    AsyncFrees scratch{st};
    const int32_t* d_depth = depth;
    if (!is_device_ptr(depth)) {
        int32_t* tmp_depth = nullptr;
        BFS_CUDA(cudaMallocAsync(&tmp_depth, (size_t)g->n * 4, st));
        scratch.p[0] = tmp_depth;
        BFS_CUDA(cudaMemcpyAsync(tmp_depth, depth, (size_t)g->n * 4, cudaMemcpyHostToDevice, st));
        d_depth = tmp_depth;
    } else {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, depth) == cudaSuccess && a.type == cudaMemoryTypeDevice && a.device != g->device)
            return fail(BFS_EINVAL, "depth lives on device %d, the graph on device %d", a.device, g->device);
    }
    int* d_max;
    BFS_CUDA(cudaMallocAsync(&d_max, 4, st));
    scratch.p[1] = d_max;
    int h_max = -1;
    BFS_CUDA(cudaMemcpyAsync(d_max, &h_max, 4, cudaMemcpyHostToDevice, st));
    int blocks = num_sms() * 4;
    max_depth_kernel<<<blocks, 256, 0, st>>>(d_depth, g->n, d_max);
    BFS_CUDA(cudaMemcpyAsync(&h_max, d_max, 4, cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    int L = 0;
    rc = depth_levels(h_max, g->n, max_levels, &L);
    if (rc != BFS_OK) return rc;
    if (levels) *levels = L;
    if (L <= 0) return BFS_OK;
    unsigned long long *d_arr, *d_const;
    BFS_CUDA(cudaMallocAsync(&d_arr, (size_t)5 * L * 8, st));
    scratch.p[2] = d_arr;
    BFS_CUDA(cudaMallocAsync(&d_const, 16, st));
    scratch.p[3] = d_const;
    BFS_CUDA(cudaMemsetAsync(d_arr, 0, (size_t)5 * L * 8, st));
    BFS_CUDA(cudaMemsetAsync(d_const, 0, 16, st));
    size_t sm = (size_t)5 * L * 8;
    if (sm <= 48 * 1024) {
        level_accum_kernel<true><<<blocks, 256, sm, st>>>(g->row_ptr, g->col, d_depth, g->n, L, d_arr, d_const);
    } else {
        level_accum_kernel<false><<<blocks, 256, 0, st>>>(g->row_ptr, g->col, d_depth, g->n, L, d_arr, d_const);
    }
    BFS_CUDA(cudaGetLastError());
    std::vector<unsigned long long> arr((size_t)5 * L), cst(2);
    BFS_CUDA(cudaMemcpyAsync(arr.data(), d_arr, arr.size() * 8, cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaMemcpyAsync(cst.data(), d_const, 16, cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    long long u = 0, eu = 0;
    for (int i = 0; i < L; ++i) {
        u += (long long)arr[2 * L + i];
        eu += (long long)arr[3 * L + i];
        int64_t* o = stats + 6 * (int64_t)i;
        o[0] = (int64_t)arr[0 * L + i];
        o[1] = (int64_t)arr[1 * L + i];
        o[2] = u + (long long)cst[0];
        o[5] = eu + (long long)cst[1];
        o[3] = o[5] - (long long)arr[4 * L + i];
        o[4] = (i + 1 < L) ? (int64_t)arr[0 * L + i + 1] : 0;
    }
    return BFS_OK;
}

// ------------------------------------------------------------ no-allocation variant
// bfs_level_stats for callers that may not allocate device memory: all of its
// scratch lives in one file-scope __device__ array of fixed size, so the call
// makes no cudaMalloc/cudaFree (nor any other allocating runtime call).
namespace bfsgb {
namespace {

constexpr int NOALLOC_MAX_LEVELS = 4096;

struct NoallocScratch {
    int max_depth;
    int pad[63];
    unsigned long long consts[2];
    unsigned long long arrays[5 * NOALLOC_MAX_LEVELS];
    long long table[6 * NOALLOC_MAX_LEVELS];
};

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

__global__ void noalloc_clear_kernel(NoallocScratch* s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 5 * NOALLOC_MAX_LEVELS; i += gridDim.x * blockDim.x)
        s->arrays[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->max_depth = -1;
        s->consts[0] = 0;
        s->consts[1] = 0;
    }
}

// The six statistics per level from the accumulated difference arrays.
__global__ void noalloc_table_kernel(NoallocScratch* s, int L) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const unsigned long long* a = s->arrays;
    long long u = 0, eu = 0;
    for (int i = 0; i < L; ++i) {
        u += (long long)a[2 * L + i];
        eu += (long long)a[3 * L + i];
        long long* o = s->table + 6 * (long long)i;
        o[0] = (long long)a[0 * L + i];
        o[1] = (long long)a[1 * L + i];
        o[2] = u + (long long)s->consts[0];
        o[5] = eu + (long long)s->consts[1];
        o[3] = o[5] - (long long)a[4 * L + i];
        o[4] = (i + 1 < L) ? (long long)a[0 * L + i + 1] : 0;
    }
}

std::mutex g_noalloc_lock;
NoallocScratch* g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device with that device current).
bfs_status noalloc_scratch(NoallocScratch** out) {
    int dev = device_id();
    if (dev < 0 || dev >= 64) return fail(BFS_EINVAL, "device index %d not supported", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_lock);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = (NoallocScratch*)p;
    }
    *out = g_noalloc_ptr[dev];
    return BFS_OK;
}

}  // namespace
}  // namespace bfsgb

extern "C" bfs_status bfs_level_stats_noalloc(const bfs_graph* g, const int32_t* depth, int32_t max_levels,
                                              int64_t* stats, int32_t* levels, void* cuda_stream) {
    if (!levels) return fail(BFS_EINVAL, "null argument");
    bfs_status rc = check_stats_args(g, depth, stats, max_levels);
    if (rc != BFS_OK) return rc;
    if (max_levels > NOALLOC_MAX_LEVELS)
        return fail(BFS_ERANGE, "max_levels %d exceeds the fixed scratch limit of %d levels", max_levels,
                    NOALLOC_MAX_LEVELS);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, depth) != cudaSuccess) cudaGetLastError();
    else if (a.type == cudaMemoryTypeDevice && a.device != g->device)
        return fail(BFS_EINVAL, "depth lives on device %d, the graph on device %d", a.device, g->device);
    if (!is_device_ptr(depth)) return fail(BFS_EINVAL, "depth must be device memory");
    NoallocScratch* s = nullptr;
    rc = noalloc_scratch(&s);
    if (rc != BFS_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = num_sms() * 4;
    noalloc_clear_kernel<<<num_sms(), 256, 0, st>>>(s);
    max_depth_kernel<<<blocks, 256, 0, st>>>(depth, g->n, &s->max_depth);
    int h_max = -1;
    BFS_CUDA(cudaMemcpyAsync(&h_max, &s->max_depth, 4, cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    int L = 0;
    rc = depth_levels(h_max, g->n, max_levels, &L);
    if (rc != BFS_OK) return rc;
    *levels = L;
    if (L <= 0) return BFS_OK;
    const size_t sm = (size_t)5 * L * 8;
    if (sm <= 48 * 1024) {
        level_accum_kernel<true><<<blocks, 256, sm, st>>>(g->row_ptr, g->col, depth, g->n, L, s->arrays, s->consts);
    } else {
        level_accum_kernel<false><<<blocks, 256, 0, st>>>(g->row_ptr, g->col, depth, g->n, L, s->arrays, s->consts);
    }
    noalloc_table_kernel<<<1, 1, 0, st>>>(s, L);
    BFS_CUDA(cudaGetLastError());
    BFS_CUDA(cudaMemcpyAsync(stats, s->table, (size_t)6 * L * sizeof(int64_t), cudaMemcpyDefault, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    return BFS_OK;
}
