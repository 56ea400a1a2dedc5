// capi.cu -- C ABI entry points: options, bfs_run dispatch, error reporting.
#include "common.cuh"

#include <cstdarg>
#include <cstring>
#include <vector>

namespace bfsgb {

static thread_local std::string t_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
}

bfs_status fail(bfs_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return s;
}

bfs_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    cudaGetLastError();  // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? BFS_ENOMEM : BFS_ECUDA;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int device_id() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

int num_sms() {
    static int cached[64] = {0};
    int d = device_id();
    if (d < 0 || d >= 64) d = 0;
    if (!cached[d]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
        cached[d] = v > 0 ? v : 1;
    }
    return cached[d];
}

bfs_status run_single(bfs_graph* g, int32_t src_value, int32_t* depth, int32_t* parent, const bfs_options& o,
                      const float* mlp_dev, cudaStream_t st);
bfs_status run_single_many(bfs_graph* g, const int32_t* src_host, int32_t k, int32_t* depth, int32_t* parent,
                           const bfs_options& o, const float* mlp_dev, cudaStream_t st);
bfs_status run_msbfs(bfs_graph* g, const int32_t* sources, int32_t k, int32_t* depth, int32_t* parent,
                     const bfs_options& o, const float* mlp_dev, cudaStream_t st);
bfs_status run_mixed(const bfs_graph* const* graphs, int32_t n_graphs, const int32_t* graph_of_query,
                     const int32_t* sources, int32_t nq, int32_t* const* depth, int32_t* const* parent,
                     const bfs_options& o, cudaStream_t st);
bfs_status sync_graph(bfs_graph* g, cudaStream_t st);
const float* policy_device_weights(const bfs_policy* p);

}  // namespace bfsgb

using namespace bfsgb;

extern "C" void bfs_options_init(bfs_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(bfs_options);
    o->mode = BFS_MODE_PERSISTENT;
    o->policy = BFS_POLICY_HEURISTIC;
    o->alpha = 14.0f;
    o->beta = 48.0f;
    o->batch_alpha = 4.0f;
    o->batch_beta = 48.0f;
    o->gamma = 16.0f;
    o->chunk = 1024;
    o->medium = 32;
    o->pull_serial = 16;
    o->block_threads = 1024;
    o->blocks_per_sm = 0;
    o->claim_aggregate = 0;
    o->push_filter = BFS_PUSH_FUSED;
    o->frontier_sort = BFS_SORT_NONE;
    o->small_levels = BFS_SMALL_AUTO;
    o->barrier_timeout_ns = 2000000000ll;
    o->batch = 1;
}

static bfs_status check_options(const bfs_options* in, bfs_options* o) {
    bfs_options_init(o);
    if (!in) return BFS_OK;
    if (in->struct_size != sizeof(bfs_options)) return fail(BFS_EINVAL, "bfs_options.struct_size mismatch (call bfs_options_init)");
    *o = *in;
    if (o->mode < 0 || o->mode > 2) return fail(BFS_EINVAL, "bad mode %d", o->mode);
    if (o->policy < 0 || o->policy > 4) return fail(BFS_EINVAL, "bad policy %d", o->policy);
    if (o->chunk < 64) return fail(BFS_EINVAL, "chunk must be >= 64");
    if (o->medium < 1) return fail(BFS_EINVAL, "medium must be >= 1");
    if (o->pull_serial < 1) return fail(BFS_EINVAL, "pull_serial must be >= 1");
    if (!(o->alpha > 0) || !(o->beta > 0) || !(o->gamma > 0) || !(o->batch_alpha > 0) || !(o->batch_beta > 0))
        return fail(BFS_EINVAL, "alpha, beta, gamma, batch_alpha, batch_beta must be > 0");
    if (o->barrier_timeout_ns <= 0) return fail(BFS_EINVAL, "barrier_timeout_ns must be > 0");
    if (o->block_threads != 256 && o->block_threads != 512 && o->block_threads != 1024)
        return fail(BFS_EINVAL, "block_threads must be 256, 512 or 1024");
    if (o->push_filter < BFS_PUSH_FUSED || o->push_filter > BFS_PUSH_FILTER_PREDICATED)
        return fail(BFS_EINVAL, "bad push_filter %d", o->push_filter);
    if (o->push_filter != BFS_PUSH_FUSED && o->mode == BFS_MODE_GRAPH)
        return fail(BFS_EINVAL, "push_filter needs the persistent or host-loop drive");
    if (o->frontier_sort < BFS_SORT_NONE || o->frontier_sort > BFS_SORT_TILE)
        return fail(BFS_EINVAL, "bad frontier_sort %d", o->frontier_sort);
    if (o->frontier_sort != BFS_SORT_NONE && o->mode == BFS_MODE_GRAPH)
        return fail(BFS_EINVAL, "frontier_sort needs the persistent or host-loop drive");
    if (o->small_levels < BFS_SMALL_AUTO || o->small_levels > BFS_SMALL_CLUSTER)
        return fail(BFS_EINVAL, "bad small_levels %d", o->small_levels);
    return BFS_OK;
}

extern "C" bfs_status bfs_run(const bfs_graph* gc, const int32_t* sources, int32_t k, int32_t* depth, int32_t* parent,
                              const bfs_options* opt, void* cuda_stream) {
    bfs_graph* g = const_cast<bfs_graph*>(gc);
    if (!g) return fail(BFS_EINVAL, "graph is NULL");
    if (!sources || !depth) return fail(BFS_EINVAL, "sources/depth is NULL");
    if (k <= 0) return fail(BFS_EINVAL, "k must be positive (got %d)", k);
    bfs_options o;
    bfs_status s = check_options(opt, &o);
    if (s != BFS_OK) return s;
    if (device_id() != g->device) return fail(BFS_EINVAL, "graph lives on device %d, current device is %d", g->device, device_id());
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<int32_t> src(k);
    if (is_device_ptr(sources)) {
        BFS_CUDA(cudaMemcpyAsync(src.data(), sources, (size_t)k * 4, cudaMemcpyDeviceToHost, st));
        BFS_CUDA(cudaStreamSynchronize(st));
    } else {
        memcpy(src.data(), sources, (size_t)k * 4);
    }
    for (int j = 0; j < k; ++j)
        if (src[j] < 0 || src[j] >= g->n) return fail(BFS_EINVAL, "source %d = %d outside [0, %d)", j, src[j], g->n);
    const float* mlp = (o.policy == BFS_POLICY_MLP) ? policy_device_weights(o.mlp) : nullptr;
    std::lock_guard<std::mutex> lk(g->lock);
    bool dev_out = is_device_ptr(depth) && (!parent || is_device_ptr(parent));
    if (k > 1 && o.batch) {
        return run_msbfs(g, src.data(), k, depth, parent, o, mlp, st);
    }
    const int64_t n = g->n;
    if (dev_out && k > 1 && o.mode == BFS_MODE_PERSISTENT && !o.level_log && !o.levels_out)
        return run_single_many(g, src.data(), k, depth, parent, o, mlp, st);
    if (dev_out) {
        for (int j = 0; j < k; ++j) {
            s = run_single(g, src[j], depth + j * n, parent ? parent + j * n : nullptr, o, mlp, st);
            if (s != BFS_OK) return s;
        }
        return BFS_OK;
    }
    // host outputs: two pairs of device staging buffers; the search of source
    // j+1 (on `st`) overlaps the copy of source j's outputs (on a copy stream),
    // and the host waits once, at the end
    int32_t *dd[2] = {nullptr, nullptr}, *dp[2] = {nullptr, nullptr};
    cudaStream_t cs = nullptr;
    cudaEvent_t searched[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaMallocAsync(&dd[b], n * 4, st) == cudaSuccess &&
             (!parent || cudaMallocAsync(&dp[b], n * 4, st) == cudaSuccess) &&
             cudaEventCreateWithFlags(&searched[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        s = fail(BFS_ENOMEM, "staging buffers");
    }
    for (int j = 0; j < k && s == BFS_OK; ++j) {
        const int b = j & 1;
        cudaError_t e = cudaSuccess;
        if (j >= 2) e = cudaStreamWaitEvent(st, copied[b], 0);  // buffer b's previous copy is done
        if (e == cudaSuccess) {
            s = run_single(g, src[j], dd[b], dp[b], o, mlp, st);
            if (s != BFS_OK) break;
            e = cudaEventRecord(searched[b], st);
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, searched[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(depth + j * n, dd[b], n * 4, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && parent) e = cudaMemcpyAsync(parent + j * n, dp[b], n * 4, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaEventRecord(copied[b], cs);
        if (e != cudaSuccess) s = cuda_fail(e, "copy outputs to host");
    }
    if (cs) {
        cudaError_t e = cudaStreamSynchronize(cs);  // every copy has landed in host memory
        if (e != cudaSuccess && s == BFS_OK) s = cuda_fail(e, "copy outputs to host");
    }
    for (int b = 0; b < 2; ++b) {
        if (dd[b]) cudaFreeAsync(dd[b], st);
        if (dp[b]) cudaFreeAsync(dp[b], st);
        if (searched[b]) cudaEventDestroy(searched[b]);
        if (copied[b]) cudaEventDestroy(copied[b]);
    }
    if (cs) cudaStreamDestroy(cs);
    if (s == BFS_OK) s = sync_graph(g, st);
    return s;
}

extern "C" bfs_status bfs_run_mixed(const bfs_graph* const* graphs, int32_t n_graphs, const int32_t* graph_of_query,
                                    const int32_t* sources, int32_t nq, int32_t* const* depth, int32_t* const* parent,
                                    const bfs_options* opt, void* cuda_stream) {
    if (!graphs || n_graphs <= 0 || !graph_of_query || !sources || nq <= 0 || !depth)
        return fail(BFS_EINVAL, "null argument or empty batch");
    bfs_options o;
    bfs_status s = check_options(opt, &o);
    if (s != BFS_OK) return s;
    for (int g = 0; g < n_graphs; ++g)
        if (!graphs[g]) return fail(BFS_EINVAL, "graphs[%d] is NULL", g);
    for (int q = 0; q < nq; ++q) {
        int gi = graph_of_query[q];
        if (gi < 0 || gi >= n_graphs) return fail(BFS_EINVAL, "graph_of_query[%d] = %d", q, gi);
        if (sources[q] < 0 || sources[q] >= graphs[gi]->n) return fail(BFS_EINVAL, "sources[%d] out of range", q);
        if (!depth[q] || !is_device_ptr(depth[q])) return fail(BFS_EINVAL, "depth[%d] must be device memory", q);
        if (parent && parent[q] && !is_device_ptr(parent[q])) return fail(BFS_EINVAL, "parent[%d] must be device memory", q);
    }
    return run_mixed(graphs, n_graphs, graph_of_query, sources, nq, depth, parent, o, (cudaStream_t)cuda_stream);
}

extern "C" bfs_status bfs_sync(const bfs_graph* g, void* cuda_stream) {
    if (!g) return fail(BFS_EINVAL, "graph is NULL");
    return sync_graph(const_cast<bfs_graph*>(g), (cudaStream_t)cuda_stream);
}

extern "C" const char* bfs_status_string(bfs_status s) {
    switch (s) {
        case BFS_OK: return "ok";
        case BFS_EINVAL: return "invalid argument";
        case BFS_ENOMEM: return "out of memory";
        case BFS_ECUDA: return "CUDA error";
        case BFS_ETIMEOUT: return "device wait timed out";
        case BFS_ERANGE: return "size out of range";
        case BFS_EVALIDATE: return "consistency check failed";
    }
    return "unknown status";
}

extern "C" const char* bfs_last_error(void) { return t_last_error.c_str(); }

extern "C" const char* bfs_version(void) { return "bfsgb 0.1 (sm_103a)"; }
