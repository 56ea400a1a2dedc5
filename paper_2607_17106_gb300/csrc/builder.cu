// builder.cu -- graph construction on the device: the S x D tensor G of
// Cascade 1 (Eq. G) in CSR form (Section 4.C), plus its rank swizzle to
// d-major order (CSC, Section 4.B, B.4) for pull levels.
//
//   edge list --(symmetrise, drop self-loops)--> 64-bit (s,d) keys
//   --(LSD radix sort, 8-bit digits)--> unique --(compaction)--> col[]
//   --(row boundaries)--> row_ptr[]
//
// The sort is a plain stable LSD radix sort (tile histogram, digit-major scan,
// stable scatter with warp match-any ranking), written for this library.
#include "common.cuh"

#include <algorithm>
#include <vector>

namespace bfsgb {

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;  // 4096 keys per tile
constexpr int RADIX = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;

// --------------------------------------------------------------- scan u32
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t x, uint32_t* tmp, uint32_t* total) {
    unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? tmp[lane] : 0, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if ((int)lane >= o) wi += y;
        }
        if (lane < nw) tmp[lane] = wi - w;
        if (lane == 31) tmp[32] = wi;
    }
    __syncthreads();
    uint32_t r = tmp[warp] + incl - x;
    *total = tmp[32];
    __syncthreads();
    return r;
}

__global__ void scan_reduce_kernel(const uint32_t* in, int64_t count, uint32_t* sums) {
    __shared__ uint32_t tmp[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < count) s += in[idx];
    }
    uint32_t total;
    block_excl_scan_u32(s, tmp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// single CTA: exclusive scan of `count` sums in place, carrying across chunks
__global__ void scan_sums_kernel(uint32_t* sums, int64_t count, uint32_t* grand_total) {
    __shared__ uint32_t tmp[33];
    uint32_t carry = 0;
    for (int64_t base = 0; base < count; base += SCAN_THREADS) {
        int64_t idx = base + threadIdx.x;
        uint32_t x = idx < count ? sums[idx] : 0, total;
        uint32_t ex = block_excl_scan_u32(x, tmp, &total);
        if (idx < count) sums[idx] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0 && grand_total) *grand_total = carry;
}

// blocked per-thread items so each thread's run is contiguous
__global__ void scan_apply_kernel(const uint32_t* in, int64_t count, const uint32_t* sums, uint32_t* out) {
    __shared__ uint32_t tmp[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS], s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < count) ? in[base + i] : 0;
        s += v[i];
    }
    uint32_t total;
    uint32_t ex = block_excl_scan_u32(s, tmp, &total) + sums[blockIdx.x];
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < count) out[base + i] = ex;
        ex += v[i];
    }
}

struct Scratch {
    std::vector<void*> ptrs;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        cudaError_t e = cudaMallocAsync((void**)p, std::max<size_t>(count, 1) * sizeof(T), st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

// exclusive scan of u32 (in may equal out); *total (device) receives the sum
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t count, uint32_t* d_total,
                               cudaStream_t st) {
    Scratch sc(st);
    int64_t tiles = div_up(std::max<int64_t>(count, 1), SCAN_TILE);
    uint32_t* sums;
    cudaError_t e = sc.alloc(&sums, tiles);
    if (e) return e;
    scan_reduce_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, count, sums);
    scan_sums_kernel<<<1, SCAN_THREADS, 0, st>>>(sums, tiles, d_total);
    scan_apply_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, count, sums, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ radix sort
__global__ void radix_upsweep_kernel(const uint64_t* keys, int64_t count, int shift, uint32_t* hist,
                                     int64_t num_tiles) {
    __shared__ uint32_t h[RADIX];
    for (int i = threadIdx.x; i < RADIX; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_ITEMS; ++r) {
        int64_t idx = base + (int64_t)r * SORT_THREADS + threadIdx.x;
        if (idx < count) atomicAdd(&h[(keys[idx] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) hist[(int64_t)d * num_tiles + blockIdx.x] = h[d];
}

// Stable scatter of one tile: items are visited in index order (round r,
// thread t <-> index r*256 + t); a key's rank among equal digits is the
// number of equal digits earlier in the tile.
__global__ void radix_downsweep_kernel(const uint64_t* keys_in, uint64_t* keys_out, int64_t count, int shift,
                                       const uint32_t* offsets, int64_t num_tiles) {
    __shared__ uint32_t s_base[RADIX];                 // global offset of each digit for this tile
    __shared__ uint32_t s_cnt[SORT_WARPS][RADIX];      // per-warp counts of the current round
    __shared__ uint32_t s_pref[SORT_WARPS][RADIX];     // exclusive prefix for (warp, digit)
    __shared__ uint32_t s_run[RADIX];                  // digits already placed in earlier rounds
    unsigned warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) {
        s_base[d] = offsets[(int64_t)d * num_tiles + blockIdx.x];
        s_run[d] = 0;
        for (int w = 0; w < SORT_WARPS; ++w) s_cnt[w][d] = 0;
    }
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_ITEMS; ++r) {
        int64_t idx = base + (int64_t)r * SORT_THREADS + threadIdx.x;
        bool valid = idx < count;
        uint64_t key = valid ? keys_in[idx] : 0;
        unsigned digit = valid ? (unsigned)((key >> shift) & (RADIX - 1)) : RADIX;  // RADIX = no item
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        unsigned rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) s_cnt[warp][digit] = __popc(peers);
        __syncthreads();
        for (int d = threadIdx.x; d < RADIX; d += blockDim.x) {
            uint32_t run = s_run[d];
            for (int w = 0; w < SORT_WARPS; ++w) {
                uint32_t c = s_cnt[w][d];
                s_pref[w][d] = run;
                run += c;
                s_cnt[w][d] = 0;
            }
            s_run[d] = run;
        }
        __syncthreads();
        if (valid) keys_out[s_base[digit] + s_pref[warp][digit] + rank] = key;
    }
}

cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t count, int bits, cudaStream_t st,
                           uint64_t** result) {
    Scratch sc(st);
    int64_t tiles = div_up(std::max<int64_t>(count, 1), SORT_TILE);
    uint32_t* hist;
    cudaError_t e = sc.alloc(&hist, (size_t)tiles * RADIX);
    if (e) return e;
    uint64_t *a = keys, *b = tmp;
    for (int shift = 0; shift < bits; shift += 8) {
        radix_upsweep_kernel<<<(unsigned)tiles, SORT_THREADS, 0, st>>>(a, count, shift, hist, tiles);
        e = exclusive_scan_u32(hist, hist, tiles * RADIX, nullptr, st);
        if (e) return e;
        radix_downsweep_kernel<<<(unsigned)tiles, SORT_THREADS, 0, st>>>(a, b, count, shift, hist, tiles);
        std::swap(a, b);
    }
    *result = a;
    return cudaGetLastError();
}

// ------------------------------------------------------------ build steps
__global__ void check_ids_kernel(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, int* bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = src[e], d = dst[e];
        if (s < 0 || s >= n || d < 0 || d >= n) atomicExch(bad, 1);
    }
}

// key = sentinel bit | s << bits | d; removed entries carry only the sentinel bit
__global__ void emit_keys_kernel(const int32_t* src, const int32_t* dst, int64_t m, int bits, int sym,
                                 int drop_self, uint64_t* keys) {
    const uint64_t sentinel = 1ull << (2 * bits);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t s = (uint32_t)src[e], d = (uint32_t)dst[e];
        bool drop = drop_self && s == d;
        if (sym) {
            keys[2 * e] = drop ? sentinel : ((s << bits) | d);
            keys[2 * e + 1] = drop ? sentinel : ((d << bits) | s);
        } else {
            keys[e] = drop ? sentinel : ((s << bits) | d);
        }
    }
}

__global__ void unique_flags_kernel(const uint64_t* keys, int64_t count, int bits, int dedup, uint32_t* flags) {
    const uint64_t sentinel = 1ull << (2 * bits);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        bool keep = k < sentinel && !(dedup && i > 0 && keys[i - 1] == k);
        flags[i] = keep ? 1u : 0u;
    }
}

__global__ void compact_kernel(const uint64_t* keys, int64_t count, int bits, const uint32_t* flags,
                               const uint32_t* pos, int32_t* rows, int32_t* cols) {
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        if (flags[i]) {
            uint64_t k = keys[i];
            rows[pos[i]] = (int32_t)(k >> bits);
            cols[pos[i]] = (int32_t)(k & mask);
        }
    }
}

// row_ptr[r] = first entry whose row is >= r
__global__ void row_ptr_kernel(const int32_t* rows, int64_t mm, int32_t n, int32_t* row_ptr) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= mm; p += (int64_t)gridDim.x * blockDim.x) {
        int32_t cur = p < mm ? rows[p] : n;
        int32_t prev = p > 0 ? rows[p - 1] : -1;
        for (int32_t r = prev + 1; r <= cur; ++r) row_ptr[r] = (int32_t)p;
    }
}

// transpose keys: (d << bits) | s for every CSR entry
__global__ void transpose_keys_kernel(const int32_t* row_ptr, const int32_t* col, int32_t n, int bits, uint64_t* keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j)
            keys[j] = ((uint64_t)(uint32_t)col[j] << bits) | (uint64_t)v;
    }
}

struct DegStats {
    unsigned long long sum;
    double sumsq;
    int max;
    int isolated;
};

__global__ void degree_stats_kernel(const int32_t* row_ptr, const int32_t* in_ptr, int32_t n, DegStats* st,
                                    uint32_t* isolated) {
    int64_t words = div_up(n, 32);
    unsigned long long sum = 0;
    double sq = 0;
    int mx = 0, iso = 0;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t bitsv = 0;
        for (int j = 0; j < 32; ++j) {
            int64_t v = w * 32 + j;
            if (v >= n) break;
            int d = row_ptr[v + 1] - row_ptr[v];
            int din = in_ptr[v + 1] - in_ptr[v];
            sum += d;
            sq += (double)d * d;
            mx = max(mx, d);
            if (din == 0) {
                bitsv |= 1u << j;
                ++iso;
            }
        }
        isolated[w] = bitsv;
    }
    sum = warp_sum(sum);
    sq = warp_sum(sq);
    iso = warp_sum(iso);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st->sum, sum);
        atomicAdd(&st->sumsq, sq);
        atomicMax(&st->max, mx);
        atomicAdd(&st->isolated, iso);
    }
}

int grid_for(int64_t count, int threads) {
    int64_t b = div_up(std::max<int64_t>(count, 1), threads);
    return (int)std::min<int64_t>(b, (int64_t)num_sms() * 32);
}

// Sort `count` keys (sentinel-terminated), keep unique ones, write CSR arrays.
bfs_status keys_to_csr(uint64_t* keys, int64_t count, int bits, int dedup, int32_t n, cudaStream_t st,
                       int32_t** row_ptr_out, int32_t** col_out, int64_t* m_out) {
    Scratch sc(st);
    uint64_t* tmp;
    BFS_CUDA(sc.alloc(&tmp, count));
    uint64_t* sorted;
    BFS_CUDA(radix_sort_u64(keys, tmp, count, 2 * bits + 1, st, &sorted));
    uint32_t *flags, *pos, *d_total;
    BFS_CUDA(sc.alloc(&flags, count));
    BFS_CUDA(sc.alloc(&pos, count));
    BFS_CUDA(sc.alloc(&d_total, 1));
    unique_flags_kernel<<<grid_for(count, 256), 256, 0, st>>>(sorted, count, bits, dedup, flags);
    BFS_CUDA(exclusive_scan_u32(flags, pos, count, d_total, st));
    uint32_t total = 0;
    BFS_CUDA(cudaMemcpyAsync(&total, d_total, 4, cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    int64_t mm = total;
    if (mm > INT32_MAX) return fail(BFS_ERANGE, "graph has %lld directed entries (> 2^31-1)", (long long)mm);
    int32_t *rows, *col, *row_ptr;
    BFS_CUDA(sc.alloc(&rows, mm));
    if (cudaMalloc(&col, std::max<int64_t>(mm, 1) * sizeof(int32_t)) != cudaSuccess)
        return fail(BFS_ENOMEM, "cannot allocate col[%lld]", (long long)mm);
    if (cudaMalloc(&row_ptr, ((int64_t)n + 1) * sizeof(int32_t)) != cudaSuccess) {
        cudaFree(col);
        return fail(BFS_ENOMEM, "cannot allocate row_ptr[%d]", n + 1);
    }
    compact_kernel<<<grid_for(count, 256), 256, 0, st>>>(sorted, count, bits, flags, pos, rows, col);
    row_ptr_kernel<<<grid_for(mm + 1, 256), 256, 0, st>>>(rows, mm, n, row_ptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(col);
        cudaFree(row_ptr);
        return cuda_fail(e, "keys_to_csr");
    }
    *row_ptr_out = row_ptr;
    *col_out = col;
    *m_out = mm;
    return BFS_OK;
}

// ------------------------------------------------------------ RCM
// Reverse Cuthill-McKee numbering (Section 7.1), computed level by level.
// rank(v) = position of v in (degree, id) order.  A component starts at its
// lowest-ranked vertex; the vertices first reached from the level whose
// positions are [lb, le) form the next level, ordered by (lowest position of
// a neighbour in [lb, le), rank) -- the order in which a FIFO queue numbering
// each dequeued vertex's unnumbered neighbours in rank order numbers them.

constexpr int RCM_SMALL_SORT = 4096;       // levels up to this size are sorted by one CTA
constexpr int64_t RCM_FIND_CHUNK = 1 << 20;  // rank-order window scanned per start search

// key = degree << bits | v
__global__ void rcm_rank_keys_kernel(const int32_t* row_ptr, int32_t n, int bits, uint64_t* keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = ((uint64_t)(uint32_t)(row_ptr[v + 1] - row_ptr[v]) << bits) | (uint64_t)v;
}

// byrank[i] = vertex of rank i, rank[v]; pos = -1, minpos = INT32_MAX; the
// degree-0 vertices (the lowest ranks, each its own component) are numbered
// at once in rank order; *n0 = their count
__global__ void rcm_init_kernel(const uint64_t* sorted, const int32_t* row_ptr, int32_t n, int bits, int32_t* byrank,
                                int32_t* rank, int32_t* pos, int32_t* order, int32_t* minpos, int* n0) {
    const uint64_t mask = (1ull << bits) - 1;
    int cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(sorted[i] & mask);
        byrank[i] = v;
        rank[v] = (int32_t)i;
        minpos[v] = INT32_MAX;
        const bool iso = row_ptr[v + 1] == row_ptr[v];
        pos[v] = iso ? (int32_t)i : -1;
        if (iso) order[i] = v;
        cnt += iso ? 1 : 0;
    }
    cnt = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n0, cnt);
}

// lowest rank index in [lo, hi) whose vertex is not numbered yet
__global__ void rcm_find_start_kernel(const int32_t* byrank, const int32_t* pos, int64_t lo, int64_t hi, int* found) {
    for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x)
        if (pos[byrank[i]] < 0) atomicMin(found, (int)i);
}

__global__ void rcm_place_start_kernel(const int32_t* byrank, const int* found, int32_t next, int32_t* pos,
                                       int32_t* order) {
    const int32_t s = byrank[*found];
    pos[s] = next;
    order[next] = s;
}

// one warp per vertex of the level [lb, le): every unnumbered neighbour v
// takes the lowest such position as its key and joins the next level once
__global__ void rcm_expand_kernel(const int32_t* row_ptr, const int32_t* col, const int32_t* order, int32_t lb,
                                  int32_t le, const int32_t* pos, int32_t* minpos, uint32_t* seen, int32_t* list,
                                  int* cnt) {
    const unsigned lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = lb + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); p < le; p += nwarps) {
        const int32_t u = order[p];
        const int32_t b = row_ptr[u], e = row_ptr[u + 1];
        for (int32_t j = b + (int32_t)lane; j < e; j += 32) {
            const int32_t v = col[j];
            if (pos[v] >= 0) continue;
            atomicMin(minpos + v, (int32_t)p);
            const uint32_t bit = 1u << (v & 31);
            if (!(atomicOr(seen + (v >> 5), bit) & bit)) list[atomicAdd(cnt, 1)] = v;
        }
    }
}

// key = minpos << bits | rank
__global__ void rcm_level_keys_kernel(const int32_t* list, int32_t cnt, const int32_t* minpos, const int32_t* rank,
                                      int bits, uint64_t* keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[i];
        keys[i] = ((uint64_t)(uint32_t)minpos[v] << bits) | (uint64_t)(uint32_t)rank[v];
    }
}

// ascending bitonic sort of up to RCM_SMALL_SORT keys in one CTA
__global__ void rcm_small_sort_kernel(uint64_t* keys, int32_t cnt) {
    __shared__ uint64_t s[RCM_SMALL_SORT];
    for (int i = threadIdx.x; i < RCM_SMALL_SORT; i += blockDim.x) s[i] = i < cnt ? keys[i] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= RCM_SMALL_SORT; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < RCM_SMALL_SORT; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const uint64_t a = s[i], c = s[ixj];
                    if ((a > c) == up) {
                        s[i] = c;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) keys[i] = s[i];
}

__global__ void rcm_assign_kernel(const uint64_t* sorted, int32_t cnt, int bits, const int32_t* byrank, int32_t next,
                                  int32_t* pos, int32_t* order) {
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = byrank[sorted[i] & mask];
        pos[v] = next + (int32_t)i;
        order[next + i] = v;
    }
}

__global__ void rcm_newid_identity_kernel(int32_t n, int32_t* newid) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        newid[v] = (int32_t)v;
}

__global__ void rcm_newid_kernel(const int32_t* pos, int32_t n, int32_t* newid) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        newid[v] = n - 1 - pos[v];
}

// (newid[s] << bits) | newid[d] for every CSR entry, one warp per row
__global__ void relabel_keys_kernel(const int32_t* row_ptr, const int32_t* col, int32_t n, const int32_t* newid,
                                    int bits, uint64_t* keys) {
    const unsigned lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nwarps) {
        const uint64_t hi = (uint64_t)(uint32_t)newid[v] << bits;
        for (int32_t j = row_ptr[v] + (int32_t)lane; j < row_ptr[v + 1]; j += 32)
            keys[j] = hi | (uint64_t)(uint32_t)newid[col[j]];
    }
}

template <typename T>
bfs_status read_scalar(const T* d, T* h, cudaStream_t st) {
    BFS_CUDA(cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    return BFS_OK;
}

// newid (device [n]) of the Reverse Cuthill-McKee numbering of a symmetric CSR
bfs_status rcm_newid(const int32_t* row_ptr, const int32_t* col, int32_t n, int bits, cudaStream_t st,
                     int32_t* newid) {
    Scratch sc(st);
    uint64_t *keys, *tmp;
    int32_t *byrank, *rank, *pos, *order, *minpos, *list;
    uint32_t* seen;
    int *d_n0, *d_cnt, *d_found;
    const int64_t words = div_up(n, 32);
    if (sc.alloc(&keys, n) || sc.alloc(&tmp, n) || sc.alloc(&byrank, n) || sc.alloc(&rank, n) || sc.alloc(&pos, n) ||
        sc.alloc(&order, n) || sc.alloc(&minpos, n) || sc.alloc(&list, n) || sc.alloc(&seen, words) ||
        sc.alloc(&d_n0, 1) || sc.alloc(&d_cnt, 1) || sc.alloc(&d_found, 1)) {
        cudaGetLastError();
        return fail(BFS_ENOMEM, "RCM scratch for n=%d", n);
    }
    rcm_rank_keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(row_ptr, n, bits, keys);
    uint64_t* sorted;
    BFS_CUDA(radix_sort_u64(keys, tmp, n, bits + 32, st, &sorted));
    BFS_CUDA(cudaMemsetAsync(d_n0, 0, 4, st));
    BFS_CUDA(cudaMemsetAsync(seen, 0, words * 4, st));
    rcm_init_kernel<<<grid_for(n, 256), 256, 0, st>>>(sorted, row_ptr, n, bits, byrank, rank, pos, order, minpos, d_n0);
    int n0 = 0;
    bfs_status s = read_scalar(d_n0, &n0, st);
    if (s != BFS_OK) return s;
    int32_t next = n0;
    int64_t cursor = n0;
    while (cursor < n) {
        const int64_t hi = std::min<int64_t>(n, cursor + RCM_FIND_CHUNK);
        const int none = INT32_MAX;
        BFS_CUDA(cudaMemcpyAsync(d_found, &none, 4, cudaMemcpyHostToDevice, st));
        rcm_find_start_kernel<<<grid_for(hi - cursor, 256), 256, 0, st>>>(byrank, pos, cursor, hi, d_found);
        int found = none;
        if ((s = read_scalar(d_found, &found, st)) != BFS_OK) return s;
        if (found == none) {
            cursor = hi;
            continue;
        }
        cursor = (int64_t)found + 1;
        rcm_place_start_kernel<<<1, 1, 0, st>>>(byrank, d_found, next, pos, order);
        int32_t lb = next, le = next + 1;
        next += 1;
        for (;;) {
            BFS_CUDA(cudaMemsetAsync(d_cnt, 0, 4, st));
            rcm_expand_kernel<<<grid_for((int64_t)(le - lb) * 32, 256), 256, 0, st>>>(row_ptr, col, order, lb, le, pos,
                                                                                     minpos, seen, list, d_cnt);
            int cnt = 0;
            if ((s = read_scalar(d_cnt, &cnt, st)) != BFS_OK) return s;
            if (cnt == 0) break;
            if (next + (int64_t)cnt > n) return fail(BFS_EVALIDATE, "RCM numbered more than n vertices");
            rcm_level_keys_kernel<<<grid_for(cnt, 256), 256, 0, st>>>(list, cnt, minpos, rank, bits, keys);
            uint64_t* lsorted = keys;
            if (cnt <= RCM_SMALL_SORT) {
                rcm_small_sort_kernel<<<1, 1024, 0, st>>>(keys, cnt);
            } else {
                BFS_CUDA(radix_sort_u64(keys, tmp, cnt, 2 * bits, st, &lsorted));
            }
            rcm_assign_kernel<<<grid_for(cnt, 256), 256, 0, st>>>(lsorted, cnt, bits, byrank, next, pos, order);
            lb = le;
            le = next + cnt;
            next += cnt;
        }
    }
    if (next != n) return fail(BFS_EVALIDATE, "RCM numbered %d of %d vertices", next, n);
    rcm_newid_kernel<<<grid_for(n, 256), 256, 0, st>>>(pos, n, newid);
    BFS_CUDA(cudaGetLastError());
    BFS_CUDA(cudaStreamSynchronize(st));
    return BFS_OK;
}

// ------------------------------------------------------------ hubs-first rows
// key = (INT32_MAX - degree) << bits | v: ascending = degree descending, id ascending
__global__ void hub_rank_keys_kernel(const int32_t* row_ptr, int32_t n, int bits, uint64_t* keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = ((uint64_t)(uint32_t)(INT32_MAX - (row_ptr[v + 1] - row_ptr[v])) << bits) | (uint64_t)v;
}

__global__ void rank_of_kernel(const uint64_t* sorted, int32_t n, int bits, int32_t* byrank, int32_t* rank) {
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(sorted[i] & mask);
        byrank[i] = v;
        rank[v] = (int32_t)i;
    }
}

// (row << bits) | rank of the entry, one warp per row
__global__ void hub_row_keys_kernel(const int32_t* ptr, const int32_t* col, int32_t n, const int32_t* rank, int bits,
                                    uint64_t* keys) {
    const unsigned lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nwarps)
        for (int32_t j = ptr[v] + (int32_t)lane; j < ptr[v + 1]; j += 32)
            keys[j] = ((uint64_t)v << bits) | (uint64_t)(uint32_t)rank[col[j]];
}

__global__ void hub_col_kernel(const uint64_t* sorted, int64_t m, int bits, const int32_t* byrank, int32_t* col) {
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        col[j] = byrank[sorted[j] & mask];
}

// Replace the d-major column array by one whose rows are ordered by the
// entries' out-degree, highest first (ties by id); row bounds are unchanged.
bfs_status pull_hubs_first(bfs_graph* g, int bits, cudaStream_t st) {
    const int32_t n = g->n;
    const int64_t m = g->m;
    Scratch sc(st);
    uint64_t *rk, *rt, *keys, *tmp;
    int32_t *byrank, *rank, *col;
    if (sc.alloc(&rk, n) || sc.alloc(&rt, n) || sc.alloc(&byrank, n) || sc.alloc(&rank, n) || sc.alloc(&keys, m) ||
        sc.alloc(&tmp, m)) {
        cudaGetLastError();
        return fail(BFS_ENOMEM, "hubs-first scratch");
    }
    if (cudaMalloc(&col, (size_t)std::max<int64_t>(m, 1) * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(BFS_ENOMEM, "hubs-first column array of %lld entries", (long long)m);
    }
    hub_rank_keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(g->row_ptr, n, bits, rk);
    uint64_t* rs;
    cudaError_t e = radix_sort_u64(rk, rt, n, bits + 32, st, &rs);
    if (e == cudaSuccess) {
        rank_of_kernel<<<grid_for(n, 256), 256, 0, st>>>(rs, n, bits, byrank, rank);
        hub_row_keys_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(g->csc_ptr, g->csc_col, n, rank, bits, keys);
        uint64_t* ks;
        e = radix_sort_u64(keys, tmp, m, 2 * bits, st, &ks);
        if (e == cudaSuccess) {
            hub_col_kernel<<<grid_for(m, 256), 256, 0, st>>>(ks, m, bits, byrank, col);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(col);
        return cuda_fail(e, "hubs-first rows");
    }
    if (g->csc_col != g->col) cudaFree(g->csc_col);
    g->csc_col = col;
    return BFS_OK;
}

// Renumber a built symmetric graph in RCM order: g->perm, then the CSR again
bfs_status rcm_reorder(bfs_graph* g, int bits, cudaStream_t st) {
    if (cudaMalloc(&g->perm, (size_t)g->n * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(BFS_ENOMEM, "permutation of n=%d", g->n);
    }
    bfs_status s = rcm_newid(g->row_ptr, g->col, g->n, bits, st, g->perm);
    if (s != BFS_OK) return s;
    Scratch sc(st);
    uint64_t* keys;
    if (sc.alloc(&keys, g->m) != cudaSuccess) {
        cudaGetLastError();
        return fail(BFS_ENOMEM, "relabel keys");
    }
    relabel_keys_kernel<<<grid_for((int64_t)g->n * 32, 256), 256, 0, st>>>(g->row_ptr, g->col, g->n, g->perm, bits, keys);
    BFS_CUDA(cudaGetLastError());
    int32_t *row_ptr, *col;
    int64_t mm = 0;
    s = keys_to_csr(keys, g->m, bits, 0, g->n, st, &row_ptr, &col, &mm);
    if (s != BFS_OK) return s;
    if (mm != g->m) {
        cudaFree(row_ptr);
        cudaFree(col);
        return fail(BFS_EVALIDATE, "relabelled graph has %lld entries, expected %lld", (long long)mm, (long long)g->m);
    }
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    g->row_ptr = g->csc_ptr = row_ptr;
    g->col = g->csc_col = col;
    return BFS_OK;
}

}  // namespace

}  // namespace bfsgb

using namespace bfsgb;

extern "C" bfs_status bfs_build_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, uint32_t flags,
                                      void* cuda_stream, bfs_graph** out) {
    if (!out) return fail(BFS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n <= 0) return fail(BFS_EINVAL, "n must be positive (got %d)", n);
    if (m < 0) return fail(BFS_EINVAL, "m must be >= 0");
    if (m > 0 && (!src || !dst)) return fail(BFS_EINVAL, "src/dst is NULL");
    int sym = (flags & BFS_SYMMETRIZE) != 0;
    if ((flags & BFS_REORDER_RCM) && !sym) return fail(BFS_EINVAL, "BFS_REORDER_RCM needs BFS_SYMMETRIZE");
    int64_t count = sym ? 2 * m : m;
    if (count > INT32_MAX) return fail(BFS_ERANGE, "%lld directed entries before deduplication (> 2^31-1)", (long long)count);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int bits = 1;
    while ((1ll << bits) < (int64_t)n) ++bits;

    Scratch sc(st);
    const int32_t *d_src = src, *d_dst = dst;
    if (m > 0 && !is_device_ptr(src)) {
        int32_t* p;
        BFS_CUDA(sc.alloc(&p, m));
        BFS_CUDA(cudaMemcpyAsync(p, src, m * 4, cudaMemcpyHostToDevice, st));
        d_src = p;
    }
    if (m > 0 && !is_device_ptr(dst)) {
        int32_t* p;
        BFS_CUDA(sc.alloc(&p, m));
        BFS_CUDA(cudaMemcpyAsync(p, dst, m * 4, cudaMemcpyHostToDevice, st));
        d_dst = p;
    }
    int* d_bad;
    BFS_CUDA(sc.alloc(&d_bad, 1));
    BFS_CUDA(cudaMemsetAsync(d_bad, 0, 4, st));
    if (m > 0) check_ids_kernel<<<grid_for(m, 256), 256, 0, st>>>(d_src, d_dst, m, n, d_bad);
    int bad = 0;
    BFS_CUDA(cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, st));
    BFS_CUDA(cudaStreamSynchronize(st));
    if (bad) return fail(BFS_EINVAL, "edge list has a vertex id outside [0, %d)", n);

    uint64_t* keys;
    BFS_CUDA(sc.alloc(&keys, count));
    if (m > 0) emit_keys_kernel<<<grid_for(m, 256), 256, 0, st>>>(d_src, d_dst, m, bits, sym, (flags & BFS_DROP_SELF) != 0, keys);
    BFS_CUDA(cudaGetLastError());

    bfs_graph* g = new (std::nothrow) bfs_graph();
    if (!g) return fail(BFS_ENOMEM, "host allocation");
    g->n = n;
    g->device = device_id();
    bfs_status s = keys_to_csr(keys, count, bits, (flags & BFS_DEDUP) != 0, n, st, &g->row_ptr, &g->col, &g->m);
    if (s != BFS_OK) {
        delete g;
        return s;
    }
    g->symmetric = sym;
    if (sym) {
        g->csc_ptr = g->row_ptr;
        g->csc_col = g->col;
        if (flags & BFS_REORDER_RCM) {
            bfs_status sr = rcm_reorder(g, bits, st);
            if (sr != BFS_OK) {
                bfs_free_graph(g);
                return sr;
            }
        }
    } else {
        // CSC = rank swizzle S,D -> D,S of the built CSR (already unique)
        uint64_t* tkeys;
        bfs_status s2 = BFS_OK;
        if (sc.alloc(&tkeys, g->m) != cudaSuccess) s2 = fail(BFS_ENOMEM, "transpose keys");
        if (s2 == BFS_OK) {
            transpose_keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(g->row_ptr, g->col, n, bits, tkeys);
            int64_t mt = 0;
            s2 = keys_to_csr(tkeys, g->m, bits, 0, n, st, &g->csc_ptr, &g->csc_col, &mt);
        }
        if (s2 != BFS_OK) {
            bfs_free_graph(g);
            return s2;
        }
    }
    if (flags & BFS_PULL_HUBS_FIRST) {
        bfs_status sh = pull_hubs_first(g, bits, st);
        if (sh != BFS_OK) {
            bfs_free_graph(g);
            return sh;
        }
    }
    int64_t words = div_up(n, 32);
    DegStats* d_st;
    bfs_status s3 = BFS_OK;
    if (cudaMalloc(&g->isolated, words * 4) != cudaSuccess || sc.alloc(&d_st, 1) != cudaSuccess)
        s3 = fail(BFS_ENOMEM, "degree statistics");
    DegStats h{};
    if (s3 == BFS_OK) {
        cudaMemsetAsync(d_st, 0, sizeof(DegStats), st);
        degree_stats_kernel<<<grid_for(words, 256), 256, 0, st>>>(g->row_ptr, g->csc_ptr, n, d_st, g->isolated);
        cudaMemcpyAsync(&h, d_st, sizeof(DegStats), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s3 = cuda_fail(e, "degree statistics");
    }
    if (s3 != BFS_OK) {
        bfs_free_graph(g);
        return s3;
    }
    g->deg_max = h.max;
    g->deg_mean = (double)h.sum / n;
    g->deg_var = h.sumsq / n - g->deg_mean * g->deg_mean;
    g->n_isolated = h.isolated;
    *out = g;
    return BFS_OK;
}

extern "C" bfs_status bfs_graph_info(const bfs_graph* g, bfs_graph_stats* out) {
    if (!g || !out) return fail(BFS_EINVAL, "null argument");
    out->n = g->n;
    out->m = g->m;
    out->symmetric = g->symmetric;
    out->n_isolated = g->n_isolated;
    out->deg_max = g->deg_max;
    out->deg_mean = g->deg_mean;
    out->deg_var = g->deg_var;
    return BFS_OK;
}

extern "C" bfs_status bfs_graph_csr(const bfs_graph* g, int32_t csc, int32_t* row_ptr, int32_t* col, void* cuda_stream) {
    if (!g) return fail(BFS_EINVAL, "graph is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int32_t* rp = csc ? g->csc_ptr : g->row_ptr;
    const int32_t* cl = csc ? g->csc_col : g->col;
    if (row_ptr) BFS_CUDA(cudaMemcpyAsync(row_ptr, rp, ((int64_t)g->n + 1) * 4, cudaMemcpyDefault, st));
    if (col && g->m > 0) BFS_CUDA(cudaMemcpyAsync(col, cl, g->m * 4, cudaMemcpyDefault, st));
    if ((row_ptr && !is_device_ptr(row_ptr)) || (col && !is_device_ptr(col))) BFS_CUDA(cudaStreamSynchronize(st));
    return BFS_OK;
}

extern "C" void bfs_free_graph(bfs_graph* g) {
    if (!g) return;
    free_ws1(g->ws1);
    free_wsms(g->wsms);
    if (g->csc_ptr && g->csc_ptr != g->row_ptr) cudaFree(g->csc_ptr);
    if (g->csc_col && g->csc_col != g->col) cudaFree(g->csc_col);
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->isolated);
    cudaFree(g->perm);
    delete g;
}

extern "C" bfs_status bfs_graph_permutation(const bfs_graph* g, int32_t* newid, void* cuda_stream) {
    if (!g || !newid) return fail(BFS_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool host = !is_device_ptr(newid);
    if (g->perm) {
        BFS_CUDA(cudaMemcpyAsync(newid, g->perm, (size_t)g->n * 4, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
        if (host) BFS_CUDA(cudaStreamSynchronize(st));
        return BFS_OK;
    }
    if (host) {
        for (int32_t v = 0; v < g->n; ++v) newid[v] = v;
        return BFS_OK;
    }
    rcm_newid_identity_kernel<<<grid_for(g->n, 256), 256, 0, st>>>(g->n, newid);
    BFS_CUDA(cudaGetLastError());
    return BFS_OK;
}
