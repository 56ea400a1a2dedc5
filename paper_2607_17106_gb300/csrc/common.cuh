// common.cuh -- internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <mutex>

#include "../../include/bfs.h"

namespace bfsgb {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
bfs_status fail(bfs_status s, const char* fmt, ...);
bfs_status cuda_fail(cudaError_t e, const char* what);

#define BFS_CUDA(call)                                          \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return ::bfsgb::cuda_fail(_e, #call); \
    } while (0)

// Pointer classification: true when p is device-accessible memory on the
// current device (device or managed); false for pageable or pinned host.
bool is_device_ptr(const void* p);

// ------------------------------------------------------ device error codes
enum : int32_t {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,     // a grid/team barrier wait exceeded its limit
    DEV_OVERFLOW = 2,    // a work list exceeded its capacity
    DEV_LEVELS = 3       // max_levels exceeded
};

// ------------------------------------------------------------------ graph
struct Workspace1;   // single-source state (bfs_single.cu)
struct WorkspaceMS;  // MS-BFS state (msbfs.cu)

}  // namespace bfsgb

struct bfs_graph {
    int32_t n = 0;
    int64_t m = 0;            // directed CSR entries
    int32_t symmetric = 0;
    int32_t device = 0;
    int32_t* row_ptr = nullptr;   // [n+1]
    int32_t* col = nullptr;       // [m]
    int32_t* csc_ptr = nullptr;   // [n+1], == row_ptr when symmetric
    int32_t* csc_col = nullptr;   // [m],   == col when symmetric
    uint32_t* isolated = nullptr; // [W] bit v set iff deg(v) == 0 (out- and in-degree)
    int32_t* perm = nullptr;      // [n] new id of each input vertex (BFS_REORDER_RCM), else null
    int32_t n_isolated = 0;
    int32_t deg_max = 0;
    double deg_mean = 0, deg_var = 0;
    int64_t n_big_units = 0;      // sizing of push chunk units, per chunk size (set on first run)
    std::mutex lock;
    bfsgb::Workspace1* ws1 = nullptr;
    bfsgb::WorkspaceMS* wsms = nullptr;
};

namespace bfsgb {

void free_ws1(Workspace1*);
void free_wsms(WorkspaceMS*);

__host__ __device__ inline int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------ device primitives
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// An L2 (cache-global) load the compiler keeps where it is written: a level's
// counters are read with three of these in a row, so that all three are in
// flight together instead of the later ones being sunk past the first test
// and costing another round trip.
__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// Control-block words a whole CTA needs (a level's counters): thread 0 loads
// them, the CTA reads them from shared memory.  When every warp of every CTA
// loaded the same words after a grid barrier, thousands of requests queued on
// one L2 sector and each level took about a microsecond longer.
// Block-uniform; both barriers are needed (the first keeps a previous call's
// readers ahead of thread 0's writes).
template <int N>
__device__ __forceinline__ void cta_load_u64(const unsigned long long* const (&src)[N], unsigned long long (&dst)[N]) {
    __shared__ unsigned long long s[N];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) s[i] = ld_cg_u64(src[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) dst[i] = s[i];
}

__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(const volatile int*)p; }

// Grid barrier state: one per persistent launch (zeroed before launch).
struct GridBarrier {
    unsigned count;  // CTA arrivals since the state was zeroed (monotonic)
    int abort;       // set by any CTA that gives up; every waiter checks it
    int err;         // DEV_* code of the first failure
    unsigned pad;
};

// Barrier over `nblocks` co-resident CTAs (cooperative launch).  Each CTA
// keeps the running arrival target in `target` (nblocks more per barrier);
// thread 0 adds its arrival to the monotonic counter and waits until the
// counter reaches the target, with a %globaltimer limit: on expiry it
// records DEV_TIMEOUT, raises the abort flag and returns false, so every CTA
// leaves its loop.  Returns false when the barrier was aborted.
// `before_arrival` runs on thread 0 after the CTA's __syncthreads and before
// the arrival, so its writes are published by the same release.
// `after_open` runs on thread 0 once the barrier is open (after the acquire,
// beside the read of the abort flag, so that their loads overlap); what it
// stores in shared memory is visible to the CTA when grid_sync returns.
struct NoArrivalWork {
    __device__ void operator()() const {}
};
template <typename F = NoArrivalWork, typename A = NoArrivalWork>
__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned nblocks, unsigned& target, int64_t timeout_ns,
                                          F before_arrival = F(), A after_open = A()) {
    __shared__ int s_ok;
    __syncthreads();
    target += nblocks;
    if (threadIdx.x == 0) {
        before_arrival();
        int ok = 1;
        // the release add publishes every write of this CTA made before the
        // __syncthreads above; the acquire load that sees the last arrival
        // makes all CTAs' writes visible to this CTA after the one below
        red_release_add_u32(&b->count, 1u);
        const uint64_t t0 = globaltimer_ns();
        unsigned spins = 0;
        while ((int)(ld_acquire_u32(&b->count) - target) < 0) {
            // limits are checked on the first poll that finds the barrier
            // open and every 32 polls after it
            if ((++spins & 31u) == 1) {
                if (ld_volatile_i32(&b->abort)) { ok = 0; break; }
                if ((int64_t)(globaltimer_ns() - t0) > timeout_ns) {
                    atomicCAS(&b->err, 0, (int)DEV_TIMEOUT);
                    atomicExch(&b->abort, 1);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok) after_open();
        if (ld_volatile_i32(&b->abort)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Block-wide exclusive scan of one int per thread (blockDim.x <= 1024).
// Returns the exclusive prefix; *total receives the block sum.  Uses `tmp`
// (>= 33 ints of shared memory).
__device__ __forceinline__ int block_exclusive_scan(int x, int* tmp, int* total) {
    unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    unsigned nw = (blockDim.x + 31) >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < nw) ? tmp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if ((int)lane >= o) wi += y;
        }
        if (lane < nw) tmp[lane] = wi - w;
        if (lane == 31) tmp[32] = wi;
    }
    __syncthreads();
    int r = tmp[warp] + incl - x;
    *total = tmp[32];
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ------------------------------------------------------------ chunk units
// A row of deg >= chunk entries is expanded as ceil(deg / chunk) units
// (v, 0), (v, 1), ... appended to out[*len ...]; a list that would pass cap
// records DEV_OVERFLOW in *err and drops the units.
__device__ __forceinline__ void append_units(int2* out, unsigned long long* len, int64_t cap, int* err, int v, int deg,
                                             int chunk) {
    const int nch = (deg + chunk - 1) / chunk;
    const unsigned long long ub = atomicAdd(len, (unsigned long long)nch);
    if (ub + nch <= (unsigned long long)cap) {
        for (int k = 0; k < nch; ++k) out[ub + k] = make_int2(v, k);
    } else {
        atomicCAS(err, 0, (int)DEV_OVERFLOW);
    }
}

// The same for the lanes of a warp with big set: one atomic per warp.  Warp-uniform call.
__device__ __forceinline__ void append_units_warp(int2* out, unsigned long long* len, int64_t cap, int* err, bool big,
                                                  int v, int deg, int chunk) {
    const unsigned bm = __ballot_sync(0xffffffffu, big);
    if (!bm) return;
    const unsigned lane = lane_id();
    const int nch = big ? (deg + chunk - 1) / chunk : 0;
    int incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(len, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + total > (unsigned long long)cap) {
        if (lane == 0) atomicCAS(err, 0, (int)DEV_OVERFLOW);
        return;
    }
    const unsigned long long off = base + (incl - nch);
    for (int k = 0; k < nch; ++k) out[off + k] = make_int2(v, k);
}

// ------------------------------------------------------------- launching
int num_sms();
int device_id();

}  // namespace bfsgb
