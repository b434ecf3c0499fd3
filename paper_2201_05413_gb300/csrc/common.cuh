// common.cuh -- shared helpers of the gbpcg CUDA library (errors, memory,
// launch geometry, deterministic block reductions).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gbpcg.h"

namespace gb {

// NVTX range over one library phase (assembly, SELL build, a solve, a serving
// chunk): profilers (nsys, ncu --nvtx) attribute the kernels to the phase.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// ---------------------------------------------------------------- errors --
void set_error(const char *fmt, ...);

// Kernel launch accounting: every launch site calls count_launches(1); launches
// recorded into a graph body are not counted at capture time (set_capturing),
// the solver adds the launches the graph actually executed.
void count_launches(int64_t k);
void set_capturing(bool on);

#define GB_CHECK_CUDA(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            ::gb::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,             \
                            cudaGetErrorString(_e));                               \
            return GB_ECUDA;                                                       \
        }                                                                          \
    } while (0)

#define GB_TRY(expr)                 \
    do {                             \
        int _rc = (expr);            \
        if (_rc != GB_OK) return _rc; \
    } while (0)

#define GB_REQUIRE(cond, ...)                 \
    do {                                      \
        if (!(cond)) {                        \
            ::gb::set_error(__VA_ARGS__);     \
            return GB_EINVAL;                 \
        }                                     \
    } while (0)

// ---------------------------------------------------------------- memory --
// Allocations go through the caller's allocator, or cudaMalloc/cudaFree when
// none was given (the stream is passed to the caller's allocator only).
void count_device_alloc();  // every device allocation Mem makes (gbpcg_device_allocations)

struct Mem {
    gb_allocator a{};
    bool has = false;
    cudaStream_t s = nullptr;
    Mem() = default;
    Mem(const gb_allocator *al, cudaStream_t st) : s(st) {
        if (al && al->alloc && al->free) { a = *al; has = true; }
    }
    int alloc(void **p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) bytes = 256;
        if (has) {
            *p = a.alloc(a.ctx, bytes, (void *)s);
            if (!*p) { set_error("allocator returned NULL for %zu bytes", bytes); return GB_ENOMEM; }
            count_device_alloc();
            return GB_OK;
        }
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            set_error("cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
            *p = nullptr;
            return e == cudaErrorMemoryAllocation ? GB_ENOMEM : GB_ECUDA;
        }
        count_device_alloc();
        return GB_OK;
    }
    template <class T> int alloc_n(T **p, size_t n) { return alloc((void **)p, n * sizeof(T)); }
    void release(void *p) {
        if (!p) return;
        if (has) a.free(a.ctx, p, (void *)s);
        else cudaFree(p);
    }
};

// Device-wide exclusive scan of n values into out[0..n] (out[n] = total),
// computed in int64; *h_total receives the total (one stream sync).
template <class In, class Out>
int scan_exclusive(const In *in, Out *out, int64_t n, int64_t *h_total, Mem &mem);

// GBPCG_USE_GRAPH=0 in the environment: solver loops run as direct launches
// instead of CUDA-graph while-nodes (same kernels; for launch-level profilers,
// which do not list the kernels a graph's device-side loop replays).
bool graphs_disabled();

// ------------------------------------------------------- launch geometry --
int num_sms();
// blocks per SM of the TMA-staged SpMV (fixed: its warp partition is built for it)
#ifndef GB_TMA_BLOCKS_PER_SM
#define GB_TMA_BLOCKS_PER_SM 4
#endif
constexpr int TMA_BLOCKS_PER_SM = GB_TMA_BLOCKS_PER_SM;
// the fp32 SpMV (smaller shared-memory ring) runs 5 blocks per SM
#ifndef GB_TMA_BLOCKS_PER_SM_NARROW
#define GB_TMA_BLOCKS_PER_SM_NARROW 5
#endif
constexpr int TMA_BLOCKS_PER_SM_NARROW = GB_TMA_BLOCKS_PER_SM_NARROW;
// Grid for a grid-stride kernel: a multiple of the SM count, at most `want`.
inline int stride_grid(int64_t work_items, int block, int per_sm) {
    int sms = num_sms();
    int64_t need = (work_items + block - 1) / block;
    int64_t g = (int64_t)sms * per_sm;
    if (need < g) g = need < 1 ? 1 : need;
    return (int)g;
}

// ------------------------------------------------------------ reductions --
// Sum over a block in a fixed order (warp shuffles, then warp 0 over the warp
// sums): deterministic for a fixed block size.  Every thread must call it.
template <int NT, class T>
__device__ __forceinline__ T block_sum(T v, T *smem /* >= NT/32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem[w] = v;
    __syncthreads();
    T r = T(0);
    if (w == 0) {
        r = (l < NT / 32) ? smem[l] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

}  // namespace gb
