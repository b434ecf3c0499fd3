// util.cu -- error reporting, device properties and the device-wide scan.
#include "common.cuh"

#include <atomic>
#include <mutex>

namespace gb {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;

void count_launches(int64_t k) {
    if (!g_capturing) g_launches.fetch_add(k, std::memory_order_relaxed);
}
void set_capturing(bool on) { g_capturing = on; }
long long launches_total() { return g_launches.load(); }

static std::atomic<long long> g_dev_allocs{0};
void count_device_alloc() { g_dev_allocs.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

bool graphs_disabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("GBPCG_USE_GRAPH");
        v = (e && e[0] == '0') ? 1 : 0;
    }
    return v == 1;
}

int num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// ------------------------------------------------------------------ scan --
// Three phases over tiles of SCAN_TILE values: tile sums, an exclusive scan of
// the tile sums by one block (looping with a carry), and the per-tile scan
// with its offset.  All sums in int64; deterministic.
constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *smem, int64_t *total) {
    // warp-inclusive scan, then scan of the warp totals
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? smem[lane] : 0;
        int64_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        smem[lane] = s - t;  // exclusive warp offsets
        if (lane == 31) smem[32] = s;
    }
    __syncthreads();
    int64_t r = x - v + smem[w];
    *total = smem[32];
    __syncthreads();
    return r;
}

template <class In>
__global__ void k_scan_tile_sums(const In *in, int64_t n, int64_t *tile_sums) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) s += (int64_t)in[i];
    }
    int64_t tot;
    block_exclusive_scan(s, sm, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_tile_offsets(int64_t *tile_sums, int64_t ntiles, int64_t *total) {
    __shared__ int64_t sm[33];
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += SCAN_BLOCK) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < ntiles ? tile_sums[i] : 0;
        int64_t tot;
        int64_t e = block_exclusive_scan(v, sm, &tot);
        if (i < ntiles) tile_sums[i] = e + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <class In, class Out>
__global__ void k_scan_apply(const In *in, Out *out, int64_t n, const int64_t *tile_off,
                             const int64_t *total) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        v[k] = i < n ? (int64_t)in[i] : 0;
        s += v[k];
    }
    int64_t tot;
    int64_t e = block_exclusive_scan(s, sm, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) out[i] = (Out)e;
        e += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (Out)*total;
}

template <class In, class Out>
int scan_exclusive(const In *in, Out *out, int64_t n, int64_t *h_total, Mem &mem) {
    const int64_t ntiles = n > 0 ? (n + SCAN_TILE - 1) / SCAN_TILE : 1;
    int64_t *tmp = nullptr;
    GB_TRY(mem.alloc_n(&tmp, (size_t)ntiles + 1));
    ::gb::count_launches(1); k_scan_tile_sums<In><<<(unsigned)ntiles, SCAN_BLOCK, 0, mem.s>>>(in, n, tmp);
    ::gb::count_launches(1); k_scan_tile_offsets<<<1, SCAN_BLOCK, 0, mem.s>>>(tmp, ntiles, tmp + ntiles);
    ::gb::count_launches(1); k_scan_apply<In, Out><<<(unsigned)ntiles, SCAN_BLOCK, 0, mem.s>>>(in, out, n, tmp, tmp + ntiles);
    cudaError_t e = cudaGetLastError();
    int64_t tot = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, tmp + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, mem.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(mem.s);
    mem.release(tmp);
    if (e != cudaSuccess) {
        set_error("scan: %s", cudaGetErrorString(e));
        return GB_ECUDA;
    }
    if (h_total) *h_total = tot;
    return GB_OK;
}

template int scan_exclusive<int32_t, int32_t>(const int32_t *, int32_t *, int64_t, int64_t *, Mem &);
template int scan_exclusive<int32_t, int64_t>(const int32_t *, int64_t *, int64_t, int64_t *, Mem &);
template int scan_exclusive<int64_t, int64_t>(const int64_t *, int64_t *, int64_t, int64_t *, Mem &);

}  // namespace gb

extern "C" const char *gbpcg_last_error(void) { return gb::g_last_error.c_str(); }
extern "C" int64_t gbpcg_kernel_launches(void) { return gb::launches_total(); }
extern "C" int64_t gbpcg_device_allocations(void) { return gb::g_dev_allocs.load(); }
extern "C" const char *gbpcg_version(void) { return "gbpcg 0.1 (sm_103a)"; }
