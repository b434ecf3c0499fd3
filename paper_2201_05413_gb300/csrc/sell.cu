// sell.cu -- CSR -> SELL-C-sigma conversion and the standalone SELL SpMV.
//
// SELL-C-sigma (sliced ELLPACK, sorted inside windows of sigma rows): the
// row order is a stable descending-length sort inside each window, the
// reordered rows are cut into chunks of C rows stored column-major and padded
// to the chunk's longest row (padding entry: the row's own index, value 0).
// The permutation is symmetric, so every solver vector lives in the new order
// and the matrix keeps its symmetry.  Column-major chunks make the C lanes of
// a warp read C consecutive indices and values per step: fully coalesced.
#include <cuda_bf16.h>

#include "common.cuh"
#include <cstring>

#include "sell.cuh"

namespace gb {

int fem_csr_view(const gb_fem_system *s, int64_t *n, const int32_t **rp, const int32_t **col,
                 const double **val, const double **diag, int *max_row);

__global__ void k_row_len_diag(int64_t n, const int32_t *rp, const int32_t *ci, const double *v,
                               int32_t *len, double *diag, int *max_len, int *bad_diag) {
    int lmax = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = rp[i], b = rp[i + 1];
        len[i] = b - a;
        lmax = max(lmax, b - a);
        double d = 0.0;
        for (int32_t k = a; k < b; ++k)
            if (ci[k] == (int32_t)i) d = v[k];
        if (!(d != 0.0)) atomicExch(bad_diag, 1);
        diag[i] = d;
    }
    atomicMax(max_len, lmax);
}

// One warp per sigma-window: histogram of row lengths, descending offsets,
// then a stable placement in row order (ties ranked with __match_any_sync).
__global__ void k_sigma_sort(int64_t n, int sigma, int max_len, const int32_t *len, int32_t *perm) {
    extern __shared__ int bins[];  // max_len + 1
    const int lane = threadIdx.x;
    const int64_t w0 = (int64_t)blockIdx.x * sigma;
    const int64_t w1 = min(n, w0 + sigma);
    for (int b = lane; b <= max_len; b += 32) bins[b] = 0;
    __syncwarp();
    for (int64_t i = w0 + lane; i < w1; i += 32) atomicAdd(&bins[len[i]], 1);
    __syncwarp();
    if (lane == 0) {  // exclusive offsets in descending length order
        int acc = 0;
        for (int b = max_len; b >= 0; --b) { int c = bins[b]; bins[b] = acc; acc += c; }
    }
    __syncwarp();
    for (int64_t t0 = w0; t0 < w1; t0 += 32) {
        const int64_t i = t0 + lane;
        const int L = i < w1 ? len[i] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, L);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (L >= 0) perm[w0 + bins[L] + rank] = (int32_t)i;
        __syncwarp();
        if (L >= 0 && rank == 0) bins[L] += __popc(peers);
        __syncwarp();
    }
}

__global__ void k_identity(int64_t n, int32_t *perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = (int32_t)i;
}

__global__ void k_perm_rows(int64_t n, const int32_t *perm, const int32_t *len, const double *diag,
                            int32_t *iperm, int32_t *row_len, double *dinv, float *dinv32) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = perm[r];
        iperm[o] = (int32_t)r;
        row_len[r] = len[o];
        const double di = 1.0 / diag[o];
        dinv[r] = di;
        dinv32[r] = (float)di;
    }
}

// max of positive doubles through their bit patterns (order-preserving)
__global__ void k_max_pos(int64_t n, const double *v, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(v[i]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_chunk_width(int64_t n, int64_t nchunks, int C, const int32_t *row_len,
                              int32_t *chunk_w, int64_t *chunk_sz) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        int w = 0;
        for (int64_t r = c * C; r < (c + 1) * C && r < n; ++r) w = max(w, row_len[r]);
        chunk_w[c] = w;
        chunk_sz[c] = (int64_t)w * C;
    }
}

__global__ void k_sell_fill(int64_t n, int64_t nchunks, int C, const int32_t *perm, const int32_t *iperm,
                            const int32_t *rp, const int32_t *ci, const double *v,
                            const int64_t *chunk_ptr, const int32_t *chunk_w, int32_t *col,
                            double *val, float *val32, __nv_bfloat16 *val16) {
    const int64_t rows = nchunks * C;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = r / C;
        const int t = (int)(r - c * C);
        const int w = chunk_w[c];
        const int64_t base = chunk_ptr[c] + t;
        int32_t a = 0, L = 0;
        if (r < n) { const int32_t o = perm[r]; a = rp[o]; L = rp[o + 1] - a; }
        for (int j = 0; j < w; ++j) {
            const int64_t k = base + (int64_t)j * C;
            int32_t cc;
            double vv;
            if (j < L) { cc = iperm[ci[a + j]]; vv = v[a + j]; }
            else { cc = r < n ? (int32_t)r : 0; vv = 0.0; }
            col[k] = cc;
            val[k] = vv;
            if (val32) val32[k] = (float)vv;
            if (val16) val16[k] = __float2bfloat16_rn((float)vv);
        }
    }
}

// 16-bit column deltas for the TMA SpMV: delta = col - min(row, n-1) for every
// padded slot (padding: the row itself, delta 0; rows past n point at n-1).
// *overflow is set if a delta does not fit in int16 (the matrix then keeps
// int32 indices only).
__global__ void k_col_delta(int64_t n, int64_t nchunks, const int64_t *chunk_ptr, const int32_t *chunk_w,
                            const int32_t *col, int16_t *col16, int *overflow) {
    const int64_t rows = nchunks * 32;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = r >> 5;
        const int t = (int)(r & 31);
        const int w = chunk_w[c];
        const int64_t base = chunk_ptr[c] + t;
        const int64_t rb = r < n ? r : n - 1;
        bool bad = false;
        for (int j = 0; j < w; ++j) {
            const int64_t k = base + (int64_t)j * 32;
            int64_t d = r < n ? (int64_t)col[k] - rb : 0;
            if (d < -32768 || d > 32767) { bad = true; d = 0; }
            col16[k] = (int16_t)d;
        }
        if (bad) atomicExch(overflow, 1);
    }
}

// Warp w of the TMA SpMV owns chunks [warp_chunk[w], warp_chunk[w+1]): the
// first chunk whose start is at or after w/nw of the padded nonzeros.
__global__ void k_warp_partition(int64_t nchunks, const int64_t *chunk_ptr, int64_t padded, int nw,
                                 int32_t *warp_chunk) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w <= nw; w += (int64_t)gridDim.x * blockDim.x) {
        if (w == nw) { warp_chunk[w] = (int32_t)nchunks; continue; }
        const int64_t target = (padded * w) / nw;
        int64_t lo = 0, hi = nchunks;  // first c in [0, nchunks] with chunk_ptr[c] >= target
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (chunk_ptr[mid] < target) lo = mid + 1; else hi = mid;
        }
        warp_chunk[w] = (int32_t)lo;
    }
}

static int build_sell(int64_t n, const int32_t *rp, const int32_t *ci, const double *v,
                      const double *diag_in, int max_row_hint, int C, int sigma, int val_types,
                      const gb_allocator *alloc, cudaStream_t st, gb_sell **out) {
    GB_REQUIRE(out, "csr_to_sell: NULL output");
    *out = nullptr;
    GB_REQUIRE(n >= 1, "csr_to_sell: empty matrix");
    GB_REQUIRE(C == 32 || C == 64 || C == 128, "csr_to_sell: C must be 32, 64 or 128");
    GB_REQUIRE(sigma >= 1, "csr_to_sell: sigma must be >= 1");
    GB_REQUIRE((val_types & ~15) == 0, "csr_to_sell: unknown val_types bits");
    gb_sell *A = new gb_sell();
    A->mem = Mem(alloc, st);
    Mem &mem = A->mem;
    A->n = n; A->C = C; A->sigma = sigma;
    A->nchunks = (n + C - 1) / C;
    int rc = GB_OK;
    int32_t *len = nullptr;
    double *diag = nullptr;
    int *flags = nullptr;  // [0] max_len, [1] bad diagonal
    int64_t *chunk_sz = nullptr;
    int hflags[2] = {0, 0};
    int64_t padded = 0;
    int32_t nnz32 = 0;
    const int grid = stride_grid(n, 256, 8);
#define STEP(x)                                  \
    do {                                         \
        rc = (x);                                \
        if (rc != GB_OK) goto fail;              \
    } while (0)
#define STEPC(x)                                                               \
    do {                                                                       \
        cudaError_t _e = (x);                                                  \
        if (_e != cudaSuccess) {                                               \
            set_error("csr_to_sell: %s: %s", #x, cudaGetErrorString(_e));     \
            rc = GB_ECUDA;                                                     \
            goto fail;                                                         \
        }                                                                      \
    } while (0)
    STEP(mem.alloc_n(&len, n));
    STEP(mem.alloc_n(&diag, n));
    STEP(mem.alloc_n(&flags, 2));
    STEPC(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st));
    ::gb::count_launches(1); k_row_len_diag<<<grid, 256, 0, st>>>(n, rp, ci, v, len, diag, flags, flags + 1);
    STEPC(cudaGetLastError());
    STEPC(cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    STEPC(cudaStreamSynchronize(st));
    if (hflags[1]) { set_error("csr_to_sell: a row has no (or a zero) diagonal entry"); rc = GB_EINVAL; goto fail; }
    if (hflags[0] > 4096) { set_error("csr_to_sell: row length %d above 4096", hflags[0]); rc = GB_EINVAL; goto fail; }
    A->max_row = hflags[0];
    (void)diag_in; (void)max_row_hint;
    STEP(mem.alloc_n(&A->perm, n));
    STEP(mem.alloc_n(&A->iperm, n));
    STEP(mem.alloc_n(&A->row_len, n));
    STEP(mem.alloc_n(&A->dinv, n));
    STEP(mem.alloc_n(&A->dinv32, n));
    if (sigma > 1) {
        const int64_t nwin = (n + sigma - 1) / sigma;
        ::gb::count_launches(1); k_sigma_sort<<<(unsigned)nwin, 32, (A->max_row + 1) * sizeof(int), st>>>(n, sigma, A->max_row, len, A->perm);
    } else {
        ::gb::count_launches(1); k_identity<<<grid, 256, 0, st>>>(n, A->perm);
    }
    STEPC(cudaGetLastError());
    ::gb::count_launches(1); k_perm_rows<<<grid, 256, 0, st>>>(n, A->perm, len, diag, A->iperm, A->row_len, A->dinv, A->dinv32);
    {
        unsigned long long *dmax = reinterpret_cast<unsigned long long *>(flags);  // 8 bytes: flags holds two ints
        unsigned long long hmax = 0;
        STEPC(cudaMemsetAsync(dmax, 0, sizeof(*dmax), st));
        ::gb::count_launches(1); k_max_pos<<<grid, 256, 0, st>>>(n, A->dinv, dmax);
        STEPC(cudaMemcpyAsync(&hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st));
        STEPC(cudaStreamSynchronize(st));
        std::memcpy(&A->dinv_max, &hmax, sizeof(double));
    }
    STEP(mem.alloc_n(&A->chunk_w, A->nchunks));
    STEP(mem.alloc_n(&A->chunk_ptr, A->nchunks + 1));
    STEP(mem.alloc_n(&chunk_sz, A->nchunks));
    ::gb::count_launches(1); k_chunk_width<<<stride_grid(A->nchunks, 256, 8), 256, 0, st>>>(n, A->nchunks, C, A->row_len, A->chunk_w, chunk_sz);
    STEPC(cudaGetLastError());
    STEP((scan_exclusive<int64_t, int64_t>(chunk_sz, A->chunk_ptr, A->nchunks, &padded, mem)));
    if (padded >= (int64_t)INT32_MAX) { set_error("csr_to_sell: padded size %lld above 2^31", (long long)padded); rc = GB_TOO_LARGE; goto fail; }
    A->padded = padded;
    STEPC(cudaMemcpyAsync(&nnz32, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    STEP(mem.alloc_n(&A->col, padded));
    STEP(mem.alloc_n(&A->val, padded));
    if (val_types & GB_VAL_F32) STEP(mem.alloc_n(&A->val32, padded));
    if (val_types & GB_VAL_BF16) STEP(mem.alloc_n(&A->val16, padded));
    ::gb::count_launches(1); k_sell_fill<<<stride_grid(A->nchunks * C, 256, 8), 256, 0, st>>>(
        n, A->nchunks, C, A->perm, A->iperm, rp, ci, v, A->chunk_ptr, A->chunk_w, A->col, A->val,
        A->val32, A->val16);
    STEPC(cudaGetLastError());
    if (C == 32 && (val_types & GB_IDX16)) {  // 16-bit column deltas where they fit
        STEP(mem.alloc_n(&A->col16, padded));
        STEPC(cudaMemsetAsync(flags, 0, sizeof(int), st));
        ::gb::count_launches(1); k_col_delta<<<stride_grid(A->nchunks * 32, 256, 8), 256, 0, st>>>(
            n, A->nchunks, A->chunk_ptr, A->chunk_w, A->col, A->col16, flags);
        STEPC(cudaGetLastError());
        STEPC(cudaMemcpyAsync(hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        STEPC(cudaStreamSynchronize(st));
        if (hflags[0]) { mem.release(A->col16); A->col16 = nullptr; }
    }
    if (C == 32) {  // chunk ranges of the TMA-staged SpMV (one per warp of its fixed grid)
        A->nwarps = num_sms() * TMA_BLOCKS_PER_SM * 8;
        STEP(mem.alloc_n(&A->warp_chunk, (size_t)A->nwarps + 1));
        ::gb::count_launches(1); k_warp_partition<<<stride_grid(A->nwarps + 1, 256, 4), 256, 0, st>>>(
            A->nchunks, A->chunk_ptr, padded, A->nwarps, A->warp_chunk);
        A->nwarps5 = num_sms() * TMA_BLOCKS_PER_SM_NARROW * 8;
        STEP(mem.alloc_n(&A->warp_chunk5, (size_t)A->nwarps5 + 1));
        ::gb::count_launches(1); k_warp_partition<<<stride_grid(A->nwarps5 + 1, 256, 4), 256, 0, st>>>(
            A->nchunks, A->chunk_ptr, padded, A->nwarps5, A->warp_chunk5);
        STEPC(cudaGetLastError());
    }
    STEPC(cudaStreamSynchronize(st));
    A->nnz = nnz32;
    mem.release(len);
    mem.release(diag);
    mem.release(flags);
    mem.release(chunk_sz);
    *out = A;
    return GB_OK;
fail:
    mem.release(len);
    mem.release(diag);
    mem.release(flags);
    mem.release(chunk_sz);
    sell_destroy(A);
    return rc;
#undef STEP
#undef STEPC
}

// ------------------------------------------------------------ SpMV (fp64) --
__global__ void k_gather(int64_t n, const int32_t *perm, const double *x, double *xp) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        xp[r] = x[perm[r]];
}
__global__ void k_scatter(int64_t n, const int32_t *perm, const double *yp, double *y) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        y[perm[r]] = yp[r];
}

__global__ void k_sell_spmv(SellView A, const double *x, double *y) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int slices = A.C >> 5;
    for (int64_t s = gw; s < A.nchunks * slices; s += nw) {
        const int64_t c = s / slices;
        const int sub = (int)(s - c * slices);
        const int64_t r = c * A.C + sub * 32 + lane;
        if (r >= A.n) continue;
        const int L = A.row_len[r];
        const int64_t base = A.chunk_ptr[c] + sub * 32 + lane;
        double acc = 0.0;
        for (int j = 0; j < L; ++j) {
            const int64_t k = base + (int64_t)j * A.C;
            acc += A.val[k] * x[A.col[k]];
        }
        y[r] = acc;
    }
}

}  // namespace gb

using namespace gb;

extern "C" int csr_to_sell(const gb_fem_system *sys, int C, int sigma, int val_types,
                           const gb_allocator *alloc, void *stream, gb_sell **out) {
    gb::Range range("gbpcg:csr_to_sell");
    GB_REQUIRE(sys, "csr_to_sell: NULL system");
    int64_t n;
    const int32_t *rp, *col;
    const double *val, *diag;
    int max_row;
    fem_csr_view(sys, &n, &rp, &col, &val, &diag, &max_row);
    return build_sell(n, rp, col, val, diag, max_row, C, sigma, val_types, alloc, (cudaStream_t)stream, out);
}

extern "C" int csr_to_sell_raw(int64_t n, const int32_t *d_rowptr, const int32_t *d_col,
                               const double *d_val, int C, int sigma, int val_types,
                               const gb_allocator *alloc, void *stream, gb_sell **out) {
    gb::Range range("gbpcg:csr_to_sell");
    GB_REQUIRE(d_rowptr && d_col && d_val, "csr_to_sell_raw: NULL array");
    return build_sell(n, d_rowptr, d_col, d_val, nullptr, 0, C, sigma, val_types, alloc,
                      (cudaStream_t)stream, out);
}

extern "C" int sell_info(const gb_sell *A, gb_sell_info *o) {
    GB_REQUIRE(A && o, "sell_info: NULL argument");
    o->n = A->n; o->nnz = A->nnz; o->padded = A->padded; o->nchunks = A->nchunks;
    o->C = A->C; o->sigma = A->sigma; o->max_row = A->max_row; o->reserved = 0;
    o->d_perm = A->perm; o->d_chunk_ptr = A->chunk_ptr; o->d_chunk_w = A->chunk_w;
    o->d_row_len = A->row_len; o->d_col = A->col; o->d_val = A->val; o->d_dinv = A->dinv;
    o->d_col16 = A->col16;
    return GB_OK;
}

extern "C" int sell_spmv(const gb_sell *A, const double *d_x, double *d_y, void *stream) {
    GB_REQUIRE(A && d_x && d_y, "sell_spmv: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    Mem mem(nullptr, st);
    double *xp = nullptr, *yp = nullptr;
    GB_TRY(mem.alloc_n(&xp, A->n));
    GB_TRY(mem.alloc_n(&yp, A->n));
    const int grid = stride_grid(A->n, 256, 8);
    ::gb::count_launches(1); k_gather<<<grid, 256, 0, st>>>(A->n, A->perm, d_x, xp);
    ::gb::count_launches(1); k_sell_spmv<<<stride_grid(A->n, 256, 8), 256, 0, st>>>(A->view(), xp, yp);
    ::gb::count_launches(1); k_scatter<<<grid, 256, 0, st>>>(A->n, A->perm, yp, d_y);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    mem.release(xp);
    mem.release(yp);
    GB_CHECK_CUDA(e);
    return GB_OK;
}

extern "C" void sell_destroy(gb_sell *A) {
    if (!A) return;
    Mem &m = A->mem;
    m.release(A->perm); m.release(A->iperm); m.release(A->row_len);
    m.release(A->dinv); m.release(A->dinv32);
    m.release(A->chunk_w); m.release(A->chunk_ptr); m.release(A->warp_chunk); m.release(A->warp_chunk5);
    m.release(A->col); m.release(A->col16); m.release(A->val); m.release(A->val32); m.release(A->val16);
    m.release(A->bj_w); m.release(A->bj_w32); m.release(A->bj_loc);
    delete A;
}
