// bjacobi.cu -- setup of the block-Jacobi preconditioner of a SELL matrix
// (the paper's Block-Jacobi, Sec. 3.2 and Sec. 4.2) and its C entry points.
// The apply runs inside the PCG kernels (bjacobi.cuh).
#include <cstring>

#include "bjacobi.cuh"

namespace gb {

constexpr int BJ_SETUP_WARPS = 4;

// One warp per block j: rows o = j bs + a, a < m = min(bs, n - j bs), in the
// free-dof order.  The dense diagonal block is gathered from the SELL rows
// (row iperm[o]; a stored column c is the free dof perm[c]), inverted in place
// by Gauss-Jordan elimination without pivoting -- the pivots of an SPD matrix
// are ratios of leading principal minors, all positive -- and the symmetric
// part of the inverse is stored packed (upper triangle, row-major) in fp64 and
// fp32, with each row's SELL position inside its 256-row window.  Rows a >= m
// of a short last block are an identity during the elimination and zero in
// the stored inverse.  lam_bits: max over rows of the absolute row sum (an
// upper bound of the largest eigenvalue of M^-1), as ordered double bits.
// bad: 1 a pivot was not positive (the block is not SPD), 2 a row's SELL
// position left its window (sigma does not divide the window).
__global__ void __launch_bounds__(32 * BJ_SETUP_WARPS)
    k_bj_setup(SellView A, const int32_t *__restrict__ perm, const int32_t *__restrict__ iperm, int bs,
               int64_t nblk, double *__restrict__ W, float *__restrict__ W32, uint8_t *__restrict__ loc,
               unsigned long long *lam_bits, int *bad) {
    extern __shared__ double bj_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * BJ_SETUP_WARPS + warp;
    if (j >= nblk) return;  // whole warps leave together
    const int ld = bs + 1;
    double *M = bj_smem + (size_t)warp * bs * ld;
    const int64_t s0 = j * bs;
    const int m = (int)(A.n - s0 < bs ? A.n - s0 : bs);
    for (int e = lane; e < bs * ld; e += 32) M[e] = 0.0;
    __syncwarp();
    if (lane < bs) {
        const int a = lane;
        const int64_t o = s0 + a;
        if (a < m) {
            const int32_t pi = __ldg(iperm + o);
            const int64_t c = pi / A.C;
            const int64_t base = A.chunk_ptr[c] + (pi - c * A.C);
            const int L = A.row_len[pi];
            for (int t = 0; t < L; ++t) {
                const int64_t k = base + (int64_t)t * A.C;
                const int64_t oj = __ldg(perm + A.col[k]);
                if (oj >= s0 && oj < s0 + m) M[a * ld + (oj - s0)] += A.val[k];
            }
            const int64_t w0 = (o / BJ_WIN) * BJ_WIN;
            if (pi < w0 || pi >= w0 + BJ_WIN) atomicExch(bad, 2);
            loc[o] = (uint8_t)((pi - w0) & (BJ_WIN - 1));
        } else {
            M[a * ld + a] = 1.0;
            loc[o] = 0;
        }
    }
    __syncwarp();
    // Gauss-Jordan: with p = M_kk, row k becomes M_kc / p (c != k) and 1/p at
    // (k,k); every other row i loses M_ik times the new row k, and its column-k
    // entry becomes -M_ik / p.  Lane c owns column c; column k (read by all
    // lanes) is rewritten by lane k only after the others are done.
    for (int k = 0; k < bs; ++k) {
        double piv = M[k * ld + k];
        if (!(piv > 0.0) || !isfinite(piv)) {
            if (lane == 0) atomicExch(bad, 1);
            piv = 1.0;
        }
        __syncwarp();
        if (lane < bs && lane != k) {
            const double rk = M[k * ld + lane] / piv;
            for (int i = 0; i < bs; ++i)
                if (i != k) M[i * ld + lane] -= M[i * ld + k] * rk;
            M[k * ld + lane] = rk;
        }
        __syncwarp();
        if (lane == k) {
            for (int i = 0; i < bs; ++i)
                if (i != k) M[i * ld + k] = -M[i * ld + k] / piv;
            M[k * ld + k] = 1.0 / piv;
        }
        __syncwarp();
    }
    const int T = bs * (bs + 1) / 2;
    double rowsum = 0.0;
    if (lane < bs) {
        const int c = lane;
        for (int a = 0; a <= c; ++a) {
            const double v = (a < m && c < m) ? 0.5 * (M[a * ld + c] + M[c * ld + a]) : 0.0;
            const int off = a * bs - (a * (a - 1)) / 2 + (c - a);
            W[j * T + off] = v;
            W32[j * T + off] = (float)v;
        }
        if (lane < m)
            for (int cc = 0; cc < m; ++cc) rowsum += fabs(0.5 * (M[lane * ld + cc] + M[cc * ld + lane]));
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) rowsum = fmax(rowsum, __shfl_xor_sync(0xffffffffu, rowsum, off));
    if (lane == 0) atomicMax(lam_bits, (unsigned long long)__double_as_longlong(rowsum));
}

__global__ void k_bj_gather(int64_t n, const int32_t *perm, const double *x, double *xp) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        xp[r] = x[perm[r]];
}
__global__ void k_bj_scatter(int64_t n, const int32_t *perm, const double *yp, double *y) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        y[perm[r]] = yp[r];
}

static void bj_release(gb_sell *A) {
    A->mem.release(A->bj_w);
    A->mem.release(A->bj_w32);
    A->mem.release(A->bj_loc);
    A->bj_w = nullptr;
    A->bj_w32 = nullptr;
    A->bj_loc = nullptr;
    A->bj_bs = 0;
    A->bj_nblk = 0;
    A->bj_lam = 0.0;
}

}  // namespace gb

using namespace gb;

extern "C" int sell_block_jacobi(gb_sell *A, int bs, void *stream) {
    gb::Range range("gbpcg:sell_block_jacobi");
    GB_REQUIRE(A, "sell_block_jacobi: NULL matrix");
    GB_REQUIRE(bs == 0 || bs == 1 || bs == 2 || bs == 4 || bs == 8 || bs == 16 || bs == 32,
               "sell_block_jacobi: block size %d is not 0, 1, 2, 4, 8, 16 or 32", bs);
    GB_REQUIRE(bs == 0 || BJ_WIN % A->sigma == 0,
               "sell_block_jacobi: sigma %d does not divide %d (a block's rows must share a window)",
               A->sigma, BJ_WIN);
    cudaStream_t st = (cudaStream_t)stream;
    GB_CHECK_CUDA(cudaStreamSynchronize(st));  // solves in flight may still read the old blocks
    bj_release(A);
    if (bs == 0) return GB_OK;
    const int64_t n = A->n;
    const int64_t nblk = (n + bs - 1) / bs;
    const int64_t T = (int64_t)bs * (bs + 1) / 2;
    Mem &mem = A->mem;
    double *W = nullptr;
    float *W32 = nullptr;
    uint8_t *loc = nullptr;
    unsigned long long *flags = nullptr;  // [0] lam bits, [1] bad flag (low 32 bits)
    int rc = GB_OK;
    struct { unsigned long long lam, bad; } h{0, 0};
    if ((rc = mem.alloc_n(&W, (size_t)(nblk * T))) != GB_OK) goto fail;
    if ((rc = mem.alloc_n(&W32, (size_t)(nblk * T))) != GB_OK) goto fail;
    if ((rc = mem.alloc_n(&loc, (size_t)(nblk * bs))) != GB_OK) goto fail;
    if ((rc = mem.alloc_n(&flags, 2)) != GB_OK) goto fail;
    {
        cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned long long), st);
        const size_t smem = (size_t)BJ_SETUP_WARPS * bs * (bs + 1) * sizeof(double);
        const int64_t grid = (nblk + BJ_SETUP_WARPS - 1) / BJ_SETUP_WARPS;
        if (e == cudaSuccess) {
            ::gb::count_launches(1);
            k_bj_setup<<<(unsigned)grid, 32 * BJ_SETUP_WARPS, smem, st>>>(A->view(), A->perm, A->iperm, bs, nblk, W,
                                                                          W32, loc, flags,
                                                                          reinterpret_cast<int *>(flags + 1));
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flags, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("sell_block_jacobi: %s", cudaGetErrorString(e));
            rc = GB_ECUDA;
            goto fail;
        }
    }
    if (h.bad & 0xffffffffu) {
        const int bad = (int)(h.bad & 0xffffffffu);
        set_error(bad == 1 ? "sell_block_jacobi: a diagonal block is not positive definite"
                           : "sell_block_jacobi: a block's rows left their 256-row window");
        rc = bad == 1 ? GB_BREAKDOWN : GB_EINVAL;
        goto fail;
    }
    mem.release(flags);
    A->bj_w = W;
    A->bj_w32 = W32;
    A->bj_loc = loc;
    A->bj_bs = bs;
    A->bj_nblk = nblk;
    std::memcpy(&A->bj_lam, &h.lam, sizeof(double));
    return GB_OK;
fail:
    mem.release(W);
    mem.release(W32);
    mem.release(loc);
    mem.release(flags);
    return rc;
}

extern "C" int sell_block_jacobi_info(const gb_sell *A, gb_bjacobi_info *out) {
    GB_REQUIRE(A && out, "sell_block_jacobi_info: NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->bs = A->bj_bs;
    out->nblk = A->bj_nblk;
    out->d_w = A->bj_w;
    out->d_w32 = A->bj_w32;
    out->d_loc = A->bj_loc;
    out->lam_bound = A->bj_lam;
    return GB_OK;
}

extern "C" int sell_block_jacobi_apply(const gb_sell *A, const double *d_x, double *d_y, void *stream) {
    GB_REQUIRE(A && d_x && d_y, "sell_block_jacobi_apply: NULL argument");
    GB_REQUIRE(A->bj_bs > 0, "sell_block_jacobi_apply: no block-Jacobi data (sell_block_jacobi)");
    cudaStream_t st = (cudaStream_t)stream;
    Mem mem(nullptr, st);
    const int64_t n = A->n;
    double *xp = nullptr, *yp = nullptr;
    GB_TRY(mem.alloc_n(&xp, n));
    int rc = mem.alloc_n(&yp, n);
    if (rc != GB_OK) { mem.release(xp); return rc; }
    const int g = stride_grid(n, 256, 8);
    ::gb::count_launches(1); k_bj_gather<<<g, 256, 0, st>>>(n, A->perm, d_x, xp);
    BjView B = A->bj_view();
    const int gw = bj_grid(n);
#define GB_BJ_APPLY(K) ::gb::count_launches(1); k_apply_bj<double, K><<<gw, BJ_WIN, 0, st>>>(n, xp, B, yp)
    GB_BJ_DISPATCH(B.bs, GB_BJ_APPLY)
#undef GB_BJ_APPLY
    ::gb::count_launches(1); k_bj_scatter<<<g, 256, 0, st>>>(n, A->perm, yp, d_y);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    mem.release(xp);
    mem.release(yp);
    if (e != cudaSuccess) {
        set_error("sell_block_jacobi_apply: %s", cudaGetErrorString(e));
        return GB_ECUDA;
    }
    return GB_OK;
}
