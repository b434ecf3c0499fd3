// bjacobi.cuh -- block-Jacobi preconditioner applied inside the PCG vector
// kernels.
//
// The paper's Block-Jacobi (Sec. 3.2; Sec. 4.2 and its accuracy-vs-epsilon
// figure): M = blockdiag(K_11, ..., K_mm) over blocks of BS consecutive
// unknowns in the free-dof order, applied as z = M^-1 r with the blocks'
// inverses.  The PCG vectors live in
// SELL order, a permutation inside windows of sigma rows; with BS and sigma
// dividing 256 every block's rows lie in one 256-row window, in both orders.
// So one CTA takes a whole window: it updates the window's x and r, keeps r in
// shared memory, applies the window's 256/BS packed inverses there and writes
// z back in SELL order -- the preconditioner costs its packed inverses
// (BS(BS+1)/2 values per block) and one byte per row, and no extra pass over r.
#pragma once
#include <cstdint>

#include "pcg.cuh"

namespace gb {

constexpr int BJ_WIN = 256;  // rows per window = threads per CTA of the window kernels

template <class TW> __device__ __forceinline__ const TW *bj_w(const BjView &B);
template <> __device__ __forceinline__ const double *bj_w<double>(const BjView &B) { return B.w; }
template <> __device__ __forceinline__ const float *bj_w<float>(const BjView &B) { return B.w32; }

// offset of (a, c), a <= c, in a row-major packed upper triangle of order BS
template <int BS>
__device__ __forceinline__ int bj_off(int a, int c) {
    return a * BS - (a * (a - 1)) / 2 + (c - a);
}

// One window: rs holds r of the window's rows (SELL order, 0 past n), ls the
// local SELL position of each row of the window in free-dof order, ws the
// window's packed inverses.  Writes z (SELL order) to zs.  Thread t computes
// row t of the free-dof order: z_t = sum_c W_b[a][c] r_(b BS + c), b = t / BS.
template <class TX, class TW, int BS>
__device__ __forceinline__ void bj_window(const TX *rs, const uint8_t *ls, const TW *ws, TX *zs,
                                          bool row_valid) {
    constexpr int T = BS * (BS + 1) / 2;
    const int t = threadIdx.x;
    if (!row_valid) return;
    const int b = t / BS, a = t - (t / BS) * BS;
    const TW *wb = ws + b * T;
    const uint8_t *lb = ls + b * BS;
    TX acc = TX(0);
#pragma unroll
    for (int c = 0; c < BS; ++c) {
        const int off = c >= a ? bj_off<BS>(a, c) : bj_off<BS>(c, a);
        acc += (TX)wb[off] * rs[lb[c]];
    }
    zs[ls[t]] = acc;
}

// Stages the window's packed inverses and row positions into shared memory.
template <class TW, int BS>
__device__ __forceinline__ void bj_stage(const BjView &B, int64_t w, int64_t n, TW *ws, uint8_t *ls) {
    constexpr int T = BS * (BS + 1) / 2;
    constexpr int NBW = BJ_WIN / BS;
    const TW *W = bj_w<TW>(B);
    const int64_t b0 = w * NBW;
    const int nb = (int)(B.nblk - b0 < NBW ? B.nblk - b0 : NBW);
    const TW *src = W + b0 * T;
    for (int e = threadIdx.x; e < nb * T; e += BJ_WIN) ws[e] = __ldg(src + e);
    const int64_t o = w * BJ_WIN + threadIdx.x;
    ls[threadIdx.x] = o < n ? __ldg(B.loc + o) : (uint8_t)0;
}

// Registers holding one window's inputs (prefetched while the previous window
// is processed): x, r, p, q of the thread's row, its share of the window's
// packed inverses, and the row position of its row.
template <class TX, class TW, int BS>
struct BjPrefetch {
    static constexpr int T = BS * (BS + 1) / 2;
    static constexpr int KW = ((BJ_WIN / BS) * T + BJ_WIN - 1) / BJ_WIN;  // inverse values per thread
    TX x, r, p, q;
    TW w[KW];
    uint8_t l;
    __device__ __forceinline__ void load(const BjView &B, int64_t win, int64_t n, const TX *xg, const TX *rg,
                                         const TX *pg, const TX *qg) {
        const int64_t i = win * BJ_WIN + threadIdx.x;
        if (i < n) {
            x = xg[i]; r = rg[i]; p = pg[i]; q = qg[i];
            l = __ldg(B.loc + i);
        } else {
            x = r = p = q = TX(0);
            l = 0;
        }
        constexpr int NBW = BJ_WIN / BS;
        const int64_t b0 = win * NBW;
        const int nb = (int)(B.nblk - b0 < NBW ? B.nblk - b0 : NBW);
        const TW *src = bj_w<TW>(B) + b0 * T;
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const int e = threadIdx.x + k * BJ_WIN;
            w[k] = e < nb * T ? __ldg(src + e) : TW(0);
        }
    }
};

// x += alpha p, r -= alpha q, z = M^-1 r (stored), r.z and r.r (see want_rr):
// k_update with the block-Jacobi apply, one 256-row window per CTA step.  The
// next window's inputs are loaded into registers before the current window's
// stores and shared-memory work, so their latency overlaps it; two barriers
// per window (the apply reads rs/ws/ls between them, zs is read after the
// second, and the next window's writes come after every thread has left it).
// (at most 51 registers for blocks of up to 8 rows: 5 CTAs per SM)
template <class TX, class TW, int BS>
__global__ void __launch_bounds__(BJ_WIN, BS <= 8 ? 5 : 1) k_update_bj(int64_t n, TX *__restrict__ x, TX *__restrict__ r,
                                                      const TX *__restrict__ p, const TX *__restrict__ q,
                                                      BjView B, TX *__restrict__ z, double *partials,
                                                      PcgScal *S) {
    if (S->done) return;
    using PF = BjPrefetch<TX, TW, BS>;
    __shared__ TX rs[BJ_WIN], zs[BJ_WIN];
    __shared__ TW ws[PF::KW * BJ_WIN];
    __shared__ uint8_t ls[BJ_WIN];
    __shared__ double sm[BJ_WIN / 32];
    const TX alpha = (TX)S->alpha;
    const bool with_rr = want_rr(S);
    TX rz = TX(0), rr = TX(0);
    const int64_t nwin = (n + BJ_WIN - 1) / BJ_WIN;
    PF cur;
    int64_t w = blockIdx.x;
    if (w < nwin) cur.load(B, w, n, x, r, p, q);
    for (; w < nwin; w += gridDim.x) {
        const int64_t i = w * BJ_WIN + threadIdx.x;
        const TX xi = cur.x + alpha * cur.p;
        const TX ri = cur.r - alpha * cur.q;
        rs[threadIdx.x] = ri;
        ls[threadIdx.x] = cur.l;
#pragma unroll
        for (int k = 0; k < PF::KW; ++k) ws[threadIdx.x + k * BJ_WIN] = cur.w[k];
        if (w + gridDim.x < nwin) cur.load(B, w + gridDim.x, n, x, r, p, q);
        if (i < n) {
            x[i] = xi;
            r[i] = ri;
        }
        __syncthreads();
        bj_window<TX, TW, BS>(rs, ls, ws, zs, i < n);
        __syncthreads();
        if (i < n) {
            const TX zi = zs[threadIdx.x];
            z[i] = zi;
            rz += ri * zi;
            if (with_rr) rr += ri * ri;
        }
    }
    const double a = block_sum<BJ_WIN>((double)rz, sm);
    const double b = with_rr ? block_sum<BJ_WIN>((double)rr, sm) : 0.0;
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
    if (arrive_last(&S->ticket)) {
        const double rz_t = sum_partials(partials, gridDim.x, 2, 0, sm);
        const double rr_t = with_rr ? sum_partials(partials, gridDim.x, 2, 1, sm) : 0.0;
        if (threadIdx.x == 0) {
            S->ticket = 0;
            S->it += 1;
            if (with_rr) S->rr = rr_t;
            if (!isfinite(rz_t) || (with_rr && !isfinite(rr_t))) stop(S, ST_BREAK);
            else if (with_rr && rr_t <= S->thresh) stop(S, ST_CONV);
            else if (S->it >= S->maxit) stop(S, ST_MAXIT);
            else {
                S->check_p = (!with_rr && rz_t <= S->dmax * S->thresh) ? 1 : 0;
                S->beta = rz_t / S->rho;
                S->rho = rz_t;
            }
        }
    }
}

// p = M^-1 r, rho = r.p: (re)starts the recurrence (k_start with block-Jacobi).
template <class TX, class TW, int BS>
__global__ void __launch_bounds__(BJ_WIN) k_start_bj(int64_t n, const TX *__restrict__ r, BjView B,
                                                     TX *__restrict__ p, double *partials, PcgScal *S) {
    constexpr int T = BS * (BS + 1) / 2;
    __shared__ TX rs[BJ_WIN], zs[BJ_WIN];
    __shared__ TW ws[(BJ_WIN / BS) * T];
    __shared__ uint8_t ls[BJ_WIN];
    __shared__ double sm[BJ_WIN / 32];
    double rz = 0.0;
    const int64_t nwin = (n + BJ_WIN - 1) / BJ_WIN;
    for (int64_t w = blockIdx.x; w < nwin; w += gridDim.x) {
        const int64_t i = w * BJ_WIN + threadIdx.x;
        const TX ri = i < n ? r[i] : TX(0);
        rs[threadIdx.x] = ri;
        bj_stage<TW, BS>(B, w, n, ws, ls);
        __syncthreads();
        bj_window<TX, TW, BS>(rs, ls, ws, zs, i < n);
        __syncthreads();
        if (i < n) {
            const TX zi = zs[threadIdx.x];
            p[i] = zi;
            rz += (double)(ri * zi);
        }
        __syncthreads();
    }
    const double a = block_sum<BJ_WIN>(rz, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
    if (arrive_last(&S->ticket)) {
        const double t = sum_partials(partials, gridDim.x, 1, 0, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            S->rho = t;
            S->done = 0;
            S->status = ST_RUN;
            S->check_p = 0;
            if (!(t > 0.0)) { S->done = 1; S->status = t == 0.0 ? ST_CONV : ST_BREAK; }
        }
    }
}

// y = M^-1 x for one vector in SELL order (sell_block_jacobi_apply).
template <class TW, int BS>
__global__ void __launch_bounds__(BJ_WIN) k_apply_bj(int64_t n, const double *__restrict__ xin, BjView B,
                                                     double *__restrict__ y) {
    constexpr int T = BS * (BS + 1) / 2;
    __shared__ double rs[BJ_WIN], zs[BJ_WIN];
    __shared__ TW ws[(BJ_WIN / BS) * T];
    __shared__ uint8_t ls[BJ_WIN];
    const int64_t nwin = (n + BJ_WIN - 1) / BJ_WIN;
    for (int64_t w = blockIdx.x; w < nwin; w += gridDim.x) {
        const int64_t i = w * BJ_WIN + threadIdx.x;
        rs[threadIdx.x] = i < n ? xin[i] : 0.0;
        bj_stage<TW, BS>(B, w, n, ws, ls);
        __syncthreads();
        bj_window<double, TW, BS>(rs, ls, ws, zs, i < n);
        __syncthreads();
        if (i < n) y[i] = zs[threadIdx.x];
        __syncthreads();
    }
}

// Grid of a window kernel: one wave of resident CTAs (the kernel's occupancy,
// queried once per instantiation), at most one CTA per window.
template <class Kern>
inline int bj_grid_of(Kern kernel, int &occ_cache, int64_t n) {
    if (occ_cache == 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, BJ_WIN, 0) != cudaSuccess || occ < 1) occ = 1;
        occ_cache = occ;
    }
    const int64_t nwin = (n + BJ_WIN - 1) / BJ_WIN;
    const int64_t g = (int64_t)num_sms() * occ_cache;
    return (int)(nwin < g ? (nwin > 0 ? nwin : 1) : g);
}
// the largest grid any window kernel takes (partial-sum slots)
inline int bj_grid(int64_t n) {
    const int64_t nwin = (n + BJ_WIN - 1) / BJ_WIN;
    const int64_t g = (int64_t)num_sms() * 8;
    return (int)(nwin < g ? (nwin > 0 ? nwin : 1) : g);
}

template <class TX, class TW, int BS> int bj_update_grid(int64_t n) {
    static int occ = 0;
    return bj_grid_of(k_update_bj<TX, TW, BS>, occ, n);
}
template <class TX, class TW, int BS> int bj_start_grid(int64_t n) {
    static int occ = 0;
    return bj_grid_of(k_start_bj<TX, TW, BS>, occ, n);
}

#define GB_BJ_DISPATCH(BSV, CALL) \
    switch (BSV) {                \
    case 1: CALL(1); break;       \
    case 2: CALL(2); break;       \
    case 4: CALL(4); break;       \
    case 8: CALL(8); break;       \
    case 16: CALL(16); break;     \
    default: CALL(32); break;     \
    }

template <class TX, class TW>
inline void launch_update_bj(const BjView &B, int64_t n, TX *x, TX *r, const TX *p, const TX *q, TX *z,
                             double *partials, PcgScal *S, cudaStream_t st) {
#define GB_BJ_UPD(K) \
    ::gb::count_launches(1);                                                                               \
    k_update_bj<TX, TW, K><<<bj_update_grid<TX, TW, K>(n), BJ_WIN, 0, st>>>(n, x, r, p, q, B, z, partials, S)
    GB_BJ_DISPATCH(B.bs, GB_BJ_UPD)
#undef GB_BJ_UPD
}

template <class TX, class TW>
inline void launch_start_bj(const BjView &B, int64_t n, const TX *r, TX *p, double *partials, PcgScal *S,
                            cudaStream_t st) {
#define GB_BJ_START(K) \
    ::gb::count_launches(1); k_start_bj<TX, TW, K><<<bj_start_grid<TX, TW, K>(n), BJ_WIN, 0, st>>>(n, r, B, p, partials, S)
    GB_BJ_DISPATCH(B.bs, GB_BJ_START)
#undef GB_BJ_START
}

}  // namespace gb
