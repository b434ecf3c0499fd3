// pcg.cu -- Jacobi-preconditioned CG on a SELL-C-sigma matrix, single RHS:
// plain fp64, and fp32/bf16-inner iterative refinement with fp64 outer
// residual, test and update.
//
// One iteration = three kernels (Hestenes-Stiefel order, as in the oracle):
//   k_spmv_pq  q = A p and the partial sums of p.q; the last block to finish
//              reduces the partials in a fixed order and sets alpha = rho/p.q
//   k_update   x += alpha p, r -= alpha q, z = D^-1 r (stored in fp64 solves),
//              partial sums of r.z and r.r; the last block sets beta, rho,
//              tests ||r||^2 <= tol^2 ||b||^2 (Eq. 2) and the iteration cap
//   k_pupdate  p = z + beta p (and the Eq. 2 test when the update deferred it)
// The scalars live on the device, so the host never waits inside the loop:
// the loop is a CUDA-graph while-node whose condition the finishing block
// clears, or (use_graph=0) direct launches polled every few iterations.  Every
// kernel returns at once when the recurrence is already done, so iterations
// enqueued past convergence cost a launch each and nothing else.
#include <chrono>
#include <cmath>
#include <mutex>
#include <vector>

#include "bicgstab.cuh"
#include "bjacobi.cuh"
#include "pcg.cuh"
#include "spmv_tma.cuh"

namespace gb {

// q = A p with TMA-staged slices (spmv_tma.cuh), one warp per balanced chunk
// range, then the same p.q reduction and alpha as k_spmv_pq.
template <class TV, class TX, class TI>
__global__ void __launch_bounds__(NT) k_spmv_tma(SellView A, const int32_t *__restrict__ wchunk,
                                                 const TV *__restrict__ val,
                                                 const TX *__restrict__ p, TX *__restrict__ q,
                                                 double *partials, PcgScal *S) {
    if (S->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && S->use_cond) cudaGraphSetConditional(S->cond, 0);
        return;
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double sm[NT / 32];
    constexpr int NB = TmaDepth<TV>::NB;
    TmaRing<TV, NB, TI> *bufs = reinterpret_cast<TmaRing<TV, NB, TI> *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + TMA_WARPS * sizeof(TmaRing<TV, NB, TI>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int b = 0; b < NB; ++b) mbar_init(&bars[NB * warp + b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncwarp();
    const int gw = blockIdx.x * TMA_WARPS + warp;
    const int c0 = __ldg(wchunk + gw), c1 = __ldg(wchunk + gw + 1);
    bool timed_out = false;
    const TX dot = spmv_warp_stream<TV, TX, NB, TI>(A, val, p, q, c0, c1, bufs[warp], &bars[NB * warp], &timed_out);
    if (timed_out && lane == 0) atomicExch(&S->err, 1);
    const double t = block_sum<NT>((double)dot, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
    if (arrive_last(&S->ticket)) {
        const double pq = sum_partials(partials, gridDim.x, 1, 0, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            S->pq = pq;
            if (S->err) stop(S, ST_TIMEOUT);
            else if (!(pq > 0.0) || !isfinite(pq)) stop(S, ST_BREAK);
            else S->alpha = S->rho / pq;
        }
    }
}

template <class TV, class TX, class TI>
static void launch_spmv_tma_t(const SellViewH &A, const TV *val, const TX *p, TX *q, double *partials,
                              PcgScal *S, cudaStream_t st) {
    static bool attr_set = false;  // per instantiation
    const int smem = (int)tma_smem_bytes<TV, TI>();
    if (!attr_set) {
        cudaFuncSetAttribute(k_spmv_tma<TV, TX, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
    }
    // the warp partition of k_spmv_tma2 for the same value type, so that both
    // index widths sum p.q in the same order
    const bool narrow = sizeof(TV) == 4 && A.warp_chunk5;
    const int32_t *wchunk = narrow ? A.warp_chunk5 : A.warp_chunk;
    const int grid = (narrow ? A.nwarps5 : A.nwarps) / TMA_WARPS;
    ::gb::count_launches(1); k_spmv_tma<TV, TX, TI><<<grid, NT, smem, st>>>(A, wchunk, val, p, q, partials, S);
}

// q = A p with the second streaming loop (32-bit indices, spmv_tma.cuh), one
// warp per chunk range of wchunk (balanced), then the p.q reduction and alpha.
// The fp32 kernel runs 5 blocks per SM on its own partition (2-deep ring); the
// fp64 (2-deep) and bf16 (3-deep) kernels 4 blocks per SM.
template <class TV, class TX>
__global__ void __launch_bounds__(NT) k_spmv_tma2(SellView A, const int32_t *__restrict__ wchunk,
                                                  const TV *__restrict__ val, const TX *__restrict__ p,
                                                  TX *__restrict__ q, double *partials, PcgScal *S) {
    if (S->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && S->use_cond) cudaGraphSetConditional(S->cond, 0);
        return;
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double sm[NT / 32];
    constexpr int NB = Tma2Cfg<TV>::NB;
    Tma2Ring<TV> *bufs = reinterpret_cast<Tma2Ring<TV> *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + TMA_WARPS * sizeof(Tma2Ring<TV>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int b = 0; b < NB; ++b) mbar_init(&bars[NB * warp + b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncwarp();
    const int gw = blockIdx.x * TMA_WARPS + warp;
    const int c0 = __ldg(wchunk + gw), c1 = __ldg(wchunk + gw + 1);
    bool timed_out = false;
    const TX dot = spmv_warp_stream2<TV, TX>(A, val, p, q, c0, c1, bufs[warp], &bars[NB * warp], &timed_out);
    if (timed_out && lane == 0) atomicExch(&S->err, 1);
    const double t = block_sum<NT>((double)dot, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
    if (arrive_last(&S->ticket)) {
        const double pq = sum_partials(partials, gridDim.x, 1, 0, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            S->pq = pq;
            if (S->err) stop(S, ST_TIMEOUT);
            else if (!(pq > 0.0) || !isfinite(pq)) stop(S, ST_BREAK);
            else S->alpha = S->rho / pq;
        }
    }
}

template <class TV, class TX>
static void launch_spmv_tma2(const SellViewH &A, const TV *val, const TX *p, TX *q, double *partials,
                             PcgScal *S, cudaStream_t st) {
    static bool attr_set = false;  // per instantiation
    const int smem = (int)tma2_smem_bytes<TV>();
    if (!attr_set) {
        cudaFuncSetAttribute(k_spmv_tma2<TV, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
    }
    // fp32 (32 KB ring per block): 5 blocks per SM; fp64 (48 KB), bf16 (36 KB): 4
    const bool narrow = sizeof(TV) == 4 && A.warp_chunk5;
    const int32_t *wchunk = narrow ? A.warp_chunk5 : A.warp_chunk;
    const int grid = (narrow ? A.nwarps5 : A.nwarps) / TMA_WARPS;
    ::gb::count_launches(1); k_spmv_tma2<TV, TX><<<grid, NT, smem, st>>>(A, wchunk, val, p, q, partials, S);
}

// 16-bit column deltas when the matrix has them (first streaming loop), 32-bit
// indices otherwise (second streaming loop)
template <class TV, class TX>
static void launch_spmv_tma(const SellViewH &A, const TV *val, const TX *p, TX *q, double *partials,
                            PcgScal *S, cudaStream_t st) {
#ifndef GB_TMA_NO_COL16
    if (A.col16) launch_spmv_tma_t<TV, TX, int16_t>(A, val, p, q, partials, S, st);
    else
#endif
#ifdef GB_TMA_OLD
        launch_spmv_tma_t<TV, TX, int32_t>(A, val, p, q, partials, S, st);
#else
        launch_spmv_tma2<TV, TX>(A, val, p, q, partials, S, st);
#endif
}

// ------------------------------------------------------------ kernels --
template <class TV, class TX, int C>
__global__ void __launch_bounds__(NT) k_spmv_pq(SellView A, const TV *__restrict__ val,
                                                const TX *__restrict__ p, TX *__restrict__ q,
                                                double *partials, PcgScal *S) {
    if (S->done) {
        // a loop entered with the recurrence already finished must still end
        if (blockIdx.x == 0 && threadIdx.x == 0 && S->use_cond) cudaGraphSetConditional(S->cond, 0);
        return;
    }
    __shared__ double sm[NT / 32];
    constexpr int SL = C / 32;
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)NT + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * NT) >> 5;
    const int64_t nsl = A.nchunks * SL;
    TX dot = TX(0);
    for (int64_t s = gw; s < nsl; s += nw) {
        const int64_t c = s / SL;
        const int sub = (int)(s - c * SL);
        const int64_t r = c * C + sub * 32 + lane;
        if (r >= A.n) continue;
        const int L = A.row_len[r];
        const int64_t base = A.chunk_ptr[c] + sub * 32 + lane;
        const TV *v = val + base;
        const int32_t *ci = A.col + base;
        TX acc = TX(0);
        int j = 0;
        for (; j + 4 <= L; j += 4) {
            const int c0 = ld_col(ci), c1 = ld_col(ci + C), c2 = ld_col(ci + 2 * C), c3 = ld_col(ci + 3 * C);
            const TX v0 = (TX)ld_val(v), v1 = (TX)ld_val(v + C), v2 = (TX)ld_val(v + 2 * C), v3 = (TX)ld_val(v + 3 * C);
            const TX p0 = p[c0], p1 = p[c1], p2 = p[c2], p3 = p[c3];
            acc += v0 * p0;
            acc += v1 * p1;
            acc += v2 * p2;
            acc += v3 * p3;
            v += 4 * C;
            ci += 4 * C;
        }
        for (; j < L; ++j) {
            acc += (TX)ld_val(v) * p[ld_col(ci)];
            v += C;
            ci += C;
        }
        q[r] = acc;
        dot += p[r] * acc;
    }
    const double t = block_sum<NT>((double)dot, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
    if (arrive_last(&S->ticket)) {
        const double pq = sum_partials(partials, gridDim.x, 1, 0, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            S->pq = pq;
            if (!(pq > 0.0) || !isfinite(pq)) stop(S, ST_BREAK);
            else S->alpha = S->rho / pq;
        }
    }
}

// Grid-stride over 16-byte groups, UPD_U groups per thread per step with every
// load issued before the arithmetic (memory-level parallelism for these
// streaming kernels); the n % VW last elements go to block 0.
#ifndef GB_UPD_U
#define GB_UPD_U 2
#endif
constexpr int UPD_U = GB_UPD_U;


// x += alpha p, r -= alpha q, r.D^-1 r (and r.r, see want_rr); z = D^-1 r is
// stored when z is given (the p update then reads it instead of D^-1 and r).
template <class TX, class TD>
__global__ void __launch_bounds__(NT) k_update(int64_t n, TX *__restrict__ x, TX *__restrict__ r,
                                               const TX *__restrict__ p, const TX *__restrict__ q,
                                               const TD *__restrict__ dinv, TX *__restrict__ z,
                                               double *partials, PcgScal *S) {
    if (S->done) return;
    __shared__ double sm[NT / 32];
    constexpr int VW = 16 / sizeof(TX);
    const TX alpha = (TX)S->alpha;
    const bool with_rr = want_rr(S);
    TX rz = TX(0), rr = TX(0);
    const int64_t ng = n / VW;
    const int64_t stride = (int64_t)gridDim.x * NT;
    for (int64_t i0 = blockIdx.x * (int64_t)NT + threadIdx.x; i0 < ng; i0 += stride * UPD_U) {
        TX xv[UPD_U][VW], rv[UPD_U][VW], pv[UPD_U][VW], qv[UPD_U][VW];
        TD dv[UPD_U][VW];
#pragma unroll
        for (int u = 0; u < UPD_U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < ng) {
                ld_pack(x, i, xv[u]);
                ld_pack(r, i, rv[u]);
                ld_pack(p, i, pv[u]);
                ld_pack(q, i, qv[u]);
                ld_pack(dinv, i, dv[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < UPD_U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < ng) {
                TX zv[VW];
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    xv[u][k] += alpha * pv[u][k];
                    rv[u][k] -= alpha * qv[u][k];
                    zv[k] = (TX)dv[u][k] * rv[u][k];
                    rz += rv[u][k] * zv[k];
                    if (with_rr) rr += rv[u][k] * rv[u][k];
                }
                st_pack(x, i, xv[u]);
                st_pack(r, i, rv[u]);
                if (z) st_pack(z, i, zv);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < n - ng * VW) {
        const int64_t i = ng * VW + threadIdx.x;
        const TX xi = x[i] + alpha * p[i];
        const TX ri = r[i] - alpha * q[i];
        const TX zi = (TX)dinv[i] * ri;
        x[i] = xi;
        r[i] = ri;
        if (z) z[i] = zi;
        rz += ri * zi;
        if (with_rr) rr += ri * ri;
    }
    const double a = block_sum<NT>((double)rz, sm);
    const double b = with_rr ? block_sum<NT>((double)rr, sm) : 0.0;
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
                // r.r skipped but the test could pass now: the p update makes it
                S->check_p = (!with_rr && rz_t <= S->dmax * S->thresh) ? 1 : 0;
                S->beta = rz_t / S->rho;
                S->rho = rz_t;
            }
        }
    }
}

// p = z + beta p with z = D^-1 r (read from z when given); when the x/r
// update left the Eq. (2) test to this kernel (S->check_p), also r.r and the
// test: a converged recurrence stops here, in the iteration that converged.
template <class TX, class TD>
__global__ void __launch_bounds__(NT) k_pupdate(int64_t n, TX *__restrict__ p, const TX *__restrict__ r,
                                                const TD *__restrict__ dinv, const TX *__restrict__ z,
                                                double *partials, PcgScal *S) {
    if (S->done) return;
    __shared__ double sm[NT / 32];
    constexpr int VW = 16 / sizeof(TX);
    const TX beta = (TX)S->beta;
    const bool check = S->check_p != 0;
    TX rr = TX(0);
    const int64_t ng = n / VW;
    const int64_t stride = (int64_t)gridDim.x * NT;
    for (int64_t i0 = blockIdx.x * (int64_t)NT + threadIdx.x; i0 < ng; i0 += stride * UPD_U) {
        TX pv[UPD_U][VW], rv[UPD_U][VW], zv[UPD_U][VW];
        TD dv[UPD_U][VW];
#pragma unroll
        for (int u = 0; u < UPD_U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < ng) {
                ld_pack(p, i, pv[u]);
                if (z) {
                    ld_pack(z, i, zv[u]);
                    if (check) ld_pack(r, i, rv[u]);
                } else {
                    ld_pack(r, i, rv[u]);
                    ld_pack(dinv, i, dv[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UPD_U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < ng) {
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    const TX zk = z ? zv[u][k] : (TX)dv[u][k] * rv[u][k];
                    pv[u][k] = zk + beta * pv[u][k];
                    if (check) rr += rv[u][k] * rv[u][k];
                }
                st_pack(p, i, pv[u]);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < n - ng * VW) {
        const int64_t i = ng * VW + threadIdx.x;
        const TX zi = z ? z[i] : (TX)dinv[i] * r[i];
        p[i] = zi + beta * p[i];
        if (check) rr += r[i] * r[i];
    }
    if (!check) return;
    const double b = block_sum<NT>((double)rr, sm);
    if (threadIdx.x == 0) partials[2 * blockIdx.x + 1] = b;
    if (arrive_last(&S->ticket)) {
        const double rr_t = sum_partials(partials, gridDim.x, 2, 1, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            S->rr = rr_t;
            S->check_p = 0;
            if (!isfinite(rr_t)) stop(S, ST_BREAK);
            else if (rr_t <= S->thresh) stop(S, ST_CONV);
        }
    }
}

// r = b - A x (fp64, x optional = 0) with ||r||^2 and ||b||^2.  The last block
// stores rr (and, when init, bb and the threshold tol^2 bb).
template <int C>
__global__ void __launch_bounds__(NT) k_residual(SellView A, const double *__restrict__ x,
                                                 const double *__restrict__ b, double *__restrict__ r,
                                                 double *partials, PcgScal *S, int init, double tol) {
    __shared__ double sm[NT / 32];
    constexpr int SL = C / 32;
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)NT + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * NT) >> 5;
    double rr = 0.0, bb = 0.0;
    for (int64_t s = gw; s < A.nchunks * SL; s += nw) {
        const int64_t c = s / SL;
        const int sub = (int)(s - c * SL);
        const int64_t row = c * C + sub * 32 + lane;
        if (row >= A.n) continue;
        double acc = 0.0;
        if (x) {
            const int L = A.row_len[row];
            const int64_t base = A.chunk_ptr[c] + sub * 32 + lane;
            for (int j = 0; j < L; ++j) acc += ld_val(A.val + base + (int64_t)j * C) * x[ld_col(A.col + base + (int64_t)j * C)];
        }
        const double bi = b[row];
        const double ri = bi - acc;
        r[row] = ri;
        rr += ri * ri;
        bb += bi * bi;
    }
    const double a = block_sum<NT>(rr, sm);
    const double c2 = block_sum<NT>(bb, sm);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = c2;
    }
    if (arrive_last(&S->ticket)) {
        const double rr_t = sum_partials(partials, gridDim.x, 2, 0, sm);
        const double bb_t = sum_partials(partials, gridDim.x, 2, 1, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            S->rr = rr_t;
            if (init) {
                S->bb = bb_t;
                S->thresh = tol * tol * bb_t;
            }
        }
    }
}

// p = D^-1 r, rho = r.z; (re)starts the recurrence.
template <class TX, class TD>
__global__ void __launch_bounds__(NT) k_start(int64_t n, const TX *__restrict__ r, const TD *__restrict__ dinv,
                                              TX *__restrict__ p, double *partials, PcgScal *S) {
    __shared__ double sm[NT / 32];
    double rz = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const TX zi = (TX)dinv[i] * r[i];
        p[i] = zi;
        rz += (double)(r[i] * zi);
    }
    const double a = block_sum<NT>(rz, sm);
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

// Residual replacement of a reliable update: r32 = (float) r64 from the fp64
// true residual, and in fp64 sums rho' = r.D^-1 r, ||r||^2 and r.p.  The last
// block prepares the step the stopped loop skipped, p = z + beta p, for the
// replaced residual: beta = rho'/rho, with p first made orthogonal to the new
// r along z (p -= (r.p / r.z) z), so p = (1 - beta c) z + beta p, c = r.p/rho'.
// Re-arms the recurrence (done = 0).  first = 1: no previous p (k_start follows).
__global__ void __launch_bounds__(NT) k_replace(int64_t n, const double *__restrict__ r64, const float *__restrict__ dinv,
                                                float *__restrict__ r32, float *__restrict__ d32,
                                                const float *__restrict__ p32, int first, double *partials, PcgScal *S) {
    __shared__ double sm[NT / 32];
    double rz = 0.0, rr = 0.0, rp = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const float ri = (float)r64[i];
        r32[i] = ri;
        d32[i] = 0.0f;
        rz += (double)(ri * (dinv[i] * ri));
        rr += (double)ri * (double)ri;
        if (!first) rp += (double)ri * (double)p32[i];
    }
    const double a = block_sum<NT>(rz, sm);
    const double b = block_sum<NT>(rr, sm);
    const double c = block_sum<NT>(rp, sm);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = a;
        partials[3 * blockIdx.x + 1] = b;
        partials[3 * blockIdx.x + 2] = c;
    }
    if (arrive_last(&S->ticket)) {
        const double rz_t = sum_partials(partials, gridDim.x, 3, 0, sm);
        const double rr_t = sum_partials(partials, gridDim.x, 3, 1, sm);
        const double rp_t = sum_partials(partials, gridDim.x, 3, 2, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            if (!first && rz_t > 0.0 && S->rho > 0.0) {
                const double beta = rz_t / S->rho;
                S->beta = beta;
                S->pz = 1.0 - beta * (rp_t / rz_t);
            }
            S->rho = rz_t;
            S->rr = rr_t;
            S->done = 0;
            S->status = ST_RUN;
            if (!(rz_t > 0.0)) { S->done = 1; S->status = rz_t == 0.0 ? ST_CONV : ST_BREAK; }
        }
    }
}

// p = pz D^-1 r + beta p (the restored direction of a reliable update)
__global__ void __launch_bounds__(NT) k_replace_p(int64_t n, const float *__restrict__ r32, const float *__restrict__ dinv,
                                                  float *__restrict__ p32, const PcgScal *S) {
    if (S->done) return;
    const float pz = (float)S->pz, beta = (float)S->beta;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
        p32[i] = pz * (dinv[i] * r32[i]) + beta * p32[i];
}

__global__ void k_gather_d(int64_t n, const int32_t *perm, const double *src, double *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src ? src[perm[i]] : 0.0;
}
__global__ void k_scatter_d(int64_t n, const int32_t *perm, const double *src, double *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[perm[i]] = src[i];
}
// r32 = (float)(s * r64)
__global__ void k_scale_down(int64_t n, const double *r, double s, float *r32, float *d32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        r32[i] = (float)(s * r[i]);
        d32[i] = 0.0f;
    }
}
// x += s * d
__global__ void k_correct(int64_t n, double *x, double s, const float *d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += s * (double)d[i];
}

// ------------------------------------------------------------- driver --
struct Grids {
    int spmv, vec, upd;
};
static Grids pick_grids(int64_t n, int C) {
    const int sms = num_sms();
    Grids g;
    const int64_t warps = ((n + C - 1) / C) * (C / 32);
    g.spmv = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, (warps + 7) / 8));
    g.vec = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, (n + 2 * NT * UPD_U - 1) / (2 * NT * UPD_U)));
    // x/r and p updates: one wave of resident blocks (4 per SM at <= 64 registers)
    g.upd = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, (n + 2 * NT * UPD_U - 1) / (2 * NT * UPD_U)));
    return g;
}

template <class TV, class TX, class TD>
static void enqueue_iteration(const SellViewH &A, const TV *val, const TD *dinv, TX *x, TX *r, TX *p,
                              TX *q, TX *z, double *partials, PcgScal *S, const Grids &g, cudaStream_t st,
                              int variant = 0, const BjView *bj = nullptr) {
    if (variant == 0 && A.C == 32 && A.warp_chunk) launch_spmv_tma<TV, TX>(A, val, p, q, partials, S, st);
    else switch (A.C) {
    case 32: ::gb::count_launches(1); k_spmv_pq<TV, TX, 32><<<g.spmv, NT, 0, st>>>(A, val, p, q, partials, S); break;
    case 64: ::gb::count_launches(1); k_spmv_pq<TV, TX, 64><<<g.spmv, NT, 0, st>>>(A, val, p, q, partials, S); break;
    default: ::gb::count_launches(1); k_spmv_pq<TV, TX, 128><<<g.spmv, NT, 0, st>>>(A, val, p, q, partials, S); break;
    }
    if (bj && bj->bs) {  // block-Jacobi: z = M^-1 r in the x/r update (z always stored)
        launch_update_bj<TX, TX>(*bj, A.n, x, r, p, q, z, partials, S, st);
    } else {
        ::gb::count_launches(1); k_update<TX, TD><<<g.upd, NT, 0, st>>>(A.n, x, r, p, q, dinv, z, partials, S);
    }
    ::gb::count_launches(1); k_pupdate<TX, TD><<<g.upd, NT, 0, st>>>(A.n, p, r, dinv, z, partials, S);
}

static void enqueue_residual(const SellView &A, const double *x, const double *b, double *r,
                             double *partials, PcgScal *S, int init, double tol, const Grids &g,
                             cudaStream_t st) {
    switch (A.C) {
    case 32: ::gb::count_launches(1); k_residual<32><<<g.spmv, NT, 0, st>>>(A, x, b, r, partials, S, init, tol); break;
    case 64: ::gb::count_launches(1); k_residual<64><<<g.spmv, NT, 0, st>>>(A, x, b, r, partials, S, init, tol); break;
    default: ::gb::count_launches(1); k_residual<128><<<g.spmv, NT, 0, st>>>(A, x, b, r, partials, S, init, tol); break;
    }
}

// Runs the CG loop until the device flag says done.  Graph mode: one launch
// of a graph holding a while-node around one iteration; the finishing block
// clears the condition.  Direct mode: `chunk` iterations per host poll.
template <class F>
static int run_loop(cudaStream_t st, PcgScal *dS, bool use_graph, int chunk, F &&enqueue, int64_t *launches,
                    int per_iter = 3) {
    if (use_graph) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaStream_t cap = nullptr;
        cudaGraphConditionalHandle h = 0;
        GB_CHECK_CUDA(cudaGraphCreate(&g, 0));
        int rc = GB_OK;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {};
        cudaGraphNode_t node;
        if (e == cudaSuccess) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            cudaGraph_t body = np.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                set_capturing(true);
                enqueue(cap);
                set_capturing(false);
                cudaGraph_t outg = nullptr;
                e = cudaStreamEndCapture(cap, &outg);
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        long long it0 = 0, it1 = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&it0, &dS->it, sizeof(it0), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            struct { int use; cudaGraphConditionalHandle h; } hs{1, h};
            e = cudaMemcpyAsync(&dS->use_cond, &hs.use, sizeof(int), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&dS->cond, &hs.h, sizeof(h), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
            int zero = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&dS->use_cond, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&it1, &dS->it, sizeof(it1), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            // the body ran once per iteration (plus once when it stopped inside SpMV)
            count_launches(per_iter * (it1 - it0) + per_iter);
        }
        if (e != cudaSuccess) { set_error("pcg loop graph: %s", cudaGetErrorString(e)); rc = GB_ECUDA; }
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (cap) cudaStreamDestroy(cap);
        (void)launches;
        return rc;
    }
    for (;;) {
        for (int i = 0; i < chunk; ++i) enqueue(st);
        if (launches) *launches += per_iter * chunk;
        int done = 0;
        GB_CHECK_CUDA(cudaGetLastError());
        GB_CHECK_CUDA(cudaMemcpyAsync(&done, &dS->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
        if (done) return GB_OK;
    }
}

// partial-sum slots every solver kernel may write (2 per block of the largest grid)
static size_t partial_slots(const gb_sell *A, const Grids &g) {
    int blocks = std::max(std::max(g.spmv, g.vec), bj_grid(A->n));
    if (A->warp_chunk) blocks = std::max(blocks, std::max(A->nwarps, A->nwarps5) / TMA_WARPS);
    return 3 * (size_t)blocks;
}

static PcgOptions defaults(const PcgOptions *o, int64_t n) {
    PcgOptions d{};
    if (o) d = *o;
    if (!(d.tol > 0)) d.tol = 1e-10;
    if (d.max_iter <= 0) d.max_iter = 20 * n + 100;
    if (d.max_outer <= 0) d.max_outer = 30;
    if (!(d.inner_tol > 0)) d.inner_tol = 1e-4;
    if (d.check_every <= 0) d.check_every = (int)std::min<int64_t>(256, std::max<int64_t>(8, (1 << 20) / std::max<int64_t>(n, 1)));
    if (graphs_disabled()) d.use_graph = 0;
    return d;
}

static int read_scal(PcgScal *dS, PcgScal *h, cudaStream_t st) {
    GB_CHECK_CUDA(cudaMemcpyAsync(h, dS, sizeof(PcgScal), cudaMemcpyDeviceToHost, st));
    GB_CHECK_CUDA(cudaStreamSynchronize(st));
    return GB_OK;
}

static int init_scal(PcgScal *dS, long long maxit, cudaStream_t st) {
    PcgScal h{};
    h.maxit = maxit;
    GB_CHECK_CUDA(cudaMemcpyAsync(dS, &h, sizeof(PcgScal), cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaStreamSynchronize(st));
    return GB_OK;
}

static int map_status(int st) {
    switch (st) {
    case ST_CONV: return GB_OK;
    case ST_TIMEOUT: return GB_TIMEOUT;
    case ST_BREAK: return GB_BREAKDOWN;
    case ST_MAXIT: return GB_NOT_CONVERGED;
    default: return GB_NOT_CONVERGED;
    }
}

// Workspace of one single-RHS solve.
struct Work {
    Mem mem;
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *b = nullptr, *partials = nullptr;
    double *z = nullptr;  // fp64 D^-1 r, when the workspace has room for it
    float *r32 = nullptr, *d32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    float *z32 = nullptr;  // fp32 M^-1 r (block-Jacobi inner solves)
    PcgScal *S = nullptr, *S2 = nullptr;
    ~Work() {
        mem.release(x); mem.release(r); mem.release(p); mem.release(q); mem.release(b); mem.release(z);
        mem.release(z32);
        mem.release(partials);
        mem.release(r32); mem.release(d32); mem.release(p32); mem.release(q32);
        mem.release(S); mem.release(S2);
    }
};

}  // namespace gb

using namespace gb;

static int solve_f64(const gb_sell *A, const PcgOptions &o, Work &w, cudaStream_t st, PcgStats *stats) {
    const SellViewH V = A->view();
    const int64_t n = A->n;
    const Grids g = pick_grids(n, A->C);
    int64_t launches = 0;
    // r = b - A x0, ||b||
    enqueue_residual(V, o.x0_zero ? nullptr : w.x, w.b, w.r, w.partials, w.S, 1, o.tol, g, st);
    ++launches;
    PcgScal h{};
    GB_TRY(read_scal(w.S, &h, st));
    stats->bnorm = std::sqrt(h.bb);
    if (h.bb == 0.0) {  // b = 0: x = 0
        GB_CHECK_CUDA(cudaMemsetAsync(w.x, 0, sizeof(double) * n, st));
        stats->relres = 0.0;
        stats->status = GB_OK;
        stats->kernel_launches = launches + 1;
        return GB_OK;
    }
    int64_t restarts = 0;
    int status = ST_RUN;
    double rel = std::sqrt(h.rr / h.bb);
    // bound of lmax(M^-1): the update defers its r.r sums while they cannot meet Eq. (2)
    const bool use_bj = o.precond == GB_PC_BLOCK_JACOBI;
    const BjView bj = A->bj_view();
    GB_CHECK_CUDA(cudaMemcpyAsync(&w.S->dmax, use_bj ? &A->bj_lam : &A->dinv_max, sizeof(double),
                                  cudaMemcpyHostToDevice, st));
    while (rel > o.tol) {
        if (use_bj) {
            launch_start_bj<double, double>(bj, n, w.r, w.p, w.partials, w.S, st);
        } else {
            ::gb::count_launches(1); k_start<double, double><<<g.vec, NT, 0, st>>>(n, w.r, A->dinv, w.p, w.partials, w.S);
        }
        ++launches;
        GB_CHECK_CUDA(cudaGetLastError());
        auto body = [&](cudaStream_t s) {
            enqueue_iteration<double, double, double>(V, A->val, A->dinv, w.x, w.r, w.p, w.q, w.z, w.partials, w.S, g, s,
                                                      o.spmv_variant ? o.spmv_variant : A->variant_hint,
                                                      use_bj ? &bj : nullptr);
        };
        GB_TRY(run_loop(st, w.S, o.use_graph != 0, o.check_every, body, nullptr));
        GB_TRY(read_scal(w.S, &h, st));
        status = h.status;
        // confirm on the true residual (Eq. 2 is stated for b - A x)
        enqueue_residual(V, w.x, w.b, w.r, w.partials, w.S, 0, o.tol, g, st);
        ++launches;
        PcgScal h2{};
        GB_TRY(read_scal(w.S, &h2, st));
        rel = std::sqrt(h2.rr / h2.bb);
        if (status != ST_CONV || rel <= o.tol || h.it >= h.maxit || ++restarts > 50) break;
    }
    if (rel <= o.tol) status = ST_CONV;
    stats->iterations = h.it;
    stats->restarts = restarts;
    stats->relres = rel;
    stats->status = map_status(status);
    stats->kernel_launches = launches + 3 * h.it;
    // block-Jacobi: the packed inverses and row positions replace D^-1
    const double bytes_iter = (double)A->nnz * 12.0 + 7.0 * n * 8.0 +
                              (use_bj ? (double)A->bj_nblk * (A->bj_bs * (A->bj_bs + 1) / 2 * 8.0 + A->bj_bs) - 8.0 * n : 0.0);
    stats->bytes_moved = bytes_iter * (double)h.it;
    return GB_OK;
}

template <class TV>
static int solve_ir(const gb_sell *A, const TV *val_in, const PcgOptions &o, Work &w, cudaStream_t st,
                    PcgStats *stats) {
    const SellViewH V = A->view();
    const int64_t n = A->n;
    const Grids g = pick_grids(n, A->C);
    int64_t launches = 0;
    Mem &mem = w.mem;
    GB_TRY(mem.alloc_n(&w.r32, n));
    GB_TRY(mem.alloc_n(&w.d32, n));
    GB_TRY(mem.alloc_n(&w.p32, n));
    GB_TRY(mem.alloc_n(&w.q32, n));
    GB_TRY(mem.alloc_n(&w.S2, 1));
    const bool use_bj = o.precond == GB_PC_BLOCK_JACOBI;
    const BjView bj = A->bj_view();
    if (use_bj) GB_TRY(mem.alloc_n(&w.z32, n));
    enqueue_residual(V, o.x0_zero ? nullptr : w.x, w.b, w.r, w.partials, w.S, 1, o.tol, g, st);
    ++launches;
    PcgScal h{};
    GB_TRY(read_scal(w.S, &h, st));
    stats->bnorm = std::sqrt(h.bb);
    if (h.bb == 0.0) {
        GB_CHECK_CUDA(cudaMemsetAsync(w.x, 0, sizeof(double) * n, st));
        stats->relres = 0.0;
        stats->status = GB_OK;
        return GB_OK;
    }
    double rel = std::sqrt(h.rr / h.bb);
    int outer = 0;
    int64_t inner_total = 0;
    double prev = rel;
    int stalls = 0;
    int status = ST_RUN;
    const double sval = sizeof(TV);
    double bytes = 0.0;
    while (rel > o.tol && outer < o.max_outer && inner_total < o.max_iter) {
        ++outer;
        const double rn = std::sqrt(h.rr);
        // inner system A d = r / ||r|| in fp32, from d = 0
        ::gb::count_launches(1); k_scale_down<<<g.vec, NT, 0, st>>>(n, w.r, 1.0 / rn, w.r32, w.d32);
        {
            // ||r32||^2 ~ 1: threshold from the inner tolerance
            PcgScal hs{};
            hs.maxit = o.max_iter - inner_total;
            hs.bb = 1.0;
            hs.thresh = o.inner_tol * o.inner_tol;
            GB_CHECK_CUDA(cudaMemcpyAsync(w.S2, &hs, sizeof(PcgScal), cudaMemcpyHostToDevice, st));
        }
        if (use_bj) {
            launch_start_bj<float, float>(bj, n, w.r32, w.p32, w.partials, w.S2, st);
        } else {
            ::gb::count_launches(1); k_start<float, float><<<g.vec, NT, 0, st>>>(n, w.r32, A->dinv32, w.p32, w.partials, w.S2);
        }
        launches += 2;
        auto body = [&](cudaStream_t s) {
            enqueue_iteration<TV, float, float>(V, val_in, A->dinv32, w.d32, w.r32, w.p32, w.q32, w.z32, w.partials, w.S2, g, s,
                                                o.spmv_variant ? o.spmv_variant : A->variant_hint,
                                                use_bj ? &bj : nullptr);
        };
        GB_TRY(run_loop(st, w.S2, o.use_graph != 0, o.check_every, body, nullptr));
        PcgScal hi{};
        GB_TRY(read_scal(w.S2, &hi, st));
        inner_total += hi.it;
        launches += 3 * hi.it;
        bytes += hi.it * ((double)A->nnz * (sval + 4.0) + 7.0 * n * 4.0 +
                          (use_bj ? (double)A->bj_nblk * (A->bj_bs * (A->bj_bs + 1) / 2 * 4.0 + A->bj_bs) - 4.0 * n : 0.0));
        // x += ||r|| d ; r = b - A x in fp64
        ::gb::count_launches(1); k_correct<<<g.vec, NT, 0, st>>>(n, w.x, rn, w.d32);
        enqueue_residual(V, w.x, w.b, w.r, w.partials, w.S, 0, o.tol, g, st);
        launches += 2;
        bytes += (double)A->nnz * 12.0 + 5.0 * n * 8.0;
        GB_TRY(read_scal(w.S, &h, st));
        rel = std::sqrt(h.rr / h.bb);
        if (!(rel < 0.9 * prev)) { if (++stalls >= 2) break; } else stalls = 0;
        prev = std::min(prev, rel);
        if (hi.status == ST_BREAK && hi.it == 0) break;
    }
    status = rel <= o.tol ? ST_CONV : ST_MAXIT;
    stats->iterations = inner_total;
    stats->outer = outer;
    stats->relres = rel;
    stats->status = map_status(status);
    stats->kernel_launches = launches;
    stats->bytes_moved = bytes;
    return GB_OK;
}

// Reliable updates (Sleijpen & van der Vorst's residual replacement, in the
// mixed-precision form used for lattice solvers): one fp32 CG recurrence on
// the correction d runs until its recursive residual has dropped by a factor
// RU_DELTA since the last replacement; then x += d and r = b - A x in fp64,
// the convergence test in fp64, and the fp32 residual is replaced by the true
// one while the search direction p is kept, so the Krylov information is not
// thrown away as in restarted refinement.
template <class TV>
static int solve_ru(const gb_sell *A, const TV *val_in, const PcgOptions &o, Work &w, cudaStream_t st,
                    PcgStats *stats) {
    constexpr double RU_DELTA = 0.1;
    const SellViewH V = A->view();
    const int64_t n = A->n;
    const Grids g = pick_grids(n, A->C);
    Mem &mem = w.mem;
    GB_TRY(mem.alloc_n(&w.r32, n));
    GB_TRY(mem.alloc_n(&w.d32, n));
    GB_TRY(mem.alloc_n(&w.p32, n));
    GB_TRY(mem.alloc_n(&w.q32, n));
    GB_TRY(mem.alloc_n(&w.S2, 1));
    int64_t launches = 0;
    enqueue_residual(V, o.x0_zero ? nullptr : w.x, w.b, w.r, w.partials, w.S, 1, o.tol, g, st);
    ++launches;
    PcgScal h{};
    GB_TRY(read_scal(w.S, &h, st));
    stats->bnorm = std::sqrt(h.bb);
    if (h.bb == 0.0) {
        GB_CHECK_CUDA(cudaMemsetAsync(w.x, 0, sizeof(double) * n, st));
        stats->relres = 0.0;
        stats->status = GB_OK;
        return GB_OK;
    }
    double rel = std::sqrt(h.rr / h.bb);
    const double target2 = 0.25 * o.tol * o.tol * h.bb;  // fp32 recursive residual goal before a final check
    int64_t inner_total = 0;
    int updates = 0, stalls = 0;
    double prev = rel;
    double bytes = 0.0;
    const double sval = sizeof(TV);
    bool first = true;
    long long last_cycle = 0;
    {
        PcgScal hs{};
        hs.maxit = o.max_iter;
        GB_CHECK_CUDA(cudaMemcpyAsync(w.S2, &hs, sizeof(PcgScal), cudaMemcpyHostToDevice, st));
    }
    while (rel > o.tol && inner_total < o.max_iter && updates < 1000) {
        // replace the fp32 residual by the fp64 one; start p on the first pass only
        ::gb::count_launches(1); k_replace<<<g.vec, NT, 0, st>>>(n, w.r, A->dinv32, w.r32, w.d32, w.p32, first ? 1 : 0,
                                                               w.partials, w.S2);
        ++launches;
        if (first) {
            ::gb::count_launches(1); k_start<float, float><<<g.vec, NT, 0, st>>>(n, w.r32, A->dinv32, w.p32, w.partials, w.S2);
            first = false;
        } else {
            ::gb::count_launches(1); k_replace_p<<<g.vec, NT, 0, st>>>(n, w.r32, A->dinv32, w.p32, w.S2);
        }
        ++launches;
        PcgScal hr{};
        GB_TRY(read_scal(w.S2, &hr, st));
        if (hr.done) break;  // r32 == 0 or not positive: nothing to iterate on
        {
            // run until ||r32||^2 <= max(delta^2 ||r32_0||^2, target), or for at
            // most a cycle budget (a recurrence that stagnates above the
            // threshold still reaches the fp64 update and the stall test)
            const double th = std::max(RU_DELTA * RU_DELTA * hr.rr, target2);
            GB_CHECK_CUDA(cudaMemcpyAsync(&w.S2->thresh, &th, sizeof(double), cudaMemcpyHostToDevice, st));
            const long long cap = 1000 + 3 * last_cycle;
            const long long mx = std::min<long long>(o.max_iter, hr.it + cap);
            GB_CHECK_CUDA(cudaMemcpyAsync(&w.S2->maxit, &mx, sizeof(long long), cudaMemcpyHostToDevice, st));
        }
        const long long it0 = hr.it;
        auto body = [&](cudaStream_t s) {
            enqueue_iteration<TV, float, float>(V, val_in, A->dinv32, w.d32, w.r32, w.p32, w.q32, (float *)nullptr, w.partials, w.S2, g, s,
                                                o.spmv_variant ? o.spmv_variant : A->variant_hint);
        };
        GB_TRY(run_loop(st, w.S2, o.use_graph != 0, o.check_every, body, nullptr));
        PcgScal hi{};
        GB_TRY(read_scal(w.S2, &hi, st));
        const long long dit = hi.it - it0;
        if (hi.status == ST_CONV) last_cycle = dit;  // the last cycle that reached its threshold
        inner_total = hi.it;
        launches += 3 * dit;
        bytes += dit * ((double)A->nnz * (sval + 4.0) + 7.0 * n * 4.0);
        // x += d ; r = b - A x (fp64)
        ::gb::count_launches(1); k_correct<<<g.vec, NT, 0, st>>>(n, w.x, 1.0, w.d32);
        enqueue_residual(V, w.x, w.b, w.r, w.partials, w.S, 0, o.tol, g, st);
        launches += 2;
        bytes += (double)A->nnz * 12.0 + 5.0 * n * 8.0;
        GB_TRY(read_scal(w.S, &h, st));
        rel = std::sqrt(h.rr / h.bb);
        ++updates;
        if (getenv("GBPCG_LOG"))
            fprintf(stderr, "[gbpcg ru] update %d: cycle its %lld status %d rel %.3e best %.3e\n", updates, dit,
                    hi.status, rel, prev);
        if (hi.status == ST_BREAK || inner_total >= o.max_iter) break;
        // a cycle that ran out of its budget, or an update without a 10% gain,
        // is a stall; two in a row hand the solve to the fp64 finish
        if (hi.status == ST_MAXIT || !(rel < 0.9 * prev)) { if (++stalls >= 2) break; } else stalls = 0;
        prev = std::min(prev, rel);
    }
    stats->iterations = inner_total;
    stats->outer = updates;
    stats->relres = rel;
    stats->status = rel <= o.tol ? GB_OK : GB_NOT_CONVERGED;
    stats->kernel_launches = launches;
    stats->bytes_moved = bytes;
    return GB_OK;
}

// BiCGSTAB (bicgstab.cuh), fp64, Jacobi or block-Jacobi on the right; the
// true residual confirms a stop (restart from it otherwise), as in solve_f64.
static int solve_bicgstab(const gb_sell *A, const PcgOptions &o, Work &w, cudaStream_t st, PcgStats *stats) {
    const SellViewH V = A->view();
    const int64_t n = A->n;
    const Grids g = pick_grids(n, A->C);
    const bool use_bj = o.precond == GB_PC_BLOCK_JACOBI;
    const BjView bj = A->bj_view();
    int64_t launches = 0;
    struct Vecs {
        Mem *m;
        double *rh = nullptr, *v = nullptr, *ph = nullptr, *s = nullptr, *sh = nullptr, *t = nullptr;
        ~Vecs() { m->release(rh); m->release(v); m->release(ph); m->release(s); m->release(sh); m->release(t); }
    } u{&w.mem};
    GB_TRY(w.mem.alloc_n(&u.rh, n));
    GB_TRY(w.mem.alloc_n(&u.v, n));
    GB_TRY(w.mem.alloc_n(&u.ph, n));
    GB_TRY(w.mem.alloc_n(&u.s, n));
    GB_TRY(w.mem.alloc_n(&u.sh, n));
    GB_TRY(w.mem.alloc_n(&u.t, n));
    enqueue_residual(V, o.x0_zero ? nullptr : w.x, w.b, w.r, w.partials, w.S, 1, o.tol, g, st);
    ++launches;
    PcgScal h{};
    GB_TRY(read_scal(w.S, &h, st));
    stats->bnorm = std::sqrt(h.bb);
    if (h.bb == 0.0) {
        GB_CHECK_CUDA(cudaMemsetAsync(w.x, 0, sizeof(double) * n, st));
        stats->relres = 0.0;
        stats->status = GB_OK;
        stats->kernel_launches = launches + 1;
        return GB_OK;
    }
    static bool attr_set[2] = {false, false};
    const int smem = (int)tma2_smem_bytes<double>();
    if (!attr_set[0]) {
        cudaFuncSetAttribute(k_spmv_bi<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_spmv_bi<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set[0] = attr_set[1] = true;
    }
    const int gs = V.nwarps / TMA_WARPS;
    const int gbj = bj_grid(n);
    int64_t restarts = 0;
    int status = ST_RUN;
    double rel = std::sqrt(h.rr / h.bb);
    double rel_start = rel;  // true residual the current recurrence started from
    while (rel > o.tol) {
        ::gb::count_launches(1); k_bi_start<<<g.vec, NT, 0, st>>>(n, w.r, u.rh, w.p, u.v, w.partials, w.S);
        ++launches;
        GB_CHECK_CUDA(cudaGetLastError());
        auto body = [&](cudaStream_t s) {
            if (use_bj) {
#define GB_BI_P(K) ::gb::count_launches(1); k_bi_p_bj<K><<<gbj, BJ_WIN, 0, s>>>(n, w.r, u.v, w.p, u.ph, bj, w.S)
                GB_BJ_DISPATCH(bj.bs, GB_BI_P)
#undef GB_BI_P
            } else {
                ::gb::count_launches(1); k_bi_p<<<g.upd, NT, 0, s>>>(n, w.r, u.v, w.p, u.ph, A->dinv, w.S);
            }
            ::gb::count_launches(1);
            k_spmv_bi<1><<<gs, NT, smem, s>>>(V, V.warp_chunk, A->val, u.ph, u.v, u.rh, w.partials, w.S);
            if (use_bj) {
#define GB_BI_S(K) ::gb::count_launches(1); k_bi_s_bj<K><<<gbj, BJ_WIN, 0, s>>>(n, w.r, u.v, u.s, u.sh, bj, w.partials, w.S)
                GB_BJ_DISPATCH(bj.bs, GB_BI_S)
#undef GB_BI_S
            } else {
                ::gb::count_launches(1); k_bi_s<<<g.upd, NT, 0, s>>>(n, w.r, u.v, u.s, u.sh, A->dinv, w.partials, w.S);
            }
            ::gb::count_launches(1);
            k_spmv_bi<2><<<gs, NT, smem, s>>>(V, V.warp_chunk, A->val, u.sh, u.t, u.s, w.partials, w.S);
            ::gb::count_launches(1);
            k_bi_x<<<g.upd, NT, 0, s>>>(n, w.x, w.r, u.ph, u.sh, u.s, u.t, u.rh, w.partials, w.S);
        };
        GB_TRY(run_loop(st, w.S, o.use_graph != 0, o.check_every, body, nullptr, 5));
        GB_TRY(read_scal(w.S, &h, st));
        status = h.status;
        enqueue_residual(V, w.x, w.b, w.r, w.partials, w.S, 0, o.tol, g, st);
        ++launches;
        PcgScal h2{};
        GB_TRY(read_scal(w.S, &h2, st));
        rel = std::sqrt(h2.rr / h2.bb);
        if (getenv("GBPCG_LOG"))
            fprintf(stderr, "[gbpcg bicgstab] stop after %lld steps: status %d (breakdown code %d), true relres %.3e\n",
                    h.it, status, h.brk, rel);
        // a stop on the recursive residual above tol, or a breakdown while the
        // true residual still falls: restart from the true residual
        const bool retry = status == ST_CONV || (status == ST_BREAK && rel < 0.9 * rel_start);
        if (!retry || rel <= o.tol || h.it >= h.maxit || ++restarts > 50) break;
        rel_start = rel;
    }
    if (rel <= o.tol) status = ST_CONV;
    stats->iterations = h.it;
    stats->restarts = restarts;
    stats->relres = rel;
    stats->status = map_status(status);
    stats->kernel_launches = launches + 5 * h.it;
    // two SpMVs and ~15 vector streams per step
    stats->bytes_moved = ((double)A->nnz * 24.0 + 15.0 * n * 8.0) * (double)h.it;
    return GB_OK;
}

extern "C" int pcg_solve(const gb_sell *A, const double *d_b, double *d_x, const PcgOptions *opt,
                         void *stream, PcgStats *stats) {
    gb::Range range("gbpcg:pcg_solve");
    GB_REQUIRE(A && d_b && d_x, "pcg_solve: NULL argument");
    PcgStats dummy{};
    if (!stats) stats = &dummy;
    *stats = PcgStats{};
    PcgOptions o = defaults(opt, A->n);
    GB_REQUIRE(o.precision >= GB_F64 && o.precision <= GB_BF16_RU, "pcg_solve: bad precision");
    GB_REQUIRE((o.precision != GB_F32_IR && o.precision != GB_F32_RU) || A->val32,
               "pcg_solve: fp32-inner precisions need fp32 values (val_types)");
    GB_REQUIRE((o.precision != GB_BF16_IR && o.precision != GB_BF16_RU) || A->val16,
               "pcg_solve: bf16-inner precisions need bf16 values (val_types)");
    GB_REQUIRE(o.precond == GB_PC_JACOBI || o.precond == GB_PC_BLOCK_JACOBI, "pcg_solve: bad precond %d",
               o.precond);
    GB_REQUIRE(o.method == GB_CG || o.method == GB_BICGSTAB, "pcg_solve: bad method %d", o.method);
    GB_REQUIRE(o.method != GB_BICGSTAB || (o.precision == GB_F64 && A->C == 32 && A->warp_chunk),
               "pcg_solve: GB_BICGSTAB runs in fp64 on C = 32 layouts");
    GB_REQUIRE(o.precond != GB_PC_BLOCK_JACOBI || A->bj_bs > 0,
               "pcg_solve: GB_PC_BLOCK_JACOBI without block-Jacobi data (sell_block_jacobi)");
    GB_REQUIRE(o.precond != GB_PC_BLOCK_JACOBI || o.precision == GB_F64 || o.precision == GB_F32_IR ||
                   o.precision == GB_BF16_IR,
               "pcg_solve: GB_PC_BLOCK_JACOBI with GB_F64, GB_F32_IR or GB_BF16_IR only");
    cudaStream_t st = (cudaStream_t)stream;
    if (o.precision == GB_F64 && o.method == GB_CG && o.precond == GB_PC_JACOBI &&
        ((o.persist_off == 0 && A->n <= GB_CLUSTER_SINGLE_MAX) || (o.persist_off == 3 && A->n <= GB_GRID_SINGLE_MAX))) {
        // a system this small is latency-bound in the loop of three grid-wide
        // launches per iteration and in its per-solve set-up: one persistent
        // launch (one thread-block cluster) solves it whole; persist_off = 3
        // asks for a group of the grid tier up to 2^18 rows
        const int rc = grid_solve_single(A, d_b, d_x, o, st, stats);
        if (rc != 1) {
            if (rc != GB_OK) return rc;
            if (stats->status != GB_OK) {
                set_error("pcg_solve: %s after %lld iterations (relres %.3e)",
                          stats->status == GB_BREAKDOWN ? "breakdown"
                          : stats->status == GB_TIMEOUT ? "a persistent-kernel barrier wait ran out"
                                                        : "not converged",
                          (long long)stats->iterations, stats->relres);
                return stats->status;
            }
            return GB_OK;
        }
    }
    Work w;
    w.mem = Mem(nullptr, st);
    const int64_t n = A->n;
    const Grids g = pick_grids(n, A->C);
    GB_TRY(w.mem.alloc_n(&w.x, n));
    GB_TRY(w.mem.alloc_n(&w.r, n));
    GB_TRY(w.mem.alloc_n(&w.p, n));
    GB_TRY(w.mem.alloc_n(&w.q, n));
    GB_TRY(w.mem.alloc_n(&w.b, n));
    GB_TRY(w.mem.alloc_n(&w.z, n));
    GB_TRY(w.mem.alloc_n(&w.partials, partial_slots(A, g)));
    GB_TRY(w.mem.alloc_n(&w.S, 1));
    GB_TRY(init_scal(w.S, o.max_iter, st));
    cudaEvent_t e0, e1;
    GB_CHECK_CUDA(cudaEventCreate(&e0));
    GB_CHECK_CUDA(cudaEventCreate(&e1));
    GB_CHECK_CUDA(cudaEventRecord(e0, st));
    ::gb::count_launches(1); k_gather_d<<<g.vec, NT, 0, st>>>(n, A->perm, d_b, w.b);
    ::gb::count_launches(1); k_gather_d<<<g.vec, NT, 0, st>>>(n, A->perm, o.x0_zero ? nullptr : d_x, w.x);
    int rc;
    if (o.method == GB_BICGSTAB) rc = solve_bicgstab(A, o, w, st, stats);
    else if (o.precision == GB_F64) rc = solve_f64(A, o, w, st, stats);
    else if (o.precision == GB_F32_IR) rc = solve_ir<float>(A, A->val32, o, w, st, stats);
    else if (o.precision == GB_BF16_IR) rc = solve_ir<__nv_bfloat16>(A, A->val16, o, w, st, stats);
    else if (o.precision == GB_F32_RU) rc = solve_ru<float>(A, A->val32, o, w, st, stats);
    else rc = solve_ru<__nv_bfloat16>(A, A->val16, o, w, st, stats);
    if (rc == GB_OK && o.precision != GB_F64 && stats->status != GB_OK && stats->iterations < o.max_iter) {
        // refinement stalled above tol: finish in fp64 from the current x
        PcgOptions o2 = o;
        o2.x0_zero = 0;
        o2.max_iter = o.max_iter - stats->iterations;
        PcgStats s2{};
        rc = init_scal(w.S, o2.max_iter, st);
        if (rc == GB_OK) rc = solve_f64(A, o2, w, st, &s2);
        if (rc == GB_OK) {
            stats->fallback_iterations = s2.iterations;
            stats->relres = s2.relres;
            stats->status = s2.status;
            stats->kernel_launches += s2.kernel_launches;
            stats->bytes_moved += s2.bytes_moved;
        }
    }
    if (rc == GB_OK) {
        ::gb::count_launches(1); k_scatter_d<<<g.vec, NT, 0, st>>>(n, A->perm, w.x, d_x);
        stats->kernel_launches += 3;
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        stats->solve_ms = ms;
        if (e != cudaSuccess) { set_error("pcg_solve: %s", cudaGetErrorString(e)); rc = GB_ECUDA; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GB_OK) return rc;
    if (stats->status != GB_OK) {
        set_error("pcg_solve: %s after %lld iterations (relres %.3e)",
                  stats->status == GB_BREAKDOWN ? "breakdown" : "not converged",
                  (long long)stats->iterations, stats->relres);
        return stats->status;
    }
    return GB_OK;
}

static int kernel_times_impl(const gb_sell *A, const double *d_b, int precision, int iters, int variant,
                             void *stream, double *h_ms) {
    GB_REQUIRE(A && d_b && h_ms, "pcg_kernel_times: NULL argument");
    GB_REQUIRE(iters >= 1 && iters <= 100000, "pcg_kernel_times: iters must be in 1..100000");
    const bool use_bj = (precision & GB_KT_BLOCK_JACOBI) != 0;
    precision &= ~GB_KT_BLOCK_JACOBI;
    GB_REQUIRE(!use_bj || A->bj_bs > 0, "pcg_kernel_times: GB_KT_BLOCK_JACOBI without block-Jacobi data");
    GB_REQUIRE(precision >= GB_F64 && precision <= GB_BF16_IR, "pcg_kernel_times: bad precision");
    GB_REQUIRE(precision != GB_F32_IR || A->val32, "pcg_kernel_times: no fp32 values");
    GB_REQUIRE(precision != GB_BF16_IR || A->val16, "pcg_kernel_times: no bf16 values");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = A->n;
    const Grids g = pick_grids(n, A->C);
    const SellViewH V = A->view();
    Work w;
    w.mem = Mem(nullptr, st);
    GB_TRY(w.mem.alloc_n(&w.x, n));
    GB_TRY(w.mem.alloc_n(&w.r, n));
    GB_TRY(w.mem.alloc_n(&w.p, n));
    GB_TRY(w.mem.alloc_n(&w.q, n));
    GB_TRY(w.mem.alloc_n(&w.b, n));
    GB_TRY(w.mem.alloc_n(&w.z, n));
    GB_TRY(w.mem.alloc_n(&w.r32, n));
    GB_TRY(w.mem.alloc_n(&w.d32, n));
    GB_TRY(w.mem.alloc_n(&w.p32, n));
    GB_TRY(w.mem.alloc_n(&w.q32, n));
    GB_TRY(w.mem.alloc_n(&w.z32, n));
    GB_TRY(w.mem.alloc_n(&w.partials, partial_slots(A, g)));
    GB_TRY(w.mem.alloc_n(&w.S, 1));
    const BjView bj = A->bj_view();
    PcgScal hs{};
    hs.maxit = (long long)iters + 1;
    hs.thresh = -1.0;  // never converges: every timed launch is a full pass
    // fp64: the solver's launch sequence (z stored, r.r sums deferred)
    if (precision == GB_F64) hs.dmax = use_bj ? A->bj_lam : A->dinv_max;
    GB_CHECK_CUDA(cudaMemcpyAsync(w.S, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    ::gb::count_launches(1); k_gather_d<<<g.vec, NT, 0, st>>>(n, A->perm, d_b, w.b);
    GB_CHECK_CUDA(cudaMemsetAsync(w.x, 0, sizeof(double) * n, st));
    enqueue_residual(V, nullptr, w.b, w.r, w.partials, w.S, 0, 0.0, g, st);
    if (precision == GB_F64) {
        if (use_bj) launch_start_bj<double, double>(bj, n, w.r, w.p, w.partials, w.S, st);
        else { ::gb::count_launches(1); k_start<double, double><<<g.vec, NT, 0, st>>>(n, w.r, A->dinv, w.p, w.partials, w.S); }
    } else {
        ::gb::count_launches(1); k_scale_down<<<g.vec, NT, 0, st>>>(n, w.r, 1.0, w.r32, w.d32);
        if (use_bj) launch_start_bj<float, float>(bj, n, w.r32, w.p32, w.partials, w.S, st);
        else { ::gb::count_launches(1); k_start<float, float><<<g.vec, NT, 0, st>>>(n, w.r32, A->dinv32, w.p32, w.partials, w.S); }
    }
    GB_CHECK_CUDA(cudaGetLastError());
    std::vector<cudaEvent_t> ev(3 * (size_t)iters + 1);
    for (auto &e : ev) GB_CHECK_CUDA(cudaEventCreate(&e));
    int rc = GB_OK;
    cudaEventRecord(ev[0], st);
    for (int i = 0; i < iters; ++i) {
        for (int k = 0; k < 3; ++k) {
            if (k == 0 && A->C == 32 && A->warp_chunk && variant == 0) {
                if (precision == GB_F64) launch_spmv_tma<double, double>(V, A->val, w.p, w.q, w.partials, w.S, st);
                else if (precision == GB_F32_IR) launch_spmv_tma<float, float>(V, A->val32, w.p32, w.q32, w.partials, w.S, st);
                else launch_spmv_tma<__nv_bfloat16, float>(V, A->val16, w.p32, w.q32, w.partials, w.S, st);
            } else if (precision == GB_F64) {
                if (k == 0) {
                    switch (A->C) {
                    case 32: ::gb::count_launches(1); k_spmv_pq<double, double, 32><<<g.spmv, NT, 0, st>>>(V, A->val, w.p, w.q, w.partials, w.S); break;
                    case 64: ::gb::count_launches(1); k_spmv_pq<double, double, 64><<<g.spmv, NT, 0, st>>>(V, A->val, w.p, w.q, w.partials, w.S); break;
                    default: ::gb::count_launches(1); k_spmv_pq<double, double, 128><<<g.spmv, NT, 0, st>>>(V, A->val, w.p, w.q, w.partials, w.S); break;
                    }
                } else if (k == 1) {
                    if (use_bj) launch_update_bj<double, double>(bj, n, w.x, w.r, w.p, w.q, w.z, w.partials, w.S, st);
                    else { ::gb::count_launches(1); k_update<double, double><<<g.upd, NT, 0, st>>>(n, w.x, w.r, w.p, w.q, A->dinv, w.z, w.partials, w.S); }
                } else {
                    ::gb::count_launches(1); k_pupdate<double, double><<<g.upd, NT, 0, st>>>(n, w.p, w.r, A->dinv, w.z, w.partials, w.S);
                }
            } else {
                if (k == 0) {
                    if (precision == GB_F32_IR) {
                        switch (A->C) {
                        case 32: ::gb::count_launches(1); k_spmv_pq<float, float, 32><<<g.spmv, NT, 0, st>>>(V, A->val32, w.p32, w.q32, w.partials, w.S); break;
                        case 64: ::gb::count_launches(1); k_spmv_pq<float, float, 64><<<g.spmv, NT, 0, st>>>(V, A->val32, w.p32, w.q32, w.partials, w.S); break;
                        default: ::gb::count_launches(1); k_spmv_pq<float, float, 128><<<g.spmv, NT, 0, st>>>(V, A->val32, w.p32, w.q32, w.partials, w.S); break;
                        }
                    } else {
                        switch (A->C) {
                        case 32: ::gb::count_launches(1); k_spmv_pq<__nv_bfloat16, float, 32><<<g.spmv, NT, 0, st>>>(V, A->val16, w.p32, w.q32, w.partials, w.S); break;
                        case 64: ::gb::count_launches(1); k_spmv_pq<__nv_bfloat16, float, 64><<<g.spmv, NT, 0, st>>>(V, A->val16, w.p32, w.q32, w.partials, w.S); break;
                        default: ::gb::count_launches(1); k_spmv_pq<__nv_bfloat16, float, 128><<<g.spmv, NT, 0, st>>>(V, A->val16, w.p32, w.q32, w.partials, w.S); break;
                        }
                    }
                } else if (k == 1) {
                    if (use_bj) launch_update_bj<float, float>(bj, n, w.d32, w.r32, w.p32, w.q32, w.z32, w.partials, w.S, st);
                    else { ::gb::count_launches(1); k_update<float, float><<<g.upd, NT, 0, st>>>(n, w.d32, w.r32, w.p32, w.q32, A->dinv32, (float *)nullptr, w.partials, w.S); }
                } else {
                    ::gb::count_launches(1); k_pupdate<float, float><<<g.upd, NT, 0, st>>>(n, w.p32, w.r32, A->dinv32, use_bj ? w.z32 : (const float *)nullptr, w.partials, w.S);
                }
            }
            cudaEventRecord(ev[3 * (size_t)i + k + 1], st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
    double tot[3] = {0, 0, 0};
    for (int i = 0; i < iters && e == cudaSuccess; ++i)
        for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[3 * (size_t)i + k], ev[3 * (size_t)i + k + 1]);
            tot[k] += ms;
        }
    for (auto &x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) { set_error("pcg_kernel_times: %s", cudaGetErrorString(e)); return GB_ECUDA; }
    PcgScal h{};
    GB_TRY(read_scal(w.S, &h, st));
    if (h.done) {
        set_error("pcg_kernel_times: the recurrence stopped (status %d) after %lld iterations; use fewer",
                  h.status, h.it);
        rc = GB_BREAKDOWN;
    }
    for (int k = 0; k < 3; ++k) h_ms[k] = tot[k] / iters;
    return rc;
}

// A bounded wait that must run out: one warp arms an mbarrier that nothing
// will complete and waits on phase 0 with the library's bounded wait.
__global__ void k_wait_selftest(unsigned long long limit_ns, int *status, unsigned long long *waited_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const unsigned long long t0 = globaltimer();
    const bool ok = mbar_wait(&bar, 0u, limit_ns);
    const bool all = __all_sync(0xffffffffu, ok);
    if (threadIdx.x == 0) {
        *status = all ? ST_CONV : ST_TIMEOUT;
        *waited_ns = globaltimer() - t0;
    }
}

extern "C" int gbpcg_wait_selftest(double limit_ms, void *stream, double *h_waited_ms) {
    GB_REQUIRE(limit_ms > 0.0 && limit_ms <= 2000.0, "gbpcg_wait_selftest: limit_ms must be in (0, 2000]");
    cudaStream_t st = (cudaStream_t)stream;
    void *buf = nullptr;
    GB_CHECK_CUDA(cudaMalloc(&buf, 16));
    int *d_status = (int *)buf;
    unsigned long long *d_waited = (unsigned long long *)((char *)buf + 8);
    ::gb::count_launches(1);
    k_wait_selftest<<<1, 32, 0, st>>>((unsigned long long)(limit_ms * 1e6), d_status, d_waited);
    int h_status = -1;
    unsigned long long h_waited = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_waited, d_waited, sizeof(h_waited), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) { set_error("gbpcg_wait_selftest: %s", cudaGetErrorString(e)); return GB_ECUDA; }
    if (h_waited_ms) *h_waited_ms = (double)h_waited * 1e-6;
    if (h_status == ST_TIMEOUT) {
        set_error("gbpcg_wait_selftest: the bounded wait gave up after %.3f ms", (double)h_waited * 1e-6);
        return GB_TIMEOUT;
    }
    return GB_OK;
}

extern "C" int pcg_kernel_times(const gb_sell *A, const double *d_b, int precision, int iters,
                                void *stream, double *h_ms) {
    GB_REQUIRE(A, "pcg_kernel_times: NULL matrix");
    return kernel_times_impl(A, d_b, precision, iters, A->variant_hint, stream, h_ms);
}

extern "C" int sell_set_variant(gb_sell *A, int variant) {
    GB_REQUIRE(A, "sell_set_variant: NULL matrix");
    GB_REQUIRE(variant == 0 || variant == 1, "sell_set_variant: variant must be 0 or 1");
    A->variant_hint = variant;
    return GB_OK;
}

// ---------------------------------------------------------------- autotune --
// Times one CG iteration (SpMV + p.q, x/r update, p update) of every candidate
// layout (chunk height C, sorting window sigma, SpMV variant) on this matrix
// and precision, and keeps the fastest.  The winner's variant is recorded in
// the matrix, so later solves use it without being told.
extern "C" int sell_autotune(const gb_fem_system *sys, const double *d_b, int precision, int val_types,
                             const gb_allocator *alloc, void *stream, SellTuneResult *best, gb_sell **out) {
    GB_REQUIRE(sys && d_b && best, "sell_autotune: NULL argument");
    GB_REQUIRE(precision == GB_F64 || precision == GB_F32_IR || precision == GB_BF16_IR,
               "sell_autotune: precision must be GB_F64, GB_F32_IR or GB_BF16_IR");
    struct Cand { int C, sigma, variant; };
    static const Cand cands[] = {{32, 256, 0}, {32, 64, 0}, {32, 1024, 0}, {32, 256, 1},
                                 {64, 256, 1}, {128, 256, 1}, {64, 1024, 1}};
    *best = SellTuneResult{};
    best->iter_ms = 1e300;
    gb_sell *keep = nullptr;
    int rc = GB_OK;
    for (const Cand &c : cands) {
        gb_sell *A = nullptr;
        rc = csr_to_sell(sys, c.C, c.sigma, val_types, alloc, stream, &A);
        if (rc != GB_OK) break;
        if (c.variant == 0 && !A->warp_chunk) { sell_destroy(A); continue; }
        double ms[3] = {0, 0, 0};
        rc = kernel_times_impl(A, d_b, precision, 2, c.variant, stream, ms);  // warm-up
        if (rc == GB_OK) rc = kernel_times_impl(A, d_b, precision, 8, c.variant, stream, ms);
        if (rc != GB_OK) { sell_destroy(A); break; }
        const double it = ms[0] + ms[1] + ms[2];
        if (it < best->iter_ms) {
            best->C = c.C; best->sigma = c.sigma; best->spmv_variant = c.variant;
            best->iter_ms = it; best->spmv_ms = ms[0];
            A->variant_hint = c.variant;
            if (keep) sell_destroy(keep);
            keep = A;
        } else {
            sell_destroy(A);
        }
        best->candidates += 1;
    }
    if (rc != GB_OK) { if (keep) sell_destroy(keep); return rc; }
    if (out) *out = keep;
    else if (keep) sell_destroy(keep);
    return GB_OK;
}

// ------------------------------------------------------- no-allocation solve --
// pcg_solve_noalloc: the fp64 pcg_solve for callers that cannot allocate
// device memory -- code that runs where cudaMalloc is forbidden or unsafe
// (inside another allocator's callbacks, in a process whose device memory is
// owned by a fixed arena it must not grow, in a real-time loop that may not
// block on the allocator).  Its scratch (the permuted b and x, r, p, q, the
// per-block partial sums and the solver scalars) lives in one file-scope
// device array of fixed size, so the call allocates nothing: it enqueues
// kernels, copies the few solver scalars back to the host and synchronises.
namespace gb {
constexpr int64_t NOALLOC_MAX_N = 262144;  // rows
constexpr int64_t NOALLOC_PARTIALS = 6144;  // doubles: 3 per block, up to 256 SMs x 8 blocks
constexpr size_t NOALLOC_BYTES = (size_t)5 * NOALLOC_MAX_N * sizeof(double) +
                                 NOALLOC_PARTIALS * sizeof(double) + 256;
// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Host code must not take the address of g_noalloc_scratch directly (that is
// a host-side stand-in).  The device address is looked up on every call, on
// the current device: a cached address could outlive the module it points
// into (a device reset or context teardown reloads it elsewhere).
static int noalloc_scratch(unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error("pcg_solve_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return GB_ECUDA;
    }
    *out = (unsigned char *)p;
    return GB_OK;
}

// A Work whose buffers are views into the static array: its fields are
// cleared on every way out of scope, before ~Work would release them.
struct NoallocWork {
    Work w;
    ~NoallocWork() {
        w.x = w.r = w.p = w.q = w.b = w.z = w.partials = nullptr;
        w.S = nullptr;
    }
};
}  // namespace gb

extern "C" int pcg_solve_noalloc(const gb_sell *A, const double *d_b, double *d_x, const PcgOptions *opt,
                                 void *stream, PcgStats *stats) {
    GB_REQUIRE(A && d_b && d_x, "pcg_solve_noalloc: NULL argument");
    if (A->n > NOALLOC_MAX_N) {
        set_error("pcg_solve_noalloc: n = %lld rows exceeds the fixed scratch limit of %lld rows; use pcg_solve",
                  (long long)A->n, (long long)NOALLOC_MAX_N);
        return GB_TOO_LARGE;
    }
    PcgStats dummy{};
    if (!stats) stats = &dummy;
    *stats = PcgStats{};
    PcgOptions o = defaults(opt, A->n);
    GB_REQUIRE(o.precision == GB_F64, "pcg_solve_noalloc: only precision GB_F64 is available");
    GB_REQUIRE(o.precond == GB_PC_JACOBI, "pcg_solve_noalloc: the Jacobi preconditioner only");
    GB_REQUIRE(o.method == GB_CG, "pcg_solve_noalloc: CG only");
    o.use_graph = 0;  // graph objects would allocate: the loop is polled direct launches
    const int64_t n = A->n;
    const Grids g = pick_grids(n, A->C);
    if ((int64_t)partial_slots(A, g) > NOALLOC_PARTIALS) {
        set_error("pcg_solve_noalloc: this device needs %lld partial sums, above the fixed %lld",
                  (long long)partial_slots(A, g), (long long)NOALLOC_PARTIALS);
        return GB_TOO_LARGE;
    }
    unsigned char *base = nullptr;
    GB_TRY(noalloc_scratch(&base));
    cudaStream_t st = (cudaStream_t)stream;
    NoallocWork nw;  // views into the static array; nothing here is released
    Work &w = nw.w;
    w.mem = Mem(nullptr, st);
    double *vec = (double *)base;
    w.x = vec;
    w.r = vec + NOALLOC_MAX_N;
    w.p = vec + 2 * NOALLOC_MAX_N;
    w.q = vec + 3 * NOALLOC_MAX_N;
    w.b = vec + 4 * NOALLOC_MAX_N;
    w.partials = vec + 5 * NOALLOC_MAX_N;
    w.S = (PcgScal *)(base + (size_t)5 * NOALLOC_MAX_N * sizeof(double) + NOALLOC_PARTIALS * sizeof(double));
    static_assert(sizeof(PcgScal) <= 256, "solver scalars must fit the reserved tail");
    int rc = init_scal(w.S, o.max_iter, st);  // the scalars (and the block ticket) start from zero
    const auto t0 = std::chrono::steady_clock::now();
    if (rc == GB_OK) {
        ::gb::count_launches(1); k_gather_d<<<g.vec, NT, 0, st>>>(n, A->perm, d_b, w.b);
        ::gb::count_launches(1); k_gather_d<<<g.vec, NT, 0, st>>>(n, A->perm, o.x0_zero ? nullptr : d_x, w.x);
        rc = solve_f64(A, o, w, st, stats);
    }
    if (rc == GB_OK) {
        ::gb::count_launches(1); k_scatter_d<<<g.vec, NT, 0, st>>>(n, A->perm, w.x, d_x);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { set_error("pcg_solve_noalloc: %s", cudaGetErrorString(e)); rc = GB_ECUDA; }
        stats->kernel_launches += 3;
    }
    stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc != GB_OK) return rc;
    if (stats->status != GB_OK) {
        set_error("pcg_solve_noalloc: %s after %lld iterations (relres %.3e)",
                  stats->status == GB_BREAKDOWN ? "breakdown" : "not converged",
                  (long long)stats->iterations, stats->relres);
        return stats->status;
    }
    return GB_OK;
}
