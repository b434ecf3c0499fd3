// bicgstab.cuh -- BiCGSTAB kernels (van der Vorst 1992), the Krylov method
// the paper runs (Sec. 3.2), right-preconditioned with Jacobi or block-Jacobi:
//   rho = r^.r;  beta = (rho/rho0)(alpha/omega);  p = r + beta (p - omega v);
//   ph = M^-1 p;  v = A ph;  alpha = rho / r^.v;  s = r - alpha v;
//   (||s|| <= tol ||b||: x += alpha ph, stop);  sh = M^-1 s;  t = A sh;
//   omega = t.s / t.t;  x += alpha ph + omega sh;  r = s - omega t.
// Five kernels per step, each fusing its vector work with the dot products
// the next scalar needs; the scalars live in PcgScal on the device (rho,
// rho0, alpha, omega, pq = r^.v), and the last block of each reduction makes
// the step's decision, so the step loop runs as a CUDA-graph while-node.
#pragma once
#include "bjacobi.cuh"
#include "pcg.cuh"
#include "spmv_tma.cuh"

namespace gb {

// ph = M^-1 p with p = r + beta (p - omega v); the first kernel of a step
// (ends the graph loop when the recurrence has stopped).  Jacobi: one pass.
__global__ void __launch_bounds__(NT) k_bi_p(int64_t n, const double *__restrict__ r, const double *__restrict__ v,
                                             double *__restrict__ p, double *__restrict__ ph,
                                             const double *__restrict__ dinv, PcgScal *S) {
    if (S->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && S->use_cond) cudaGraphSetConditional(S->cond, 0);
        return;
    }
    const double beta = (S->rho / S->rho0) * (S->alpha / S->omega), omega = S->omega;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const double pi = r[i] + beta * (p[i] - omega * v[i]);
        p[i] = pi;
        ph[i] = dinv[i] * pi;
    }
}

// the same with block-Jacobi: one 256-row window per CTA step
template <int BS>
__global__ void __launch_bounds__(BJ_WIN) k_bi_p_bj(int64_t n, const double *__restrict__ r,
                                                    const double *__restrict__ v, double *__restrict__ p,
                                                    double *__restrict__ ph, BjView B, PcgScal *S) {
    if (S->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && S->use_cond) cudaGraphSetConditional(S->cond, 0);
        return;
    }
    constexpr int T = BS * (BS + 1) / 2;
    __shared__ double rs[BJ_WIN], zs[BJ_WIN];
    __shared__ double ws[(BJ_WIN / BS) * T];
    __shared__ uint8_t ls[BJ_WIN];
    const double beta = (S->rho / S->rho0) * (S->alpha / S->omega), omega = S->omega;
    const int64_t nwin = (n + BJ_WIN - 1) / BJ_WIN;
    for (int64_t w = blockIdx.x; w < nwin; w += gridDim.x) {
        const int64_t i = w * BJ_WIN + threadIdx.x;
        double pi = 0.0;
        if (i < n) {
            pi = r[i] + beta * (p[i] - omega * v[i]);
            p[i] = pi;
        }
        rs[threadIdx.x] = pi;
        bj_stage<double, BS>(B, w, n, ws, ls);
        __syncthreads();
        bj_window<double, double, BS>(rs, ls, ws, zs, i < n);
        __syncthreads();
        if (i < n) ph[i] = zs[threadIdx.x];
        __syncthreads();
    }
}

// v = A ph and r^.v -> alpha = rho / r^.v (DM 1); t = A sh, t.s and t.t ->
// omega = t.s / t.t (DM 2, skipped after an early stop on s).  TMA-staged
// streams as k_spmv_tma2 (fp64 warp partition).
template <int DM>
__global__ void __launch_bounds__(NT) k_spmv_bi(SellView A, const int32_t *__restrict__ wchunk,
                                                const double *__restrict__ val, const double *__restrict__ xin,
                                                double *__restrict__ y, const double *__restrict__ d1,
                                                double *partials, PcgScal *S) {
    if (S->done || (DM == 2 && S->early)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double sm[NT / 32];
    constexpr int NB = Tma2Cfg<double>::NB;
    Tma2Ring<double> *bufs = reinterpret_cast<Tma2Ring<double> *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + TMA_WARPS * sizeof(Tma2Ring<double>));
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
    double d2 = 0.0;
    const double d = spmv_warp_stream2<double, double, DM>(A, val, xin, y, c0, c1, bufs[warp], &bars[NB * warp],
                                                           &timed_out, d1, &d2);
    if (timed_out && lane == 0) atomicExch(&S->err, 1);
    const double a = block_sum<NT>(d, sm);
    const double b = DM == 2 ? block_sum<NT>(d2, sm) : 0.0;
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
    if (arrive_last(&S->ticket)) {
        const double ta = sum_partials(partials, gridDim.x, 2, 0, sm);
        const double tb = DM == 2 ? sum_partials(partials, gridDim.x, 2, 1, sm) : 0.0;
        if (threadIdx.x == 0) {
            S->ticket = 0;
            if (S->err) stop(S, ST_TIMEOUT);
            else if (DM == 1) {
                S->pq = ta;
                if (ta == 0.0 || !isfinite(ta)) { S->brk = 1; stop(S, ST_BREAK); }
                else S->alpha = S->rho / ta;
            } else {
                if (tb == 0.0 || !isfinite(tb) || !isfinite(ta)) { S->brk = 2; stop(S, ST_BREAK); }
                else S->omega = ta / tb;
            }
        }
    }
}

// last block of k_bi_s: counts the step, ||s||^2 -> early stop flag
__device__ __forceinline__ void bi_s_decide(double ss_t, PcgScal *S) {
    S->ticket = 0;
    S->it += 1;
    if (!isfinite(ss_t)) { S->brk = 3; stop(S, ST_BREAK); }
    else if (ss_t <= S->thresh) S->early = 1;
}

// s = r - alpha v, sh = M^-1 s (Jacobi), ||s||^2
__global__ void __launch_bounds__(NT) k_bi_s(int64_t n, const double *__restrict__ r, const double *__restrict__ v,
                                             double *__restrict__ s, double *__restrict__ sh,
                                             const double *__restrict__ dinv, double *partials, PcgScal *S) {
    if (S->done) return;
    __shared__ double sm[NT / 32];
    const double alpha = S->alpha;
    double ss = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const double si = r[i] - alpha * v[i];
        s[i] = si;
        sh[i] = dinv[i] * si;
        ss += si * si;
    }
    const double a = block_sum<NT>(ss, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
    if (arrive_last(&S->ticket)) {
        const double t = sum_partials(partials, gridDim.x, 1, 0, sm);
        if (threadIdx.x == 0) bi_s_decide(t, S);
    }
}

template <int BS>
__global__ void __launch_bounds__(BJ_WIN) k_bi_s_bj(int64_t n, const double *__restrict__ r,
                                                    const double *__restrict__ v, double *__restrict__ s,
                                                    double *__restrict__ sh, BjView B, double *partials,
                                                    PcgScal *S) {
    if (S->done) return;
    constexpr int T = BS * (BS + 1) / 2;
    __shared__ double rs[BJ_WIN], zs[BJ_WIN];
    __shared__ double ws[(BJ_WIN / BS) * T];
    __shared__ uint8_t ls[BJ_WIN];
    __shared__ double sm[BJ_WIN / 32];
    const double alpha = S->alpha;
    double ss = 0.0;
    const int64_t nwin = (n + BJ_WIN - 1) / BJ_WIN;
    for (int64_t w = blockIdx.x; w < nwin; w += gridDim.x) {
        const int64_t i = w * BJ_WIN + threadIdx.x;
        double si = 0.0;
        if (i < n) {
            si = r[i] - alpha * v[i];
            s[i] = si;
            ss += si * si;
        }
        rs[threadIdx.x] = si;
        bj_stage<double, BS>(B, w, n, ws, ls);
        __syncthreads();
        bj_window<double, double, BS>(rs, ls, ws, zs, i < n);
        __syncthreads();
        if (i < n) sh[i] = zs[threadIdx.x];
        __syncthreads();
    }
    const double a = block_sum<BJ_WIN>(ss, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
    if (arrive_last(&S->ticket)) {
        const double t = sum_partials(partials, gridDim.x, 1, 0, sm);
        if (threadIdx.x == 0) bi_s_decide(t, S);
    }
}

// x += alpha ph + omega sh, r = s - omega t, rho' = r^.r, ||r||^2 and the
// step's decision; after an early stop on s only x += alpha ph.
__global__ void __launch_bounds__(NT) k_bi_x(int64_t n, double *__restrict__ x, double *__restrict__ r,
                                             const double *__restrict__ ph, const double *__restrict__ sh,
                                             const double *__restrict__ s, const double *__restrict__ t,
                                             const double *__restrict__ rh, double *partials, PcgScal *S) {
    if (S->done) return;
    __shared__ double sm[NT / 32];
    const double alpha = S->alpha, omega = S->omega;
    const bool early = S->early != 0;
    double rho = 0.0, rr = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        if (early) {
            x[i] += alpha * ph[i];
        } else {
            x[i] += alpha * ph[i] + omega * sh[i];
            const double ri = s[i] - omega * t[i];
            r[i] = ri;
            rho += rh[i] * ri;
            rr += ri * ri;
        }
    }
    const double a = early ? 0.0 : block_sum<NT>(rho, sm);
    const double b = early ? 0.0 : block_sum<NT>(rr, sm);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
    if (arrive_last(&S->ticket)) {
        const double rho_t = early ? 0.0 : sum_partials(partials, gridDim.x, 2, 0, sm);
        const double rr_t = early ? 0.0 : sum_partials(partials, gridDim.x, 2, 1, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            if (early) {
                stop(S, ST_CONV);
            } else {
                S->rr = rr_t;
                if (!isfinite(rr_t) || !isfinite(rho_t)) { S->brk = 4; stop(S, ST_BREAK); }
                else if (rr_t <= S->thresh) stop(S, ST_CONV);
                else if (S->it >= S->maxit) stop(S, ST_MAXIT);
                else if (rho_t == 0.0) { S->brk = 4; stop(S, ST_BREAK); }
                else if (S->omega == 0.0 || !isfinite(S->omega)) { S->brk = 5; stop(S, ST_BREAK); }
                else {
                    S->rho0 = S->rho;
                    S->rho = rho_t;
                }
            }
        }
    }
}

// (re)start: r^ = r, p = v = 0, rho = r.r, rho0 = alpha = omega = 1
__global__ void __launch_bounds__(NT) k_bi_start(int64_t n, const double *__restrict__ r, double *__restrict__ rh,
                                                 double *__restrict__ p, double *__restrict__ v, double *partials,
                                                 PcgScal *S) {
    __shared__ double sm[NT / 32];
    double rho = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const double ri = r[i];
        rh[i] = ri;
        p[i] = 0.0;
        v[i] = 0.0;
        rho += ri * ri;
    }
    const double a = block_sum<NT>(rho, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
    if (arrive_last(&S->ticket)) {
        const double t = sum_partials(partials, gridDim.x, 1, 0, sm);
        if (threadIdx.x == 0) {
            S->ticket = 0;
            S->rho = t;
            S->rho0 = 1.0;
            S->alpha = 1.0;
            S->omega = 1.0;
            S->early = 0;
            S->brk = 0;
            S->done = 0;
            S->status = ST_RUN;
            if (!(t > 0.0)) { S->done = 1; S->status = t == 0.0 ? ST_CONV : ST_BREAK; }
        }
    }
}

}  // namespace gb
