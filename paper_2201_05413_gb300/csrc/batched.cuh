// batched.cuh -- kernels and host helpers shared by pcg_solve_batched and the
// serving engine: k independent Jacobi-PCG recurrences per system, many
// systems per launch (see batched.cu for the decomposition).
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "pcg.cuh"

namespace gb {

constexpr int KMAX = 32;

struct ColState {  // per-column scalars of one system, arrays of length k
    double *rho, *pq, *alpha, *beta, *rr, *bb, *thresh, *scale;
    double *pz, *target;  // reliable updates: z-coefficient of the restored p; fp32 residual floor
    long long *it;
    int *done, *status;
};

struct BSys {
    SellView A;
    const void *val;  // matrix values of the recurrence's precision
    void *X, *R, *P, *Q;  // permuted row-major n x k (element type of the recurrence)
    const double *B64;    // permuted right-hand side (fp64)
    double *X64, *R64;    // fp64 solution / residual (refinement and fp64 solves)
    ColState c;
    int k, kw;
    int unit0, nunits;
    int64_t rows_per_unit;
    unsigned int ticket;
    int active;  // columns still iterating
};

struct BGlobal {
    long long maxit;
    int active_systems;
    int done;
    int use_cond;
    int stop_req;        // a stop requested during this iteration (applied at its end)
    int stop_on_retire;  // stop the loop as soon as any system retires (serving)
    int budget;          // iterations left in this launch sequence; < 0 = unlimited
    unsigned int ticket; // end-of-iteration counter of k_bpupdate
    cudaGraphConditionalHandle cond;
};

__device__ __forceinline__ void bstop_all(BGlobal *G) {
    G->done = 1;
    if (G->use_cond) cudaGraphSetConditional(G->cond, 0);
}

// system's last block: count active columns; a system whose columns are all
// frozen retires, and the loop is asked to stop at the end of this iteration
// when it was the last one (or when the caller wants to see every retirement)
__device__ __forceinline__ void retire_if_idle(BSys &S, BGlobal *G) {
    int a = 0;
    for (int j = 0; j < S.k; ++j) a += S.c.done[j] ? 0 : 1;
    if (S.active > 0 && a == 0) {
        const int left = atomicSub(&G->active_systems, 1) - 1;
        if (left == 0 || G->stop_on_retire) G->stop_req = 1;
    }
    S.active = a;
}

__device__ __forceinline__ bool sys_arrive_last(unsigned int *ticket, int nunits) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned)nunits - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// per-column block reduction: smem[NT] holds one value per thread; column j
// sums the groups' entries in group order.  Result in threads j < kw.
__device__ __forceinline__ double col_block_sum(double v, double *smem, int kw) {
    __syncthreads();
    smem[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < (unsigned)kw)
        for (int g = 0; g < NT / kw; ++g) s += smem[g * kw + threadIdx.x];
    return s;
}

// deterministic per-column sum of a system's unit partials
__device__ __forceinline__ double col_unit_sum(const double *partials, int unit0, int nunits, int j, int slot) {
    double s = 0.0;
    for (int u = 0; u < nunits; ++u) s += __ldcg(partials + ((size_t)(unit0 + u) * 2 + slot) * KMAX + j);
    return s;
}

template <class T> __device__ __forceinline__ float ldv(const T *p);
template <> __device__ __forceinline__ float ldv<float>(const float *p) { return __ldcs(p); }
template <> __device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16 *p) { return ld_val(p); }

template <class TX, class TV>
__device__ __forceinline__ TX ldval_as(const TV *p) {
    if constexpr (sizeof(TV) == 8) return (TX)__ldcs((const double *)p);
    else return (TX)ldv<TV>(p);
}

// ---------------------------------------------------------------- SpMM --
template <class TX, class TV>
__global__ void __launch_bounds__(NT) k_bspmm(BSys *sys, const int *unit_sys, BGlobal *G, double *partials) {
    if (G->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && G->use_cond) cudaGraphSetConditional(G->cond, 0);
        return;
    }
    __shared__ double sm[NT];
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    if (S.active == 0) return;
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    const bool on = j < k && !S.c.done[j];
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    const TX *P = (const TX *)S.P;
    TX *Q = (TX *)S.Q;
    const TV *val = (const TV *)S.val;
    const int C = S.A.C;
    TX dot = TX(0);
    if (on) {
        for (int64_t r = r0 + grp; r < r1; r += ngrp) {
            const int64_t c = r / C;
            const int L = S.A.row_len[r];
            const int64_t base = S.A.chunk_ptr[c] + (r - c * C);
            TX acc = TX(0);
            int jj = 0;
            for (; jj + 4 <= L; jj += 4) {
                const int64_t b0 = base + (int64_t)jj * C;
                const int c0 = __ldg(S.A.col + b0), c1 = __ldg(S.A.col + b0 + C);
                const int c2 = __ldg(S.A.col + b0 + 2 * C), c3 = __ldg(S.A.col + b0 + 3 * C);
                const TX v0 = ldval_as<TX>(val + b0), v1 = ldval_as<TX>(val + b0 + C);
                const TX v2 = ldval_as<TX>(val + b0 + 2 * C), v3 = ldval_as<TX>(val + b0 + 3 * C);
                acc += v0 * P[(int64_t)c0 * k + j];
                acc += v1 * P[(int64_t)c1 * k + j];
                acc += v2 * P[(int64_t)c2 * k + j];
                acc += v3 * P[(int64_t)c3 * k + j];
            }
            for (; jj < L; ++jj) {
                const int64_t b0 = base + (int64_t)jj * C;
                acc += ldval_as<TX>(val + b0) * P[(int64_t)__ldg(S.A.col + b0) * k + j];
            }
            Q[r * k + j] = acc;
            dot += P[r * k + j] * acc;
        }
    }
    const double t = col_block_sum((double)dot, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 2) * KMAX + threadIdx.x] = t;
    if (sys_arrive_last(&S.ticket, S.nunits)) {
        if (threadIdx.x < (unsigned)k && !S.c.done[threadIdx.x]) {
            const int jj = threadIdx.x;
            const double pq = col_unit_sum(partials, S.unit0, S.nunits, jj, 0);
            S.c.pq[jj] = pq;
            if (!(pq > 0.0) || !isfinite(pq)) { S.c.status[jj] = ST_BREAK; S.c.done[jj] = 1; }
            else S.c.alpha[jj] = S.c.rho[jj] / pq;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.ticket = 0;
            retire_if_idle(S, G);
        }
    }
}

// --------------------------------------------------------------- update --
template <class TX>
__global__ void __launch_bounds__(NT) k_bupdate(BSys *sys, const int *unit_sys, BGlobal *G, double *partials) {
    if (G->done) return;
    __shared__ double sm[NT];
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    if (S.active == 0) return;
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    const bool on = j < k && !S.c.done[j];
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    TX *X = (TX *)S.X, *R = (TX *)S.R;
    const TX *P = (const TX *)S.P, *Q = (const TX *)S.Q;
    const bool f64 = sizeof(TX) == 8;
    TX rz = TX(0), rr = TX(0);
    if (on) {
        const TX alpha = (TX)S.c.alpha[j];
        for (int64_t r = r0 + grp; r < r1; r += ngrp) {
            const int64_t e = r * k + j;
            const TX d = f64 ? (TX)S.A.dinv[r] : (TX)S.A.dinv32[r];
            const TX xi = X[e] + alpha * P[e];
            const TX ri = R[e] - alpha * Q[e];
            X[e] = xi;
            R[e] = ri;
            rz += ri * (d * ri);
            rr += ri * ri;
        }
    }
    const double a = col_block_sum((double)rz, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 2) * KMAX + threadIdx.x] = a;
    const double b = col_block_sum((double)rr, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 2 + 1) * KMAX + threadIdx.x] = b;
    if (sys_arrive_last(&S.ticket, S.nunits)) {
        if (threadIdx.x < (unsigned)k && !S.c.done[threadIdx.x]) {
            const int jj = threadIdx.x;
            const double rz_t = col_unit_sum(partials, S.unit0, S.nunits, jj, 0);
            const double rr_t = col_unit_sum(partials, S.unit0, S.nunits, jj, 1);
            S.c.it[jj] += 1;
            S.c.rr[jj] = rr_t;
            if (!isfinite(rz_t) || !isfinite(rr_t)) { S.c.status[jj] = ST_BREAK; S.c.done[jj] = 1; }
            else if (rr_t <= S.c.thresh[jj]) { S.c.status[jj] = ST_CONV; S.c.done[jj] = 1; }
            else if (S.c.it[jj] >= G->maxit) { S.c.status[jj] = ST_MAXIT; S.c.done[jj] = 1; }
            else {
                S.c.beta[jj] = rz_t / S.c.rho[jj];
                S.c.rho[jj] = rz_t;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.ticket = 0;
            retire_if_idle(S, G);
        }
    }
}

// P = D^-1 R + beta P for the active columns; the block that ends the
// iteration last applies a pending stop (retirement, budget, all done), so a
// loop only ever stops between complete iterations.
template <class TX>
__global__ void __launch_bounds__(NT) k_bpupdate(BSys *sys, const int *unit_sys, BGlobal *G) {
    if (G->done) return;
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    if (S.active != 0 && j < k && !S.c.done[j]) {
        const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
        const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
        TX *P = (TX *)S.P;
        const TX *R = (const TX *)S.R;
        const TX beta = (TX)S.c.beta[j];
        const bool f64 = sizeof(TX) == 8;
        for (int64_t r = r0 + grp; r < r1; r += ngrp) {
            const int64_t e = r * k + j;
            const TX d = f64 ? (TX)S.A.dinv[r] : (TX)S.A.dinv32[r];
            P[e] = d * R[e] + beta * P[e];
        }
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&G->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        G->ticket = 0;
        if (G->budget > 0) G->budget -= 1;
        if (G->stop_req || G->budget == 0 || G->active_systems <= 0) bstop_all(G);
    }
}

// ------------------------------------------------------ start / residual --
// P = D^-1 R, rho_j = R_j.Z_j for the columns selected by `mask` (restart),
// and every other column left as it is.
template <class TX>
__global__ void __launch_bounds__(NT) k_bstart(BSys *sys, const int *unit_sys, double *partials, const int *mask) {
    __shared__ double sm[NT];
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    const bool on = j < k && mask[s * KMAX + j];
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    TX *P = (TX *)S.P;
    const TX *R = (const TX *)S.R;
    const bool f64 = sizeof(TX) == 8;
    double rz = 0.0;
    if (on)
        for (int64_t r = r0 + grp; r < r1; r += ngrp) {
            const int64_t e = r * k + j;
            const TX d = f64 ? (TX)S.A.dinv[r] : (TX)S.A.dinv32[r];
            const TX z = d * R[e];
            P[e] = z;
            rz += (double)(R[e] * z);
        }
    const double a = col_block_sum(rz, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 2) * KMAX + threadIdx.x] = a;
    if (sys_arrive_last(&S.ticket, S.nunits)) {
        if (threadIdx.x < (unsigned)k) {
            const int jj = threadIdx.x;
            if (mask[s * KMAX + jj]) {
                const double t = col_unit_sum(partials, S.unit0, S.nunits, jj, 0);
                S.c.rho[jj] = t;
                S.c.done[jj] = 0;
                S.c.status[jj] = ST_RUN;
                if (!(t > 0.0)) { S.c.done[jj] = 1; S.c.status[jj] = t == 0.0 ? ST_CONV : ST_BREAK; }
            } else {
                S.c.done[jj] = 1;  // not part of this loop
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.ticket = 0;
            int a2 = 0;
            for (int q = 0; q < k; ++q) a2 += S.c.done[q] ? 0 : 1;
            S.active = a2;
        }
    }
}

// R64 = B - A X64 (fp64) per column with ||R_j||^2 (and ||B_j||^2, threshold
// when init).  Skips the product when X64 is known to be zero.
static __global__ void __launch_bounds__(NT) k_bresid(BSys *sys, const int *unit_sys, double *partials, int init,
                                               int x_zero, double tol) {
    __shared__ double sm[NT];
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    const int C = S.A.C;
    double rr = 0.0, bb = 0.0;
    if (j < k)
        for (int64_t r = r0 + grp; r < r1; r += ngrp) {
            double acc = 0.0;
            if (!x_zero) {
                const int64_t c = r / C;
                const int L = S.A.row_len[r];
                const int64_t base = S.A.chunk_ptr[c] + (r - c * C);
                for (int jj = 0; jj < L; ++jj) {
                    const int64_t b0 = base + (int64_t)jj * C;
                    acc += __ldcs(S.A.val + b0) * S.X64[(int64_t)__ldg(S.A.col + b0) * k + j];
                }
            }
            const double bi = S.B64[r * k + j];
            const double ri = bi - acc;
            S.R64[r * k + j] = ri;
            rr += ri * ri;
            bb += bi * bi;
        }
    const double a = col_block_sum(rr, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 2) * KMAX + threadIdx.x] = a;
    const double b = col_block_sum(bb, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 2 + 1) * KMAX + threadIdx.x] = b;
    if (sys_arrive_last(&S.ticket, S.nunits)) {
        if (threadIdx.x < (unsigned)k) {
            const int jj = threadIdx.x;
            S.c.rr[jj] = col_unit_sum(partials, S.unit0, S.nunits, jj, 0);
            if (init) {
                const double bt = col_unit_sum(partials, S.unit0, S.nunits, jj, 1);
                S.c.bb[jj] = bt;
                S.c.thresh[jj] = tol * tol * bt;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) S.ticket = 0;
    }
}

// refinement helpers (fp32 recurrences): R32 = R64 / ||R64_j||, D32 = 0 for
// the masked columns; X64 += ||R64_j|| D32 for the masked columns.
static __global__ void k_bscale_down(BSys *sys, const int *unit_sys, const int *mask) {
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    if (!(j < k) || !mask[s * KMAX + j]) return;
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    const double sc = 1.0 / S.c.scale[j];
    float *R = (float *)S.R, *X = (float *)S.X;
    for (int64_t r = r0 + grp; r < r1; r += ngrp) {
        const int64_t e = r * k + j;
        R[e] = (float)(sc * S.R64[e]);
        X[e] = 0.0f;
    }
}
static __global__ void k_bcorrect(BSys *sys, const int *unit_sys, const int *mask) {
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    if (!(j < k) || !mask[s * KMAX + j]) return;
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    const double sc = S.c.scale[j];
    const float *X = (const float *)S.X;
    for (int64_t r = r0 + grp; r < r1; r += ngrp) {
        const int64_t e = r * k + j;
        S.X64[e] += sc * (double)X[e];
    }
}

// Reliable update, batched: for the masked columns (mask 1: keep and restore
// p, mask 2: fresh start p = z) R32 = (float) R64, D32 = 0 and fp64 sums of
// R.D^-1 R, ||R||^2, R.P; the system's last block sets beta and the
// z-coefficient of the restored direction, rho, rr, and the next inner
// threshold max(delta^2 ||r||^2, target), and re-arms the columns.
static __global__ void __launch_bounds__(NT) k_breplace(BSys *sys, const int *unit_sys, double *partials,
                                                         const int *mask, double delta2) {
    __shared__ double sm[NT];
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    const int m = j < k ? mask[s * KMAX + j] : 0;
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    float *R = (float *)S.R, *X = (float *)S.X;
    const float *P = (const float *)S.P;
    double rz = 0.0, rr = 0.0, rp = 0.0;
    if (m)
        for (int64_t r = r0 + grp; r < r1; r += ngrp) {
            const int64_t e = r * k + j;
            const float ri = (float)S.R64[e];
            R[e] = ri;
            X[e] = 0.0f;
            rz += (double)(ri * (S.A.dinv32[r] * ri));
            rr += (double)ri * (double)ri;
            if (m == 1) rp += (double)ri * (double)P[e];
        }
    const double a = col_block_sum(rz, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 3) * KMAX + threadIdx.x] = a;
    const double b = col_block_sum(rr, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 3 + 1) * KMAX + threadIdx.x] = b;
    const double c = col_block_sum(rp, sm, kw);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 3 + 2) * KMAX + threadIdx.x] = c;
    if (sys_arrive_last(&S.ticket, S.nunits)) {
        if (threadIdx.x < (unsigned)k) {
            const int jj = threadIdx.x;
            const int mm = mask[s * KMAX + jj];
            if (mm) {
                double rz_t = 0.0, rr_t = 0.0, rp_t = 0.0;
                for (int u = 0; u < S.nunits; ++u) {
                    const size_t base = (size_t)(S.unit0 + u) * 3;
                    rz_t += __ldcg(partials + (base + 0) * KMAX + jj);
                    rr_t += __ldcg(partials + (base + 1) * KMAX + jj);
                    rp_t += __ldcg(partials + (base + 2) * KMAX + jj);
                }
                if (mm == 1 && rz_t > 0.0 && S.c.rho[jj] > 0.0) {
                    const double beta = rz_t / S.c.rho[jj];
                    S.c.beta[jj] = beta;
                    S.c.pz[jj] = 1.0 - beta * (rp_t / rz_t);
                } else {
                    S.c.beta[jj] = 0.0;
                    S.c.pz[jj] = 1.0;
                }
                S.c.rho[jj] = rz_t;
                S.c.rr[jj] = rr_t;
                S.c.thresh[jj] = fmax(delta2 * rr_t, S.c.target[jj]);
                S.c.done[jj] = 0;
                S.c.status[jj] = ST_RUN;
                if (!(rz_t > 0.0)) { S.c.done[jj] = 1; S.c.status[jj] = rz_t == 0.0 ? ST_CONV : ST_BREAK; }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.ticket = 0;
            int a2 = 0;
            for (int q = 0; q < k; ++q) a2 += S.c.done[q] ? 0 : 1;
            S.active = a2;
        }
    }
}

// P = pz D^-1 R + beta P for the masked columns (mask 1), P = D^-1 R for a
// fresh start (mask 2); fp32 recurrences
static __global__ void k_breplace_p(BSys *sys, const int *unit_sys, const int *mask) {
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    if (!(j < k) || !mask[s * KMAX + j] || S.c.done[j]) return;
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    const float pz = (float)S.c.pz[j], beta = (float)S.c.beta[j];
    float *P = (float *)S.P;
    const float *R = (const float *)S.R;
    if (mask[s * KMAX + j] == 2) {  // fresh start: P = z (never 0 * P: P may hold stale bits)
        for (int64_t r = r0 + grp; r < r1; r += ngrp) P[r * k + j] = S.A.dinv32[r] * R[r * k + j];
        return;
    }
    for (int64_t r = r0 + grp; r < r1; r += ngrp) {
        const int64_t e = r * k + j;
        P[e] = pz * (S.A.dinv32[r] * R[e]) + beta * P[e];
    }
}

static __global__ void k_gather_rows(int64_t n, int k, const int32_t *perm, const double *src, double *dst) {
    const int64_t tot = n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / k;
        const int j = (int)(t - r * k);
        dst[t] = src ? src[(int64_t)perm[r] * k + j] : 0.0;
    }
}
static __global__ void k_scatter_rows(int64_t n, int k, const int32_t *perm, const double *src, double *dst) {
    const int64_t tot = n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / k;
        const int j = (int)(t - r * k);
        dst[(int64_t)perm[r] * k + j] = src[t];
    }
}

// ----------------------------------------------------------------- host --
struct Batch {
    Mem mem;
    std::vector<BSys> h;
    BSys *d_sys = nullptr;
    int *d_unit_sys = nullptr, *d_mask = nullptr;
    BGlobal *d_G = nullptr;
    double *partials = nullptr;
    std::vector<void *> owned;
    int units = 0;
    template <class T> int take(T **p, size_t n) {
        int rc = mem.alloc_n(p, n);
        if (rc == GB_OK) owned.push_back((void *)*p);
        return rc;
    }
    ~Batch() {
        for (void *p : owned) mem.release(p);
    }
};

static int kw_of(int k) {
    int w = 1;
    while (w < k) w <<= 1;
    return w;
}

template <class TX, class TV>
static void enqueue_biter(Batch &b, cudaStream_t s) {
    ::gb::count_launches(1); k_bspmm<TX, TV><<<b.units, NT, 0, s>>>(b.d_sys, b.d_unit_sys, b.d_G, b.partials);
    ::gb::count_launches(1); k_bupdate<TX><<<b.units, NT, 0, s>>>(b.d_sys, b.d_unit_sys, b.d_G, b.partials);
    ::gb::count_launches(1); k_bpupdate<TX><<<b.units, NT, 0, s>>>(b.d_sys, b.d_unit_sys, b.d_G);
}

// Runs the batched loop until every system is retired (graph while-node, or
// direct launches polled every `chunk` iterations).
template <class F>
static int run_bloop(cudaStream_t st, BGlobal *dG, bool use_graph, int chunk, F &&enqueue) {
    if (use_graph) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaStream_t cap = nullptr;
        cudaGraphConditionalHandle h = 0;
        int rc = GB_OK;
        GB_CHECK_CUDA(cudaGraphCreate(&g, 0));
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
            e = cudaStreamBeginCaptureToGraph(cap, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                set_capturing(true);
                enqueue(cap);
                set_capturing(false);
                cudaGraph_t outg = nullptr;
                e = cudaStreamEndCapture(cap, &outg);
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (e == cudaSuccess) {
            struct { int use; cudaGraphConditionalHandle h; } hs{1, h};
            e = cudaMemcpyAsync(&dG->use_cond, &hs.use, sizeof(int), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&dG->cond, &hs.h, sizeof(h), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
            int zero = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&dG->use_cond, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
        if (e != cudaSuccess) { set_error("batched loop graph: %s", cudaGetErrorString(e)); rc = GB_ECUDA; }
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (cap) cudaStreamDestroy(cap);
        return rc;
    }
    for (;;) {
        for (int i = 0; i < chunk; ++i) enqueue(st);
        int done = 0;
        GB_CHECK_CUDA(cudaGetLastError());
        GB_CHECK_CUDA(cudaMemcpyAsync(&done, &dG->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
        if (done) return GB_OK;
    }
}

// host copy of every system's column state
struct HostCols {
    std::vector<std::vector<double>> rr, bb;
    std::vector<std::vector<long long>> it;
    std::vector<std::vector<int>> done, status;
};

static int pull_cols(Batch &b, HostCols &hc, cudaStream_t st) {
    const size_t ns = b.h.size();
    hc.rr.resize(ns); hc.bb.resize(ns); hc.it.resize(ns); hc.done.resize(ns); hc.status.resize(ns);
    for (size_t s = 0; s < ns; ++s) {
        const int k = b.h[s].k;
        hc.rr[s].resize(k); hc.bb[s].resize(k); hc.it[s].resize(k); hc.done[s].resize(k); hc.status[s].resize(k);
        GB_CHECK_CUDA(cudaMemcpyAsync(hc.rr[s].data(), b.h[s].c.rr, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(hc.bb[s].data(), b.h[s].c.bb, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(hc.it[s].data(), b.h[s].c.it, sizeof(long long) * k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(hc.done[s].data(), b.h[s].c.done, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(hc.status[s].data(), b.h[s].c.status, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
    }
    GB_CHECK_CUDA(cudaStreamSynchronize(st));
    return GB_OK;
}

// Starts the recurrences of the masked columns (P = D^-1 R, rho) and launches
// the loop until all of them stop.  Returns after the loop.
template <class TX, class TV>
static int start_and_loop(Batch &b, const std::vector<int> &mask, long long maxit, const PcgOptions &o,
                          cudaStream_t st) {
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
    ::gb::count_launches(1); k_bstart<TX><<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, b.d_mask);
    GB_CHECK_CUDA(cudaGetLastError());
    // count systems with an active column
    std::vector<BSys> hs(b.h.size());
    GB_CHECK_CUDA(cudaMemcpyAsync(hs.data(), b.d_sys, sizeof(BSys) * hs.size(), cudaMemcpyDeviceToHost, st));
    GB_CHECK_CUDA(cudaStreamSynchronize(st));
    int act = 0;
    for (auto &x : hs) act += x.active > 0 ? 1 : 0;
    if (act == 0) return GB_OK;
    BGlobal g{};
    g.maxit = maxit;
    g.active_systems = act;
    g.budget = -1;
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_G, &g, sizeof(g), cudaMemcpyHostToDevice, st));
    GB_TRY(run_bloop(st, b.d_G, o.use_graph != 0, o.check_every, [&](cudaStream_t s) { enqueue_biter<TX, TV>(b, s); }));
    return GB_OK;
}

}  // namespace gb
