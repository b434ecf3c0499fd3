// batched.cuh -- kernels and host helpers shared by pcg_solve_batched and the
// serving engine: k independent Jacobi-PCG recurrences per system, many
// systems per launch (see batched.cu for the decomposition).
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "bsys.cuh"
#include "bspmm_tma.cuh"
#include "bpersist.cuh"

namespace gb {

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

template <class T> __device__ __forceinline__ float ldv(const T *p);
template <> __device__ __forceinline__ float ldv<float>(const float *p) { return __ldcs(p); }
template <> __device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16 *p) { return ld_val(p); }

template <class TX, class TV>
__device__ __forceinline__ TX ldval_as(const TV *p) {
    if constexpr (sizeof(TV) == 8) return (TX)__ldcs((const double *)p);
    else return (TX)ldv<TV>(p);
}

// ---------------------------------------------------------------- SpMM --
// Q = A P for the active columns.  A group of lanes owns one row; lane l of
// the group owns VW consecutive columns (VW = 4 fp32 / 2 fp64 when k allows
// 16-byte row segments, else 1), so one gather P[col][VW l .. VW l + VW) is one
// vector load feeding VW FMAs.  The group's lanes load as many of the row's
// entries at once, broadcast them within the group with shuffles and issue
// the gathers back to back, so the index load is off the gathers' critical
// path.  Warps process 32/group rows side by side.
template <class TX, int VW> struct VecN;
template <> struct VecN<double, 1> { using T = double; };
template <> struct VecN<double, 2> { using T = double2; };
template <> struct VecN<float, 1> { using T = float; };
template <> struct VecN<float, 2> { using T = float2; };
template <> struct VecN<float, 4> { using T = float4; };

template <class V> __device__ __forceinline__ void vfma(V &acc, float v, const V &p);
template <> __device__ __forceinline__ void vfma<float>(float &a, float v, const float &p) { a += v * p; }
template <> __device__ __forceinline__ void vfma<float2>(float2 &a, float v, const float2 &p) { a.x += v * p.x; a.y += v * p.y; }
template <> __device__ __forceinline__ void vfma<float4>(float4 &a, float v, const float4 &p) {
    a.x += v * p.x; a.y += v * p.y; a.z += v * p.z; a.w += v * p.w;
}
__device__ __forceinline__ void vfmad(double &a, double v, const double &p) { a += v * p; }
__device__ __forceinline__ void vfmad(double2 &a, double v, const double2 &p) { a.x += v * p.x; a.y += v * p.y; }
template <class V, class TX> __device__ __forceinline__ void vfma_any(V &a, TX v, const V &p) {
    if constexpr (sizeof(TX) == 8) vfmad(a, v, p); else vfma<V>(a, v, p);
}
template <class V> __device__ __forceinline__ V vzero() { V v; memset(&v, 0, sizeof(V)); return v; }
template <class V, class TX> __device__ __forceinline__ TX vdot(const V &a, const V &b) {
    const TX *x = reinterpret_cast<const TX *>(&a), *y = reinterpret_cast<const TX *>(&b);
    TX t = TX(0);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(V) / sizeof(TX)); ++i) t += x[i] * y[i];
    return t;
}

// columns per lane for a system: the widest of 4 (fp32) / 2 (fp64) that divides k
template <class TX> __host__ __device__ __forceinline__ int vec_width(int k) {
    if (sizeof(TX) == 4) return (k % 4 == 0) ? 4 : ((k % 2 == 0) ? 2 : 1);
    return (k % 2 == 0) ? 2 : 1;
}

template <class TX, class TV, int VW>
__device__ __forceinline__ void bspmm_rows(BSys &S, int unit, int k, TX *colsum /* per-lane dot partials, VW */) {
    using V = typename VecN<TX, VW>::T;
    const int kv = k / VW;                 // vector columns
    int gw = 1;
    while (gw < kv) gw <<= 1;              // lanes per row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int jv = lane % gw, grp = lane / gw, gpw = 32 / gw;
    TX ccomp[VW];
#pragma unroll
    for (int u = 0; u < VW; ++u) ccomp[u] = TX(0);
    bool on = jv < kv;
    if (on) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < VW; ++u) any |= !S.c.done[jv * VW + u];
        on = any;
    }
    const int64_t r0 = (int64_t)(unit - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    const V *P = reinterpret_cast<const V *>(S.P);
    V *Q = reinterpret_cast<V *>(S.Q);
    const TV *val = (const TV *)S.val;
    const int C = S.A.C;
    for (int64_t rb = r0 + (int64_t)warp * gpw; rb < r1; rb += (int64_t)(NT / 32) * gpw) {
        const int64_t r = rb + grp;
        const bool rv = r < r1;
        const int L = rv ? S.A.row_len[r] : 0;
        const int64_t c = rv ? r / C : 0;
        const int64_t base = rv ? S.A.chunk_ptr[c] + (r - c * C) : 0;
        const int Lmax = __reduce_max_sync(0xffffffffu, L);
        V acc = vzero<V>();
        constexpr int PRE = 4;  // entries each lane holds: one round trip for rows up to PRE*gw long
        for (int e0 = 0; e0 < Lmax; e0 += PRE * gw) {
            int mycol[PRE];
            TX myval[PRE];
#pragma unroll
            for (int q = 0; q < PRE; ++q) {
                const int e = e0 + q * gw + jv;
                mycol[q] = 0;
                myval[q] = TX(0);
                if (e < L) {
                    mycol[q] = __ldg(S.A.col + base + (int64_t)e * C);
                    myval[q] = ldval_as<TX>(val + base + (int64_t)e * C);
                }
            }
#pragma unroll
            for (int q = 0; q < PRE; ++q) {
                const int eq = e0 + q * gw;
                if (eq >= Lmax) break;
                const int nb = min(gw, Lmax - eq);
#pragma unroll 8
                for (int ee = 0; ee < nb; ++ee) {
                    const int src = grp * gw + ee;
                    const int cc = __shfl_sync(0xffffffffu, mycol[q], src);
                    const TX vv = __shfl_sync(0xffffffffu, myval[q], src);
                    if (on && eq + ee < L) vfma_any<V, TX>(acc, vv, P[(int64_t)cc * kv + jv]);
                }
            }
        }
        if (rv && on) {
            Q[r * kv + jv] = acc;
            const V pr = P[r * kv + jv];
            const TX *a = reinterpret_cast<const TX *>(&acc), *b = reinterpret_cast<const TX *>(&pr);
#pragma unroll
            for (int u = 0; u < VW; ++u) kadd(colsum[u], ccomp[u], a[u] * b[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < VW; ++u) colsum[u] -= ccomp[u];
}

// Per-column block sums of lane partials (lane jv = lane % gw owns columns
// jv*VW .. jv*VW+VW-1): an xor tree over the lanes of a column inside each warp
// in the recurrence's precision, then the warps in order in fp64.  Fixed
// order: deterministic.  All threads call; valid in threads j < k.
template <class TX, int VW>
__device__ __forceinline__ double col_tree_sum(TX (&v)[VW], int k, double *csum /* NT/32 x KMAX */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kv = k / VW;
    int gw = 1;
    while (gw < kv) gw <<= 1;
    for (int o = gw; o < 32; o <<= 1)
#pragma unroll
        for (int u = 0; u < VW; ++u) v[u] += __shfl_xor_sync(0xffffffffu, v[u], o);
    __syncthreads();  // csum may still be read by a previous call
    if (lane < kv)
#pragma unroll
        for (int u = 0; u < VW; ++u) csum[warp * KMAX + lane * VW + u] = (double)v[u];
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < (unsigned)k)
        for (int w = 0; w < NT / 32; ++w) t += csum[w * KMAX + threadIdx.x];
    return t;
}

template <class TX, class TV, int VW>
__device__ __forceinline__ void bspmm_block(BSys &S, int unit, int k, double *partials, double *csum) {
    TX colsum[VW];
#pragma unroll
    for (int u = 0; u < VW; ++u) colsum[u] = TX(0);
    bspmm_rows<TX, TV, VW>(S, unit, k, colsum);
    const double t = col_tree_sum<TX, VW>(colsum, k, csum);
    if (threadIdx.x < (unsigned)k) partials[((size_t)unit * 2) * KMAX + threadIdx.x] = t;
}

// General SpMM (any chunk height): groups of lanes own rows, lanes own VW
// consecutive columns; over the units [unit_base, unit_base + gridDim.x).
template <class TX, class TV>
__global__ void __launch_bounds__(NT, 4) k_bspmm(BSys *sys, const int *unit_sys, int unit_base, BGlobal *G,
                                                 double *partials) {
    if (G->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && G->use_cond) cudaGraphSetConditional(G->cond, 0);
        return;
    }
    __shared__ double sm[NT];
    __shared__ double csum[NT / 32 * KMAX];  // per warp, per column
    const int unit = unit_base + blockIdx.x;
    const int s = unit_sys[unit];
    BSys &S = sys[s];
    if (S.active == 0) return;
    const int k = S.k, kw = S.kw;
    const int VW = vec_width<TX>(k);
    if (VW == 4) bspmm_block<TX, TV, (sizeof(TX) == 4 ? 4 : 2)>(S, unit, k, partials, csum);
    else if (VW == 2) bspmm_block<TX, TV, 2>(S, unit, k, partials, csum);
    else bspmm_block<TX, TV, 1>(S, unit, k, partials, csum);
    if (sys_arrive_last(&S.ticket, S.nunits)) {
        const double pq = col_unit_sum_block(partials, S.unit0, S.nunits, 0, 2, kw, sm);
        if (threadIdx.x < (unsigned)k && !S.c.done[threadIdx.x]) {
            const int jj = threadIdx.x;
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
// X += alpha P, R -= alpha Q per active column, with the fp64 partial sums of
// R.D^-1 R and R.R; lanes own VW consecutive columns of a row (vector loads),
// groups of lanes own rows.  The system's last block reduces in a fixed order.
template <class TX, int VW>
__device__ __forceinline__ void bupdate_rows(BSys &S, int k, TX (&rz)[VW], TX (&rr)[VW]) {
    // per-lane partial sums in the recurrence's precision (zero on entry)
    using V = typename VecN<TX, VW>::T;
    const int kv = k / VW;
    int gw = 1;
    while (gw < kv) gw <<= 1;
    const int jv = (threadIdx.x & 31) % gw, grp = threadIdx.x / gw, ngrp = NT / gw;
    if (jv >= kv) return;
    TX cz[VW], cr[VW];  // compensation of rz, rr (kadd)
#pragma unroll
    for (int u = 0; u < VW; ++u) { cz[u] = TX(0); cr[u] = TX(0); }
    TX alpha[VW];
    bool on[VW];
    bool any = false;
#pragma unroll
    for (int u = 0; u < VW; ++u) {
        on[u] = !S.c.done[jv * VW + u];
        alpha[u] = on[u] ? (TX)S.c.alpha[jv * VW + u] : TX(0);
        any |= on[u];
    }
    if (!any) return;
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    V *X = reinterpret_cast<V *>(S.X), *R = reinterpret_cast<V *>(S.R);
    const V *P = reinterpret_cast<const V *>(S.P), *Q = reinterpret_cast<const V *>(S.Q);
    const bool f64 = sizeof(TX) == 8;
    constexpr int RU4 = sizeof(V) >= 8 ? 2 : 4;  // rows in flight per thread
    for (int64_t rb = r0 + grp; rb < r1; rb += (int64_t)RU4 * ngrp) {
        V xv[RU4], rv[RU4], pv[RU4], qv[RU4];
        TX dd[RU4];
#pragma unroll
        for (int t = 0; t < RU4; ++t) {
            const int64_t r = rb + (int64_t)t * ngrp;
            if (r < r1) {
                const int64_t e = r * kv + jv;
                dd[t] = f64 ? (TX)S.A.dinv[r] : (TX)S.A.dinv32[r];
                xv[t] = X[e]; rv[t] = R[e]; pv[t] = P[e]; qv[t] = Q[e];
            }
        }
#pragma unroll
        for (int t = 0; t < RU4; ++t) {
            const int64_t r = rb + (int64_t)t * ngrp;
            if (r < r1) {
                const int64_t e = r * kv + jv;
                TX *x = reinterpret_cast<TX *>(&xv[t]), *rr_ = reinterpret_cast<TX *>(&rv[t]);
                const TX *pp = reinterpret_cast<const TX *>(&pv[t]), *qq = reinterpret_cast<const TX *>(&qv[t]);
#pragma unroll
                for (int u = 0; u < VW; ++u) {  // frozen columns keep their values (alpha 0)
                    x[u] += alpha[u] * pp[u];
                    rr_[u] -= alpha[u] * qq[u];
                    kadd(rz[u], cz[u], rr_[u] * (dd[t] * rr_[u]));
                    kadd(rr[u], cr[u], rr_[u] * rr_[u]);
                }
                X[e] = xv[t];
                R[e] = rv[t];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < VW; ++u) { rz[u] -= cz[u]; rr[u] -= cr[u]; }
}

template <class TX, int VW>
__device__ __forceinline__ void bupdate_block(BSys &S, int k, double *partials, double *csum) {
    TX rz[VW], rr[VW];
#pragma unroll
    for (int u = 0; u < VW; ++u) { rz[u] = TX(0); rr[u] = TX(0); }
    bupdate_rows<TX, VW>(S, k, rz, rr);
    const double a = col_tree_sum<TX, VW>(rz, k, csum);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 2) * KMAX + threadIdx.x] = a;
    const double b = col_tree_sum<TX, VW>(rr, k, csum);
    if (threadIdx.x < (unsigned)k) partials[((size_t)blockIdx.x * 2 + 1) * KMAX + threadIdx.x] = b;
}

template <class TX>
__global__ void __launch_bounds__(NT, 4) k_bupdate(BSys *sys, const int *unit_sys, BGlobal *G, double *partials) {
    if (G->done) return;
    __shared__ double sm[NT];
    __shared__ double csum[NT / 32 * KMAX];
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    if (S.active == 0) return;
    const int k = S.k, kw = S.kw;
    const int VW = vec_width<TX>(k);
    if (VW == 4) bupdate_block<TX, (sizeof(TX) == 4 ? 4 : 2)>(S, k, partials, csum);
    else if (VW == 2) bupdate_block<TX, 2>(S, k, partials, csum);
    else bupdate_block<TX, 1>(S, k, partials, csum);
    if (sys_arrive_last(&S.ticket, S.nunits)) {
        const double rz_t = col_unit_sum_block(partials, S.unit0, S.nunits, 0, 2, kw, sm);
        const double rr_t = col_unit_sum_block(partials, S.unit0, S.nunits, 1, 2, kw, sm);
        if (threadIdx.x < (unsigned)k && !S.c.done[threadIdx.x]) {
            const int jj = threadIdx.x;
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

template <class TX, int VW>
__device__ __forceinline__ void bpupdate_rows(BSys &S, int k) {
    using V = typename VecN<TX, VW>::T;
    const int kv = k / VW;
    int gw = 1;
    while (gw < kv) gw <<= 1;
    const int jv = (threadIdx.x & 31) % gw, grp = threadIdx.x / gw, ngrp = NT / gw;
    if (jv >= kv) return;
    TX beta[VW];
    bool on[VW];
    bool any = false;
#pragma unroll
    for (int u = 0; u < VW; ++u) {
        on[u] = !S.c.done[jv * VW + u];
        beta[u] = (TX)S.c.beta[jv * VW + u];
        any |= on[u];
    }
    if (!any) return;
    const int64_t r0 = (int64_t)(blockIdx.x - S.unit0) * S.rows_per_unit;
    const int64_t r1 = min(S.A.n, r0 + S.rows_per_unit);
    V *P = reinterpret_cast<V *>(S.P);
    const V *R = reinterpret_cast<const V *>(S.R);
    const bool f64 = sizeof(TX) == 8;
    constexpr int RU4 = 4;  // rows in flight per thread
    for (int64_t rb = r0 + grp; rb < r1; rb += (int64_t)RU4 * ngrp) {
        V pv[RU4], rv[RU4];
        TX dd[RU4];
#pragma unroll
        for (int t = 0; t < RU4; ++t) {
            const int64_t r = rb + (int64_t)t * ngrp;
            if (r < r1) {
                const int64_t e = r * kv + jv;
                dd[t] = f64 ? (TX)S.A.dinv[r] : (TX)S.A.dinv32[r];
                pv[t] = P[e];
                rv[t] = R[e];
            }
        }
#pragma unroll
        for (int t = 0; t < RU4; ++t) {
            const int64_t r = rb + (int64_t)t * ngrp;
            if (r < r1) {
                TX *pp = reinterpret_cast<TX *>(&pv[t]);
                const TX *rp = reinterpret_cast<const TX *>(&rv[t]);
#pragma unroll
                for (int u = 0; u < VW; ++u)
                    if (on[u]) pp[u] = dd[t] * rp[u] + beta[u] * pp[u];
                P[r * kv + jv] = pv[t];
            }
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
    const int k = S.k;
    if (S.active != 0) {
        const int VW = vec_width<TX>(k);
        if (VW == 4) bpupdate_rows<TX, (sizeof(TX) == 4 ? 4 : 2)>(S, k);
        else if (VW == 2) bpupdate_rows<TX, 2>(S, k);
        else bpupdate_rows<TX, 1>(S, k);
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
        const double t = col_unit_sum_block(partials, S.unit0, S.nunits, 0, 2, kw, sm);
        if (threadIdx.x < (unsigned)k) {
            const int jj = threadIdx.x;
            if (mask[s * KMAX + jj]) {
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
        const double rr_t = col_unit_sum_block(partials, S.unit0, S.nunits, 0, 2, kw, sm);
        const double bb_t = col_unit_sum_block(partials, S.unit0, S.nunits, 1, 2, kw, sm);
        if (threadIdx.x < (unsigned)k) {
            const int jj = threadIdx.x;
            S.c.rr[jj] = rr_t;
            if (init) {
                S.c.bb[jj] = bb_t;
                S.c.thresh[jj] = tol * tol * bb_t;
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
        const double rz_t = col_unit_sum_block(partials, S.unit0, S.nunits, 0, 3, kw, sm);
        const double rr_t = col_unit_sum_block(partials, S.unit0, S.nunits, 1, 3, kw, sm);
        const double rp_t = col_unit_sum_block(partials, S.unit0, S.nunits, 2, 3, kw, sm);
        if (threadIdx.x < (unsigned)k) {
            const int jj = threadIdx.x;
            const int mm = mask[s * KMAX + jj];
            if (mm) {
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
    std::vector<int *> grid_err;  // error words of the grid-tier launches
    bool tma = false;  // every system has 32-row chunks: the TMA-streamed SpMM applies
    ClassRanges cls;   // the unit table ordered by width class
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

// Units of a system (one block of the batched kernels each): consecutive
// whole chunks of 32 rows, about 32 chunks per unit, at most 2048 units.  The
// split depends on the system's own size only.
static inline int units_of_rows(int64_t n, int64_t *rows_per_unit) {
    const int64_t chunks = (n + 31) / 32;
    const int64_t units = std::max<int64_t>(1, std::min<int64_t>((chunks + 31) / 32, 2048));
    int64_t cpu = (chunks + units - 1) / units;
    // whole groups of 8 chunks (the 256-row sorting windows of the default
    // layout), which the wide SpMM hands out to its 8 warps one group at a time
    if (chunks > 8) cpu = (cpu + 7) / 8 * 8;
    *rows_per_unit = cpu * 32;
    return (int)((chunks + cpu - 1) / cpu);
}

// ------------------------------------------------------------- grid tier --
inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Blocks of k_bgrid<TX> the current device holds at once: the size bound of
// its cooperative launches (0 if the kernel cannot be resident).
template <class TX> int grid_resident_blocks() {
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (cache[dev] <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bgrid<TX>, PNT, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            per_sm = 0;
        }
        cache[dev] = per_sm * num_sms();
    }
    return cache[dev];
}

// Blocks per group for n rows with kp columns each: about one block per
// GB_GRID_ROWS row-columns, rounded up to a power of two and at most the
// largest power of two the device holds (and at most PNT: one polling thread
// per block of the group).  A system's group size, and with it the order of
// its sums, depends on its own size only.
inline int grid_blocks_for(int64_t n, int kp, int resident) {
    const int64_t want = (n * kp + GB_GRID_ROWS - 1) / GB_GRID_ROWS;
    int64_t cap = 1;
    while (cap * 2 <= resident && cap * 2 <= PNT) cap *= 2;
    int64_t g = 1;
    while (g < want && g < cap) g *= 2;
    return (int)g;
}

// Bytes of a grid launch's workspace: per group two phases of G exchange
// slots, then the kernel's error word (grid_ws_err).
inline size_t grid_ws_bytes(int groups, int G) {
    return align256(sizeof(double) * 2 * GRID_SLOT * (size_t)G * groups) + 256;
}
inline int *grid_ws_err(void *ws, int groups, int G) {
    return (int *)((char *)ws + align256(sizeof(double) * 2 * GRID_SLOT * (size_t)G * groups));
}

// One cooperative launch of k_bgrid<TX>: `groups` groups of G blocks over the
// list (d_next zeroed, ws zeroed: grid_ws_bytes(groups, G)).  *d_err_out
// receives the address of the error word.
template <class TX>
int launch_grid(BSys *d_sys, const int *d_list, int nlist, int *d_next, int G, int groups, void *ws,
                const PersistOpts &po, cudaStream_t st, int **d_err_out = nullptr) {
    double *gslots = (double *)ws;
    int *err = grid_ws_err(ws, groups, G);
    if (d_err_out) *d_err_out = err;
    PersistOpts o = po;
    void *args[] = {(void *)&d_sys, (void *)&d_list, (void *)&nlist, (void *)&d_next, (void *)&gslots,
                    (void *)&G,     (void *)&err,    (void *)&o};
    ::gb::count_launches(1);
    const cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_bgrid<TX>, dim3((unsigned)(groups * G)),
                                                      dim3(PNT), args, 0, st);
    if (e != cudaSuccess) {
        set_error("grid-tier launch (%d groups of %d blocks): %s", groups, G, cudaGetErrorString(e));
        return GB_ECUDA;
    }
    return GB_OK;
}

// Widest width class (0: k = 1 .. 5: k <= 32) that takes the TMA-streamed SpMM;
// wider classes take the general kernel, whose lane groups gather a P row as
// one coalesced segment.  Measured on 2D P2 1024^2 (SpMM ms, TMA / general):
// fp32 k=1 0.16/0.27, k=8 0.31/0.43, k=16 0.48/0.71, k=32 0.92/1.09 (2048^2:
// 3.36/4.31); fp64 k=1 0.21/0.30, k=8 0.86/0.94, k=16 1.83/1.80, k=32 4.00/3.52.
#ifndef GB_BSPMM_TMA_MAXC32
#define GB_BSPMM_TMA_MAXC32 5
#endif
#ifndef GB_BSPMM_TMA_MAXC64
#define GB_BSPMM_TMA_MAXC64 3
#endif

// SpMM of one iteration: one launch per width class present, over that
// class's units, of the kernel the class takes (the TMA-streamed one needs
// 32-row chunks in every system of the batch).
template <class TX, class TV>
static void launch_bspmm(bool tma, const ClassRanges &cr, int units, BSys *d_sys, const int *d_unit_sys,
                         BGlobal *d_G, double *partials, cudaStream_t s) {
    (void)units;
    constexpr int maxc = sizeof(TX) == 8 ? GB_BSPMM_TMA_MAXC64 : GB_BSPMM_TMA_MAXC32;
    for (int c = 0; c < ClassRanges::N; ++c) {
        if (cr.count[c] <= 0) continue;
        if (tma && c <= maxc) {
            launch_bspmm_tma<TX, TV>(1 << c, cr.base[c], cr.count[c], d_sys, d_unit_sys, d_G, partials, s);
        } else {
            ::gb::count_launches(1);
            k_bspmm<TX, TV><<<cr.count[c], NT, 0, s>>>(d_sys, d_unit_sys, cr.base[c], d_G, partials);
        }
    }
}

template <class TX, class TV>
static void enqueue_biter(Batch &b, cudaStream_t s) {
    launch_bspmm<TX, TV>(b.tma, b.cls, b.units, b.d_sys, b.d_unit_sys, b.d_G, b.partials, s);
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
