// batched.cu -- pcg_solve_batched: many systems, each with k <= 32 right-hand
// sides (Eq. MRH of Sec. 4.3, "block of r.h.s. terms"), solved by k
// independent Jacobi-PCG recurrences per system that share one SELL pass per
// iteration (SpMM), all systems advancing in the same three launches.
//
// Work decomposition: every system is cut into "units" of consecutive rows;
// one block owns one unit.  Inside a block, threads form groups of kw lanes
// (kw = the power of two >= k): a group owns one row and lane j owns column j,
// so the k values of a row-major block row are read and written together.
// Each unit writes per-column partial sums; the last block of a system (per-
// system ticket) reduces them in unit order -- deterministic -- and updates
// that system's per-column scalars.  A column that meets Eq. (2) is frozen
// (convergence mask); a system whose columns are all frozen leaves the loop,
// and the block that retires the last system clears the while-node condition.
//
// precision GB_F64 runs the recurrences in fp64; GB_F32_IR / GB_BF16_IR wrap
// fp32 recurrences (fp32 or bf16 values) in fp64 iterative refinement: outer
// residual B - A X, convergence test and update X += ||r_j|| D_j in fp64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pcg.cuh"

namespace gb {

constexpr int KMAX = 32;

struct ColState {  // per-column scalars of one system, arrays of length k
    double *rho, *pq, *alpha, *beta, *rr, *bb, *thresh, *scale;
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
    cudaGraphConditionalHandle cond;
};

__device__ __forceinline__ void bstop_all(BGlobal *G) {
    G->done = 1;
    if (G->use_cond) cudaGraphSetConditional(G->cond, 0);
}

// system's last block: count active columns, retire the system if none remain
__device__ __forceinline__ void retire_if_idle(BSys &S, BGlobal *G) {
    int a = 0;
    for (int j = 0; j < S.k; ++j) a += S.c.done[j] ? 0 : 1;
    if (S.active > 0 && a == 0) {
        if (atomicSub(&G->active_systems, 1) == 1) bstop_all(G);
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

template <class TX>
__global__ void __launch_bounds__(NT) k_bpupdate(BSys *sys, const int *unit_sys, BGlobal *G) {
    if (G->done) return;
    const int s = unit_sys[blockIdx.x];
    BSys &S = sys[s];
    if (S.active == 0) return;
    const int k = S.k, kw = S.kw;
    const int j = threadIdx.x % kw, grp = threadIdx.x / kw, ngrp = NT / kw;
    if (!(j < k) || S.c.done[j]) return;
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
__global__ void __launch_bounds__(NT) k_bresid(BSys *sys, const int *unit_sys, double *partials, int init,
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
__global__ void k_bscale_down(BSys *sys, const int *unit_sys, const int *mask) {
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
__global__ void k_bcorrect(BSys *sys, const int *unit_sys, const int *mask) {
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

__global__ void k_gather_rows(int64_t n, int k, const int32_t *perm, const double *src, double *dst) {
    const int64_t tot = n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / k;
        const int j = (int)(t - r * k);
        dst[t] = src ? src[(int64_t)perm[r] * k + j] : 0.0;
    }
}
__global__ void k_scatter_rows(int64_t n, int k, const int32_t *perm, const double *src, double *dst) {
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
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_G, &g, sizeof(g), cudaMemcpyHostToDevice, st));
    GB_TRY(run_bloop(st, b.d_G, o.use_graph != 0, o.check_every, [&](cudaStream_t s) { enqueue_biter<TX, TV>(b, s); }));
    return GB_OK;
}

}  // namespace gb

using namespace gb;

template <class TV>
static int batched_ir(Batch &b, const PcgOptions &o, cudaStream_t st, std::vector<int> &outer_cnt,
                      std::vector<long long> &inner_its) {
    const size_t ns = b.h.size();
    HostCols hc;
    std::vector<int> mask(ns * KMAX, 0);
    std::vector<double> prev;
    outer_cnt.assign(ns, 0);
    inner_its.assign(ns, 0);
    // scale = ||r_j|| kept in c.scale; the fp32 recurrence works on R/||r||
    for (int outer = 0; outer < o.max_outer; ++outer) {
        GB_TRY(pull_cols(b, hc, st));
        bool any = false;
        std::vector<double> scale;
        for (size_t s = 0; s < ns; ++s) {
            const int k = b.h[s].k;
            scale.assign(k, 1.0);
            for (int j = 0; j < k; ++j) {
                const bool need = hc.bb[s][j] > 0 && hc.rr[s][j] > o.tol * o.tol * hc.bb[s][j];
                mask[s * KMAX + j] = need ? 1 : 0;
                scale[j] = need ? std::sqrt(hc.rr[s][j]) : 1.0;
                any |= need;
                if (need) outer_cnt[s] += 1;
            }
            GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.scale, scale.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
            // inner threshold: ||r32|| = 1, stop at inner_tol
            std::vector<double> th(k, o.inner_tol * o.inner_tol);
            std::vector<long long> z(k, 0);
            GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.thresh, th.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
            GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.it, z.data(), sizeof(long long) * k, cudaMemcpyHostToDevice, st));
            GB_CHECK_CUDA(cudaStreamSynchronize(st));
        }
        if (!any) break;
        GB_CHECK_CUDA(cudaMemcpyAsync(b.d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
        ::gb::count_launches(1); k_bscale_down<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_mask);
        GB_TRY((start_and_loop<float, TV>(b, mask, o.max_iter, o, st)));
        HostCols hi;
        GB_TRY(pull_cols(b, hi, st));
        for (size_t s = 0; s < ns; ++s) {
            long long mx = 0;
            for (int j = 0; j < b.h[s].k; ++j) if (mask[s * KMAX + j]) mx = std::max(mx, hi.it[s][j]);
            inner_its[s] += mx;
        }
        ::gb::count_launches(1); k_bcorrect<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_mask);
        ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 0, 0, o.tol);
        GB_CHECK_CUDA(cudaGetLastError());
        // restore the outer thresholds (tol^2 ||b||^2) for the next test
        for (size_t s = 0; s < ns; ++s) {
            std::vector<double> th(b.h[s].k);
            for (int j = 0; j < b.h[s].k; ++j) th[j] = o.tol * o.tol * hc.bb[s][j];
            GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.thresh, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, st));
        }
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    return GB_OK;
}

extern "C" int pcg_solve_batched(int nsys, const gb_sell *const *A, const double *const *d_B,
                                 double *const *d_X, const int *k, const PcgOptions *opt, void *stream,
                                 PcgStats *stats) {
    GB_REQUIRE(nsys >= 1 && A && d_B && d_X && k && stats, "pcg_solve_batched: NULL argument");
    for (int s = 0; s < nsys; ++s) {
        GB_REQUIRE(A[s] && d_B[s] && d_X[s], "pcg_solve_batched: system %d has a NULL pointer", s);
        GB_REQUIRE(k[s] >= 1 && k[s] <= KMAX, "pcg_solve_batched: k[%d]=%d not in 1..%d", s, k[s], KMAX);
    }
    PcgOptions o{};
    if (opt) o = *opt;
    if (!(o.tol > 0)) o.tol = 1e-10;
    int64_t nmax = 0;
    for (int s = 0; s < nsys; ++s) nmax = std::max<int64_t>(nmax, A[s]->n);
    if (o.max_iter <= 0) o.max_iter = 20 * nmax + 100;
    if (o.max_outer <= 0) o.max_outer = 30;
    if (!(o.inner_tol > 0)) o.inner_tol = 1e-4;
    if (o.check_every <= 0) o.check_every = 16;
    GB_REQUIRE(o.precision >= GB_F64 && o.precision <= GB_BF16_IR, "pcg_solve_batched: bad precision");
    for (int s = 0; s < nsys; ++s) {
        GB_REQUIRE(o.precision != GB_F32_IR || A[s]->val32, "pcg_solve_batched: system %d has no fp32 values", s);
        GB_REQUIRE(o.precision != GB_BF16_IR || A[s]->val16, "pcg_solve_batched: system %d has no bf16 values", s);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool ir = o.precision != GB_F64;
    Batch b;
    b.mem = Mem(nullptr, st);
    b.h.resize(nsys);
    std::vector<int> unit_sys;
    for (int s = 0; s < nsys; ++s) {
        BSys &S = b.h[s];
        const gb_sell *M = A[s];
        const int64_t n = M->n;
        S = BSys{};
        S.A = M->view();
        S.k = k[s];
        S.kw = kw_of(k[s]);
        const int64_t groups = NT / S.kw;
        int64_t units = (n + groups * 4 - 1) / (groups * 4);
        units = std::max<int64_t>(1, std::min<int64_t>(units, 2048));
        S.rows_per_unit = (n + units - 1) / units;
        units = (n + S.rows_per_unit - 1) / S.rows_per_unit;
        S.unit0 = (int)unit_sys.size();
        S.nunits = (int)units;
        for (int64_t u = 0; u < units; ++u) unit_sys.push_back(s);
        const size_t nk = (size_t)n * S.k;
        double *B64, *X64, *R64;
        GB_TRY(b.take(&B64, nk));
        GB_TRY(b.take(&X64, nk));
        GB_TRY(b.take(&R64, nk));
        S.B64 = B64; S.X64 = X64; S.R64 = R64;
        if (!ir) {
            double *P, *Q;
            GB_TRY(b.take(&P, nk));
            GB_TRY(b.take(&Q, nk));
            S.X = X64; S.R = R64; S.P = P; S.Q = Q;
            S.val = M->val;
        } else {
            float *X, *R, *P, *Q;
            GB_TRY(b.take(&X, nk));
            GB_TRY(b.take(&R, nk));
            GB_TRY(b.take(&P, nk));
            GB_TRY(b.take(&Q, nk));
            S.X = X; S.R = R; S.P = P; S.Q = Q;
            S.val = o.precision == GB_F32_IR ? (const void *)M->val32 : (const void *)M->val16;
        }
        double *cd;
        GB_TRY(b.take(&cd, (size_t)8 * KMAX));
        S.c.rho = cd; S.c.pq = cd + KMAX; S.c.alpha = cd + 2 * KMAX; S.c.beta = cd + 3 * KMAX;
        S.c.rr = cd + 4 * KMAX; S.c.bb = cd + 5 * KMAX; S.c.thresh = cd + 6 * KMAX; S.c.scale = cd + 7 * KMAX;
        long long *ci;
        GB_TRY(b.take(&ci, (size_t)KMAX));
        S.c.it = ci;
        int *cs;
        GB_TRY(b.take(&cs, (size_t)2 * KMAX));
        S.c.done = cs; S.c.status = cs + KMAX;
        GB_CHECK_CUDA(cudaMemsetAsync(cd, 0, sizeof(double) * 8 * KMAX, st));
        GB_CHECK_CUDA(cudaMemsetAsync(ci, 0, sizeof(long long) * KMAX, st));
        GB_CHECK_CUDA(cudaMemsetAsync(cs, 0, sizeof(int) * 2 * KMAX, st));
        const int g = stride_grid((int64_t)nk, 256, 8);
        ::gb::count_launches(1); k_gather_rows<<<g, 256, 0, st>>>(n, S.k, M->perm, d_B[s], B64);
        ::gb::count_launches(1); k_gather_rows<<<g, 256, 0, st>>>(n, S.k, M->perm, o.x0_zero ? nullptr : d_X[s], X64);
    }
    b.units = (int)unit_sys.size();
    GB_TRY(b.take(&b.d_sys, (size_t)nsys));
    GB_TRY(b.take(&b.d_unit_sys, unit_sys.size()));
    GB_TRY(b.take(&b.d_mask, (size_t)nsys * KMAX));
    GB_TRY(b.take(&b.d_G, 1));
    GB_TRY(b.take(&b.partials, (size_t)b.units * 2 * KMAX));
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_sys, b.h.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_unit_sys, unit_sys.data(), sizeof(int) * unit_sys.size(), cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaMemsetAsync(b.d_G, 0, sizeof(BGlobal), st));

    cudaEvent_t e0, e1;
    GB_CHECK_CUDA(cudaEventCreate(&e0));
    GB_CHECK_CUDA(cudaEventCreate(&e1));
    GB_CHECK_CUDA(cudaEventRecord(e0, st));
    // R = B - A X0, ||B_j||, thresholds
    ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 1, o.x0_zero ? 1 : 0, o.tol);
    GB_CHECK_CUDA(cudaGetLastError());
    HostCols hc;
    GB_TRY(pull_cols(b, hc, st));
    std::vector<int> mask(nsys * KMAX, 0);
    std::vector<int> outer_cnt(nsys, 0);
    std::vector<long long> inner_its(nsys, 0);
    std::vector<long long> restarts(nsys, 0);
    std::vector<long long> fallback_its(nsys, 0);
    int rc = GB_OK;
    if (!ir) {
        // fp64 recurrences; restart columns whose true residual misses tol
        for (int round = 0; round < 50; ++round) {
            bool any = false;
            for (int s = 0; s < nsys; ++s)
                for (int j = 0; j < k[s]; ++j) {
                    const bool need = hc.bb[s][j] > 0 && hc.rr[s][j] > o.tol * o.tol * hc.bb[s][j] &&
                                      (round == 0 || hc.status[s][j] == ST_CONV);
                    mask[s * KMAX + j] = need ? 1 : 0;
                    any |= need;
                    if (need && round > 0) restarts[s] += 1;
                }
            if (!any) break;
            rc = start_and_loop<double, double>(b, mask, o.max_iter, o, st);
            if (rc != GB_OK) break;
            ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 0, 0, o.tol);
            GB_CHECK_CUDA(cudaGetLastError());
            HostCols h2;
            rc = pull_cols(b, h2, st);
            if (rc != GB_OK) break;
            // keep status from the loop, residuals from the true residual
            for (int s = 0; s < nsys; ++s) { hc.rr[s] = h2.rr[s]; hc.status[s] = h2.status[s]; hc.it[s] = h2.it[s]; }
        }
    } else {
        rc = o.precision == GB_F32_IR ? batched_ir<float>(b, o, st, outer_cnt, inner_its)
                                      : batched_ir<__nv_bfloat16>(b, o, st, outer_cnt, inner_its);
        if (rc == GB_OK) rc = pull_cols(b, hc, st);
        // columns the refinement left above tol finish in fp64 from their X
        bool fb = false;
        for (int s2 = 0; s2 < nsys && rc == GB_OK; ++s2)
            for (int j = 0; j < k[s2]; ++j) {
                const bool need = hc.bb[s2][j] > 0 && hc.rr[s2][j] > o.tol * o.tol * hc.bb[s2][j];
                mask[s2 * KMAX + j] = need ? 1 : 0;
                fb |= need;
            }
        if (rc == GB_OK && fb) {
            for (int s2 = 0; s2 < nsys && rc == GB_OK; ++s2) {
                BSys &S = b.h[s2];
                const size_t nk = (size_t)S.A.n * S.k;
                double *P, *Q;
                rc = b.take(&P, nk);
                if (rc == GB_OK) rc = b.take(&Q, nk);
                if (rc != GB_OK) break;
                S.X = S.X64; S.R = S.R64; S.P = P; S.Q = Q; S.val = A[s2]->val;
                std::vector<long long> z(S.k, 0);
                cudaMemcpyAsync(S.c.it, z.data(), sizeof(long long) * S.k, cudaMemcpyHostToDevice, st);
                cudaStreamSynchronize(st);
            }
            if (rc == GB_OK) {
                cudaMemcpyAsync(b.d_sys, b.h.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, st);
                rc = start_and_loop<double, double>(b, mask, o.max_iter, o, st);
            }
            if (rc == GB_OK) {
                ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 0, 0, o.tol);
                HostCols h3;
                rc = pull_cols(b, h3, st);
                for (int s2 = 0; s2 < nsys && rc == GB_OK; ++s2) {
                    hc.rr[s2] = h3.rr[s2];
                    hc.status[s2] = h3.status[s2];
                    long long mx = 0;
                    for (int j = 0; j < k[s2]; ++j) if (mask[s2 * KMAX + j]) mx = std::max(mx, h3.it[s2][j]);
                    fallback_its[s2] = mx;
                }
            }
        }
    }
    if (rc != GB_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    for (int s = 0; s < nsys; ++s) {
        const int g = stride_grid((int64_t)A[s]->n * k[s], 256, 8);
        ::gb::count_launches(1); k_scatter_rows<<<g, 256, 0, st>>>(A[s]->n, k[s], A[s]->perm, b.h[s].X64, d_X[s]);
    }
    GB_CHECK_CUDA(cudaEventRecord(e1, st));
    GB_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int worst = GB_OK;
    for (int s = 0; s < nsys; ++s) {
        PcgStats &S = stats[s];
        S = PcgStats{};
        double rel = 0.0, bn = 0.0;
        long long its = 0;
        int status = GB_OK;
        for (int j = 0; j < k[s]; ++j) {
            const double bb = hc.bb[s][j];
            const double r = bb > 0 ? std::sqrt(hc.rr[s][j] / bb) : 0.0;
            rel = std::max(rel, r);
            bn = std::max(bn, std::sqrt(bb));
            its = std::max(its, hc.it[s][j]);
            if (r > o.tol) status = (hc.status[s][j] == ST_BREAK) ? GB_BREAKDOWN : GB_NOT_CONVERGED;
        }
        S.iterations = ir ? inner_its[s] : its;
        S.restarts = restarts[s];
        S.outer = outer_cnt[s];
        S.relres = rel;
        S.bnorm = bn;
        S.status = status;
        S.solve_ms = ms;
        const double sv = ir ? (o.precision == GB_F32_IR ? 4.0 : 2.0) : 8.0;
        const double sx = ir ? 4.0 : 8.0;
        S.bytes_moved = (double)S.iterations * ((double)A[s]->nnz * (sv + 4.0) + 7.0 * A[s]->n * k[s] * sx);
        S.kernel_launches = 3 * (S.iterations + fallback_its[s]);
        S.fallback_iterations = fallback_its[s];
        if (fallback_its[s]) S.bytes_moved += (double)fallback_its[s] * ((double)A[s]->nnz * 12.0 + 7.0 * A[s]->n * k[s] * 8.0);
        if (status != GB_OK && worst == GB_OK) worst = status;
    }
    if (worst != GB_OK) {
        set_error("pcg_solve_batched: a column did not reach tol (status %d)", worst);
        return worst;
    }
    return GB_OK;
}
