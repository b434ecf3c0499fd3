// bsys.cuh -- the system table of the batched solvers (pcg_solve_batched and
// the serving engine): per-system descriptors, per-column recurrence state,
// the loop-wide control block, and the per-system completion helpers.
#pragma once
#include "pcg.cuh"

namespace gb {

constexpr int KMAX = 32;

// Compensated (Kahan) accumulation of the per-lane column partials of the
// fp32 recurrences: a lane adds up hundreds of products of a column (its rows
// of a unit), and plain fp32 sums of that length perturb the recurrences'
// alpha and beta by ~1e-6 -- enough to cost iterations on the ill-conditioned
// systems (2D P2 2048^2).  s holds the sum, c the lost low part (the sum is
// s - c); fp64 partials add plainly.
template <class TX> __device__ __forceinline__ void kadd(TX &s, TX &c, TX v) {
    if constexpr (sizeof(TX) == 4) {
        const TX y = v - c;
        const TX t = s + y;
        c = (t - s) - y;
        s = t;
    } else {
        s += v;
    }
}

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
    int outer;   // refinement steps made by the persistent kernel
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
    int err;             // a bounded wait in a kernel ran out
    cudaGraphConditionalHandle cond;
};

// The unit table of a batch ordered by width class (class c: systems with
// 2^(c-1) < k <= 2^c, class 0: k = 1): class c owns units [base[c], base[c] + count[c]).
struct ClassRanges {
    static constexpr int N = 6;
    int base[N] = {0, 0, 0, 0, 0, 0};
    int count[N] = {0, 0, 0, 0, 0, 0};
};
__host__ __device__ __forceinline__ int width_class(int k) {
    return k <= 1 ? 0 : k <= 2 ? 1 : k <= 4 ? 2 : k <= 8 ? 3 : k <= 16 ? 4 : 5;
}

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

// Per-column sum of a system's unit partials by the whole block: thread t
// sums units t/kw, t/kw + NT/kw, ... of column t%kw, then column j adds the
// NT/kw part sums in order.  Fixed order: deterministic.  All threads call;
// the result is valid in threads j < kw.  stride = partial slots per unit.
__device__ __forceinline__ double col_unit_sum_block(const double *partials, int unit0, int nunits, int slot,
                                                     int stride, int kw, double *smem) {
    const int j = threadIdx.x % kw, part = threadIdx.x / kw, nparts = NT / kw;
    double s = 0.0;
    for (int u = part; u < nunits; u += nparts) s += __ldcg(partials + ((size_t)(unit0 + u) * stride + slot) * KMAX + j);
    __syncthreads();
    smem[threadIdx.x] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < (unsigned)kw)
        for (int q = 0; q < nparts; ++q) t += smem[q * kw + threadIdx.x];
    __syncthreads();
    return t;
}

}  // namespace gb
