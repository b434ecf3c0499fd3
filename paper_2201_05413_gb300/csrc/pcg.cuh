// pcg.cuh -- device-side Jacobi-PCG building blocks shared by the single-,
// multi-RHS and batched solvers.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "sell.cuh"

namespace gb {

constexpr int NT = 256;  // threads per block of every solver kernel

// Device-resident scalars of one CG recurrence (fp64 whatever the vector type).
struct PcgScal {
    double rho;     // r.z
    double pq;      // p.Ap
    double alpha, beta;
    double rr;      // ||r||^2 (recursive)
    double bb;      // ||b||^2
    double thresh;  // tol^2 ||b||^2
    double pz;      // reliable update: coefficient of z in the restored p
    double dmax;    // bound of lmax(M^-1) for the deferred r.r test (0: r.r every iteration)
    long long it, maxit;
    int done, status;
    unsigned int ticket;  // last-block counter
    int err;              // set by a kernel whose bounded wait ran out
    int use_cond;
    int check_p;          // the p update makes this iteration's Eq. (2) test
    cudaGraphConditionalHandle cond;
    double omega, rho0;   // BiCGSTAB: omega, the previous rho
    int early;            // BiCGSTAB: the step stopped on ||s|| (x += alpha ph only)
    int brk;              // BiCGSTAB: which quantity broke down (1 r^.v, 2 t.t, 3 ||s||, 4 rho, 5 omega)
};
enum { ST_RUN = 0, ST_CONV = 1, ST_BREAK = 2, ST_MAXIT = 3, ST_TIMEOUT = 4 };

// Streaming loads for the matrix (read once per iteration: evict first).
__device__ __forceinline__ double ld_val(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16 *p) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float(((unsigned int)u) << 16);
}
__device__ __forceinline__ int ld_col(const int32_t *p) { return __ldcs(p); }

// True in every thread of the block that arrives last at `ticket` (after all
// other blocks have published their partial sums).
__device__ __forceinline__ bool arrive_last(unsigned int *ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Deterministic sum of partials[i*stride+off], i < G (fixed order per thread,
// fixed tree across threads).  Valid in thread 0; all threads must call.
__device__ __forceinline__ double sum_partials(const double *partials, int G, int stride, int off,
                                               double *smem) {
    double s = 0.0;
    for (int i = threadIdx.x; i < G; i += NT) s += __ldcg(partials + (size_t)i * stride + off);
    return block_sum<NT>(s, smem);
}

// 16-byte accesses of the streaming vector kernels: VW elements of T per load
// (4 fp32 / 2 fp64); a type narrower than the step's element count (fp32
// D^-1 beside fp64 vectors) takes fewer bytes per access.
template <class T, int N> struct alignas(sizeof(T) * N) Pack { T v[N]; };
template <class T, int N>
__device__ __forceinline__ void ld_pack(const T *p, int64_t i, T (&o)[N]) {
    if constexpr (sizeof(T) * N <= 16) {
        const Pack<T, N> v = reinterpret_cast<const Pack<T, N> *>(p)[i];
#pragma unroll
        for (int k = 0; k < N; ++k) o[k] = v.v[k];
    } else {
        constexpr int H = N / 2;
        const Pack<T, H> a = reinterpret_cast<const Pack<T, H> *>(p)[2 * i];
        const Pack<T, H> b = reinterpret_cast<const Pack<T, H> *>(p)[2 * i + 1];
#pragma unroll
        for (int k = 0; k < H; ++k) { o[k] = a.v[k]; o[H + k] = b.v[k]; }
    }
}
template <class T, int N>
__device__ __forceinline__ void st_pack(T *p, int64_t i, const T (&o)[N]) {
    Pack<T, N> v;
#pragma unroll
    for (int k = 0; k < N; ++k) v.v[k] = o[k];
    reinterpret_cast<Pack<T, N> *>(p)[i] = v;
}

// ||r||^2 is needed only when it can meet the Eq. (2) threshold: since
// r.M^-1 r <= lmax(M^-1) ||r||^2, while rho = r.z stays above an upper bound of
// lmax(M^-1) times the threshold (S->dmax > 0: max(D^-1) for Jacobi, the
// largest absolute row sum of the inverses for block-Jacobi) the x/r update skips
// the r.r sums; when this iteration's r.z falls below that bound with r.r
// skipped, the p update computes r.r from the r it reads anyway and makes the
// test there, in the same iteration -- the stopping iteration is unchanged.
__device__ __forceinline__ bool want_rr(const PcgScal *S) {
    return !(S->dmax > 0.0) || S->rho <= S->dmax * S->thresh;
}

__device__ __forceinline__ void stop(PcgScal *S, int status) {
    S->status = status;
    S->done = 1;
    if (S->use_cond) cudaGraphSetConditional(S->cond, 0);
}

// Rows (times the column power of two) per block of a grid-tier group, and
// the largest single system pcg_solve hands to the grid tier when asked to
// (PcgOptions.persist_off = 3).
#ifndef GB_GRID_ROWS
#define GB_GRID_ROWS 2048
#endif
#ifndef GB_GRID_SINGLE_MAX
#define GB_GRID_SINGLE_MAX (1 << 18)
#endif
// the largest single system pcg_solve solves by one thread-block cluster by
// default (64^2 P1, 3969 rows: 1.52 against 2.30 ms per solve in the
// multi-kernel loop; at 16129 rows the loop is faster, 14.0 against 20.1 ms)
#ifndef GB_CLUSTER_SINGLE_MAX
#define GB_CLUSTER_SINGLE_MAX (1 << 13)
#endif

// fp64 Jacobi-PCG of one system by one group of the grid-tier persistent
// kernel (batched.cu): returns GB_OK with *stats filled, an error code, or 1
// when the tier is not available (the caller takes the multi-kernel loop).
int grid_solve_single(const gb_sell *M, const double *d_b, double *d_x, const PcgOptions &o, cudaStream_t st,
                      PcgStats *stats);

}  // namespace gb
