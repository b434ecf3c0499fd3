// bpersist.cuh -- persistent, CTA-local Jacobi-PCG for the small systems of a
// batch: one launch over a list of systems; each block takes the next system
// from the list (atomic counter) and runs every iteration of all its columns
// itself, with __syncthreads between the phases and block-level reductions,
// until each column has met Eq. (2), hit the iteration cap or broken down.
// No block waits on another, so there is nothing to spin on.
//
// A small system costs one block a few microseconds per iteration instead of
// the three grid-wide launches of the batched loop, and many small systems
// proceed side by side on different SMs.  A system's arithmetic depends only
// on its own data (one block, fixed reduction order), so its result is the
// same alone and in any batch.
//
// TX = double: fp64 CG on X64/R64 with D^-1 in fp64, restarted from the true
// residual b - A x when the recursive one has met the threshold but the true
// one has not (as the multi-kernel fp64 path).
// TX = float: iterative refinement -- the fp64 residual r = b - A x, the test
// and x += ||r|| d stay in fp64; the correction d solves A d = r / ||r|| by fp32
// CG (fp32 values and vectors) to the relative residual inner_tol.
//
// Thread layout: kp = the power of two >= k; thread t of the group owns
// column t mod kp (idle when >= k) of rows t / kp, t / kp + GN / kp, ...;
// per-column sums run an xor tree over the lanes of a column and then the
// warps in order.
//
// The phases are written once for a "group" of threads that solves one
// system together:
//   CtaGroup      one block (k_bpersist, small systems: n kp <= 2^15);
//   ClusterGroup  the CS = 8 blocks of a thread-block cluster (k_bcluster,
//                 medium systems: 2^15 < n kp <= 2^16).  Each block reduces
//                 its partial sums itself, publishes them in its shared
//                 memory, and after a cluster barrier every block reads the 8
//                 partials through distributed shared memory in rank order,
//                 so all blocks hold the same sums and take the same
//                 decisions.  The barrier (barrier.cluster, release/acquire)
//                 also orders the blocks' global writes of the vectors other
//                 blocks gather next (p, x); those gathers read L2 (ld.cg).
//                 The blocks of a cluster are co-scheduled by the hardware,
//                 so its barrier is not a spin on memory.
//   GridGroup     G blocks of a cooperative launch (k_bgrid, systems too large
//                 for one cluster): the same exchange through global memory --
//                 each block publishes its column sums and an exchange number
//                 in a slot of its own (release store), waits until the G
//                 slots show this exchange (acquire loads, one thread per
//                 slot, bounded by %globaltimer), and adds the G slots in
//                 rank order.  A cooperative launch keeps all blocks resident,
//                 so every exchange completes; a wait that runs out all the
//                 same sets the kernel's error word, the blocks stop, and the
//                 columns report ST_TIMEOUT.
#pragma once
#include <cooperative_groups.h>

#include "bsys.cuh"
#include "spmv_tma.cuh"

namespace gb {

constexpr int PNT = 512;                         // threads per block
constexpr int64_t PERSIST_MAX_ELEMS = 1 << 15;   // n * kp of a system the CTA-local kernel takes
constexpr int CLUSTER_CS = 8;                    // blocks per cluster (the portable maximum)
// n * kp of a system the cluster kernel takes: above 2^15 one block is too
// slow, and above ~2^16 the multi-launch loop over every SM is faster than
// 8 SMs per system even with 19 such systems side by side (2D P1 200^2: 47
// against 53 ms alone, 97 against 90 ms for 19; 3D P1 48^3 with 2 columns: 51
// against 14 ms alone, 134 against 61 ms for 19)
constexpr int64_t CLUSTER_MAX_ELEMS = 1 << 16;

struct PersistOpts {
    long long maxit;    // iterations per column (fp64) / inner iterations per outer step (fp32)
    double tol;         // Eq. (2) threshold
    double inner_tol;   // fp32 inner relative residual
    int max_outer;      // refinement steps (fp32) / true-residual restarts (fp64)
    int init;           // cluster / grid tiers: form R64 = B64 - A X64, ||b|| and the thresholds itself
    int x0_zero;        // with init: X64 = 0 (R64 = B64)
    unsigned long long wait_ns;  // grid tier: bound of a barrier wait (0: WAIT_LIMIT_NS)
};

// Shared-memory scratch of the group's reductions.
struct GrpSmem {
    double red[PNT / 32][32];  // warp partials
    double xs[2][32];          // this block's per-column sums, published to the cluster (two phases)
    int ph;                    // phase of the next cluster exchange
};

// Per-column block sum; every thread passes its value, threads j < k read
// out[j] after the call.  kp divides 32.
__device__ __forceinline__ void p_colsum(double v, int kp, double (*red)[32], double *out) {
    for (int o = kp; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < kp) red[warp][lane] = v;
    __syncthreads();
    if (threadIdx.x < (unsigned)kp) {
        double s = 0.0;
        for (int w = 0; w < PNT / 32; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

struct CtaGroup {
    static constexpr int GN = PNT;  // threads of the group
    static __device__ __forceinline__ int gn() { return GN; }
    static __device__ __forceinline__ bool failed() { return false; }
    static __device__ __forceinline__ int gtid() { return threadIdx.x; }
    static __device__ __forceinline__ bool leader() { return true; }
    // the group's global writes before the call are seen by its reads after it
    static __device__ __forceinline__ void sync() { __syncthreads(); }
    template <class T> static __device__ __forceinline__ T ldv(const T *p) { return *p; }
    static __device__ __forceinline__ void colsum(double v, int kp, GrpSmem &g, double *out) {
        p_colsum(v, kp, g.red, out);
    }
    static __device__ __forceinline__ void colsum2(double v, double w, int kp, GrpSmem &g, double *out,
                                                   double *out2) {
        colsum(v, kp, g, out);
        colsum(w, kp, g, out2);
    }
};

struct ClusterGroup {
    static constexpr int GN = CLUSTER_CS * PNT;
    static __device__ __forceinline__ int gn() { return GN; }
    static __device__ __forceinline__ bool failed() { return false; }
    static __device__ __forceinline__ int rank() { return (int)cooperative_groups::this_cluster().block_rank(); }
    static __device__ __forceinline__ int gtid() { return rank() * PNT + (int)threadIdx.x; }
    static __device__ __forceinline__ bool leader() { return rank() == 0; }
    static __device__ __forceinline__ void sync() { cooperative_groups::this_cluster().sync(); }
    template <class T> static __device__ __forceinline__ T ldv(const T *p) { return __ldcg(p); }
    // block sums, published in xs[ph]; after the cluster barrier each block
    // adds the CS blocks' sums in rank order.  The next exchange writes the
    // other phase, and a block can only reach the one after that once every
    // block has passed the barrier of the next one, i.e. finished reading.
    static __device__ __forceinline__ void colsum(double v, int kp, GrpSmem &g, double *out) {
        const int ph = g.ph;
        p_colsum(v, kp, g.red, g.xs[ph]);
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        cl.sync();
        if (threadIdx.x < (unsigned)kp) {
            double s = 0.0;
            for (int r = 0; r < CLUSTER_CS; ++r) s += cl.map_shared_rank(&g.xs[ph][0], r)[threadIdx.x];
            out[threadIdx.x] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) g.ph = ph ^ 1;
        __syncthreads();
    }
    static __device__ __forceinline__ void colsum2(double v, double w, int kp, GrpSmem &g, double *out,
                                                   double *out2) {
        colsum(v, kp, g, out);
        colsum(w, kp, g, out2);
    }
};

// ---------------------------------------------------------- grid groups --
// Exchange slots of one group of the grid tier (global memory, zeroed before
// the launch): [2 phases][G blocks][GRID_SLOT doubles]; a slot holds the
// exchange number its block last published (first 4 bytes of its first 128)
// and up to 64 values after that.  Exchange e uses phase e mod 2.
constexpr int GRID_SLOT = 80;
constexpr int GRID_SLOT_VALS = 16;  // first value (doubles into the slot)

// Per-block context of the grid tier (one copy per block, in shared memory).
struct GridCtx {
    int rank, G, gn;  // rank in the group, blocks per group, threads per group
    int failed;       // a wait of this block ran out (the group stops)
    unsigned int seq; // number of the block's next exchange (from 1)
    double *slots;    // the group's exchange slots
    int *err;         // kernel-wide error word
    unsigned long long limit_ns;
};
__shared__ GridCtx g_gctx;

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One exchange of the group: the block publishes nv values (vals, shared
// memory, nv <= 64) in its slot and then its exchange number with a release
// store; threads 0 .. G-1 each wait, with acquire loads, for one block's
// number to reach this exchange; after the block barrier every block's values
// are visible to every thread (read them with grid_slot_value).  No counter,
// no read-modify-write: the G flags are polled in parallel.  A block can only
// publish exchange e + 2 (the same phase) once every block has published
// e + 1, i.e. has finished reading exchange e, so the two phases never
// overlap.  Every wait is bounded: past limit_ns the block marks itself
// failed and sets the kernel's error word; a failed block publishes nothing
// more and returns from later exchanges at once, so the others' waits run out
// too and the whole group stops.  Returns the slots of this exchange.
__device__ __forceinline__ const double *grid_exchange(const double *vals, int nv) {
    GridCtx &c = g_gctx;
    __syncthreads();
    const unsigned int e = c.seq;
    double *base = c.slots + (size_t)(e & 1u) * c.G * GRID_SLOT;
    if (!c.failed) {
        double *mine = base + (size_t)c.rank * GRID_SLOT;
        if ((int)threadIdx.x < nv) mine[GRID_SLOT_VALS + threadIdx.x] = vals[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) st_release_u32(reinterpret_cast<unsigned int *>(mine), e);
        if ((int)threadIdx.x < c.G) {
            const unsigned int *flag = reinterpret_cast<const unsigned int *>(base + (size_t)threadIdx.x * GRID_SLOT);
            unsigned long long t0 = 0;
            for (unsigned int polls = 0; (int)(ld_acquire_u32(flag) - e) < 0; ++polls) {
                if ((polls & 63u) == 63u) {
                    const unsigned long long t = globaltimer();
                    if (t0 == 0) {
                        t0 = t;
                    } else if (t - t0 > c.limit_ns) {
                        c.failed = 1;
                        atomicExch(c.err, 1);
                        break;
                    }
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) c.seq = e + 1u;
    return base;
}
// value v of block r's slot (after grid_exchange returned `base`): L2 loads,
// never an L1 copy of an earlier exchange
__device__ __forceinline__ double grid_slot_value(const double *base, int r, int v) {
    return __ldcg(base + (size_t)r * GRID_SLOT + GRID_SLOT_VALS + v);
}

__device__ __forceinline__ void grid_group_sync() { (void)grid_exchange(nullptr, 0); }

struct GridGroup {
    static __device__ __forceinline__ int gn() { return g_gctx.gn; }
    static __device__ __forceinline__ bool failed() { return g_gctx.failed != 0; }
    static __device__ __forceinline__ int gtid() { return g_gctx.rank * PNT + (int)threadIdx.x; }
    static __device__ __forceinline__ bool leader() { return g_gctx.rank == 0; }
    static __device__ __forceinline__ void sync() { grid_group_sync(); }
    template <class T> static __device__ __forceinline__ T ldv(const T *p) { return __ldcg(p); }
    // nv values per column (1 or 2): the block sums (g.xs[t][j]) published in
    // one exchange, then every block adds the G blocks' sums -- thread
    // (seg, j) the ranks seg, seg + PNT/kp, ... in order, then the fixed tree
    // of p_colsum -- so all blocks hold the same sums.
    static __device__ __forceinline__ void exchange(const double *v, int nv, int kp, GrpSmem &g, double *const *out) {
        for (int t = 0; t < nv; ++t) p_colsum(v[t], kp, g.red, g.xs[t]);
        const double *base = grid_exchange(&g.xs[0][0], 32 * nv);
        const int j = (int)threadIdx.x % kp, seg = (int)threadIdx.x / kp, nseg = PNT / kp;
        const int G = g_gctx.G;
        for (int t = 0; t < nv; ++t) {
            double s = 0.0;
            for (int r = seg; r < G; r += nseg) s += grid_slot_value(base, r, t * 32 + j);
            p_colsum(s, kp, g.red, out[t]);
        }
    }
    static __device__ __forceinline__ void colsum(double v, int kp, GrpSmem &g, double *out) {
        double *o[1] = {out};
        exchange(&v, 1, kp, g, o);
    }
    static __device__ __forceinline__ void colsum2(double v, double w, int kp, GrpSmem &g, double *out,
                                                   double *out2) {
        const double vw[2] = {v, w};
        double *o[2] = {out, out2};
        exchange(vw, 2, kp, g, o);
    }
};

struct PState {  // per-column scalars of the running recurrence (shared memory)
    double alpha[32], beta[32], rho[32], thresh[32], rr[32], scale[32], t0[32], t1[32];
    double bb[32], othresh[32];  // ||b_j||^2 and the Eq. (2) threshold tol^2 ||b_j||^2
    long long it[32];
    int run[32];     // column iterating in the current recurrence
    int status[32];  // ST_*
};

// q = A p for the columns of this thread, partial p.q; TV values, TX vectors.
// The vectors are rewritten inside this kernel, so they are read with plain
// (coherent) loads: no __restrict__ / read-only-cache loads on them.  Two
// rows per step, each walked to its chunk's width (a padded slot holds value
// 0 and points at the row itself, so it adds exactly zero), four slots of
// both rows loaded before their gathers: fewer dependent trips to L2 per row
// (four rows per step spill registers and were slower: 1.87 against 1.52 ms
// for the 64^2 P1 solve on one cluster).
template <class Grp, class TV, class TX>
__device__ __forceinline__ double p_spmv(const SellView &A, const TV *__restrict__ val, const TX *P, TX *Q,
                                         int64_t n, int k, int kp, int j, bool on) {
    double pq = 0.0;
    if (!on) return pq;
    const int C = A.C;
    const int64_t step = Grp::gn() / kp;
    for (int64_t r0 = Grp::gtid() / kp; r0 < n; r0 += 2 * step) {
        const int64_t rw[2] = {r0, r0 + step};
        int w[2];
        int64_t base[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            w[u] = 0;
            base[u] = 0;
            if (rw[u] < n) {
                const int64_t c = rw[u] / C;
                w[u] = __ldg(A.chunk_w + c);
                base[u] = __ldg(A.chunk_ptr + c) + (rw[u] - c * C);
            }
        }
        TX acc[2] = {TX(0), TX(0)};
        const int wm = w[0] > w[1] ? w[0] : w[1];
        for (int s = 0; s < wm; s += 4) {
            int cl[2][4];
            TX vl[2][4], pv[2][4];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    cl[u][t] = 0;
                    vl[u][t] = TX(0);
                    if (s + t < w[u]) {
                        const int64_t e = base[u] + (int64_t)(s + t) * C;
                        cl[u][t] = __ldg(A.col + e);
                        vl[u][t] = (TX)ld_val(val + e);
                    }
                }
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    pv[u][t] = (s + t < w[u]) ? Grp::ldv(P + (int64_t)cl[u][t] * k + j) : TX(0);
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (s + t < w[u]) acc[u] += vl[u][t] * pv[u][t];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (rw[u] < n) {
                Q[rw[u] * k + j] = acc[u];
                pq += (double)(P[rw[u] * k + j] * acc[u]);
            }
    }
    return pq;
}

// Runs CG on (X, R, P, Q) for the columns with st.run[j] set, stopping each at
// ||R_j||^2 <= st.thresh[j], at st.it[j] == maxit, or on breakdown.  R holds the
// starting residual; X is updated in place.
template <class Grp, class TV, class TX, class TD>
__device__ void p_cg(const SellView &A, const TV *__restrict__ val, const TD *__restrict__ dinv, TX *X, TX *R, TX *P,
                     TX *Q, int64_t n, int k, int kp, long long maxit, PState &st, GrpSmem &gs) {
    const int j = threadIdx.x % kp;
    const int64_t row0 = Grp::gtid() / kp, rstep = Grp::gn() / kp;
    // start: P = D^-1 R, rho = R.D^-1 R
    {
        const bool on = j < k && st.run[j];
        double rz = 0.0;
        if (on)
            for (int64_t r = row0; r < n; r += rstep) {
                const TX z = (TX)dinv[r] * R[r * k + j];
                P[r * k + j] = z;
                rz += (double)(R[r * k + j] * z);
            }
        Grp::colsum(rz, kp, gs, st.t0);  // (in a cluster: also publishes P before the first gathers)
        if (threadIdx.x < (unsigned)k && st.run[threadIdx.x]) {
            const double t = st.t0[threadIdx.x];
            st.rho[threadIdx.x] = t;
            if (!(t > 0.0)) { st.run[threadIdx.x] = 0; st.status[threadIdx.x] = t == 0.0 ? ST_CONV : ST_BREAK; }
        }
        __syncthreads();
    }
    for (;;) {
        if (Grp::failed()) {  // a group barrier wait ran out: the columns stop here
            if (threadIdx.x < (unsigned)k && st.run[threadIdx.x]) {
                st.run[threadIdx.x] = 0;
                st.status[threadIdx.x] = ST_TIMEOUT;
            }
            __syncthreads();
            break;
        }
        int any = 0;
        for (int q = 0; q < k; ++q) any |= st.run[q];
        if (!any) break;
        const bool on = j < k && st.run[j];
        // q = A p, alpha = rho / p.q
        const double pq = p_spmv<Grp, TV, TX>(A, val, P, Q, n, k, kp, j, on);
        Grp::colsum(pq, kp, gs, st.t0);
        if (threadIdx.x < (unsigned)k && st.run[threadIdx.x]) {
            const double t = st.t0[threadIdx.x];
            if (!(t > 0.0) || !isfinite(t)) { st.run[threadIdx.x] = 0; st.status[threadIdx.x] = ST_BREAK; }
            else st.alpha[threadIdx.x] = st.rho[threadIdx.x] / t;
        }
        __syncthreads();
        // x += alpha p, r -= alpha q, r.D^-1 r, r.r
        const bool on2 = j < k && st.run[j];
        double rz = 0.0, rr = 0.0;
        if (on2) {
            const TX a = (TX)st.alpha[j];
            constexpr int U = 4;  // rows in flight per thread
            const int64_t step = rstep;
            for (int64_t r0 = row0; r0 < n; r0 += U * step) {
                TX xv[U], pv[U], rv[U], qv[U], dv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t r = r0 + u * step;
                    if (r < n) {
                        const int64_t e = r * k + j;
                        xv[u] = X[e]; pv[u] = P[e]; rv[u] = R[e]; qv[u] = Q[e]; dv[u] = (TX)dinv[r];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t r = r0 + u * step;
                    if (r < n) {
                        const int64_t e = r * k + j;
                        X[e] = xv[u] + a * pv[u];
                        const TX rn = rv[u] - a * qv[u];
                        R[e] = rn;
                        rz += (double)(rn * (dv[u] * rn));
                        rr += (double)(rn * rn);
                    }
                }
            }
        }
        Grp::colsum2(rz, rr, kp, gs, st.t0, st.t1);
        if (threadIdx.x < (unsigned)k && st.run[threadIdx.x]) {
            const int q = threadIdx.x;
            st.it[q] += 1;
            st.rr[q] = st.t1[q];
            if (!isfinite(st.t0[q]) || !isfinite(st.t1[q])) { st.run[q] = 0; st.status[q] = ST_BREAK; }
            else if (st.t1[q] <= st.thresh[q]) { st.run[q] = 0; st.status[q] = ST_CONV; }
            else if (st.it[q] >= maxit) { st.run[q] = 0; st.status[q] = ST_MAXIT; }
            else { st.beta[q] = st.t0[q] / st.rho[q]; st.rho[q] = st.t0[q]; }
        }
        __syncthreads();
        // p = D^-1 r + beta p
        const bool on3 = j < k && st.run[j];
        if (on3) {
            const TX b = (TX)st.beta[j];
            constexpr int U = 4;
            const int64_t step = rstep;
            for (int64_t r0 = row0; r0 < n; r0 += U * step) {
                TX pv[U], rv[U], dv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t r = r0 + u * step;
                    if (r < n) { const int64_t e = r * k + j; pv[u] = P[e]; rv[u] = R[e]; dv[u] = (TX)dinv[r]; }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t r = r0 + u * step;
                    if (r < n) P[r * k + j] = dv[u] * rv[u] + b * pv[u];
                }
            }
        }
        Grp::sync();  // the new P before the next gathers
    }
}

// R64 = B64 - A X64 in fp64 for the columns in `sel`; ||R64_j||^2 into st.rr.
template <class Grp>
static __device__ void p_resid(const BSys &S, int64_t n, int k, int kp, const int *sel, PState &st, GrpSmem &gs) {
    const int j = threadIdx.x % kp;
    double rr = 0.0;
    if (j < k && sel[j]) {
        const SellView &A = S.A;
        const int C = A.C;
        for (int64_t r = Grp::gtid() / kp; r < n; r += Grp::gn() / kp) {
            const int64_t c = r / C;
            const int L = A.row_len[r];
            const int64_t base = A.chunk_ptr[c] + (r - c * C);
            double acc = 0.0;
            for (int s = 0; s < L; ++s) {
                const int64_t e = base + (int64_t)s * C;
                acc += ld_val(A.val + e) * Grp::ldv(S.X64 + (int64_t)__ldg(A.col + e) * k + j);
            }
            const double ri = S.B64[r * k + j] - acc;
            S.R64[r * k + j] = ri;
            rr += ri * ri;
        }
    }
    Grp::colsum(rr, kp, gs, st.t1);
    if (threadIdx.x < (unsigned)k && sel[threadIdx.x]) st.rr[threadIdx.x] = st.t1[threadIdx.x];
    __syncthreads();
}

// Entry state of a system from the batch's initial residual kernel
// (R64 = B - A X0 there): ||r_j||^2, ||b_j||^2 and the thresholds.
static __device__ void p_load_state(const BSys &S, PState &st) {
    if (threadIdx.x < (unsigned)S.k) {
        const int q = threadIdx.x;
        st.rr[q] = S.c.rr[q];
        st.bb[q] = S.c.bb[q];
        st.othresh[q] = S.c.thresh[q];
    }
    __syncthreads();
}

// The same entry state computed by the group itself: R64 = B64 - A X64 (or
// B64 when x0_zero), ||r_j||^2, ||b_j||^2, thresholds tol^2 ||b_j||^2; the
// leader also leaves them in the column state for the host.
template <class Grp>
static __device__ void p_init(BSys &S, int x0_zero, double tol, PState &st, GrpSmem &gs) {
    const int64_t n = S.A.n;
    const int k = S.k;
    int kp = 1;
    while (kp < k) kp <<= 1;
    const int j = threadIdx.x % kp;
    double rr = 0.0, bb = 0.0;
    if (j < k) {
        const SellView &A = S.A;
        const int C = A.C;
        for (int64_t r = Grp::gtid() / kp; r < n; r += Grp::gn() / kp) {
            double acc = 0.0;
            if (!x0_zero) {
                const int64_t c = r / C;
                const int L = A.row_len[r];
                const int64_t base = A.chunk_ptr[c] + (r - c * C);
                for (int s = 0; s < L; ++s) {
                    const int64_t e = base + (int64_t)s * C;
                    acc += ld_val(A.val + e) * Grp::ldv(S.X64 + (int64_t)__ldg(A.col + e) * k + j);
                }
            }
            const double bi = S.B64[r * k + j];
            const double ri = bi - acc;
            S.R64[r * k + j] = ri;
            rr += ri * ri;
            bb += bi * bi;
        }
    }
    Grp::colsum2(rr, bb, kp, gs, st.t0, st.t1);
    if (threadIdx.x < (unsigned)k) {
        const int q = threadIdx.x;
        st.rr[q] = st.t0[q];
        st.bb[q] = st.t1[q];
        st.othresh[q] = tol * tol * st.t1[q];
        if (Grp::leader()) {
            S.c.rr[q] = st.rr[q];
            S.c.bb[q] = st.bb[q];
            S.c.thresh[q] = st.othresh[q];
        }
    }
    __syncthreads();
}

// One system, fp64 recurrences, from the entry state in st (p_load_state or
// p_init): CG rounds restarted from the true residual.
template <class Grp>
static __device__ void p_solve_f64(BSys &S, const PersistOpts &o, PState &st, GrpSmem &gs, int *sel) {
    const int64_t n = S.A.n;
    const int k = S.k;
    int kp = 1;
    while (kp < k) kp <<= 1;
    if (threadIdx.x < 32) {
        const int q = threadIdx.x;
        st.it[q] = 0;
        st.run[q] = 0;
        st.status[q] = ST_CONV;
        if (q < k) st.thresh[q] = st.othresh[q];
    }
    __syncthreads();
    int rounds = 0;
    for (int round = 0; round <= o.max_outer; ++round) {
        if (Grp::failed()) break;
        // columns whose true residual is above the threshold and that may go on
        if (threadIdx.x < 32) {
            const int q = threadIdx.x;
            const bool go = q < k && st.bb[q] > 0.0 && st.rr[q] > st.thresh[q] &&
                            (round == 0 || st.status[q] == ST_CONV) && st.it[q] < o.maxit;
            st.run[q] = go ? 1 : 0;
            sel[q] = go ? 1 : 0;
            if (go) st.status[q] = ST_RUN;
        }
        __syncthreads();
        int any = 0;
        for (int q = 0; q < k; ++q) any |= sel[q];
        if (!any) break;
        rounds = round + 1;
        p_cg<Grp, double, double, double>(S.A, S.A.val, S.A.dinv, S.X64, S.R64, (double *)S.P, (double *)S.Q, n, k,
                                          kp, o.maxit, st, gs);
        p_resid<Grp>(S, n, k, kp, sel, st, gs);  // true residual of the columns just run
        if (round == o.max_outer && threadIdx.x < (unsigned)k && sel[threadIdx.x] &&
            st.rr[threadIdx.x] > st.thresh[threadIdx.x] && st.status[threadIdx.x] == ST_CONV)
            st.status[threadIdx.x] = ST_MAXIT;
        __syncthreads();
    }
    if (Grp::failed() && threadIdx.x < (unsigned)k && st.rr[threadIdx.x] > st.thresh[threadIdx.x])
        st.status[threadIdx.x] = ST_TIMEOUT;
    if (threadIdx.x == 0 && Grp::leader()) S.outer = rounds;  // CG rounds (restarts + 1)
    __syncthreads();
}

// One system, fp32 correction solves inside fp64 refinement.
template <class Grp>
static __device__ void p_solve_ir(BSys &S, const PersistOpts &o, PState &st, GrpSmem &gs, int *sel) {
    const int64_t n = S.A.n;
    const int k = S.k;
    int kp = 1;
    while (kp < k) kp <<= 1;
    const int j = threadIdx.x % kp;
    float *D = (float *)S.X, *R = (float *)S.R, *P = (float *)S.P, *Q = (float *)S.Q;
    if (threadIdx.x < 32) {
        const int q = threadIdx.x;
        st.it[q] = 0;
        st.status[q] = ST_CONV;
    }
    __syncthreads();
    long long inner_total = 0;
    int outer = 0;
    for (; outer < o.max_outer; ++outer) {
        if (Grp::failed()) break;
        // columns above the threshold: scale their residual down to unit norm
        if (threadIdx.x < 32) {
            const int q = threadIdx.x;
            const bool go = q < k && st.bb[q] > 0.0 && st.rr[q] > st.othresh[q];
            sel[q] = go ? 1 : 0;
            st.run[q] = go ? 1 : 0;
            st.scale[q] = go ? sqrt(st.rr[q]) : 1.0;
            st.thresh[q] = o.inner_tol * o.inner_tol;  // ||R32||^2 relative to 1
            if (go) st.status[q] = ST_RUN;
        }
        __syncthreads();
        int any = 0;
        for (int q = 0; q < k; ++q) any |= sel[q];
        if (!any) break;
        if (j < k && sel[j]) {
            const double sc = 1.0 / st.scale[j];
            for (int64_t r = Grp::gtid() / kp; r < n; r += Grp::gn() / kp) {
                R[r * k + j] = (float)(sc * S.R64[r * k + j]);
                D[r * k + j] = 0.0f;
            }
        }
        if (threadIdx.x < 32) st.it[threadIdx.x] = 0;
        __syncthreads();
        p_cg<Grp, float, float, float>(S.A, S.A.val32, S.A.dinv32, D, R, P, Q, n, k, kp, o.maxit, st, gs);
        long long mx = 0;
        for (int q = 0; q < k; ++q) if (sel[q]) mx = max(mx, st.it[q]);
        inner_total += mx;
        // x += ||r|| d in fp64, then the true residual
        if (j < k && sel[j]) {
            const double sc = st.scale[j];
            for (int64_t r = Grp::gtid() / kp; r < n; r += Grp::gn() / kp) S.X64[r * k + j] += sc * (double)D[r * k + j];
        }
        Grp::sync();  // the new X64 before p_resid gathers it
        p_resid<Grp>(S, n, k, kp, sel, st, gs);
    }
    if (threadIdx.x < (unsigned)k) {
        const int q = threadIdx.x;
        st.status[q] = (st.bb[q] == 0.0 || st.rr[q] <= st.othresh[q]) ? ST_CONV
                       : Grp::failed()                              ? ST_TIMEOUT
                                                                    : ST_MAXIT;
        st.it[q] = inner_total;
    }
    if (threadIdx.x == 0 && Grp::leader()) S.outer = outer;
    __syncthreads();
}

// The column state a finished system leaves for the host, as the batched
// loop leaves it (written by the group's leader block).
template <class Grp>
static __device__ void p_publish(BSys &S, const PState &st) {
    if (Grp::leader()) {
        if (threadIdx.x < (unsigned)S.k) {
            const int q = threadIdx.x;
            S.c.rr[q] = st.rr[q];
            S.c.status[q] = st.status[q];
            S.c.it[q] = st.it[q];
            S.c.done[q] = 1;
        }
        if (threadIdx.x == 0) S.active = 0;
    }
    __syncthreads();
}

template <class TX>
__global__ void __launch_bounds__(PNT) k_bpersist(BSys *sys, const int *list, int nlist, int *next, PersistOpts o) {
    __shared__ PState st;
    __shared__ GrpSmem gs;
    __shared__ int sel[32];
    __shared__ int idx;
    for (;;) {
        if (threadIdx.x == 0) idx = atomicAdd(next, 1);
        __syncthreads();
        const int i = idx;
        __syncthreads();
        if (i >= nlist) break;
        BSys &S = sys[list[i]];
        p_load_state(S, st);
        if (sizeof(TX) == 8) p_solve_f64<CtaGroup>(S, o, st, gs, sel);
        else p_solve_ir<CtaGroup>(S, o, st, gs, sel);
        p_publish<CtaGroup>(S, st);
    }
}

// The cluster tier: each cluster of CLUSTER_CS blocks takes the next system
// of the list (the rank-0 block draws it, the others read it through
// distributed shared memory) and solves it whole.
template <class TX>
__global__ void __cluster_dims__(CLUSTER_CS, 1, 1) __launch_bounds__(PNT)
    k_bcluster(BSys *sys, const int *list, int nlist, int *next, PersistOpts o) {
    __shared__ PState st;
    __shared__ GrpSmem gs;
    __shared__ int sel[32];
    __shared__ int idx;
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    if (threadIdx.x == 0) gs.ph = 0;
    for (;;) {
        if (threadIdx.x == 0 && cl.block_rank() == 0) idx = atomicAdd(next, 1);
        cl.sync();
        const int i = *cl.map_shared_rank(&idx, 0);
        cl.sync();  // every block has read idx before rank 0 draws again
        if (i >= nlist) break;
        BSys &S = sys[list[i]];
        if (o.init) p_init<ClusterGroup>(S, o.x0_zero, o.tol, st, gs);
        else p_load_state(S, st);
        if (sizeof(TX) == 8) p_solve_f64<ClusterGroup>(S, o, st, gs, sel);
        else p_solve_ir<ClusterGroup>(S, o, st, gs, sel);
        p_publish<ClusterGroup>(S, st);
    }
}

// The grid tier: groups of G blocks of one cooperative launch (all blocks
// resident), each group drawing the next system of the list (rank 0 draws and
// publishes the entry in an exchange) and solving it whole with the phases
// above.  An exchange wait that runs out (GridGroup) leaves the kernel's
// error word set; the group stops at its next exchange.
template <class TX>
__global__ void __launch_bounds__(PNT) k_bgrid(BSys *sys, const int *list, int nlist, int *next, double *gslots,
                                               int G, int *err, PersistOpts o) {
    __shared__ PState st;
    __shared__ GrpSmem gs;
    __shared__ int sel[32];
    __shared__ double item;
    const int group = (int)blockIdx.x / G;
    if (threadIdx.x == 0) {
        g_gctx.rank = (int)blockIdx.x % G;
        g_gctx.G = G;
        g_gctx.gn = G * PNT;
        g_gctx.failed = 0;
        g_gctx.seq = 1u;
        g_gctx.slots = gslots + (size_t)group * 2 * G * GRID_SLOT;
        g_gctx.err = err;
        g_gctx.limit_ns = o.wait_ns ? o.wait_ns : WAIT_LIMIT_NS;
        item = 0.0;
    }
    __syncthreads();
    for (;;) {
        // rank 0 draws the next entry and publishes it; the others publish nothing
        if (threadIdx.x == 0 && g_gctx.rank == 0) item = (double)atomicAdd(next, 1);
        const double *base = grid_exchange(&item, g_gctx.rank == 0 ? 1 : 0);
        const int i = GridGroup::failed() ? nlist : (int)grid_slot_value(base, 0, 0);
        if (i >= nlist) break;
        BSys &S = sys[list[i]];
        if (o.init) p_init<GridGroup>(S, o.x0_zero, o.tol, st, gs);
        else p_load_state(S, st);
        if (sizeof(TX) == 8) p_solve_f64<GridGroup>(S, o, st, gs, sel);
        else p_solve_ir<GridGroup>(S, o, st, gs, sel);
        p_publish<GridGroup>(S, st);
    }
}

// Which persistent tier takes a system: 0 none (the multi-launch loop),
// 1 CTA-local, 2 cluster, 3 grid groups.
#ifndef GB_GRID_BATCH_MAX_LOG2
#define GB_GRID_BATCH_MAX_LOG2 18
#endif
constexpr int64_t GRID_MAX_ELEMS = (int64_t)1 << GB_GRID_BATCH_MAX_LOG2;
inline int persist_tier(int64_t n, int k) {
    int kp = 1;
    while (kp < k) kp <<= 1;
    if (n * kp <= PERSIST_MAX_ELEMS) return 1;
    if (n * kp <= CLUSTER_MAX_ELEMS) return 2;
    if (n * kp <= GRID_MAX_ELEMS) return 3;  // taken only on request (PcgOptions.persist_off = 3)
    return 0;
}
inline bool persist_eligible(int64_t n, int k) { return persist_tier(n, k) == 1; }

}  // namespace gb
