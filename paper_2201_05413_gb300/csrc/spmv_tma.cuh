// spmv_tma.cuh -- SELL-32 SpMV with TMA-staged matrix streams.
//
// Each warp owns a contiguous range of chunks, balanced by padded nonzeros
// (gb_sell::warp_chunk).  Because chunks are stored back to back, the range's
// column indices and values are two contiguous arrays; the warp streams them
// in stages of SJ column-steps (SJ*32 entries): one lane issues two 1-D bulk
// copies (cp.async.bulk, the TMA's non-tensor form) per stage into a ring of
// NB shared-memory buffers, each completing on its own mbarrier, with NB
// stages in flight.  While the copies land, the lanes gather p for the stage
// they hold (SJ independent loads back to back) and accumulate.  Waits use a
// suspend-time hint and are bounded by %globaltimer: a wait that runs out
// sets S->err (-> GB_TIMEOUT) and the warp stops, after letting its copies
// in flight land.
#pragma once
#include "pcg.cuh"

namespace gb {

#ifndef GB_TMA_SJ
#define GB_TMA_SJ 8
#endif
#ifndef GB_TMA_HINT_NS
#define GB_TMA_HINT_NS 0
#endif
#ifndef GB_TMA_NB64
#define GB_TMA_NB64 2
#endif
#ifndef GB_TMA_NB32
#define GB_TMA_NB32 3
#endif
#ifndef GB_TMA_PREFETCH
#define GB_TMA_PREFETCH 0  // stages beyond the ring prefetched into L2 (0 = off)
#endif
constexpr int SJ = GB_TMA_SJ;  // column-steps per staged slice
constexpr int TMA_WARPS = 8;   // warps per block (TMA_BLOCKS_PER_SM blocks per SM)
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps (up to the hint) until
// the phase completes instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
#if GB_TMA_HINT_NS > 0
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(GB_TMA_HINT_NS)
        : "memory");
#else
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
#endif
    return ok != 0;
}
// bounded wait; true when the phase completed, false when limit_ns passed
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = WAIT_LIMIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 8; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ring depth (stages in flight per warp): fp64 stages are 3 KB, fp32 2 KB, bf16 1.5 KB
template <class TV> struct TmaDepth { static constexpr int NB = sizeof(TV) == 8 ? GB_TMA_NB64 : GB_TMA_NB32; };

// TI: int32_t (column indices) or int16_t (column - min(row, n-1) deltas)
template <class TV, int NB, class TI = int32_t>
struct TmaRing {
    TI col[NB][SJ * 32];
    TV val[NB][SJ * 32];
};

template <class TV, class TI = int32_t>
constexpr size_t tma_smem_bytes() {
    return TMA_WARPS * sizeof(TmaRing<TV, TmaDepth<TV>::NB, TI>) + TMA_WARPS * TmaDepth<TV>::NB * sizeof(uint64_t);
}

template <class TX> __device__ __forceinline__ TX ldg_vec(const TX *p) { return __ldg(p); }

template <class TX, class TV>
__device__ __forceinline__ TX to_tx(TV v) {
    if constexpr (sizeof(TV) == 2) return (TX)__bfloat162float(v);
    else return (TX)v;
}

// One warp's chunk range as a linear stream.  The range's indices and values
// are contiguous (chunks are stored back to back), so the warp walks them in
// stages of SJ column-steps (SJ*32 entries) through a ring of NB shared-memory
// buffers, NB stages in flight, independently of where chunks begin or end.
// Inside a stage the SJ gathers of p are issued first, then the products are
// accumulated; a chunk ends when its column counter reaches the chunk width.
// Returns the warp's partial p.q (per lane); *timed_out on a wait that ran out.
template <class TV, class TX, int NB, class TI>
__device__ __forceinline__ TX spmv_warp_stream(const SellView &A, const TV *__restrict__ val,
                                               const TX *__restrict__ p, TX *__restrict__ q,
                                               int c0, int c1, TmaRing<TV, NB, TI> &sm, uint64_t *bars,
                                               bool *timed_out) {
    constexpr bool DELTA = sizeof(TI) == 2;
    const TI *colsrc = DELTA ? (const TI *)A.col16 : (const TI *)A.col;
    const int lane = threadIdx.x & 31;
    TX dot = TX(0);
    if (c0 >= c1) return dot;
    const int64_t e0 = __ldg(A.chunk_ptr + c0), e1 = __ldg(A.chunk_ptr + c1);
    const int64_t nsteps = (e1 - e0) >> 5;
    const int64_t nstages = (nsteps + SJ - 1) / SJ;
    auto issue = [&](int64_t st) {
        if (lane == 0) {
            const int b = (int)(st % NB);
            const int sj = (int)min((int64_t)SJ, nsteps - st * SJ);
            const int64_t off = e0 + st * SJ * 32;
            const uint32_t bc = (uint32_t)(sj * 32 * sizeof(TI));
            const uint32_t bv = (uint32_t)(sj * 32 * sizeof(TV));
            mbar_expect_tx(&bars[b], bc + bv);
            bulk_g2s(sm.col[b], colsrc + off, bc, &bars[b]);
            bulk_g2s(sm.val[b], val + off, bv, &bars[b]);
            if (GB_TMA_PREFETCH > 0 && st + GB_TMA_PREFETCH < nstages) {
                // warm L2 with a stage beyond the ring: more bytes in flight than shared memory holds
                const int64_t pst = st + GB_TMA_PREFETCH;
                const int psj = (int)min((int64_t)SJ, nsteps - pst * SJ);
                const int64_t poff = e0 + pst * SJ * 32;
                bulk_prefetch_l2(colsrc + poff, (uint32_t)(psj * 32 * sizeof(TI)));
                bulk_prefetch_l2(val + poff, (uint32_t)(psj * 32 * sizeof(TV)));
            }
        }
    };
    for (int64_t st = 0; st < nstages && st < NB; ++st) issue(st);
    // current chunk (skip empty ones: they own no steps, their rows get q = 0)
    int c = c0, w = __ldg(A.chunk_w + c);
    while (w == 0) {
        const int64_t rr = (int64_t)c * 32 + lane;
        if (rr < A.n) q[rr] = TX(0);
        ++c;
        w = c < c1 ? __ldg(A.chunk_w + c) : 1;
    }
    int64_t r = (int64_t)c * 32 + lane;
    int L = r < A.n ? __ldg(A.row_len + r) : 0;
    int32_t rb = (int32_t)(r < A.n ? r : A.n - 1);  // base of the column deltas
    int j = 0;
    TX acc = TX(0);
    int64_t st_fail = -1;
    for (int64_t st = 0; st < nstages; ++st) {
        const int b = (int)(st % NB);
        const uint32_t parity = (uint32_t)((st / NB) & 1);
        bool ok = true;
        if (lane == 0) ok = mbar_wait(&bars[b], parity);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) {
            *timed_out = true;
            st_fail = st;
            break;
        }
        const int sj = (int)min((int64_t)SJ, nsteps - st * SJ);
        TX pv[SJ];
        {
            // gather pass: a stage may cross chunk boundaries, so 16-bit
            // deltas take the row base of the chunk each step belongs to
            int jg = j, wg = w, cg = c;
            int32_t rbg = rb;
#pragma unroll
            for (int jj = 0; jj < SJ; ++jj)
                if (jj < sj) {
                    const int32_t cj = DELTA ? rbg + (int32_t)sm.col[b][jj * 32 + lane] : (int32_t)sm.col[b][jj * 32 + lane];
                    pv[jj] = __ldg(p + cj);
                    if (DELTA && ++jg == wg) {
                        jg = 0;
                        do {
                            ++cg;
                            wg = cg < c1 ? __ldg(A.chunk_w + cg) : 1;
                        } while (wg == 0);
                        const int64_t rr = (int64_t)cg * 32 + lane;
                        rbg = (int32_t)(rr < A.n ? rr : A.n - 1);
                    }
                }
        }
#pragma unroll
        for (int jj = 0; jj < SJ; ++jj) {
            if (jj < sj) {
                if (j < L) acc += to_tx<TX>(sm.val[b][jj * 32 + lane]) * pv[jj];
                if (++j == w) {  // chunk complete (warp-uniform)
                    if (r < A.n) {
                        q[r] = acc;
                        dot += __ldg(p + r) * acc;
                    }
                    acc = TX(0);
                    j = 0;
                    ++c;
                    w = c < c1 ? __ldg(A.chunk_w + c) : 1;
                    while (w == 0) {
                        const int64_t rr = (int64_t)c * 32 + lane;
                        if (rr < A.n) q[rr] = TX(0);
                        ++c;
                        w = c < c1 ? __ldg(A.chunk_w + c) : 1;
                    }
                    r = (int64_t)c * 32 + lane;
                    L = (c < c1 && r < A.n) ? __ldg(A.row_len + r) : 0;
                    rb = (int32_t)(r < A.n ? r : A.n - 1);
                }
            }
        }
        __syncwarp();
        fence_proxy_async();  // our reads of buffer b precede the next bulk write into it
        if (st + NB < nstages) issue(st + NB);
    }
    if (st_fail >= 0 && lane == 0) {
        // stages [st_fail, st_fail + NB) were issued and not consumed: let
        // their copies land before the buffers go away (bounded waits)
        for (int64_t s2 = st_fail; s2 < nstages && s2 < st_fail + NB; ++s2)
            (void)mbar_wait(&bars[s2 % NB], (uint32_t)((s2 / NB) & 1));
    }
    __syncwarp();
    return dot;
}


// ------------------------------------------------------------------------
// Second streaming loop (32-bit indices): the per-entry work is one shared-
// memory index load, one gather of p, one shared-memory value load and one
// FMA.  No per-lane length test: a padded slot holds value 0 and points at
// the row itself (or at row 0 past n), so it adds exactly zero.  The chunk
// widths of the warp's range are held 32 at a time in a register (lane l:
// chunk cb + l) and broadcast by shuffle when a chunk completes.  The matrix
// copies carry an L2 evict-first policy: the matrix is read once per
// iteration and should not push the solver's vectors out of L2.
#ifndef GB_TMA2_SJ32
#define GB_TMA2_SJ32 8
#endif
#ifndef GB_TMA2_NB32
#define GB_TMA2_NB32 2
#endif
#ifndef GB_TMA2_NB16
#define GB_TMA2_NB16 3
#endif
#ifndef GB_TMA2_SJ64
#define GB_TMA2_SJ64 8
#endif
#ifndef GB_TMA2_NB64
#define GB_TMA2_NB64 2
#endif
#ifndef GB_TMA2_EVICT_FIRST
#define GB_TMA2_EVICT_FIRST 1
#endif

template <class TV> struct Tma2Cfg {
    static constexpr int SJ = sizeof(TV) == 8 ? GB_TMA2_SJ64 : GB_TMA2_SJ32;
    static constexpr int NB = sizeof(TV) == 8 ? GB_TMA2_NB64 : (sizeof(TV) == 4 ? GB_TMA2_NB32 : GB_TMA2_NB16);
};

template <class TV>
struct Tma2Ring {
    static constexpr int SJ = Tma2Cfg<TV>::SJ, NB = Tma2Cfg<TV>::NB;
    int32_t col[NB][SJ * 32];
    TV val[NB][SJ * 32];
};

template <class TV>
constexpr size_t tma2_smem_bytes() {
    return TMA_WARPS * sizeof(Tma2Ring<TV>) + TMA_WARPS * Tma2Cfg<TV>::NB * sizeof(uint64_t);
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_g2s_pol(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                             uint64_t pol) {
#if GB_TMA2_EVICT_FIRST
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
#else
    (void)pol;
    bulk_g2s(dst, src, bytes, bar);
#endif
}

// DM (dot mode): 0 returns sum_r p_r q_r (CG's p.Ap); 1 returns sum_r d1_r q_r;
// 2 also adds sum_r q_r q_r into *dot2 (BiCGSTAB's r^.v, and t.s with t.t).
template <class TV, class TX, int DM = 0>
__device__ __forceinline__ TX spmv_warp_stream2(const SellView &A, const TV *__restrict__ val,
                                                const TX *__restrict__ p, TX *__restrict__ q, int c0, int c1,
                                                Tma2Ring<TV> &sm, uint64_t *bars, bool *timed_out,
                                                const TX *__restrict__ d1 = nullptr, TX *dot2 = nullptr) {
    constexpr int SJ = Tma2Cfg<TV>::SJ, NB = Tma2Cfg<TV>::NB;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    TX dot = TX(0);
    if (c0 >= c1) return dot;
    const int64_t e0 = __ldg(A.chunk_ptr + c0), e1 = __ldg(A.chunk_ptr + c1);
    const int64_t nsteps = (e1 - e0) >> 5;
    const int64_t nstages = (nsteps + SJ - 1) / SJ;
    uint64_t pol = 0;
    if (GB_TMA2_EVICT_FIRST && lane == 0) pol = l2_policy_evict_first();
    int64_t issued = 0;  // stages whose copies have been started
    auto issue = [&](int64_t st) {
        issued = st + 1;
        if (lane == 0) {
            const int b = (int)(st % NB);
            const int sj = (int)min((int64_t)SJ, nsteps - st * SJ);
            const int64_t off = e0 + st * SJ * 32;
            const uint32_t bc = (uint32_t)(sj * 32 * sizeof(int32_t));
            const uint32_t bv = (uint32_t)(sj * 32 * sizeof(TV));
            mbar_expect_tx(&bars[b], bc + bv);
            bulk_g2s_pol(sm.col[b], A.col + off, bc, &bars[b], pol);
            bulk_g2s_pol(sm.val[b], val + off, bv, &bars[b], pol);
        }
    };
    for (int64_t st = 0; st < nstages && st < NB; ++st) issue(st);

    // chunk cursor: current chunk cb + ci, `left` steps of it still to come
    int cb = c0, ci = -1, left = 0;
    int wv = (cb + lane < c1) ? __ldg(A.chunk_w + cb + lane) : 0;
    int64_t r = (int64_t)c0 * 32 + lane - 32;
    TX pr = TX(0);
    auto next_chunk = [&]() {
        do {
            if (++ci == 32) {
                cb += 32;
                ci = 0;
                wv = (cb + lane < c1) ? __ldg(A.chunk_w + cb + lane) : 0;
            }
            left = __shfl_sync(FULL, wv, ci);
            r += 32;
            if (left == 0 && cb + ci < c1 && r < A.n) q[r] = TX(0);  // an all-empty chunk
        } while (left == 0 && cb + ci < c1);
        if constexpr (DM == 0) pr = (cb + ci < c1 && r < A.n) ? __ldg(p + r) : TX(0);
        else pr = (cb + ci < c1 && r < A.n) ? __ldg(d1 + r) : TX(0);
    };
    next_chunk();
    TX acc = TX(0);
    auto step = [&](TV v, TX pv) {
        acc += to_tx<TX>(v) * pv;
        if (--left == 0) {  // chunk complete (warp-uniform)
            if (r < A.n) {
                q[r] = acc;
                dot += pr * acc;
                if constexpr (DM == 2) *dot2 += acc * acc;
            }
            acc = TX(0);
            next_chunk();
        }
    };
    int64_t st_fail = -1;
    for (int64_t st = 0; st < nstages; ++st) {
        const int b = (int)(st % NB);
        const uint32_t parity = (uint32_t)((st / NB) & 1);
        const bool ok = mbar_wait(&bars[b], parity);
        if (!__all_sync(FULL, ok)) {
            *timed_out = true;
            st_fail = st;
            break;
        }
        const int32_t *cs = sm.col[b];
        const TV *vs = sm.val[b];
        const int sj = (int)min((int64_t)SJ, nsteps - st * SJ);
        if (sj == SJ) {
            TX pv[SJ];
#pragma unroll
            for (int jj = 0; jj < SJ; ++jj) pv[jj] = __ldg(p + cs[jj * 32 + lane]);
#pragma unroll
            for (int jj = 0; jj < SJ; ++jj) step(vs[jj * 32 + lane], pv[jj]);
        } else {
            for (int jj = 0; jj < sj; ++jj) step(vs[jj * 32 + lane], __ldg(p + cs[jj * 32 + lane]));
        }
        __syncwarp();
        fence_proxy_async();  // our reads of buffer b precede the next bulk write into it
        if (st + NB < nstages) issue(st + NB);
    }
    if (st_fail >= 0 && lane == 0) {
        for (int64_t s2 = st_fail; s2 < issued; ++s2)
            (void)mbar_wait(&bars[s2 % NB], (uint32_t)((s2 / NB) & 1));
    }
    __syncwarp();
    return dot;
}

}  // namespace gb
