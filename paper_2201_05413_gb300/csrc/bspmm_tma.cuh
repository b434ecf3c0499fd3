// bspmm_tma.cuh -- blocked multi-RHS SpMM Q = A P for the batched solvers,
// with the matrix streamed through shared memory by the TMA (as the single-RHS
// SpMV of spmv_tma.cuh).
//
// A unit (one block) is a range of whole 32-row chunks of one system; its 8
// warps take consecutive sub-ranges of it and stream their entries in stages
// of SJ column-steps through a ring of NB buffers.  For every entry the lane
// gathers the k values of row `col` of P (row-major n x k: one contiguous
// segment, vector loads when k is the class width K) and adds val * P[col]
// into its accumulators; when a chunk completes the lane writes its part of the
// row of Q and folds P[row] . Q[row] into its per-column dot products.  Wide
// rows are split across G lanes (16 bytes of the row each, so a row is gathered
// as one coalesced segment) and the chunk's 32 rows are then taken in G passes.
// The unit's per-column sums are reduced in a fixed order (lanes, then warps),
// and a system always runs in the kernel of its own width class: a unit's
// partial depends on its own rows only, and a system's result is the same
// alone and in any batch.
#pragma once
#include "bsys.cuh"
#include "spmv_tma.cuh"

namespace gb {

// Lanes per matrix row for width K: one 16-byte slice of a P row per lane
// (VW = 16 / sizeof(TX) columns), so that the g lanes of a row gather it as one
// coalesced segment; narrow widths take one lane per row.
template <class TX, int K> struct BSlice {
    static constexpr int G = (K * (int)sizeof(TX) / 16) < 1 ? 1 : K * (int)sizeof(TX) / 16;  // lanes per row
    static constexpr int VW = K / G;                                                          // columns per lane
    static constexpr int R = 32 / G;                                                          // rows per pass
};

// Resident blocks per SM for width K: accumulators (K columns) + the gather
// buffer + ~44 registers of addressing must fit 65536 / (NT x blocks).
#ifndef GB_BSPMM_INTERLEAVE
#define GB_BSPMM_INTERLEAVE 1
#endif
constexpr bool BSPMM_INTERLEAVE = GB_BSPMM_INTERLEAVE != 0;
#ifndef GB_BSPMM_WIDE_GBUF
#define GB_BSPMM_WIDE_GBUF 32
#endif
template <class TX, int K> struct BspmmOcc {
    static constexpr int ACC = K * (int)sizeof(TX) / 4;  // accumulator registers
    // gather buffer: 16 registers; fp32 rows of 64 bytes or more (G >= 4
    // lanes per row) take GB_BSPMM_WIDE_GBUF when it still fits 128 registers
    // (fp32, k = 32 on 2D P2 1024^2: 0.93 ms with 32, 1.17 ms with 24, 1.22 ms
    // with 16); fp64 keeps 16, which leaves k = 8 three blocks per SM (0.865
    // against 0.895 ms with 32)
    static constexpr int GBUF =
        (sizeof(TX) == 4 && K * (int)sizeof(TX) >= 64 && ACC + GB_BSPMM_WIDE_GBUF + 44 <= 128) ? GB_BSPMM_WIDE_GBUF
                                                                                              : 16;
    static constexpr int R = ACC + GBUF + 44;
    static constexpr int blocks = R <= 64 ? 4 : (R <= 84 ? 3 : 2);
};

// One warp's chunks c0, c0 + cs, ..., c0 + (nc - 1) cs of system S (cs = 1:
// a contiguous range, streamed as one linear array; cs > 1: the chunks are
// copied piece by piece, a stage never mixing two chunks' bytes in one copy).
// rot >= 0 (cs a power of two): chunk i is c0 + i cs + ((rot + i) mod cs)
// instead, i.e. the warp takes a different position in each group of cs
// chunks.
// For each column-step of a chunk the 32 rows are taken in G passes of R
// rows; in pass q lane l works on row q R + l / G and columns (l mod G) VW ..
// +VW.  Returns the lane's partial P.Q for its VW columns in dot[].
template <class TX, class TV, int K>
__device__ __forceinline__ void bspmm_warp_stream(const BSys &S, int64_t c0, int64_t nc, int cs, int rot, Tma2Ring<TV> &sm,
                                                  uint64_t *bars, bool *timed_out, TX (&dot)[BSlice<TX, K>::VW]) {
    constexpr int SJ = Tma2Cfg<TV>::SJ, NB = Tma2Cfg<TV>::NB;
    constexpr int G = BSlice<TX, K>::G, VW = BSlice<TX, K>::VW, R = BSlice<TX, K>::R;
    // gathers issued back to back: a buffer of BspmmOcc<TX, K>::GBUF registers
    constexpr int RG = VW * (int)sizeof(TX) / 4;  // registers per gather
    constexpr int GU = (BspmmOcc<TX, K>::GBUF / RG) < 1 ? 1 : BspmmOcc<TX, K>::GBUF / RG;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int k = S.k;
    const int sub = lane / G, slice = lane % G;
    const int c0col = slice * VW;  // first column of this lane
    const SellView &A = S.A;
    const TV *__restrict__ val = (const TV *)S.val;
    const TX *__restrict__ P = (const TX *)S.P;
    TX *__restrict__ Q = (TX *)S.Q;
#pragma unroll
    for (int u = 0; u < VW; ++u) dot[u] = TX(0);
    if (nc <= 0) return;
    auto chunk_of = [&](int64_t i) -> int64_t {
        return rot < 0 ? c0 + i * cs : c0 + i * cs + ((rot + i) & (int64_t)(cs - 1));
    };
    TX dcomp[VW];  // compensation of dot (kadd)
#pragma unroll
    for (int u = 0; u < VW; ++u) dcomp[u] = TX(0);
    const int64_t e0 = __ldg(A.chunk_ptr + c0);
    int64_t nsteps;
    if (cs == 1) {
        nsteps = (__ldg(A.chunk_ptr + c0 + nc) - e0) >> 5;
    } else {
        int64_t t = 0;
        for (int64_t i = lane; i < nc; i += 32) t += __ldg(A.chunk_w + chunk_of(i));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
        nsteps = t;
    }
    const int64_t nstages = (nsteps + SJ - 1) / SJ;
    uint64_t pol = 0;
    if (GB_TMA2_EVICT_FIRST && lane == 0) pol = l2_policy_evict_first();
    int64_t issued = 0;
    int64_t ic = 0, ioff = 0;  // issue cursor (lane 0, cs > 1): chunk index, steps of it already issued
    auto issue = [&](int64_t st) {
        issued = st + 1;
        if (lane == 0) {
            const int b = (int)(st % NB);
            const int sj = (int)min((int64_t)SJ, nsteps - st * SJ);
            mbar_expect_tx(&bars[b], (uint32_t)(sj * 32 * (sizeof(int32_t) + sizeof(TV))));
            if (cs == 1) {
                const int64_t off = e0 + st * SJ * 32;
                bulk_g2s_pol(sm.col[b], A.col + off, (uint32_t)(sj * 32 * sizeof(int32_t)), &bars[b], pol);
                bulk_g2s_pol(sm.val[b], val + off, (uint32_t)(sj * 32 * sizeof(TV)), &bars[b], pol);
            } else {
                // the stage's sj steps from the chunks at the cursor, one piece per chunk
                int filled = 0;
                while (filled < sj && ic < nc) {
                    const int64_t c = chunk_of(ic);
                    const int64_t w = __ldg(A.chunk_w + c);
                    const int take = (int)min((int64_t)(sj - filled), w - ioff);
                    if (take > 0) {
                        const int64_t off = __ldg(A.chunk_ptr + c) + ioff * 32;
                        bulk_g2s_pol(sm.col[b] + filled * 32, A.col + off, (uint32_t)(take * 32 * sizeof(int32_t)),
                                     &bars[b], pol);
                        bulk_g2s_pol(sm.val[b] + filled * 32, val + off, (uint32_t)(take * 32 * sizeof(TV)),
                                     &bars[b], pol);
                        filled += take;
                        ioff += take;
                    }
                    if (ioff >= w) {
                        ++ic;
                        ioff = 0;
                    }
                }
            }
        }
    };
    for (int64_t st = 0; st < nstages && st < NB; ++st) issue(st);

    // VW values of row `row` of a row-major n x k block from column c0col
    auto ld = [&](int64_t row, TX (&v)[VW]) {
        if (k == K) {
            const Pack<TX, VW> t = *reinterpret_cast<const Pack<TX, VW> *>(P + row * K + c0col);
#pragma unroll
            for (int u = 0; u < VW; ++u) v[u] = t.v[u];
        } else {
#pragma unroll
            for (int u = 0; u < VW; ++u) v[u] = c0col + u < k ? __ldg(P + row * k + c0col + u) : TX(0);
        }
    };
    auto stq = [&](int64_t row, const TX (&v)[VW]) {
        if (k == K) {
            Pack<TX, VW> t;
#pragma unroll
            for (int u = 0; u < VW; ++u) t.v[u] = v[u];
            *reinterpret_cast<Pack<TX, VW> *>(Q + row * K + c0col) = t;
        } else {
#pragma unroll
            for (int u = 0; u < VW; ++u)
                if (c0col + u < k) Q[row * k + c0col + u] = v[u];
        }
    };

    // consume cursor: chunk tb + ci of the warp's list (widths of tb .. tb + 31
    // held one per lane), `left` steps of it still to come
    int64_t tb = 0;
    int ci = -1, left = 0;
    int wv = (lane < nc) ? __ldg(A.chunk_w + chunk_of(lane)) : 0;
    int64_t rbase = 0;  // first row of the current chunk
    TX acc[G][VW];
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
        for (int u = 0; u < VW; ++u) acc[q][u] = TX(0);
    auto next_chunk = [&]() {
        do {
            if (++ci == 32) {
                tb += 32;
                ci = 0;
                wv = (tb + lane < nc) ? __ldg(A.chunk_w + chunk_of(tb + lane)) : 0;
            }
            left = __shfl_sync(FULL, wv, ci);
            rbase = chunk_of(tb + ci) * 32;
            if (left == 0 && tb + ci < nc) {  // an all-empty chunk: its rows of Q are zero
                TX z[VW];
#pragma unroll
                for (int u = 0; u < VW; ++u) z[u] = TX(0);
#pragma unroll
                for (int q = 0; q < G; ++q)
                    if (rbase + q * R + sub < A.n) stq(rbase + q * R + sub, z);
            }
        } while (left == 0 && tb + ci < nc);
    };
    next_chunk();
    auto flush = [&]() {  // chunk complete (warp-uniform)
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int64_t row = rbase + q * R + sub;
            if (row < A.n) {
                stq(row, acc[q]);
                TX pr[VW];
                ld(row, pr);
#pragma unroll
                for (int u = 0; u < VW; ++u) kadd(dot[u], dcomp[u], pr[u] * acc[q][u]);
            }
#pragma unroll
            for (int u = 0; u < VW; ++u) acc[q][u] = TX(0);
        }
        next_chunk();
    };
    int64_t st_fail = -1;
    for (int64_t st = 0; st < nstages; ++st) {
        const int b = (int)(st % NB);
        const bool ok = mbar_wait(&bars[b], (uint32_t)((st / NB) & 1));
        if (!__all_sync(FULL, ok)) {
            *timed_out = true;
            st_fail = st;
            break;
        }
        const int32_t *cs = sm.col[b];
        const TV *vs = sm.val[b];
        const int sj = (int)min((int64_t)SJ, nsteps - st * SJ);
        if constexpr (G == 1) {
            // one lane per row: GU consecutive steps' gathers back to back
#pragma unroll
            for (int j0 = 0; j0 < SJ; j0 += GU) {
                TX pr[GU][VW];
#pragma unroll
                for (int t = 0; t < GU; ++t)
                    if (j0 + t < sj) ld(cs[(j0 + t) * 32 + sub], pr[t]);
#pragma unroll
                for (int t = 0; t < GU; ++t)
                    if (j0 + t < sj) {
                        const TX v = to_tx<TX>(vs[(j0 + t) * 32 + sub]);
#pragma unroll
                        for (int u = 0; u < VW; ++u) acc[0][u] += v * pr[t][u];
                        if (--left == 0) flush();
                    }
            }
        } else if constexpr (GU >= G) {
            // G lanes per row, SU = GU / G whole steps' gathers back to back
            constexpr int SU = GU / G;
#pragma unroll 1
            for (int j0 = 0; j0 < sj; j0 += SU) {
                TX pr[SU][G][VW];
#pragma unroll
                for (int t = 0; t < SU; ++t)
                    if (j0 + t < sj)
#pragma unroll
                        for (int q = 0; q < G; ++q) ld(cs[(j0 + t) * 32 + q * R + sub], pr[t][q]);
#pragma unroll
                for (int t = 0; t < SU; ++t)
                    if (j0 + t < sj) {
#pragma unroll
                        for (int q = 0; q < G; ++q) {
                            const TX v = to_tx<TX>(vs[(j0 + t) * 32 + q * R + sub]);
#pragma unroll
                            for (int u = 0; u < VW; ++u) acc[q][u] += v * pr[t][q][u];
                        }
                        if (--left == 0) flush();
                    }
            }
        } else {
            // G lanes per row: a step's G passes, GU gathers at a time; the
            // step loop is kept rolled so the chunk end has one code path
#pragma unroll 1
            for (int jj = 0; jj < sj; ++jj) {
#pragma unroll
                for (int q0 = 0; q0 < G; q0 += GU) {
                    TX pr[GU][VW];
#pragma unroll
                    for (int t = 0; t < GU; ++t)
                        if (q0 + t < G) ld(cs[jj * 32 + (q0 + t) * R + sub], pr[t]);
#pragma unroll
                    for (int t = 0; t < GU; ++t)
                        if (q0 + t < G) {
                            const TX v = to_tx<TX>(vs[jj * 32 + (q0 + t) * R + sub]);
#pragma unroll
                            for (int u = 0; u < VW; ++u) acc[q0 + t][u] += v * pr[t][u];
                        }
                }
                if (--left == 0) flush();
            }
        }
        __syncwarp();
        fence_proxy_async();  // our reads of buffer b precede the next bulk write into it
        if (st + NB < nstages) issue(st + NB);
    }
    if (st_fail >= 0 && lane == 0) {
        for (int64_t s2 = st_fail; s2 < issued; ++s2)
            (void)mbar_wait(&bars[s2 % NB], (uint32_t)((s2 / NB) & 1));
    }
#pragma unroll
    for (int u = 0; u < VW; ++u) dot[u] -= dcomp[u];
    __syncwarp();
}

template <class TV> constexpr size_t bspmm_tma_smem() { return tma2_smem_bytes<TV>(); }

template <class TX, class TV, int K>
__global__ void __launch_bounds__(NT, (BspmmOcc<TX, K>::blocks))
    k_bspmm_tma(BSys *sys, const int *unit_sys, int unit_base, BGlobal *G_, double *partials) {
    if (G_->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && G_->use_cond) cudaGraphSetConditional(G_->cond, 0);
        return;
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double sm[NT];
    __shared__ double csum[NT / 32][32];
    const int u = unit_base + blockIdx.x;  // this block's unit of the batch's unit table
    const int s = unit_sys[u];
    BSys &S = sys[s];
    if (S.active == 0) return;
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
    const int64_t cpu = S.rows_per_unit >> 5;  // chunks per unit
    const int64_t uc0 = (int64_t)(u - S.unit0) * cpu;
    const int64_t uc1 = min(S.A.nchunks, uc0 + cpu);
    bool timed_out = false;
    constexpr int G = BSlice<TX, K>::G, VW = BSlice<TX, K>::VW;
    TX dot[VW];
    if (BSPMM_INTERLEAVE && G > 1 && sizeof(TX) == 4) {
        // fp32 rows of wide P blocks (G lanes per row): the block's 8 warps
        // work on the 8 chunks of one sorting window (256 rows) at a time,
        // so they gather overlapping sets of P rows, and warp w takes chunk
        // (w + m) mod 8 of the unit's m-th window: the sort puts a window's
        // longest rows in its first chunk, and the rotation gives every warp
        // each position once per 8 windows, so the warps finish together
        // (2D P2, k = 32: 0.773 against 0.916 ms with contiguous ranges at
        // 1024^2, 2.69 against 3.34 ms at 2048^2)
        int64_t nc = 0;
        while (nc < cpu && uc0 + nc * TMA_WARPS + ((warp + nc) & (TMA_WARPS - 1)) < uc1) ++nc;
        bspmm_warp_stream<TX, TV, K>(S, uc0, nc, TMA_WARPS, warp, bufs[warp], &bars[NB * warp], &timed_out, dot);
    } else {
        const int64_t cpw = (cpu + TMA_WARPS - 1) / TMA_WARPS;
        const int64_t wc0 = min(uc1, uc0 + warp * cpw), wc1 = min(uc1, wc0 + cpw);
        bspmm_warp_stream<TX, TV, K>(S, wc0, wc1 - wc0, 1, -1, bufs[warp], &bars[NB * warp], &timed_out, dot);
    }
    if (timed_out && lane == 0) atomicExch(&G_->err, 1);
    // per-column unit sums in a fixed order: the lanes of a column inside the
    // warp (xor tree over the lane bits above the slice), then warps in order
#pragma unroll
    for (int o = G; o < 32; o <<= 1)
#pragma unroll
        for (int u = 0; u < VW; ++u) dot[u] += __shfl_xor_sync(0xffffffffu, dot[u], o);
    if (lane < G)
#pragma unroll
        for (int u = 0; u < VW; ++u) csum[warp][lane * VW + u] = (double)dot[u];
    __syncthreads();
    const int k = S.k, kw = S.kw;
    if (threadIdx.x < (unsigned)k) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += csum[w][threadIdx.x];
        partials[((size_t)u * 2) * KMAX + threadIdx.x] = t;
    }
    if (sys_arrive_last(&S.ticket, S.nunits)) {
        const double pq = col_unit_sum_block(partials, S.unit0, S.nunits, 0, 2, kw, sm);
        if (threadIdx.x < (unsigned)k && !S.c.done[threadIdx.x]) {
            const int jj = threadIdx.x;
            S.c.pq[jj] = pq;
            if (G_->err) { S.c.status[jj] = ST_TIMEOUT; S.c.done[jj] = 1; }
            else if (!(pq > 0.0) || !isfinite(pq)) { S.c.status[jj] = ST_BREAK; S.c.done[jj] = 1; }
            else S.c.alpha[jj] = S.c.rho[jj] / pq;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.ticket = 0;
            retire_if_idle(S, G_);
        }
    }
}

// SpMM over the units [unit_base, unit_base + units) of the unit table, all
// of systems of width class K (32-row chunks).
template <class TX, class TV>
static void launch_bspmm_tma(int K, int unit_base, int units, BSys *d_sys, const int *d_unit_sys, BGlobal *d_G,
                             double *partials, cudaStream_t s) {
    if (units <= 0) return;
#define GB_BSPMM_CASE(KK)                                                                                     \
    case KK: {                                                                                                \
        constexpr int smem = (int)bspmm_tma_smem<TV>();                                                      \
        static bool attr = false;                                                                             \
        if (!attr) {                                                                                          \
            cudaFuncSetAttribute(k_bspmm_tma<TX, TV, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
            attr = true;                                                                                      \
        }                                                                                                     \
        ::gb::count_launches(1);                                                                              \
        k_bspmm_tma<TX, TV, KK><<<units, NT, smem, s>>>(d_sys, d_unit_sys, unit_base, d_G, partials);         \
        break;                                                                                                \
    }
    switch (K) {
        GB_BSPMM_CASE(1)
        GB_BSPMM_CASE(2)
        GB_BSPMM_CASE(4)
        GB_BSPMM_CASE(8)
        GB_BSPMM_CASE(16)
        GB_BSPMM_CASE(32)
    }
#undef GB_BSPMM_CASE
}

}  // namespace gb
