// sell.cuh -- SELL-C-sigma matrix object shared by the builder and the solvers.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace gb {

// Plain view passed by value to kernels.
struct SellView {
    int64_t n, nchunks;
    int C;
    const int64_t *chunk_ptr;
    const int32_t *row_len;
    const int32_t *col;
    const double *val;
    const float *val32;
    const __nv_bfloat16 *val16;
    const double *dinv;
    const float *dinv32;
    const int32_t *chunk_w;
    const int32_t *warp_chunk;  // nwarps+1 chunk bounds, balanced by padded nonzeros (C == 32)
    int nwarps;
    const int16_t *col16;       // column - min(row, n-1) per padded slot, or null (C == 32)
};

// Host-side view: the kernel view plus the warp partition of the fp32
// SpMV's 5-blocks-per-SM grid, passed to that kernel as its own argument.
// (Kept out of SellView: every kernel takes SellView by value, and a larger
// SellView changed the fp64 SpMV's code -- 54 instead of 52 registers -- and
// slowed it from 120 to 137-142 us on 2D P2 1024^2.)
struct SellViewH : SellView {
    const int32_t *warp_chunk5 = nullptr;
    int nwarps5 = 0;
};

// Block-Jacobi data of a matrix (bjacobi.cuh), passed by value to kernels.
struct BjView {
    int bs = 0;                    // 0: no block-Jacobi data
    int64_t nblk = 0;
    const double *w = nullptr;     // nblk x bs(bs+1)/2: upper triangle of each inverse, row-major
    const float *w32 = nullptr;    // the same in fp32
    const uint8_t *loc = nullptr;  // nblk*bs: SELL position of free dof o minus 256 floor(o/256)
    double lam = 0.0;              // upper bound of the largest eigenvalue of M^-1 (row sums)
};

}  // namespace gb

struct gb_sell {
    int64_t n = 0, nnz = 0, padded = 0, nchunks = 0;
    int C = 32, sigma = 1, max_row = 0;
    int32_t *perm = nullptr, *iperm = nullptr, *row_len = nullptr, *chunk_w = nullptr, *col = nullptr;
    int32_t *warp_chunk = nullptr, *warp_chunk5 = nullptr;
    int16_t *col16 = nullptr;
    int nwarps = 0, nwarps5 = 0;
    int variant_hint = 0;  // SpMV variant solves use by default (set by sell_autotune)
    // block-Jacobi preconditioner (sell_block_jacobi): packed inverses, row positions
    int bj_bs = 0;
    int64_t bj_nblk = 0;
    double *bj_w = nullptr;
    float *bj_w32 = nullptr;
    uint8_t *bj_loc = nullptr;
    double bj_lam = 0.0;
    double dinv_max = 0.0; // max_i 1/K_ii (host copy)
    int64_t *chunk_ptr = nullptr;
    double *val = nullptr, *dinv = nullptr;
    float *val32 = nullptr, *dinv32 = nullptr;
    __nv_bfloat16 *val16 = nullptr;
    gb::Mem mem;
    gb::SellViewH view() const {
        gb::SellViewH v;
        static_cast<gb::SellView &>(v) = gb::SellView{n, nchunks, C, chunk_ptr, row_len, col, val, val32, val16,
                                                      dinv, dinv32, chunk_w, warp_chunk, nwarps, col16};
        v.warp_chunk5 = warp_chunk5;
        v.nwarps5 = nwarps5;
        return v;
    }
    gb::BjView bj_view() const {
        gb::BjView b;
        b.bs = bj_bs; b.nblk = bj_nblk; b.w = bj_w; b.w32 = bj_w32; b.loc = bj_loc; b.lam = bj_lam;
        return b;
    }
};
