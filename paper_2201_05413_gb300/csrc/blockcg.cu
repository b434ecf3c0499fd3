// blockcg.cu -- block conjugate gradients for A X = B, the block of
// right-hand sides of Sec. 4.3 (Eq. MRH) solved in one shared Krylov space.
//
// The method (O'Leary 1980) in the breakdown-free form of Ji and Li (2017):
// the search block P is orthonormalised with a rank test every step, so
// dependent directions -- a rank-deficient B, columns converging at different
// rates -- are dropped instead of making P^T A P singular.  Per step:
//   Q = A P;  alpha = (P^T Q)^-1 P^T R;  X += P alpha;  R -= Q alpha;
//   Z = M^-1 R;  beta = -(P^T Q)^-1 Q^T Z;  W = Z + P beta;  P = orth(W),
// orth(W) = W T with T from the eigen-decomposition of the (column-scaled)
// Gram matrix W^T W, keeping eigenvalues above a relative threshold.
//
// GB300 mapping: the n-sized work -- the SpMM, the tall-skinny Gram products
// U^T V and the block combinations -- runs in the kernels below on row-major
// n x KW blocks (KW = 4, 8, 16 or 32); the k x k algebra (a Cholesky factor of
// P^T Q, the eigen-decomposition) is done on the host between them, three
// host round trips per step.  The Gram products cost O(n k^2) operations per
// step, which GB300's fp64 units make the dominant cost at k = 32; the fp32
// inner solve of the refinement mode (fp32 products, tile sums carried in
// fp64) runs them at fp32 rate.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pcg.cuh"

namespace gb {
namespace {

constexpr int BC_NT = 256;
constexpr int BC_TR = 32;  // rows per Gram tile

template <class T> struct alignas(4 * sizeof(T)) Quad { T v[4]; };

// ---------------------------------------------------------------- kernels --
// Y = A X for row-major n x KW blocks in SELL order; one thread per (row,
// column quad).  The threads of a row read the same matrix entries in the
// same instruction (one request).
template <class TV, class TX, int KW>
__global__ void __launch_bounds__(BC_NT) k_bc_spmm(SellView A, const TV *__restrict__ val,
                                                   const TX *__restrict__ X, TX *__restrict__ Y) {
    constexpr int QW = KW / 4;
    const int64_t items = A.n * QW;
    for (int64_t t = blockIdx.x * (int64_t)BC_NT + threadIdx.x; t < items; t += (int64_t)gridDim.x * BC_NT) {
        const int64_t r = t / QW;
        const int q = (int)(t - r * QW);
        const int64_t c = r / A.C;
        const int64_t base = A.chunk_ptr[c] + (r - c * A.C);
        const int L = A.row_len[r];
        TX acc[4] = {TX(0), TX(0), TX(0), TX(0)};
        for (int j = 0; j < L; ++j) {
            const int64_t e = base + (int64_t)j * A.C;
            const TX a = (TX)ld_val(val + e);
            const int col = ld_col(A.col + e);
            const Quad<TX> x = reinterpret_cast<const Quad<TX> *>(X + (int64_t)col * KW)[q];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += a * x.v[u];
        }
        Quad<TX> o;
#pragma unroll
        for (int u = 0; u < 4; ++u) o.v[u] = acc[u];
        reinterpret_cast<Quad<TX> *>(Y + r * KW)[q] = o;
    }
}

// Per-block partial sums of U^T V (KW x KW) over tiles of BC_TR rows: each
// tile's products are summed in TX and added to an fp64 accumulator.
template <class TX, int KW>
__global__ void __launch_bounds__(BC_NT) k_bc_gram(int64_t n, const TX *__restrict__ U, const TX *__restrict__ V,
                                                   double *__restrict__ part) {
    constexpr int E = KW * KW;
    constexpr int PER = (E + BC_NT - 1) / BC_NT;
    __shared__ TX us[BC_TR][KW], vs[BC_TR][KW];
    double acc[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) acc[p] = 0.0;
    const int64_t ntiles = (n + BC_TR - 1) / BC_TR;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * BC_TR;
        for (int e = threadIdx.x; e < BC_TR * KW; e += BC_NT) {
            const int rr = e / KW, cc = e - (e / KW) * KW;
            const int64_t r = r0 + rr;
            us[rr][cc] = r < n ? U[r * KW + cc] : TX(0);
            vs[rr][cc] = r < n ? V[r * KW + cc] : TX(0);
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int e = threadIdx.x + p * BC_NT;
            if (e < E) {
                const int a = e / KW, c = e - (e / KW) * KW;
                TX s = TX(0);
#pragma unroll 8
                for (int rr = 0; rr < BC_TR; ++rr) s += us[rr][a] * vs[rr][c];
                acc[p] += (double)s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = threadIdx.x + p * BC_NT;
        if (e < E) part[(size_t)blockIdx.x * E + e] = acc[p];
    }
}

// Per-block partial column sums of squares of U (n x KW).
template <class TX, int KW>
__global__ void __launch_bounds__(BC_NT) k_bc_colsq(int64_t n, const TX *__restrict__ U, double *__restrict__ part) {
    __shared__ double sm[BC_NT];
    constexpr int RPB = BC_NT / KW;  // rows per block step
    const int c = threadIdx.x % KW, rr = threadIdx.x / KW;
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * RPB + rr; r < n; r += (int64_t)gridDim.x * RPB) {
        const double u = (double)U[r * KW + c];
        acc += u * u;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < KW) {
        double s = 0.0;
        for (int q = 0; q < RPB; ++q) s += sm[q * KW + threadIdx.x];
        part[(size_t)blockIdx.x * KW + threadIdx.x] = s;
    }
}

// out[e] = sum over blocks b (in order) of part[b*E + e]
__global__ void k_bc_sum(int nb, int E, const double *__restrict__ part, double *__restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[(size_t)b * E + e];
        out[e] = s;
    }
}

// X += P alpha, R -= Q alpha, Z = D^-1 R (alpha: KW x KW fp64, row-major)
template <class TX, class TD, int KW>
__global__ void __launch_bounds__(BC_NT) k_bc_update(int64_t n, const TX *__restrict__ P, const TX *__restrict__ Q,
                                                     const double *__restrict__ alpha, TX *__restrict__ X,
                                                     TX *__restrict__ R, const TD *__restrict__ dinv,
                                                     TX *__restrict__ Z) {
    constexpr int QW = KW / 4;
    __shared__ TX al[KW][KW];
    for (int e = threadIdx.x; e < KW * KW; e += BC_NT) al[e / KW][e % KW] = (TX)alpha[e];
    __syncthreads();
    const int64_t items = n * QW;
    for (int64_t t = blockIdx.x * (int64_t)BC_NT + threadIdx.x; t < items; t += (int64_t)gridDim.x * BC_NT) {
        const int64_t r = t / QW;
        const int q = (int)(t - r * QW);
        TX dx[4] = {TX(0), TX(0), TX(0), TX(0)}, dr[4] = {TX(0), TX(0), TX(0), TX(0)};
#pragma unroll 1
        for (int m4 = 0; m4 < QW; ++m4) {
            const Quad<TX> pm = reinterpret_cast<const Quad<TX> *>(P + r * KW)[m4];
            const Quad<TX> qm = reinterpret_cast<const Quad<TX> *>(Q + r * KW)[m4];
#pragma unroll
            for (int mm = 0; mm < 4; ++mm)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    dx[u] += pm.v[mm] * al[4 * m4 + mm][4 * q + u];
                    dr[u] += qm.v[mm] * al[4 * m4 + mm][4 * q + u];
                }
        }
        Quad<TX> xo = reinterpret_cast<const Quad<TX> *>(X + r * KW)[q];
        Quad<TX> ro = reinterpret_cast<const Quad<TX> *>(R + r * KW)[q];
        Quad<TX> zo;
        const TX d = (TX)dinv[r];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            xo.v[u] += dx[u];
            ro.v[u] -= dr[u];
            zo.v[u] = d * ro.v[u];
        }
        reinterpret_cast<Quad<TX> *>(X + r * KW)[q] = xo;
        reinterpret_cast<Quad<TX> *>(R + r * KW)[q] = ro;
        reinterpret_cast<Quad<TX> *>(Z + r * KW)[q] = zo;
    }
}

// Y = U T1 + V T2 (T1, T2: KW x KW fp64; V may be null); or with diag_u,
// Y = U + V T2 (T1 the identity).
template <class TX, int KW>
__global__ void __launch_bounds__(BC_NT) k_bc_comb(int64_t n, const TX *__restrict__ U, const double *__restrict__ T1,
                                                   int diag_u, const TX *__restrict__ V,
                                                   const double *__restrict__ T2, TX *__restrict__ Y) {
    constexpr int QW = KW / 4;
    __shared__ TX t1[KW][KW], t2[KW][KW];
    for (int e = threadIdx.x; e < KW * KW; e += BC_NT) {
        t1[e / KW][e % KW] = diag_u ? (TX)(e / KW == e % KW ? 1.0 : 0.0) : (TX)T1[e];
        t2[e / KW][e % KW] = V ? (TX)T2[e] : TX(0);
    }
    __syncthreads();
    const int64_t items = n * QW;
    for (int64_t t = blockIdx.x * (int64_t)BC_NT + threadIdx.x; t < items; t += (int64_t)gridDim.x * BC_NT) {
        const int64_t r = t / QW;
        const int q = (int)(t - r * QW);
        TX y[4] = {TX(0), TX(0), TX(0), TX(0)};
        if (diag_u) {
            const Quad<TX> um = reinterpret_cast<const Quad<TX> *>(U + r * KW)[q];
#pragma unroll
            for (int u = 0; u < 4; ++u) y[u] = um.v[u];
        } else {
    #pragma unroll 1
        for (int m4 = 0; m4 < QW; ++m4) {
                const Quad<TX> um = reinterpret_cast<const Quad<TX> *>(U + r * KW)[m4];
#pragma unroll
                for (int mm = 0; mm < 4; ++mm)
#pragma unroll
                    for (int u = 0; u < 4; ++u) y[u] += um.v[mm] * t1[4 * m4 + mm][4 * q + u];
            }
        }
        if (V) {
    #pragma unroll 1
        for (int m4 = 0; m4 < QW; ++m4) {
                const Quad<TX> vm = reinterpret_cast<const Quad<TX> *>(V + r * KW)[m4];
#pragma unroll
                for (int mm = 0; mm < 4; ++mm)
#pragma unroll
                    for (int u = 0; u < 4; ++u) y[u] += vm.v[mm] * t2[4 * m4 + mm][4 * q + u];
            }
        }
        Quad<TX> o;
#pragma unroll
        for (int u = 0; u < 4; ++u) o.v[u] = y[u];
        reinterpret_cast<Quad<TX> *>(Y + r * KW)[q] = o;
    }
}

// Z = D^-1 R
template <class TX, class TD, int KW>
__global__ void k_bc_precond(int64_t n, const TX *__restrict__ R, const TD *__restrict__ dinv, TX *__restrict__ Z) {
    const int64_t items = n * KW;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x)
        Z[t] = (TX)dinv[t / KW] * R[t];
}

// Bp (SELL order, n x KW, zero-padded) = B[perm] (n x k, original order)
__global__ void k_bc_gather(int64_t n, int k, int KW, const int32_t *__restrict__ perm, const double *__restrict__ B,
                            double *__restrict__ Bp) {
    const int64_t items = n * KW;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / KW;
        const int j = (int)(t - r * KW);
        Bp[t] = j < k ? B[(int64_t)perm[r] * k + j] : 0.0;
    }
}
__global__ void k_bc_scatter(int64_t n, int k, int KW, const int32_t *__restrict__ perm, const double *__restrict__ Xp,
                             double *__restrict__ X) {
    const int64_t items = n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / k;
        const int j = (int)(t - r * k);
        X[(int64_t)perm[r] * k + j] = Xp[r * KW + j];
    }
}

// R = B - Y (fp64)
__global__ void k_bc_sub(int64_t m, const double *__restrict__ B, const double *__restrict__ Y, double *__restrict__ R) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
        R[t] = B[t] - Y[t];
}
// R32 = R64 * s_j (column scale), X32 = 0
__global__ void k_bc_scale_down(int64_t n, int KW, const double *__restrict__ R64, const double *__restrict__ s,
                                float *__restrict__ R32, float *__restrict__ X32) {
    const int64_t items = n * KW;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x) {
        R32[t] = (float)(R64[t] * s[t % KW]);
        X32[t] = 0.0f;
    }
}
// X64 += X32 * s_j
__global__ void k_bc_correct(int64_t n, int KW, double *__restrict__ X64, const float *__restrict__ X32,
                             const double *__restrict__ s) {
    const int64_t items = n * KW;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x)
        X64[t] += (double)X32[t] * s[t % KW];
}

// ------------------------------------------------------------- host side --
// Symmetric eigen-decomposition of an m x m row-major matrix (overwritten) by
// Jacobi rotations, sweeping the off-diagonal pairs in cyclic order; on return
// the diagonal holds the eigenvalues and the columns of V the eigenvectors.
static void jacobi_eig(int m, std::vector<double> &S, std::vector<double> &V) {
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    auto at = [&](int i, int j) -> double & { return S[(size_t)i * m + j]; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < m; ++i) {
            diag += at(i, i) * at(i, i);
            for (int j = i + 1; j < m; ++j) off += 2.0 * at(i, j) * at(i, j);
        }
        if (off == 0.0 || off <= 1e-32 * (off + diag)) break;
        for (int p = 0; p + 1 < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double b = at(p, q);
                if (b == 0.0) continue;
                // choose c, s with c^2 + s^2 = 1 so that the rotated (p, q) entry vanishes
                const double zeta = (at(q, q) - at(p, p)) / (2.0 * b);
                const double t = std::copysign(1.0, zeta) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < m; ++i) {
                    const double xp = at(i, p), xq = at(i, q);
                    at(i, p) = c * xp - s * xq;
                    at(i, q) = s * xp + c * xq;
                }
                for (int i = 0; i < m; ++i) {
                    const double xp = at(p, i), xq = at(q, i);
                    at(p, i) = c * xp - s * xq;
                    at(q, i) = s * xp + c * xq;
                }
                for (int i = 0; i < m; ++i) {
                    const double xp = V[(size_t)i * m + p], xq = V[(size_t)i * m + q];
                    V[(size_t)i * m + p] = c * xp - s * xq;
                    V[(size_t)i * m + q] = s * xp + c * xq;
                }
            }
    }
}

// Cholesky factor (lower, in place) of the leading s x s block of G (row
// stride ld); false if not positive definite.
static bool chol_lower(int s, std::vector<double> &G, int ld) {
    for (int j = 0; j < s; ++j) {
        double d = G[(size_t)j * ld + j];
        for (int q = 0; q < j; ++q) d -= G[(size_t)j * ld + q] * G[(size_t)j * ld + q];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        d = std::sqrt(d);
        G[(size_t)j * ld + j] = d;
        for (int i = j + 1; i < s; ++i) {
            double t = G[(size_t)i * ld + j];
            for (int q = 0; q < j; ++q) t -= G[(size_t)i * ld + q] * G[(size_t)j * ld + q];
            G[(size_t)i * ld + j] = t / d;
        }
    }
    return true;
}
// Y (s x ncol of a KW-wide row-major array) <- (L L^T)^-1 Y
static void chol_apply(int s, const std::vector<double> &L, int ld, std::vector<double> &Y, int ldy, int ncol) {
    for (int c = 0; c < ncol; ++c) {
        for (int i = 0; i < s; ++i) {
            double t = Y[(size_t)i * ldy + c];
            for (int q = 0; q < i; ++q) t -= L[(size_t)i * ld + q] * Y[(size_t)q * ldy + c];
            Y[(size_t)i * ldy + c] = t / L[(size_t)i * ld + i];
        }
        for (int i = s - 1; i >= 0; --i) {
            double t = Y[(size_t)i * ldy + c];
            for (int q = i + 1; q < s; ++q) t -= L[(size_t)q * ld + i] * Y[(size_t)q * ldy + c];
            Y[(size_t)i * ldy + c] = t / L[(size_t)i * ld + i];
        }
    }
}

// Device workspace of one block solve.
template <class TX>
struct BcWork {
    TX *X = nullptr, *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr, *W = nullptr;
    double *part = nullptr, *small = nullptr;  // Gram partials; 4 KW x KW fp64 matrices
};

template <class TV, class TX, int KW>
struct BcOps {
    const SellView A;
    const TV *val;
    cudaStream_t st;
    int grid_rows, grid_gram;
    double *part, *out;  // Gram partials and the device copy of one KW x KW result
    int64_t *launches;

    void spmm(const TX *X, TX *Y) const {
        ::gb::count_launches(1); ++*launches;
        k_bc_spmm<TV, TX, KW><<<grid_rows, BC_NT, 0, st>>>(A, val, X, Y);
    }
    // h = U^T V (KW x KW), synchronises
    int gram(const TX *U, const TX *V, std::vector<double> &h) const {
        ::gb::count_launches(2); *launches += 2;
        k_bc_gram<TX, KW><<<grid_gram, BC_NT, 0, st>>>(A.n, U, V, part);
        k_bc_sum<<<(KW * KW + 255) / 256, 256, 0, st>>>(grid_gram, KW * KW, part, out);
        h.resize((size_t)KW * KW);
        GB_CHECK_CUDA(cudaGetLastError());
        GB_CHECK_CUDA(cudaMemcpyAsync(h.data(), out, sizeof(double) * KW * KW, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
        return GB_OK;
    }
    // squared column norms of U, synchronises
    int colsq(const TX *U, std::vector<double> &h) const {
        ::gb::count_launches(2); *launches += 2;
        k_bc_colsq<TX, KW><<<grid_gram, BC_NT, 0, st>>>(A.n, U, part);
        k_bc_sum<<<1, 256, 0, st>>>(grid_gram, KW, part, out);
        h.resize(KW);
        GB_CHECK_CUDA(cudaGetLastError());
        GB_CHECK_CUDA(cudaMemcpyAsync(h.data(), out, sizeof(double) * KW, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
        return GB_OK;
    }
};

// orth: from G = W^T W (host), column weights cw (0: column left out), the
// transform T (KW x KW, columns >= s zero) with W T orthonormal; returns s.
template <int KW>
static int orth_transform(const std::vector<double> &G, const std::vector<double> &cw, double eps,
                          std::vector<double> &T) {
    std::vector<double> S((size_t)KW * KW), V;
    for (int i = 0; i < KW; ++i)
        for (int j = 0; j < KW; ++j) S[(size_t)i * KW + j] = G[(size_t)i * KW + j] * cw[i] * cw[j];
    jacobi_eig(KW, S, V);
    std::vector<int> ord(KW);
    for (int i = 0; i < KW; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int a, int b) { return S[(size_t)a * KW + a] > S[(size_t)b * KW + b]; });
    const double lmax = S[(size_t)ord[0] * KW + ord[0]];
    int s = 0;
    if (lmax > 0.0 && std::isfinite(lmax))
        while (s < KW && S[(size_t)ord[s] * KW + ord[s]] > eps * lmax) ++s;
    T.assign((size_t)KW * KW, 0.0);
    for (int j = 0; j < s; ++j) {
        const double inv = 1.0 / std::sqrt(S[(size_t)ord[j] * KW + ord[j]]);
        for (int i = 0; i < KW; ++i) T[(size_t)i * KW + j] = cw[i] * V[(size_t)i * KW + ord[j]] * inv;
    }
    return s;
}

struct BcResult {
    long long it = 0;
    int status = ST_RUN;  // ST_CONV, ST_MAXIT, ST_BREAK
};

// The block-CG recurrence on (X, R) in TX: runs until every column j with
// thr[j] >= 0 has ||R_j|| <= thr[j] (columns with thr[j] < 0 are left out of
// the search block), or maxit steps.  X and R are updated in place.
template <class TV, class TX, class TD, int KW>
static int bc_recurrence(const BcOps<TV, TX, KW> &ops, const TD *dinv, BcWork<TX> &w, const std::vector<double> &thr,
                         double eps, long long maxit, BcResult *res) {
    const int64_t n = ops.A.n;
    cudaStream_t st = ops.st;
    double *d_m1 = w.small, *d_m2 = w.small + KW * KW;
    std::vector<double> rn2, cw(KW), G, T, PtQ, L, al, be;
    auto col_weights = [&](const std::vector<double> &r2) {
        bool any = false;
        for (int j = 0; j < KW; ++j) {
            const double rnj = std::sqrt(r2[j]);
            cw[j] = (thr[j] >= 0.0 && rnj > thr[j] && rnj > 0.0) ? 1.0 / rnj : 0.0;
            any = any || cw[j] > 0.0;
        }
        return any;
    };
    ::gb::count_launches(1); ++*ops.launches;
    k_bc_precond<TX, TD, KW><<<ops.grid_rows, BC_NT, 0, st>>>(n, w.R, dinv, w.Z);
    GB_TRY(ops.colsq(w.R, rn2));
    if (!col_weights(rn2)) { res->status = ST_CONV; return GB_OK; }
    GB_TRY(ops.gram(w.Z, w.Z, G));
    int s = orth_transform<KW>(G, cw, eps, T);
    GB_CHECK_CUDA(cudaMemcpyAsync(d_m1, T.data(), sizeof(double) * KW * KW, cudaMemcpyHostToDevice, st));
    ::gb::count_launches(1); ++*ops.launches;
    k_bc_comb<TX, KW><<<ops.grid_rows, BC_NT, 0, st>>>(n, w.Z, d_m1, 0, (const TX *)nullptr, nullptr, w.P);
    while (res->it < maxit) {
        if (s == 0) { res->status = ST_BREAK; return GB_OK; }
        ops.spmm(w.P, w.Q);
        GB_TRY(ops.gram(w.P, w.Q, PtQ));
        GB_TRY(ops.gram(w.P, w.R, al));
        L = PtQ;
        if (!chol_lower(s, L, KW)) { res->status = ST_BREAK; return GB_OK; }
        for (int i = s; i < KW; ++i)
            for (int j = 0; j < KW; ++j) al[(size_t)i * KW + j] = 0.0;
        chol_apply(s, L, KW, al, KW, KW);
        GB_CHECK_CUDA(cudaMemcpyAsync(d_m1, al.data(), sizeof(double) * KW * KW, cudaMemcpyHostToDevice, st));
        ::gb::count_launches(1); ++*ops.launches;
        k_bc_update<TX, TD, KW><<<ops.grid_rows, BC_NT, 0, st>>>(n, w.P, w.Q, d_m1, w.X, w.R, dinv, w.Z);
        res->it += 1;
        GB_TRY(ops.colsq(w.R, rn2));
        bool done = true;
        for (int j = 0; j < KW; ++j)
            if (thr[j] >= 0.0 && !(std::sqrt(rn2[j]) <= thr[j])) done = false;
        for (int j = 0; j < KW; ++j)
            if (!std::isfinite(rn2[j])) { res->status = ST_BREAK; return GB_OK; }
        if (done) { res->status = ST_CONV; return GB_OK; }
        // beta = -(P^T Q)^-1 Q^T Z ;  W = Z + P beta ;  P = orth(W)
        GB_TRY(ops.gram(w.Q, w.Z, be));
        for (int i = 0; i < KW; ++i)
            for (int j = 0; j < KW; ++j) be[(size_t)i * KW + j] = i < s ? -be[(size_t)i * KW + j] : 0.0;
        chol_apply(s, L, KW, be, KW, KW);
        GB_CHECK_CUDA(cudaMemcpyAsync(d_m2, be.data(), sizeof(double) * KW * KW, cudaMemcpyHostToDevice, st));
        ::gb::count_launches(1); ++*ops.launches;
        k_bc_comb<TX, KW><<<ops.grid_rows, BC_NT, 0, st>>>(n, w.Z, nullptr, 1, w.P, d_m2, w.W);
        if (!col_weights(rn2)) { res->status = ST_CONV; return GB_OK; }
        GB_TRY(ops.gram(w.W, w.W, G));
        s = orth_transform<KW>(G, cw, eps, T);
        GB_CHECK_CUDA(cudaMemcpyAsync(d_m1, T.data(), sizeof(double) * KW * KW, cudaMemcpyHostToDevice, st));
        ::gb::count_launches(1); ++*ops.launches;
        k_bc_comb<TX, KW><<<ops.grid_rows, BC_NT, 0, st>>>(n, w.W, d_m1, 0, (const TX *)nullptr, nullptr, w.P);
    }
    res->status = ST_MAXIT;
    return GB_OK;
}

template <int KW>
static int block_solve(const gb_sell *Ah, const double *d_B, double *d_X, int k, const PcgOptions &o,
                       cudaStream_t st, PcgStats *stats) {
    const SellView A = Ah->view();
    const int64_t n = A.n;
    const size_t nk = (size_t)n * KW;
    Mem mem(nullptr, st);
    const int sms = num_sms();
    const int grid_rows = stride_grid(n * (KW / 4), BC_NT, 8);
    const int grid_gram = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, (n + BC_TR - 1) / BC_TR));
    const int grid_vec = stride_grid((int64_t)nk, BC_NT, 8);
    int64_t launches = 0;
    struct Bufs {
        Mem *m;
        std::vector<void *> ptrs;
        ~Bufs() { for (void *p : ptrs) m->release(p); }
    } bufs{&mem, {}};
    auto alloc = [&](auto **p, size_t cnt) {
        int rc = mem.alloc_n(p, cnt);
        if (rc == GB_OK) bufs.ptrs.push_back((void *)*p);
        return rc;
    };
    double *B64, *X64, *R64, *Y64, *part, *small, *scale;
    GB_TRY(alloc(&B64, nk));
    GB_TRY(alloc(&X64, nk));
    GB_TRY(alloc(&R64, nk));
    GB_TRY(alloc(&Y64, nk));
    GB_TRY(alloc(&part, (size_t)grid_gram * KW * KW));
    GB_TRY(alloc(&small, (size_t)4 * KW * KW));
    GB_TRY(alloc(&scale, KW));
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
    } ev;
    GB_CHECK_CUDA(cudaEventCreate(&ev.a));
    GB_CHECK_CUDA(cudaEventCreate(&ev.b));
    GB_CHECK_CUDA(cudaEventRecord(ev.a, st));
    ::gb::count_launches(1); ++launches;
    k_bc_gather<<<grid_vec, BC_NT, 0, st>>>(n, k, KW, Ah->perm, d_B, B64);
    if (o.x0_zero) {
        GB_CHECK_CUDA(cudaMemsetAsync(X64, 0, sizeof(double) * nk, st));
    } else {
        ::gb::count_launches(1); ++launches;
        k_bc_gather<<<grid_vec, BC_NT, 0, st>>>(n, k, KW, Ah->perm, d_X, X64);
    }
    BcOps<double, double, KW> ops64{A, Ah->val, st, grid_rows, grid_gram, part, small + 2 * KW * KW, &launches};
    std::vector<double> bn2, rn2;
    GB_TRY(ops64.colsq(B64, bn2));
    std::vector<double> bn(KW);
    for (int j = 0; j < KW; ++j) bn[j] = std::sqrt(bn2[j]);
    auto true_residual = [&](std::vector<double> &rel) -> int {
        ops64.spmm(X64, Y64);
        ::gb::count_launches(1); ++launches;
        k_bc_sub<<<grid_vec, BC_NT, 0, st>>>((int64_t)nk, B64, Y64, R64);
        GB_TRY(ops64.colsq(R64, rn2));
        rel.assign(KW, 0.0);
        for (int j = 0; j < k; ++j) {
            const double r = std::sqrt(rn2[j]);
            rel[j] = bn[j] > 0.0 ? r / bn[j] : r;
        }
        return GB_OK;
    };
    std::vector<double> rel;
    GB_TRY(true_residual(rel));
    auto worst = [&]() { double w = 0.0; for (int j = 0; j < k; ++j) w = std::max(w, rel[j]); return w; };
    long long it_total = 0;
    int outer = 0, restarts = 0, status = ST_RUN;
    const long long maxit = o.max_iter;
    if (o.precision == GB_F64) {
        BcWork<double> w;
        w.X = X64;
        w.R = R64;
        GB_TRY(alloc(&w.Z, nk));
        GB_TRY(alloc(&w.P, nk));
        GB_TRY(alloc(&w.Q, nk));
        GB_TRY(alloc(&w.W, nk));
        w.small = small;
        while (!(worst() <= o.tol)) {
            if (it_total >= maxit || restarts > 50) { status = ST_MAXIT; break; }
            std::vector<double> thr(KW, -1.0);
            for (int j = 0; j < k; ++j) thr[j] = bn[j] > 0.0 ? o.tol * bn[j] : 0.0;
            BcResult res;
            res.it = it_total;
            GB_TRY((bc_recurrence<double, double, double, KW>(ops64, Ah->dinv, w, thr, 1e-12, maxit, &res)));
            it_total = res.it;
            GB_TRY(true_residual(rel));
            if (res.status == ST_BREAK) { status = worst() <= o.tol ? ST_CONV : ST_BREAK; break; }
            if (!(worst() <= o.tol)) ++restarts;
        }
    } else {
        // fp32 block CG on the scaled residual, fp64 refinement outside
        BcWork<float> w;
        GB_TRY(alloc(&w.X, nk));
        GB_TRY(alloc(&w.R, nk));
        GB_TRY(alloc(&w.Z, nk));
        GB_TRY(alloc(&w.P, nk));
        GB_TRY(alloc(&w.Q, nk));
        GB_TRY(alloc(&w.W, nk));
        w.small = small;
        BcOps<float, float, KW> ops32{A, Ah->val32, st, grid_rows, grid_gram, part, small + 2 * KW * KW, &launches};
        double prev = worst();
        int stalls = 0;
        while (!(worst() <= o.tol)) {
            if (it_total >= maxit || outer >= o.max_outer) { status = ST_MAXIT; break; }
            ++outer;
            std::vector<double> sc(KW, 0.0), thr(KW, -1.0), back(KW, 0.0);
            for (int j = 0; j < k; ++j) {
                const double r = std::sqrt(rn2[j]);
                if (rel[j] > o.tol && r > 0.0) {
                    sc[j] = 1.0 / r;
                    back[j] = r;
                    thr[j] = o.inner_tol;
                }
            }
            GB_CHECK_CUDA(cudaMemcpyAsync(scale, sc.data(), sizeof(double) * KW, cudaMemcpyHostToDevice, st));
            ::gb::count_launches(1); ++launches;
            k_bc_scale_down<<<grid_vec, BC_NT, 0, st>>>(n, KW, R64, scale, w.R, w.X);
            BcResult res;
            res.it = it_total;
            GB_TRY((bc_recurrence<float, float, float, KW>(ops32, Ah->dinv32, w, thr, 1e-6, maxit, &res)));
            it_total = res.it;
            GB_CHECK_CUDA(cudaMemcpyAsync(scale, back.data(), sizeof(double) * KW, cudaMemcpyHostToDevice, st));
            ::gb::count_launches(1); ++launches;
            k_bc_correct<<<grid_vec, BC_NT, 0, st>>>(n, KW, X64, w.X, scale);
            GB_TRY(true_residual(rel));
            const double wv = worst();
            if (!(wv < 0.9 * prev)) { if (++stalls >= 2) { status = ST_MAXIT; break; } } else stalls = 0;
            prev = std::min(prev, wv);
        }
    }
    if (worst() <= o.tol) status = ST_CONV;
    ::gb::count_launches(1); ++launches;
    k_bc_scatter<<<grid_vec, BC_NT, 0, st>>>(n, k, KW, Ah->perm, X64, d_X);
    GB_CHECK_CUDA(cudaGetLastError());
    GB_CHECK_CUDA(cudaEventRecord(ev.b, st));
    GB_CHECK_CUDA(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    stats->iterations = it_total;
    stats->outer = outer;
    stats->restarts = restarts;
    stats->relres = worst();
    double bmax = 0.0;
    for (int j = 0; j < k; ++j) bmax = std::max(bmax, bn[j]);
    stats->bnorm = bmax;
    stats->solve_ms = ms;
    stats->kernel_launches = launches;
    stats->status = status == ST_CONV ? GB_OK : (status == ST_BREAK ? GB_BREAKDOWN : GB_NOT_CONVERGED);
    return GB_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" int pcg_solve_block(const gb_sell *A, const double *d_B, double *d_X, int k, const PcgOptions *opt,
                               void *stream, PcgStats *stats) {
    gb::Range range("gbpcg:pcg_solve_block");
    GB_REQUIRE(A && d_B && d_X, "pcg_solve_block: NULL argument");
    GB_REQUIRE(k >= 1 && k <= 32, "pcg_solve_block: k=%d not in 1..32", k);
    PcgStats dummy{};
    if (!stats) stats = &dummy;
    *stats = PcgStats{};
    PcgOptions o{};
    if (opt) o = *opt;
    if (!(o.tol > 0)) o.tol = 1e-10;
    if (o.max_iter <= 0) o.max_iter = 20 * A->n + 100;
    if (o.max_outer <= 0) o.max_outer = 30;
    if (!(o.inner_tol > 0)) o.inner_tol = 1e-4;
    GB_REQUIRE(o.precision == GB_F64 || o.precision == GB_F32_IR,
               "pcg_solve_block: precision GB_F64 or GB_F32_IR");
    GB_REQUIRE(o.precision != GB_F32_IR || A->val32, "pcg_solve_block: GB_F32_IR needs fp32 values (val_types)");
    GB_REQUIRE(o.precond == GB_PC_JACOBI, "pcg_solve_block: the Jacobi preconditioner only");
    GB_REQUIRE(o.method == GB_CG, "pcg_solve_block: block CG (method GB_CG) only");
    cudaStream_t st = (cudaStream_t)stream;
    const int KW = k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
    switch (KW) {
    case 4: return block_solve<4>(A, d_B, d_X, k, o, st, stats);
    case 8: return block_solve<8>(A, d_B, d_X, k, o, st, stats);
    case 16: return block_solve<16>(A, d_B, d_X, k, o, st, stats);
    default: return block_solve<32>(A, d_B, d_X, k, o, st, stats);
    }
}
