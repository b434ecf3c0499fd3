/*
 * gbpcg.h -- C ABI of the GB300 (sm_103a) FEM-Laplace Jacobi-PCG library.
 *
 * The library solves the sparse SPD systems that come from discretising
 * Laplace's equation with Dirichlet data (paper Sec. 2.2) by P1/P2 finite
 * elements on lattice meshes, with one or many right-hand sides (Eq. MRH,
 * Sec. 4.3), by Jacobi-preconditioned conjugate gradients (the preconditioned
 * Krylov solve of Sec. 2.1) stopped by the relative residual of Eq. (2).
 * Every step runs in CUDA kernels of this library; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Pointers prefixed d_ are device pointers, h_ host pointers.  The caller
 *    owns every buffer it passes; the library owns the opaque handles it
 *    returns and everything reachable from them, and allocates through the
 *    caller's gb_allocator (NULL = cudaMalloc/cudaFree).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; entry points that must return sizes or statistics
 *    synchronise that stream before returning (stated per function).
 *  - Return value: GB_OK (0) or a negative GB_E* code; gbpcg_last_error()
 *    returns a thread-local message for the last failure.  Arguments are
 *    validated before any work is enqueued.
 *  - Vectors passed to the solvers are in the free-dof order of the system
 *    (increasing lexicographic dof-lattice index, x fastest); multi-RHS blocks
 *    are row-major n x k.  The library's internal row permutation never shows.
 *  - Index type is int32: a system needs n, nnz and padded nnz below 2^31.
 */
#ifndef GBPCG_H
#define GBPCG_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GB_OK = 0,
    GB_EINVAL = -1,          /* bad argument */
    GB_ENOMEM = -2,          /* allocator returned NULL */
    GB_ECUDA = -3,           /* a CUDA runtime call failed */
    GB_NOT_CONVERGED = -4,   /* max_iter reached; x and stats are still written */
    GB_BREAKDOWN = -5,       /* p.Ap <= 0 or non-finite: matrix not SPD or bad data */
    GB_TIMEOUT = -6,         /* a device-side bounded wait ran out */
    GB_TOO_LARGE = -7,       /* request exceeds a size limit or the memory budget */
    GB_PENDING = 1           /* serve_poll: request not finished yet */
};

/* Thread-local message of the last failing call on this thread. */
const char *gbpcg_last_error(void);
/* Library version string. */
const char *gbpcg_version(void);
/* Kernels this process has launched through the library so far (launches
 * replayed by a CUDA graph's loop included). */
int64_t gbpcg_kernel_launches(void);
/* Device allocations the library's solvers, assembly and format conversion
 * have made so far in this process (through a caller's gb_allocator or
 * cudaMalloc); a call that allocates nothing leaves it unchanged. */
int64_t gbpcg_device_allocations(void);

/* Device memory supplier.  alloc(ctx, bytes, stream) returns a device pointer
 * aligned to at least 256 bytes, or NULL; free(ctx, ptr, stream) releases it.
 * Both are called from the calling thread only, never from a kernel. */
typedef struct gb_allocator {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, void *stream);
} gb_allocator;

/* ------------------------------------------------------------ assembly --
 * Mesh of the unit square (dim 2) or cube (dim 3) with `cells` cells per side
 * (Sec. 2.2 case study).  2D: each cell is cut into two triangles by its
 * SW-NE diagonal, or by a per-cell random diagonal (diag_mode 1: the NW-SE one
 * when the cell's draw is below 1/2); with jitter=1 every interior vertex moves
 * by (2u-1)h/4 per coordinate.  3D: Kuhn split of each cube into six
 * tetrahedra along its main diagonal (diag_mode must be 0); with jitter=1 every
 * interior vertex moves by (2u-1)h/8 per coordinate (at h/4 a tetrahedron
 * could invert) -- an irregular tetrahedral mesh.  The draws u come from the
 * counter-based SplitMix64 generator: output i of stream s of run `seed` is
 * mix64(key + (i+1)*0x9E3779B97F4A7C15), key = seed*2^40 xor s*2^32,
 * u = (output >> 11) * 2^-53; streams 0/1/3 jitter x/y/z (i = vertex id),
 * stream 2 the diagonal (i = cell id).  degree 1..4 (P1-P4 Lagrange elements,
 * the degree study of Sec. 4.2 / Table 7): dofs are the points of the lattice
 * with degree*cells+1 points per side (the Lagrange nodes of every simplex lie
 * on it); boundary dofs are those with a coordinate 0 or degree*cells.  A
 * P3/P4 node's coordinates are (sum of beta_a P_a over its smallest face, in
 * ascending vertex id) / degree, correctly rounded, a vertex node the vertex. */
typedef struct gb_fem_spec {
    int32_t dim;        /* 2 or 3 */
    int32_t degree;     /* 1, 2, 3 or 4 */
    int32_t cells;      /* cells per side, >= 2 */
    int32_t jitter;     /* 0 or 1 */
    int32_t diag_mode;  /* 0 fixed SW-NE, 1 random per cell (2D only) */
    int32_t reserved;   /* must be 0 */
    uint64_t seed;
} gb_fem_spec;

typedef struct gb_fem_system gb_fem_system;

/* Read-only views of an assembled system (device pointers owned by it). */
typedef struct gb_fem_info {
    int64_t n_dof, n_free, n_bnd;
    int64_t nnz;        /* stored entries of K_II (structural: never value-dropped) */
    int64_t nnz_ib;     /* stored entries of K_IB */
    int32_t dim, degree, cells, side;  /* side = dof-lattice points per side */
    int32_t max_row;    /* longest row of K_II */
    int32_t reserved;
    const int32_t *d_rowptr;     /* K_II CSR, n_free+1, columns ascending */
    const int32_t *d_col;
    const double *d_val;
    const int32_t *d_rowptr_ib;  /* K_IB CSR (columns = boundary ids) */
    const int32_t *d_col_ib;
    const double *d_val_ib;
    const double *d_diag;        /* diag(K_II), n_free */
} gb_fem_info;

/* Builds the mesh, numbers the dofs, assembles the stiffness
 * K_ij = sum_T int_T grad(phi_i).grad(phi_j) and splits it into the free block
 * K_II and the coupling K_IB (Dirichlet elimination, Sec. 2.2).  Each row is
 * gathered over its incident elements in a fixed order, so K_II is
 * bit-exactly symmetric and the result is deterministic.  Synchronises
 * `stream` once (to size the column arrays). */
int fem_assemble(const gb_fem_spec *spec, const gb_allocator *alloc, void *stream,
                 gb_fem_system **out);
int fem_system_info(const gb_fem_system *sys, gb_fem_info *out);
/* Free-dof <-> full-dof maps (device int32 arrays of n_free / n_bnd / n_dof). */
int fem_dof_maps(const gb_fem_system *sys, int32_t *d_full_of_free, int32_t *d_full_of_bnd,
                 int32_t *d_free_of_full, void *stream);
/* Coordinates of the boundary (which=0, n_bnd rows) or free (which=1, n_free
 * rows) dofs, row-major rows x dim.  P2 edge dofs sit at edge midpoints. */
int fem_boundary_coords(const gb_fem_system *sys, int which, double *d_xyz, void *stream);
/* Dirichlet data g at the boundary (which=0) or free (which=1) dofs for k
 * columns, row-major rows x k.  gid: 0 sin(pi x)sinh(pi y)/sinh(pi);
 * 1 x^2-y^2; 2 x^2+y^2-2z^2; 3 c0+c1 x+c2 y+c3 z (4 coefficients per column);
 * 4 sum_{m=0..4} a_m Re(x+iy)^m + b_m Im(x+iy)^m (10 coefficients per column,
 * ordered a_0,b_0,a_1,b_1,...).  h_coef: host array, k*ncoef values (NULL when
 * ncoef is 0).  Synchronous in h_coef only (copied before return). */
int fem_dirichlet(const gb_fem_system *sys, int gid, const double *h_coef, int k, int which,
                  double *d_out, void *stream);
/* b = -K_IB g_B for k columns (row-major: d_gB n_bnd x k, d_b n_free x k). */
int fem_lift_rhs(const gb_fem_system *sys, const double *d_gB, int k, double *d_b, void *stream);
void fem_system_destroy(gb_fem_system *sys);

/* ---------------------------------------------------------- SELL-C-sigma --
 * Sliced ELLPACK with sorting window sigma: rows are ordered by descending
 * length inside windows of sigma consecutive rows (stable), cut into chunks of
 * C rows, each chunk stored column-major and padded to its longest row
 * (padding: the row's own index, value 0).  The permutation is applied
 * symmetrically (rows and columns).  val_types: bit 0 fp64, bit 1 fp32,
 * bit 2 bf16 value copies (fp64 is always kept; fp32/bf16 serve the mixed-
 * precision inner solve).  GB_IDX16 (C = 32 only): also store 16-bit column
 * deltas (column - min(row, n-1)) when they all fit; the SpMV then streams
 * those instead of 32-bit indices (6 instead of 8 bytes per fp32 entry).
 * C in {32, 64, 128}; sigma >= 1. */
enum { GB_VAL_F64 = 1, GB_VAL_F32 = 2, GB_VAL_BF16 = 4, GB_IDX16 = 8 };

typedef struct gb_sell gb_sell;

typedef struct gb_sell_info {
    int64_t n, nnz, padded, nchunks;
    int32_t C, sigma, max_row, reserved;
    const int32_t *d_perm;       /* perm[new] = old */
    const int64_t *d_chunk_ptr;  /* nchunks+1 */
    const int32_t *d_chunk_w;    /* nchunks */
    const int32_t *d_row_len;    /* n, new order */
    const int32_t *d_col;        /* padded, new numbering */
    const double *d_val;         /* padded fp64 */
    const double *d_dinv;        /* 1/diag, new order */
    const int16_t *d_col16;      /* GB_IDX16: column - min(row, n-1) per padded slot when every
                                    delta fits in 16 bits (the SpMV then streams these), else NULL */
} gb_sell_info;

/* From an assembled system's K_II.  Asynchronous except for one sync to read
 * the padded size. */
int csr_to_sell(const gb_fem_system *sys, int C, int sigma, int val_types,
                const gb_allocator *alloc, void *stream, gb_sell **out);
/* From any CSR matrix with a non-zero diagonal (device arrays; int32 rowptr). */
int csr_to_sell_raw(int64_t n, const int32_t *d_rowptr, const int32_t *d_col, const double *d_val,
                    int C, int sigma, int val_types, const gb_allocator *alloc, void *stream,
                    gb_sell **out);
int sell_info(const gb_sell *A, gb_sell_info *out);
/* y = A x through the SELL storage (x, y in the original order). */
int sell_spmv(const gb_sell *A, const double *d_x, double *d_y, void *stream);
void sell_destroy(gb_sell *A);

/* Autotuner: builds the matrix in each candidate layout -- chunk height C
 * (32, 64, 128), sorting window sigma (64, 256, 1024), SpMV variant (TMA-
 * staged streams or one row per lane) -- times a CG iteration of each for
 * `precision` (GB_F64, GB_F32_IR or GB_BF16_IR; d_b: a right-hand side, n
 * doubles, original order) with CUDA events, and returns the fastest in
 * *best.  With out != NULL the winning matrix is returned (its SpMV variant
 * becomes the default of later solves on it), else it is destroyed.
 * Synchronises `stream`. */
typedef struct SellTuneResult {
    int32_t C, sigma, spmv_variant, candidates;
    double iter_ms;   /* one CG iteration of the winner (sum of its three kernels) */
    double spmv_ms;   /* its SpMV + p.q kernel */
} SellTuneResult;
int sell_autotune(const gb_fem_system *sys, const double *d_b, int precision, int val_types,
                  const gb_allocator *alloc, void *stream, SellTuneResult *best, gb_sell **out);
/* Sets the SpMV variant later solves on A use when PcgOptions.spmv_variant is
 * 0 (the autotuner's choice, replayed from a cache): 0 = TMA-staged streams
 * where the layout has them (C = 32), 1 = one row per lane.  GB_EINVAL for
 * another value. */
int sell_set_variant(gb_sell *A, int variant);

/* Block-Jacobi preconditioner (the paper's Block-Jacobi, Sec. 3.2 and Sec.
 * 4.2): M = blockdiag(K_11, ..., K_mm), K_jj the diagonal block of the bs
 * consecutive free dofs [j bs, min(n, (j+1) bs)) in the original (free-dof)
 * order; the last block is shorter when bs does not divide n.
 * sell_block_jacobi computes each block's inverse on the device (Gauss-Jordan
 * elimination in fp64, symmetrised) and attaches it to A, replacing any
 * earlier one; bs = 0 detaches it.  bs in {0, 1, 2, 4, 8, 16, 32}, and A's
 * sigma must divide 256: then the rows of a block share one 256-row window of
 * the SELL permutation, which the fused PCG update works on.  Synchronises
 * `stream` (also before freeing earlier blocks).  Errors: GB_EINVAL (bs or
 * sigma), GB_ENOMEM, GB_BREAKDOWN (a block is not positive definite).  A
 * solve uses it with PcgOptions.precond = GB_PC_BLOCK_JACOBI.
 * sell_block_jacobi_info: the attached data (device pointers, owned by A):
 * d_w holds per block the upper triangle of its inverse, row-major (bs(bs+1)/2
 * doubles per block, rows and columns past a short block's end 0), d_w32 the
 * same in fp32, d_loc per free dof o the SELL position of o minus
 * 256 floor(o/256) (nblk * bs bytes); lam_bound = max absolute row sum of the
 * inverses (>= the largest eigenvalue of M^-1).  bs = 0 when none is attached.
 * sell_block_jacobi_apply: y = M^-1 x (n doubles each, free-dof order);
 * GB_EINVAL without attached blocks; synchronises `stream`. */
typedef struct gb_bjacobi_info {
    int32_t bs, reserved;
    int64_t nblk;
    const double *d_w;
    const float *d_w32;
    const uint8_t *d_loc;
    double lam_bound;
} gb_bjacobi_info;
int sell_block_jacobi(gb_sell *A, int bs, void *stream);
int sell_block_jacobi_info(const gb_sell *A, gb_bjacobi_info *out);
int sell_block_jacobi_apply(const gb_sell *A, const double *d_x, double *d_y, void *stream);

/* ------------------------------------------------------------------ PCG --
 * Jacobi-PCG: r = b - A x0, z = D^{-1} r, p = z; iterate q = A p,
 * alpha = r.z / p.q, x += alpha p, r -= alpha q, z = D^{-1} r, beta = r.z'/r.z,
 * p = z + beta p; stop when ||r||/||b|| <= tol (Eq. 2), then confirm on the
 * true residual b - A x in fp64 (restart from it if it is above tol).
 * precision GB_F64: everything in fp64.  GB_F32_IR / GB_BF16_IR: iterative
 * refinement -- fp64 outer residual b - A x, convergence test and update
 * x += d; the correction d solves A d = r approximately by an inner PCG with
 * fp32 vectors, fp32 accumulation and fp32 (or bf16-stored) matrix values to
 * relative residual inner_tol.  If the refinement stalls (two outer steps
 * without a 10% residual reduction) or runs out of outer steps above tol, the
 * solve continues with fp64 PCG from the current x on the device, and
 * stats.fallback_iterations counts those iterations.
 * GB_F32_RU / GB_BF16_RU: the same split of precisions with reliable updates
 * instead of restarts -- one fp32 recurrence keeps its search direction; each
 * time its residual has dropped tenfold, x += d and r = b - A x are formed in
 * fp64, the test is made in fp64 and the fp32 residual is replaced by the
 * true one (stats.outer counts these updates).  pcg_solve only.
 * precond GB_PC_BLOCK_JACOBI replaces D^{-1} by the block inverses attached
 * with sell_block_jacobi (pcg_solve with GB_F64, GB_F32_IR or GB_BF16_IR --
 * the inner solve then applies the fp32 copy; GB_EINVAL otherwise, and in
 * pcg_solve_batched and pcg_solve_noalloc). */
enum { GB_F64 = 0, GB_F32_IR = 1, GB_BF16_IR = 2, GB_F32_RU = 3, GB_BF16_RU = 4 };
enum { GB_PC_JACOBI = 0, GB_PC_BLOCK_JACOBI = 1 };
/* method GB_BICGSTAB: BiCGSTAB (van der Vorst), the Krylov method of the
 * paper's experiments (Sec. 3.2), preconditioned on the right with the
 * Jacobi or block-Jacobi M: two SpMVs and two preconditioner applications per
 * step (stats.iterations counts steps); the stop is confirmed on the true
 * residual as for CG.  pcg_solve with GB_F64 on C = 32 layouts (GB_EINVAL
 * otherwise, and in the batched, block and no-allocation solvers). */
enum { GB_CG = 0, GB_BICGSTAB = 1 };

typedef struct PcgOptions {
    double tol;            /* Eq. (2) threshold, e.g. 1e-10 */
    int64_t max_iter;      /* total (inner) iterations cap; 0 = 20 n + 100 */
    int32_t precision;     /* GB_F64 | GB_F32_IR | GB_BF16_IR | GB_F32_RU | GB_BF16_RU */
    int32_t max_outer;     /* refinement steps cap (IR only); 0 = 30 */
    double inner_tol;      /* inner relative residual (IR only); 0 = 1e-4 */
    int32_t check_every;   /* iterations per host convergence poll; 0 = auto */
    int32_t use_graph;     /* 1 = replay captured CUDA graphs (default), 0 = direct launches;
                              GBPCG_USE_GRAPH=0 in the environment forces 0 (for launch-level
                              profilers, which do not list a graph loop's replayed kernels) */
    int32_t x0_zero;       /* 1 = ignore d_x on entry and start from 0 */
    int32_t spmv_variant;  /* 0 = auto (TMA-staged slices for C = 32), 1 = one-row-per-lane loads */
    int32_t persist_off;   /* pcg_solve_batched: 0 (default) = systems with n * k2 <= 32768 (k2: the
                              power of two >= k) are solved whole by one CTA each in a single
                              persistent launch, and systems with n * k2 <= 65536 by one
                              thread-block cluster of 8 CTAs each in another; 1 = every system in
                              the multi-launch loop; 2 = the CTA-local tier only; 3 = as 0, and
                              systems with n * k2 <= 262144 by one group of CTAs each (about one
                              CTA per 2048 rows x k2, a power of two) in one cooperative launch
                              per group size, whose group exchanges are bounded waits
                              (GB_TIMEOUT if one runs out).
                              pcg_solve (GB_F64, Jacobi, CG): 0 = a system of n <= 8192 rows is
                              solved whole by one 8-CTA cluster in one launch; 3 = one group of
                              the grid tier for n <= 262144; 1 = always the multi-kernel loop.
                              (On GB300 the multi-kernel loop is faster than the grid tier at
                              every size measured, so the grid tier is not the default.) */
    int32_t precond;       /* GB_PC_JACOBI (0, default) or GB_PC_BLOCK_JACOBI */
    int32_t method;        /* GB_CG (0, default) or GB_BICGSTAB (pcg_solve, GB_F64, C = 32) */
} PcgOptions;

typedef struct PcgStats {
    int64_t iterations;    /* CG iterations (inner ones for IR) */
    int64_t restarts;      /* true-residual restarts (F64) */
    int32_t outer;         /* refinement steps (IR) */
    int32_t status;        /* GB_OK / GB_NOT_CONVERGED / GB_BREAKDOWN */
    double relres;         /* final true relative residual ||b - A x|| / ||b|| (fp64) */
    double bnorm;          /* ||b||_2 */
    double solve_ms;       /* device time of the solve (events on `stream`) */
    int64_t kernel_launches;  /* kernels this solve launched */
    double bytes_moved;    /* algorithmic bytes of the solve (matrix + vector streams) */
    int64_t fallback_iterations;  /* IR only: fp64 PCG iterations run after the
                                     refinement stalled above tol (0 if none) */
} PcgStats;

/* Solves A x = b for one right-hand side (Sec. 2.1: preconditioned Krylov
 * solve; Eq. 2: stop at ||b - A x|| <= tol ||b||, confirmed on the true
 * residual).  d_b, d_x: n doubles in the original free-dof order (x in: x0
 * unless x0_zero).  GB_F64 Jacobi-CG: the CG loop is a CUDA-graph while-node
 * of three kernels per iteration, or, for n <= 8192 (persist_off = 0), one
 * launch of a persistent kernel on one 8-CTA thread-block cluster that forms
 * the residual and runs every iteration (its memory comes from the
 * stream-ordered pool); persist_off = 1 always takes the graph loop.
 * Synchronises `stream` (convergence polling and statistics). */
int pcg_solve(const gb_sell *A, const double *d_b, double *d_x, const PcgOptions *opt,
              void *stream, PcgStats *stats);

/* Solves nsys systems, system s with k[s] right-hand sides (row-major
 * n_s x k_s blocks d_B[s], d_X[s]).  Systems with k > 1 run blocked multi-RHS
 * PCG: one SpMM pass per iteration serves all columns, each column keeps its
 * own alpha, beta and convergence mask.  All systems advance in the same
 * launches.  opt->precision: GB_F64; GB_F32_IR / GB_BF16_IR (fp32
 * recurrences inside fp64 iterative refinement); GB_F32_RU (one fp32
 * recurrence per column with fp64 reliable updates -- x += d, r = b - A x,
 * residual replacement -- every 10x decrease; stats.outer = updates).  The
 * persistent tiers (PcgOptions.persist_off) solve their systems in fp64, or
 * with fp32 correction solves inside fp64 refinement for the fp32
 * precisions.  Columns a mixed-precision solve leaves above tol finish in
 * fp64 (stats.fallback_iterations).  Synchronises `stream`; stats[s] per
 * system (iterations = max over its columns). */
int pcg_solve_batched(int nsys, const gb_sell *const *A, const double *const *d_B,
                      double *const *d_X, const int *k, const PcgOptions *opt, void *stream,
                      PcgStats *stats);

/* Block CG for A X = B (Sec. 4.3, Eq. MRH: the k right-hand sides known
 * together): one Krylov space shared by the k columns (O'Leary's block
 * conjugate gradients) in a breakdown-free form -- the search block is
 * orthonormalised every step with a rank test (eigenvalues of its Gram
 * matrix, columns scaled by their residual norms, below a relative threshold
 * dropped), so a rank-deficient B or columns converging at different rates
 * reduce the block instead of breaking the recurrence.  Jacobi
 * preconditioner.  d_B, d_X: n x k row-major in the original free-dof order
 * (d_X in: x0 unless x0_zero, out: X), 1 <= k <= 32.  precision GB_F64 (the
 * recurrence in fp64, restarted from the true residual until every column
 * meets Eq. 2) or GB_F32_IR (fp32 block recurrence on the column-scaled fp64
 * residual to inner_tol, fp64 refinement outside).  stats (one for the
 * block): iterations = block steps, outer = refinement steps, relres = the
 * largest column relative residual, status GB_OK / GB_NOT_CONVERGED /
 * GB_BREAKDOWN.  Synchronises `stream` (the k x k algebra runs on the host,
 * three round trips per step). */
int pcg_solve_block(const gb_sell *A, const double *d_B, double *d_X, int k, const PcgOptions *opt,
                    void *stream, PcgStats *stats);

/* ------------------------------------------------------------- serving --
 * A solve server with continuous batching.  Requests (mesh spec, k right-
 * hand sides) are admitted as resident "slots" while max_slots and the device
 * memory budget allow; every resident slot advances in the same launches (the
 * batched kernels), arrivals are assembled on a side stream while the others
 * iterate, and finished slots free their memory for the next ones.  Each
 * request's arithmetic depends only on its own data: its result is the same
 * alone and in a mix.  precision GB_F32_RU (fp32 recurrences with fp64
 * reliable updates, test and solution) or GB_F64.  One server thread per
 * server; submit/poll/stats are thread-safe. */
typedef struct gb_server gb_server;

typedef struct ServeOptions {
    size_t mem_budget;       /* device bytes the admitted requests may hold */
    int32_t max_slots;       /* requests resident at once (1..4096) */
    int32_t precision;       /* GB_F32_RU or GB_F64 */
    double tol;              /* Eq. (2) threshold (0 = 1e-10) */
    int64_t max_iter;        /* iterations per column (0 = 10^6) */
    int32_t iters_per_step;  /* CG iterations between scheduling points; 0 = adaptive (default):
                                about 10 ms of the resident requests' iterations, 4 to 200 */
    int32_t device;          /* CUDA device, -1 = the current one */
    int32_t cluster_lane;    /* 1 = requests with 2^15 < n * k2 <= 2^16 are solved whole by one
                                8-CTA cluster each in the persistent lane; 0 (default) = they
                                advance in the lock-step loop with the large ones */
} ServeOptions;

typedef struct ServeRequest {
    gb_fem_spec spec;        /* the system (fem_assemble) */
    int32_t k;               /* right-hand sides, 1..32 */
    int32_t gid;             /* Dirichlet data id (fem_dirichlet) when h_gB is NULL */
    const double *h_coef;    /* coefficients for gid 3/4 (k x ncoef); copied at submit */
    const double *h_gB;      /* or boundary values, n_bnd x k row-major (valid until done) */
    double *h_x;             /* result, n_free x k row-major in free-dof order (valid until done) */
} ServeRequest;

typedef struct ServeResult {
    int32_t status;          /* GB_OK, GB_NOT_CONVERGED, GB_BREAKDOWN, GB_TOO_LARGE, ... */
    int32_t k;
    int64_t n;               /* free dofs */
    int64_t iterations;      /* max over the request's columns */
    int32_t updates;         /* reliable updates made (GB_F32_RU) */
    int32_t reserved;
    double relres;           /* max over columns of ||b - A x|| / ||b|| (fp64) */
    double queue_ms;         /* submit -> admitted (assembled, on the device) */
    double latency_ms;       /* submit -> result written to h_x */
    double bytes;            /* device bytes the request held */
} ServeResult;

typedef struct ServeStats {
    int64_t submitted, completed, rejected, pending, resident, steps;
    double mem_in_use, mem_peak;  /* bytes */
    int32_t max_resident, reserved;
} ServeStats;

/* alloc: where the requests' device memory (their matrices, right-hand sides
 * and Krylov state) comes from -- the caller's allocator, called from the
 * server's own thread (so it must be thread-safe), or NULL for a
 * stream-ordered pool (cudaMallocAsync).  Either way the bytes are counted
 * against mem_budget.  The server's fixed tables (max_slots descriptors) use
 * cudaMalloc.  The caller's current device is left as it was.  Errors:
 * GB_EINVAL (options, an allocator without alloc/free), GB_ENOMEM, GB_ECUDA;
 * nothing stays allocated after an error. */
int serve_create(const ServeOptions *opt, const gb_allocator *alloc, gb_server **out);
/* Non-blocking: queues the request and returns its ticket (> 0). */
int serve_submit(gb_server *srv, const ServeRequest *req, uint64_t *ticket);
/* GB_PENDING while the request runs; then its final status with *out filled
 * (once: the result is released by the call that returns it). */
int serve_poll(gb_server *srv, uint64_t ticket, ServeResult *out);
int serve_stats(gb_server *srv, ServeStats *out);
/* Finishes resident work, fails queued requests, joins the thread. */
void serve_destroy(gb_server *srv);

/* pcg_solve_noalloc -- the paper has no counterpart; this is a service for
 * callers that cannot allocate device memory: code running inside another
 * allocator's callbacks, in a process whose device memory belongs to a fixed
 * arena that must not grow, or in a loop that may not block on cudaMalloc.
 * It is pcg_solve with precision GB_F64 only, but it allocates nothing: its
 * scratch (permuted b and x, r, p, q, partial sums, solver scalars) lives in a
 * file-scope device array sized for at most 262144 rows (about 10.5 MB),
 * which every GPU that loads the library holds until the process exits.
 * The caller still passes A, d_b and d_x (n doubles each, x in: x0 unless
 * opt->x0_zero).  Larger systems return GB_TOO_LARGE with a message naming the
 * limit; other precisions return GB_EINVAL.  The CG loop is always direct
 * launches polled from the host (opt->use_graph is ignored), the call
 * synchronises `stream`, and stats->solve_ms is host wall time.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing once the library's module is
 * loaded there); the first call on a device may be what loads the module,
 * which reserves the array, so make that first call before any stream capture
 * begins.  All calls share the one array and the solver scalars are reset at
 * the start of every call; two calls whose work overlaps on the GPU
 * (different streams or threads) race on that array and give wrong results. */
int pcg_solve_noalloc(const gb_sell *A, const double *d_b, double *d_x, const PcgOptions *opt,
                      void *stream, PcgStats *stats);

/* Measurement entry point (no counterpart in the paper): runs `iters` fp64
 * (precision GB_F64) or fp32-inner (GB_F32_IR / GB_BF16_IR) CG iterations on
 * A with right-hand side d_b from x = 0, as direct launches on `stream`, with
 * a CUDA event pair around every launch, and writes the mean duration in
 * milliseconds of each of the iteration's three kernels to h_ms[0] (SpMV +
 * p.Ap), h_ms[1] (x, r update + r.z, r.r) and h_ms[2] (p update).  The
 * iterations run even past convergence (the scalars are reset each time), so
 * every timed launch does a full pass.  precision | GB_KT_BLOCK_JACOBI times
 * the block-Jacobi iteration instead (h_ms[1]: the x, r update with z = M^-1 r;
 * GB_EINVAL without sell_block_jacobi data).  Synchronises `stream`. */
enum { GB_KT_BLOCK_JACOBI = 256 };
int pcg_kernel_times(const gb_sell *A, const double *d_b, int precision, int iters, void *stream,
                     double *h_ms);

/* Measurement entry point (no counterpart in the paper): the batched
 * counterpart of pcg_kernel_times.  Runs `iters` iterations of the blocked
 * multi-RHS recurrences of pcg_solve_batched on nsys systems (system s with
 * k[s] right-hand sides, d_B[s] row-major n_s x k_s) from X = 0, in fp64
 * (GB_F64) or with fp32 recurrences (GB_F32_IR: fp32 values, GB_BF16_IR: bf16
 * values), as direct launches on `stream` with a CUDA event pair around every
 * launch, and writes the mean milliseconds of the iteration's three kernels to
 * h_ms[0] (SpMM + per-column p.Ap), h_ms[1] (X, R update + R.Z, R.R) and
 * h_ms[2] (P update).  Every column keeps iterating for the whole run.
 * Synchronises `stream`. */
int pcg_batched_kernel_times(int nsys, const gb_sell *const *A, const double *const *d_B, const int *k,
                             int precision, int iters, void *stream, double *h_ms);

/* RHS block width autotuner for blocked multi-RHS solves: the k columns of
 * d_B (n x k row-major, original order, 1 <= k <= 256) are cut into groups of
 * w = 1, 2, 4, 8, 16, 32 columns (w <= k); for each w one blocked iteration
 * of that batch (pcg_solve_batched's kernels) is timed with CUDA events and
 * *best_width receives the width with the least time; h_ms (6 doubles, may be
 * NULL) the iteration time per width (0 where w > k).  Pass groups of
 * *best_width columns to pcg_solve_batched.  Synchronises `stream`. */
int pcg_batched_autotune_width(const gb_sell *A, const double *d_B, int k, int precision, void *stream,
                               int *best_width, double *h_ms);

/* Diagnostic entry point (no counterpart in the paper): exercises, on the
 * GPU, the bounded wait that the library's kernels use on their shared-memory
 * transaction barriers.  One warp arms a barrier that nothing completes and
 * waits on it with a limit of limit_ms milliseconds (0 < limit_ms <= 2000); the
 * wait gives up, the kernel records how long it waited and returns, and the
 * call returns GB_TIMEOUT -- the status a solve reports when one of its waits
 * runs out -- with *h_waited_ms set (may be NULL).  The device stays usable
 * afterwards.  Allocates 16 bytes with cudaMalloc; synchronises `stream`. */
int gbpcg_wait_selftest(double limit_ms, void *stream, double *h_waited_ms);

/* Diagnostic entry point (no counterpart in the paper): exercises, on the
 * GPU, the bounded wait of the grid-tier persistent kernel's group exchange
 * (each block of a group publishes its partial sums and an exchange number in
 * a slot of global memory and waits until every block's slot shows the same
 * exchange).  The grid kernel runs with an empty system list and one block of
 * a group of two, so the second block's number never appears; the wait gives
 * up after limit_ms milliseconds (0 < limit_ms <= 2000), sets the kernel's
 * error word and returns, and the call returns GB_TIMEOUT -- what a solve
 * reports when a group exchange wait runs out -- with the kernel's duration
 * in *h_waited_ms (may be NULL).  The device stays usable afterwards.
 * Allocates a few KB with cudaMalloc; synchronises `stream`. */
int gbpcg_grid_wait_selftest(double limit_ms, void *stream, double *h_waited_ms);

#ifdef __cplusplus
}
#endif
#endif
