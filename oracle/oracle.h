/*
 * oracle.h -- plain, slow, single-threaded CPU oracle for the FEM-Laplace
 * Jacobi-PCG path.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product library never
 * does, and the two share no source.
 *
 * What it computes (all fp64):
 *   - the Laplace problem with Dirichlet data (paper Sec. 2.2): lattice meshes
 *     (regular or jittered triangles in 2D, Kuhn tetrahedra in 3D), P1/P2
 *     Lagrange elements, stiffness K_ij = int grad(phi_i).grad(phi_j);
 *   - elimination of the Dirichlet dofs: K_II u_I = -K_IB g_B;
 *   - Jacobi-preconditioned CG with the stopping rule of Eq. (2);
 *   - a dense Cholesky solve for tiny systems;
 *   - the SELL-C-sigma index structure (row permutation, chunk widths, padded
 *     column array) used by the device SpMV.
 * Every function states the passage or the definition it follows.
 */
#ifndef GBPCG_ORACLE_H
#define GBPCG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* SplitMix64 (Steele, Lea, Flood 2014): the i-th (0-based) output of the
 * sequential generator started at state `key` is mix64(key + (i+1)*gamma). */
uint64_t orc_rng_u64(uint64_t key, uint64_t i);
/* key of stream `stream` of run `seed`: seed*2^40 xor stream*2^32 (mod 2^64) */
uint64_t orc_rng_key(uint64_t seed, uint32_t stream);

typedef struct orc_sys orc_sys;

/* Mesh + dofs + elements (Sec. 2.2 case study).  dim 2|3, degree 1|2,
 * cells per side >= 1, jitter 0|1 (2D only), diag_mode 0 fixed SW-NE, 1 random.
 * Returns NULL on invalid arguments. */
orc_sys *orc_mesh(int dim, int degree, int cells, int jitter, int diag_mode, uint64_t seed);
void orc_free(orc_sys *s);

/* sizes: [0]=n_vertices [1]=n_dof [2]=n_elements [3]=n_loc [4]=n_free
 *        [5]=n_bnd [6]=nnz_full [7]=nnz_ii [8]=nnz_ib */
void orc_sizes(const orc_sys *s, int64_t out[9]);

void orc_get_vertex_coords(const orc_sys *s, double *out);      /* n_vertices*dim */
void orc_get_dof_coords(const orc_sys *s, double *out);         /* n_dof*dim */
void orc_get_elements(const orc_sys *s, int32_t *out);          /* n_elements*n_loc dof ids */
void orc_get_maps(const orc_sys *s, int32_t *free_of_full, int32_t *bnd_of_full,
                  int32_t *full_of_free, int32_t *full_of_bnd);

/* Element stiffness of element e (n_loc x n_loc, row-major). */
void orc_element_matrix(const orc_sys *s, int64_t e, double *out);

/* Assemble the full stiffness over all dofs for the rows selected by
 * row_mask (n_dof bytes, non-zero = keep; NULL = every row), then split the
 * selected free rows into K_II and K_IB.  Returns 0 on success. */
int orc_assemble(orc_sys *s, const uint8_t *row_mask);

void orc_get_full(const orc_sys *s, int64_t *rp, int32_t *ci, double *v);
void orc_get_ii(const orc_sys *s, int64_t *rp, int32_t *ci, double *v);
void orc_get_ib(const orc_sys *s, int64_t *rp, int32_t *ci, double *v);

/* Dirichlet data g evaluated at dof coordinates.  gid: 0 sin(pi x)sinh(pi y)/sinh(pi),
 * 1 x^2-y^2, 2 x^2+y^2-2z^2, 3 linear c0+c1 x+c2 y+c3 z (coef[4]),
 * 4 harmonic basis sum_k a_k Re(x+iy)^k + b_k Im(x+iy)^k, k=0..4 (coef[10] per column).
 * which: 0 boundary dofs (n_bnd rows), 1 free dofs (n_free rows).  out is
 * row-major rows x k; coef holds ncoef(gid) values per column. */
int orc_eval_g(const orc_sys *s, int gid, const double *coef, int k, int which, double *out);

/* b = -K_IB g_B for k columns (row-major n_free x k). */
void orc_lift(const orc_sys *s, const double *gB, int k, double *b);

/* y = A x for a CSR matrix. */
void orc_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
              const double *x, double *y);

/* Jacobi-PCG (Hestenes-Stiefel CG with M = diag(A)), x in: x0, out: x.
 * Stops when ||b - A x||_2 / ||b||_2 <= tol (Eq. 2), checked on the recursive
 * residual and confirmed on the true residual.  Returns 0 converged,
 * 1 not converged in maxit, 2 breakdown (p.Ap <= 0 or non-finite). */
int orc_pcg(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
            const double *b, double *x, double tol, int64_t maxit,
            int64_t *iters, double *relres);

/* Block-Jacobi (Sec. 3.2, Sec. 4.2): M = blockdiag of the diagonal blocks of
 * bs consecutive rows (the last one shorter when bs does not divide n).
 * orc_bjacobi writes each block's inverse, dense row-major, into W
 * (ceil(n/bs) x bs x bs; a short block fills its leading corner, the rest 0);
 * returns 0, or 1 if a block is not SPD.  orc_bjacobi_apply: z = M^{-1} r.
 * orc_pcg_bj: orc_pcg with this M (returns 2 if a block is not SPD). */
int orc_bjacobi(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int bs,
                double *W);
void orc_bjacobi_apply(int64_t n, int bs, const double *W, const double *r, double *z);
int orc_pcg_bj(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int bs,
               const double *b, double *x, double tol, int64_t maxit, int64_t *iters,
               double *relres);

/* BiCGSTAB (Sec. 3.2's Krylov method), right-preconditioned: bs <= 1 Jacobi,
 * bs >= 2 block-Jacobi over blocks of bs rows (orc_bjacobi).  Any nonsingular
 * CSR matrix.  Stops on Eq. (2), confirmed on the true residual (restart from
 * it otherwise).  Returns 0 converged, 1 not converged in maxit steps, 2
 * breakdown; relres: the true relative residual of the x returned. */
int orc_bicgstab(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int bs,
                 const double *b, double *x, double tol, int64_t maxit, int64_t *iters,
                 double *relres);

/* Block CG for A X = B (Sec. 4.3's block of right-hand sides; B, X n x k
 * row-major, X in: X0, out: X): one shared Krylov space (O'Leary), in the
 * breakdown-free form of Ji and Li (rank-revealing orthonormalisation of the
 * search block), Jacobi preconditioner.  Stops when every column meets Eq. (2)
 * on the true residual; relres[k] receives the final relative residuals.
 * Returns 0 converged, 1 not converged in maxit steps, 2 breakdown (no
 * search direction left above the rank threshold, or P^T A P not SPD). */
int orc_block_cg(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int k,
                 const double *B, double *X, double tol, int64_t maxit, int64_t *iters,
                 double *relres);

/* Dense Cholesky solve A x = b (n small).  Returns 0, or 1 if A is not SPD. */
int orc_cholesky_solve(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                       const double *b, double *x);

/* SELL-C-sigma structure of a CSR pattern.  orc_sell_size gives the number of
 * chunks and the padded length; orc_sell_fill writes perm[new]=old,
 * chunk_ptr[nchunks+1], chunk_w[nchunks], row_len[n] (new order) and the padded
 * column array in new numbering (column-major inside a chunk). */
void orc_sell_size(int64_t n, const int64_t *rp, int C, int sigma,
                   int64_t *nchunks, int64_t *padded);
void orc_sell_fill(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                   int C, int sigma, int32_t *perm, int64_t *chunk_ptr,
                   int32_t *chunk_w, int32_t *row_len, int32_t *col, double *val);

#ifdef __cplusplus
}
#endif
#endif
