/*
 * oracle.c -- plain CPU oracle (fp64, single thread).  TEST INFRASTRUCTURE:
 * loaded only by the tests, the smoke check and the benchmark's CPU-baseline
 * leg.  It shares no code with the CUDA library.  Build: gcc -O2 -std=c11
 * -ffp-contract=off (no FMA contraction, so the jittered coordinates are
 * reproducible bit for bit from their defining expression).
 *
 * The problem (paper Sec. 2.2): Laplace's equation Delta u = 0 on the unit
 * square/cube with u = g on the boundary, discretised with P1 (the paper's
 * linear case, whose 2D/3D weights are the cotangent formula of Sec. 2.2) or
 * P2 Lagrange elements (the polynomial-degree study of Sec. 4.2, Table 7).
 * The stiffness matrix is K_ij = sum_T int_T grad(phi_i).grad(phi_j); the
 * Dirichlet dofs are eliminated, leaving the SPD system K_II u = -K_IB g_B,
 * which is solved by CG with the Jacobi preconditioner M = diag(K_II)
 * (preconditioned Krylov solve, Sec. 2.1) to the relative residual of Eq. (2).
 *
 * The `omp` pragmas on the CG loops are inert in the pinned build above (no
 * -fopenmp); the benchmark's all-core CPU baseline compiles this same source
 * a second time with -fopenmp for timing only (its dot products then sum in
 * per-thread pieces, so its rounding differs from the single-thread build's).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG -- */
/* SplitMix64: state advances by the golden-ratio increment gamma; each state
 * is passed through the mix64 finaliser (shift-xor, multiply, twice). */
static const uint64_t GAMMA = 0x9E3779B97F4A7C15ULL;

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_rng_u64(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GAMMA); }

uint64_t orc_rng_key(uint64_t seed, uint32_t stream) {
    return (seed << 40) ^ ((uint64_t)stream << 32);
}

/* uniform double in [0,1) from the top 53 bits */
static double u01(uint64_t r) { return (double)(r >> 11) * 0x1p-53; }

/* --------------------------------------------------------------- system -- */
struct orc_sys {
    int dim, degree, cells, jitter, diag_mode;
    uint64_t seed;
    int V;          /* vertices per side: cells+1 */
    int S;          /* dof-lattice points per side: degree*cells+1 */
    int64_t nv, ndof, nel;
    int nvert_el;   /* dim+1 */
    int nloc;       /* dofs per element */
    int beta[35][4]; /* degree >= 3: local dof l = Lagrange node sum_a beta[l][a] P_a / degree */
    double *vx;     /* nv*dim */
    double *dx;     /* ndof*dim */
    int32_t *elv;   /* nel*nvert_el vertex ids */
    int32_t *eld;   /* nel*nloc dof ids: vertices first, then edges (a,b), a<b */
    int32_t *free_of_full, *bnd_of_full, *full_of_free, *full_of_bnd;
    int64_t nfree, nbnd;
    /* assembled (selected rows) */
    int64_t nnz_full, nnz_ii, nnz_ib;
    int64_t *rp_full, *rp_ii, *rp_ib;
    int32_t *ci_full, *ci_ii, *ci_ib;
    double *v_full, *v_ii, *v_ib;
};

static void free_assembly(orc_sys *s) {
    free(s->rp_full); free(s->ci_full); free(s->v_full);
    free(s->rp_ii); free(s->ci_ii); free(s->v_ii);
    free(s->rp_ib); free(s->ci_ib); free(s->v_ib);
    s->rp_full = s->rp_ii = s->rp_ib = NULL;
    s->ci_full = s->ci_ii = s->ci_ib = NULL;
    s->v_full = s->v_ii = s->v_ib = NULL;
    s->nnz_full = s->nnz_ii = s->nnz_ib = 0;
}

void orc_free(orc_sys *s) {
    if (!s) return;
    free_assembly(s);
    free(s->vx); free(s->dx); free(s->elv); free(s->eld);
    free(s->free_of_full); free(s->bnd_of_full); free(s->full_of_free); free(s->full_of_bnd);
    free(s);
}

/* local edge list of a simplex: (a,b) with a<b in lexicographic order */
static const int EDGES2[3][2] = {{0, 1}, {0, 2}, {1, 2}};
static const int EDGES3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
/* Kuhn split of a cube: one tetrahedron per ordering of the three axes; the
 * path v000 -> +e_p0 -> +e_p1 -> +e_p2 = v111. */
static const int KUHN[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

orc_sys *orc_mesh(int dim, int degree, int cells, int jitter, int diag_mode, uint64_t seed) {
    if ((dim != 2 && dim != 3) || degree < 1 || degree > 4 || cells < 1) return NULL;
    orc_sys *s = (orc_sys *)calloc(1, sizeof(orc_sys));
    s->dim = dim; s->degree = degree; s->cells = cells; s->jitter = jitter;
    s->diag_mode = diag_mode; s->seed = seed;
    s->V = cells + 1;
    s->S = degree * cells + 1;
    s->nv = 1; s->ndof = 1;
    for (int d = 0; d < dim; ++d) { s->nv *= s->V; s->ndof *= s->S; }
    s->nvert_el = dim + 1;
    s->nloc = degree == 1 ? dim + 1 : (dim == 2 ? 6 : 10);
    if (degree >= 3) {
        /* Lagrange nodes of degree m: multi-indices beta in N^(d+1), |beta| = m,
         * enumerated with beta_1 slowest ... beta_d fastest, beta_0 = m - rest */
        int l = 0;
        if (dim == 2) {
            for (int b1 = 0; b1 <= degree; ++b1)
                for (int b2 = 0; b1 + b2 <= degree; ++b2, ++l) {
                    s->beta[l][0] = degree - b1 - b2; s->beta[l][1] = b1; s->beta[l][2] = b2; s->beta[l][3] = 0;
                }
        } else {
            for (int b1 = 0; b1 <= degree; ++b1)
                for (int b2 = 0; b1 + b2 <= degree; ++b2)
                    for (int b3 = 0; b1 + b2 + b3 <= degree; ++b3, ++l) {
                        s->beta[l][0] = degree - b1 - b2 - b3;
                        s->beta[l][1] = b1; s->beta[l][2] = b2; s->beta[l][3] = b3;
                    }
        }
        s->nloc = l; /* (m+1)(m+2)/2 in 2D, (m+1)(m+2)(m+3)/6 in 3D */
    }
    int64_t ncell = 1;
    for (int d = 0; d < dim; ++d) ncell *= cells;
    s->nel = ncell * (dim == 2 ? 2 : 6);

    /* vertex coordinates: lattice point i/cells, interior points of a jittered
     * mesh moved by (2u-1)*q per coordinate, u from streams 0 (x), 1 (y) and
     * 3 (z), counter = vertex id; q = h/4 in 2D and h/8 in 3D, the largest
     * amplitude h/2^m at which no Kuhn tetrahedron can invert (at h/4 one can:
     * the determinant of its edge vectors reaches -h^3/2 over the corners of
     * the jitter box, against >= h^3/4 at h/8). */
    s->vx = (double *)malloc(sizeof(double) * s->nv * dim);
    const uint64_t keys[3] = {orc_rng_key(seed, 0), orc_rng_key(seed, 1), orc_rng_key(seed, 3)};
    const double q = (dim == 3 ? 0.125 : 0.25) / (double)cells;
    for (int64_t v = 0; v < s->nv; ++v) {
        int64_t t = v;
        int idx[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) { idx[d] = (int)(t % s->V); t /= s->V; }
        int interior = 1;
        for (int d = 0; d < dim; ++d) if (idx[d] == 0 || idx[d] == cells) interior = 0;
        for (int d = 0; d < dim; ++d) {
            double x = (double)idx[d] / (double)cells;
            if (jitter && interior) {
                uint64_t r = orc_rng_u64(keys[d], (uint64_t)v);
                double dd = 2.0 * u01(r) - 1.0;
                x = x + dd * q;
            }
            s->vx[v * dim + d] = x;
        }
    }

    /* elements */
    s->elv = (int32_t *)malloc(sizeof(int32_t) * s->nel * s->nvert_el);
    s->eld = (int32_t *)malloc(sizeof(int32_t) * s->nel * s->nloc);
    const uint64_t kf = orc_rng_key(seed, 2);
    int64_t e = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        int ci[3] = {0, 0, 0};
        int64_t t = c;
        for (int d = 0; d < dim; ++d) { ci[d] = (int)(t % cells); t /= cells; }
        if (dim == 2) {
            int32_t v00 = ci[0] + s->V * ci[1];
            int32_t v10 = v00 + 1, v01 = v00 + s->V, v11 = v00 + s->V + 1;
            int flip = 0;
            if (diag_mode == 1) flip = (orc_rng_u64(kf, (uint64_t)c) >> 63) == 0; /* u < 1/2 */
            int32_t tri[2][3];
            if (!flip) { /* diagonal v00-v11 */
                tri[0][0] = v00; tri[0][1] = v10; tri[0][2] = v11;
                tri[1][0] = v00; tri[1][1] = v11; tri[1][2] = v01;
            } else {     /* diagonal v10-v01 */
                tri[0][0] = v00; tri[0][1] = v10; tri[0][2] = v01;
                tri[1][0] = v10; tri[1][1] = v11; tri[1][2] = v01;
            }
            for (int k = 0; k < 2; ++k, ++e)
                for (int a = 0; a < 3; ++a) s->elv[e * 3 + a] = tri[k][a];
        } else {
            for (int k = 0; k < 6; ++k, ++e) {
                int p[3] = {ci[0], ci[1], ci[2]};
                s->elv[e * 4 + 0] = p[0] + s->V * (p[1] + s->V * p[2]);
                for (int m = 0; m < 3; ++m) {
                    p[KUHN[k][m]] += 1;
                    s->elv[e * 4 + m + 1] = p[0] + s->V * (p[1] + s->V * p[2]);
                }
            }
        }
    }

    /* dof ids: vertex (i,j,k) -> dof-lattice point degree*(i,j,k); edge midpoint
     * -> the mean of its endpoints' dof-lattice points. */
    s->dx = (double *)malloc(sizeof(double) * s->ndof * dim);
    for (int64_t i = 0; i < s->ndof * dim; ++i) s->dx[i] = NAN;
    for (e = 0; e < s->nel; ++e) {
        int lat[4][3];
        for (int a = 0; a < s->nvert_el; ++a) {
            int64_t t = s->elv[e * s->nvert_el + a];
            for (int d = 0; d < 3; ++d) { lat[a][d] = 0; }
            for (int d = 0; d < dim; ++d) { lat[a][d] = (int)(t % s->V) * degree; t /= s->V; }
        }
        for (int a = 0; a < s->nvert_el; ++a) {
            int64_t id = 0, mul = 1;
            for (int d = 0; d < dim; ++d) { id += lat[a][d] * mul; mul *= s->S; }
            s->eld[e * s->nloc + a] = (int32_t)id;
            const int32_t v = s->elv[e * s->nvert_el + a];
            for (int d = 0; d < dim; ++d) s->dx[id * dim + d] = s->vx[(int64_t)v * dim + d];
        }
        if (degree >= 3) {
            /* node beta sits at dof-lattice point sum_a beta_a v_a (vertex v_a in
             * cell units): the degree-refined lattice.  Its coordinates are
             * (sum_a beta_a P_a) / degree over the vertices with beta_a > 0 -- the
             * smallest mesh face holding the node, the same from every element
             * around it -- summed in ascending vertex id with correctly rounded
             * operations; a vertex node is the vertex itself. */
            int vc[4][3];
            for (int a = 0; a < s->nvert_el; ++a)
                for (int d = 0; d < dim; ++d) vc[a][d] = lat[a][d] / degree;
            for (int l = 0; l < s->nloc; ++l) {
                int64_t id = 0, mul = 1;
                int N[3] = {0, 0, 0};
                for (int d = 0; d < dim; ++d) {
                    for (int a = 0; a < s->nvert_el; ++a) N[d] += s->beta[l][a] * vc[a][d];
                    id += N[d] * mul;
                    mul *= s->S;
                }
                s->eld[e * s->nloc + l] = (int32_t)id;
                int32_t fv[4];
                int fb[4], nf = 0;
                for (int a = 0; a < s->nvert_el; ++a)
                    if (s->beta[l][a] > 0) { fv[nf] = s->elv[e * s->nvert_el + a]; fb[nf] = s->beta[l][a]; ++nf; }
                for (int i = 1; i < nf; ++i) { /* ascending vertex id */
                    int32_t tv = fv[i]; int tb = fb[i], j = i;
                    while (j > 0 && fv[j - 1] > tv) { fv[j] = fv[j - 1]; fb[j] = fb[j - 1]; --j; }
                    fv[j] = tv; fb[j] = tb;
                }
                for (int d = 0; d < dim; ++d) {
                    if (nf == 1) { s->dx[id * dim + d] = s->vx[(int64_t)fv[0] * dim + d]; continue; }
                    double t = 0.0;
                    for (int i = 0; i < nf; ++i) t = t + (double)fb[i] * s->vx[(int64_t)fv[i] * dim + d];
                    s->dx[id * dim + d] = t / (double)degree;
                }
            }
        }
        if (degree == 2) {
            const int ne = dim == 2 ? 3 : 6;
            for (int m = 0; m < ne; ++m) {
                const int a = dim == 2 ? EDGES2[m][0] : EDGES3[m][0];
                const int b = dim == 2 ? EDGES2[m][1] : EDGES3[m][1];
                int64_t id = 0, mul = 1;
                for (int d = 0; d < dim; ++d) { id += ((lat[a][d] + lat[b][d]) / 2) * mul; mul *= s->S; }
                s->eld[e * s->nloc + s->nvert_el + m] = (int32_t)id;
                const int32_t va = s->elv[e * s->nvert_el + a], vb = s->elv[e * s->nvert_el + b];
                for (int d = 0; d < dim; ++d)
                    s->dx[id * dim + d] = (s->vx[(int64_t)va * dim + d] + s->vx[(int64_t)vb * dim + d]) * 0.5;
            }
        }
    }

    /* boundary: a dof-lattice coordinate equal to 0 or S-1.  Free and boundary
     * dofs keep the order of the full numbering. */
    s->free_of_full = (int32_t *)malloc(sizeof(int32_t) * s->ndof);
    s->bnd_of_full = (int32_t *)malloc(sizeof(int32_t) * s->ndof);
    s->nfree = s->nbnd = 0;
    for (int64_t i = 0; i < s->ndof; ++i) {
        int64_t t = i;
        int onb = 0;
        for (int d = 0; d < dim; ++d) {
            int c = (int)(t % s->S); t /= s->S;
            if (c == 0 || c == s->S - 1) onb = 1;
        }
        if (onb) { s->bnd_of_full[i] = (int32_t)s->nbnd++; s->free_of_full[i] = -1; }
        else { s->free_of_full[i] = (int32_t)s->nfree++; s->bnd_of_full[i] = -1; }
    }
    s->full_of_free = (int32_t *)malloc(sizeof(int32_t) * (s->nfree ? s->nfree : 1));
    s->full_of_bnd = (int32_t *)malloc(sizeof(int32_t) * (s->nbnd ? s->nbnd : 1));
    for (int64_t i = 0; i < s->ndof; ++i) {
        if (s->free_of_full[i] >= 0) s->full_of_free[s->free_of_full[i]] = (int32_t)i;
        else s->full_of_bnd[s->bnd_of_full[i]] = (int32_t)i;
    }
    return s;
}

void orc_sizes(const orc_sys *s, int64_t out[9]) {
    out[0] = s->nv; out[1] = s->ndof; out[2] = s->nel; out[3] = s->nloc;
    out[4] = s->nfree; out[5] = s->nbnd; out[6] = s->nnz_full; out[7] = s->nnz_ii; out[8] = s->nnz_ib;
}

void orc_get_vertex_coords(const orc_sys *s, double *out) {
    memcpy(out, s->vx, sizeof(double) * s->nv * s->dim);
}
void orc_get_dof_coords(const orc_sys *s, double *out) {
    memcpy(out, s->dx, sizeof(double) * s->ndof * s->dim);
}
void orc_get_elements(const orc_sys *s, int32_t *out) {
    memcpy(out, s->eld, sizeof(int32_t) * s->nel * s->nloc);
}
void orc_get_maps(const orc_sys *s, int32_t *fof, int32_t *bof, int32_t *foff, int32_t *fofb) {
    if (fof) memcpy(fof, s->free_of_full, sizeof(int32_t) * s->ndof);
    if (bof) memcpy(bof, s->bnd_of_full, sizeof(int32_t) * s->ndof);
    if (foff) memcpy(foff, s->full_of_free, sizeof(int32_t) * s->nfree);
    if (fofb) memcpy(fofb, s->full_of_bnd, sizeof(int32_t) * s->nbnd);
}

/* ------------------------------------------------------ element matrix -- */
/* Barycentric gradients of a simplex with vertices P[0..d]: with J the matrix
 * whose columns are P[a]-P[0] (a=1..d), lambda_a for a>=1 are the entries of
 * J^{-1}(x-P[0]), so grad(lambda_a) is row a-1 of J^{-1}, and
 * grad(lambda_0) = -sum_{a>=1} grad(lambda_a).  |T| = |det J| / d!. */
static double simplex_gradients(int dim, const double P[4][3], double g[4][3]) {
    double J[3][3] = {{0}};
    for (int a = 1; a <= dim; ++a)
        for (int r = 0; r < dim; ++r) J[r][a - 1] = P[a][r] - P[0][r];
    double det, inv[3][3];
    if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        inv[0][0] = J[1][1] / det;  inv[0][1] = -J[0][1] / det;
        inv[1][0] = -J[1][0] / det; inv[1][1] = J[0][0] / det;
    } else {
        /* inverse = adjugate / det; adjugate = transpose of the cofactors */
        double cof[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, c1 = (c + 1) % 3, c2 = (c + 2) % 3;
                cof[r][c] = J[r1][c1] * J[r2][c2] - J[r1][c2] * J[r2][c1];
            }
        det = J[0][0] * cof[0][0] + J[0][1] * cof[0][1] + J[0][2] * cof[0][2];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) inv[r][c] = cof[c][r] / det;
    }
    for (int a = 1; a <= dim; ++a)
        for (int c = 0; c < dim; ++c) g[a][c] = inv[a - 1][c];
    for (int c = 0; c < dim; ++c) {
        double t = 0.0;
        for (int a = 1; a <= dim; ++a) t += g[a][c];
        g[0][c] = -t;
    }
    return fabs(det) / (dim == 2 ? 2.0 : 6.0);
}

/* Gradient of local basis function i written as sum_{m,c} C[m][c] lambda_m grad(lambda_c)
 * (homogeneous in lambda because sum_m lambda_m = 1):
 *   P2 vertex a: phi = lambda_a (2 lambda_a - 1), grad = (4 lambda_a - 1) g_a
 *                -> C[m][a] = 3 if m == a else -1;
 *   P2 edge (a,b): phi = 4 lambda_a lambda_b, grad = 4 lambda_a g_b + 4 lambda_b g_a. */
static void p2_grad_coeffs(int dim, int i, double C[4][4]) {
    for (int m = 0; m < 4; ++m)
        for (int c = 0; c < 4; ++c) C[m][c] = 0.0;
    const int nv = dim + 1;
    if (i < nv) {
        for (int m = 0; m < nv; ++m) C[m][i] = (m == i) ? 3.0 : -1.0;
    } else {
        const int k = i - nv;
        const int a = dim == 2 ? EDGES2[k][0] : EDGES3[k][0];
        const int b = dim == 2 ? EDGES2[k][1] : EDGES3[k][1];
        C[a][b] = 4.0;
        C[b][a] = 4.0;
    }
}

/* Degree m >= 3: Silvester's form of the Lagrange basis,
 *   phi_beta(lambda) = prod_a P_{beta_a}(lambda_a),  P_k(t) = prod_{j<k} (m t - j)/(j + 1),
 * and grad phi = sum_a (d phi / d lambda_a) grad lambda_a, so
 *   K_{beta,gamma} = sum_{a,b} (g_a . g_b) int_T (d_a phi_beta)(d_b phi_gamma)
 * with every integrand a product over c of polynomials in lambda_c alone,
 * integrated monomial by monomial: int_T prod lambda_c^e_c = |T| d! prod e_c! / (d + sum e)!.
 * The reference integrals (per unit |T|) depend on (d, m) only: tabulated once. */
#define PMAX 4
static int ref_dim = 0, ref_deg = 0, ref_nloc = 0;
static double *ref_tab = NULL; /* [i][j][a][b] */

/* coefficients (degree <= PMAX) of P_k and its derivative */
static void silvester(int m, int k, double *c, double *dc) {
    for (int i = 0; i <= PMAX; ++i) c[i] = 0.0;
    c[0] = 1.0;
    for (int j = 0; j < k; ++j) { /* multiply by (m t - j)/(j+1) */
        double nc[PMAX + 1] = {0};
        for (int i = 0; i <= PMAX; ++i) {
            if (c[i] == 0.0) continue;
            if (i + 1 <= PMAX) nc[i + 1] += c[i] * (double)m / (double)(j + 1);
            nc[i] -= c[i] * (double)j / (double)(j + 1);
        }
        for (int i = 0; i <= PMAX; ++i) c[i] = nc[i];
    }
    for (int i = 0; i <= PMAX; ++i) dc[i] = (i + 1 <= PMAX) ? (double)(i + 1) * c[i + 1] : 0.0;
}

static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }

static void build_ref_table(const orc_sys *s) {
    const int d = s->dim, nv = d + 1, m = s->degree, nl = s->nloc;
    if (ref_tab && ref_dim == d && ref_deg == m) return;
    free(ref_tab);
    ref_tab = (double *)calloc((size_t)nl * nl * nv * nv, sizeof(double));
    ref_dim = d; ref_deg = m; ref_nloc = nl;
    double P[PMAX + 1][PMAX + 1], dP[PMAX + 1][PMAX + 1];
    for (int k = 0; k <= m; ++k) silvester(m, k, P[k], dP[k]);
    for (int i = 0; i < nl; ++i)
        for (int j = 0; j < nl; ++j)
            for (int a = 0; a < nv; ++a)
                for (int b = 0; b < nv; ++b) {
                    /* u_c = f_c h_c, f_c = (c == a ? P' : P)_{beta_i c}, h_c likewise for j, b */
                    double u[4][2 * PMAX + 1];
                    for (int c = 0; c < nv; ++c) {
                        const double *f = (c == a) ? dP[s->beta[i][c]] : P[s->beta[i][c]];
                        const double *h = (c == b) ? dP[s->beta[j][c]] : P[s->beta[j][c]];
                        for (int t = 0; t <= 2 * PMAX; ++t) u[c][t] = 0.0;
                        for (int p = 0; p <= PMAX; ++p)
                            for (int q = 0; q <= PMAX; ++q) u[c][p + q] += f[p] * h[q];
                    }
                    /* sum over exponent tuples, each e_c up to the degree of u_c */
                    int E[4] = {1, 1, 1, 1};
                    for (int c = 0; c < nv; ++c) {
                        int top = 0;
                        for (int t = 0; t <= 2 * PMAX; ++t) if (u[c][t] != 0.0) top = t;
                        E[c] = top + 1;
                    }
                    double tot = 0.0;
                    int e[4] = {0, 0, 0, 0};
                    int64_t ncomb = 1;
                    for (int c = 0; c < nv; ++c) ncomb *= E[c];
                    for (int64_t z = 0; z < ncomb; ++z) {
                        int64_t t = z;
                        double coef = 1.0, pf = 1.0;
                        int se = 0;
                        for (int c = 0; c < nv; ++c) {
                            e[c] = (int)(t % E[c]); t /= E[c];
                            coef *= u[c][e[c]];
                            pf *= factorial(e[c]);
                            se += e[c];
                        }
                        if (coef == 0.0) continue;
                        tot += coef * factorial(d) * pf / factorial(d + se);
                    }
                    ref_tab[(((size_t)i * nl + j) * nv + a) * nv + b] = tot;
                }
}

void orc_element_matrix(const orc_sys *s, int64_t e, double *out) {
    const int dim = s->dim, nv = dim + 1, nloc = s->nloc;
    double P[4][3] = {{0}}, g[4][3] = {{0}};
    for (int a = 0; a < nv; ++a) {
        const int32_t v = s->elv[e * nv + a];
        for (int d = 0; d < dim; ++d) P[a][d] = s->vx[(int64_t)v * dim + d];
    }
    const double vol = simplex_gradients(dim, P, g);
    double G[4][4];
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) {
            double t = 0.0;
            for (int d = 0; d < dim; ++d) t += g[a][d] * g[b][d];
            G[a][b] = t;
        }
    if (s->degree == 1) {
        /* K_ab = |T| grad(lambda_a).grad(lambda_b) */
        for (int a = 0; a < nv; ++a)
            for (int b = 0; b < nv; ++b) out[a * nloc + b] = vol * G[a][b];
        return;
    }
    if (s->degree >= 3) {
        build_ref_table(s);
        for (int i = 0; i < nloc; ++i)
            for (int j = i; j < nloc; ++j) { /* K_ji = K_ij: computed once */
                double t = 0.0;
                for (int a = 0; a < nv; ++a)
                    for (int b = 0; b < nv; ++b) t += G[a][b] * ref_tab[(((size_t)i * nloc + j) * nv + a) * nv + b];
                out[i * nloc + j] = vol * t;
                out[j * nloc + i] = vol * t;
            }
        return;
    }
    /* int_T lambda_m lambda_n = |T| d! (1 + delta_mn) / (d+2)! */
    const double fact = dim == 2 ? 2.0 / 24.0 : 6.0 / 120.0;
    double M[4][4];
    for (int m = 0; m < nv; ++m)
        for (int n = 0; n < nv; ++n) M[m][n] = vol * fact * (m == n ? 2.0 : 1.0);
    double Ci[4][4], Cj[4][4];
    for (int i = 0; i < nloc; ++i) {
        p2_grad_coeffs(dim, i, Ci);
        for (int j = i; j < nloc; ++j) {
            p2_grad_coeffs(dim, j, Cj);
            /* K_ij = sum_{m,c,n,e} Ci[m][c] Cj[n][e] (g_c.g_e) int lambda_m lambda_n */
            double t = 0.0;
            for (int m = 0; m < nv; ++m)
                for (int c = 0; c < nv; ++c) {
                    if (Ci[m][c] == 0.0) continue;
                    for (int n = 0; n < nv; ++n)
                        for (int ee = 0; ee < nv; ++ee) {
                            if (Cj[n][ee] == 0.0) continue;
                            t += Ci[m][c] * Cj[n][ee] * G[c][ee] * M[m][n];
                        }
                }
            out[i * nloc + j] = t;
            out[j * nloc + i] = t;
        }
    }
}

/* ------------------------------------------------------------ assembly -- */
typedef struct { int32_t col; double val; } trip;

/* stable insertion sort by column (keeps element order among duplicates) */
static void sort_row(trip *t, int64_t m) {
    for (int64_t i = 1; i < m; ++i) {
        trip x = t[i];
        int64_t j = i - 1;
        while (j >= 0 && t[j].col > x.col) { t[j + 1] = t[j]; --j; }
        t[j + 1] = x;
    }
}

int orc_assemble(orc_sys *s, const uint8_t *row_mask) {
    free_assembly(s);
    const int nloc = s->nloc;
    /* pass 1: triplet count per selected row */
    int64_t *cnt = (int64_t *)calloc((size_t)s->ndof + 1, sizeof(int64_t));
    for (int64_t e = 0; e < s->nel; ++e)
        for (int a = 0; a < nloc; ++a) {
            const int32_t i = s->eld[e * nloc + a];
            if (!row_mask || row_mask[i]) cnt[i + 1] += nloc;
        }
    for (int64_t i = 0; i < s->ndof; ++i) cnt[i + 1] += cnt[i];
    const int64_t ntrip = cnt[s->ndof];
    trip *T = (trip *)malloc(sizeof(trip) * (ntrip ? ntrip : 1));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (s->ndof ? s->ndof : 1));
    memcpy(pos, cnt, sizeof(int64_t) * s->ndof);
    /* pass 2: scatter element matrices in element order */
    double Ke[35 * 35];
    for (int64_t e = 0; e < s->nel; ++e) {
        int any = !row_mask;
        for (int a = 0; a < nloc && !any; ++a) any = row_mask[s->eld[e * nloc + a]] != 0;
        if (!any) continue;
        orc_element_matrix(s, e, Ke);
        for (int a = 0; a < nloc; ++a) {
            const int32_t i = s->eld[e * nloc + a];
            if (row_mask && !row_mask[i]) continue;
            for (int b = 0; b < nloc; ++b) {
                T[pos[i]].col = s->eld[e * nloc + b];
                T[pos[i]].val = Ke[a * nloc + b];
                pos[i]++;
            }
        }
    }
    free(pos);
    /* pass 3: per row, sort by column and sum duplicates in element order */
    s->rp_full = (int64_t *)malloc(sizeof(int64_t) * (s->ndof + 1));
    s->rp_full[0] = 0;
    int64_t nnz = 0;
    for (int64_t i = 0; i < s->ndof; ++i) {
        trip *t = T + cnt[i];
        const int64_t m = cnt[i + 1] - cnt[i];
        sort_row(t, m);
        int64_t w = 0;
        for (int64_t k = 0; k < m; ++k) {
            if (w > 0 && t[w - 1].col == t[k].col) t[w - 1].val += t[k].val;
            else t[w++] = t[k];
        }
        nnz += w;
        s->rp_full[i + 1] = nnz;
    }
    s->nnz_full = nnz;
    s->ci_full = (int32_t *)malloc(sizeof(int32_t) * (nnz ? nnz : 1));
    s->v_full = (double *)malloc(sizeof(double) * (nnz ? nnz : 1));
    for (int64_t i = 0; i < s->ndof; ++i) {
        const trip *t = T + cnt[i];
        const int64_t w = s->rp_full[i + 1] - s->rp_full[i];
        for (int64_t k = 0; k < w; ++k) {
            s->ci_full[s->rp_full[i] + k] = t[k].col;
            s->v_full[s->rp_full[i] + k] = t[k].val;
        }
    }
    free(T);
    free(cnt);

    /* split: free rows; free columns -> K_II (free numbering), boundary
     * columns -> K_IB (boundary numbering).  Both keep ascending columns. */
    s->rp_ii = (int64_t *)malloc(sizeof(int64_t) * (s->nfree + 1));
    s->rp_ib = (int64_t *)malloc(sizeof(int64_t) * (s->nfree + 1));
    s->rp_ii[0] = s->rp_ib[0] = 0;
    for (int64_t f = 0; f < s->nfree; ++f) {
        const int32_t i = s->full_of_free[f];
        int64_t a = 0, b = 0;
        for (int64_t k = s->rp_full[i]; k < s->rp_full[i + 1]; ++k) {
            if (s->free_of_full[s->ci_full[k]] >= 0) ++a; else ++b;
        }
        s->rp_ii[f + 1] = s->rp_ii[f] + a;
        s->rp_ib[f + 1] = s->rp_ib[f] + b;
    }
    s->nnz_ii = s->rp_ii[s->nfree];
    s->nnz_ib = s->rp_ib[s->nfree];
    s->ci_ii = (int32_t *)malloc(sizeof(int32_t) * (s->nnz_ii ? s->nnz_ii : 1));
    s->v_ii = (double *)malloc(sizeof(double) * (s->nnz_ii ? s->nnz_ii : 1));
    s->ci_ib = (int32_t *)malloc(sizeof(int32_t) * (s->nnz_ib ? s->nnz_ib : 1));
    s->v_ib = (double *)malloc(sizeof(double) * (s->nnz_ib ? s->nnz_ib : 1));
    for (int64_t f = 0; f < s->nfree; ++f) {
        const int32_t i = s->full_of_free[f];
        int64_t a = s->rp_ii[f], b = s->rp_ib[f];
        for (int64_t k = s->rp_full[i]; k < s->rp_full[i + 1]; ++k) {
            const int32_t j = s->ci_full[k];
            if (s->free_of_full[j] >= 0) { s->ci_ii[a] = s->free_of_full[j]; s->v_ii[a++] = s->v_full[k]; }
            else { s->ci_ib[b] = s->bnd_of_full[j]; s->v_ib[b++] = s->v_full[k]; }
        }
    }
    return 0;
}

void orc_get_full(const orc_sys *s, int64_t *rp, int32_t *ci, double *v) {
    if (rp) memcpy(rp, s->rp_full, sizeof(int64_t) * (s->ndof + 1));
    if (ci) memcpy(ci, s->ci_full, sizeof(int32_t) * s->nnz_full);
    if (v) memcpy(v, s->v_full, sizeof(double) * s->nnz_full);
}
void orc_get_ii(const orc_sys *s, int64_t *rp, int32_t *ci, double *v) {
    if (rp) memcpy(rp, s->rp_ii, sizeof(int64_t) * (s->nfree + 1));
    if (ci) memcpy(ci, s->ci_ii, sizeof(int32_t) * s->nnz_ii);
    if (v) memcpy(v, s->v_ii, sizeof(double) * s->nnz_ii);
}
void orc_get_ib(const orc_sys *s, int64_t *rp, int32_t *ci, double *v) {
    if (rp) memcpy(rp, s->rp_ib, sizeof(int64_t) * (s->nfree + 1));
    if (ci) memcpy(ci, s->ci_ib, sizeof(int32_t) * s->nnz_ib);
    if (v) memcpy(v, s->v_ib, sizeof(double) * s->nnz_ib);
}

/* ------------------------------------------------------- Dirichlet data -- */
static int ncoef(int gid) { return gid == 3 ? 4 : (gid == 4 ? 10 : 0); }

static double gfun(int gid, const double *c, const double *p, int dim) {
    const double x = p[0], y = p[1], z = dim == 3 ? p[2] : 0.0;
    const double PI = 3.14159265358979323846;
    switch (gid) {
    case 0: return sin(PI * x) * sinh(PI * y) / sinh(PI);
    case 1: return x * x - y * y;
    case 2: return x * x + y * y - 2.0 * z * z;
    case 3: return c[0] + c[1] * x + c[2] * y + c[3] * z;
    case 4: {
        /* Re/Im of (x+iy)^k, k=0..4, written out as real polynomials */
        const double re[5] = {1.0, x, x * x - y * y, x * x * x - 3.0 * x * y * y,
                              x * x * x * x - 6.0 * x * x * y * y + y * y * y * y};
        const double im[5] = {0.0, y, 2.0 * x * y, 3.0 * x * x * y - y * y * y,
                              4.0 * x * x * x * y - 4.0 * x * y * y * y};
        double t = 0.0;
        for (int k = 0; k < 5; ++k) t += c[2 * k] * re[k] + c[2 * k + 1] * im[k];
        return t;
    }
    default: return NAN;
    }
}

int orc_eval_g(const orc_sys *s, int gid, const double *coef, int k, int which, double *out) {
    if (gid < 0 || gid > 4 || k < 1) return 1;
    const int nc = ncoef(gid);
    const int64_t rows = which == 0 ? s->nbnd : s->nfree;
    for (int64_t r = 0; r < rows; ++r) {
        const int32_t i = which == 0 ? s->full_of_bnd[r] : s->full_of_free[r];
        for (int c = 0; c < k; ++c)
            out[r * k + c] = gfun(gid, coef ? coef + (int64_t)c * nc : NULL, s->dx + (int64_t)i * s->dim, s->dim);
    }
    return 0;
}

void orc_lift(const orc_sys *s, const double *gB, int k, double *b) {
    for (int64_t f = 0; f < s->nfree; ++f)
        for (int c = 0; c < k; ++c) {
            double t = 0.0;
            for (int64_t q = s->rp_ib[f]; q < s->rp_ib[f + 1]; ++q)
                t += s->v_ib[q] * gB[(int64_t)s->ci_ib[q] * k + c];
            b[f * k + c] = -t;
        }
}

/* -------------------------------------------------------------- solvers -- */
void orc_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
              const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double t = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) t += v[k] * x[ci[k]];
        y[i] = t;
    }
}

static double dot(int64_t n, const double *a, const double *b) {
    double t = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : t)
    for (int64_t i = 0; i < n; ++i) t += a[i] * b[i];
    return t;
}

/* z = M^{-1} r for one preconditioner M (its data in ctx). */
typedef void (*precond_fn)(int64_t n, const void *ctx, const double *r, double *z);

/* Jacobi: M = diag(A), ctx = 1/A_ii */
static void jacobi_apply(int64_t n, const void *ctx, const double *r, double *z) {
    const double *dinv = (const double *)ctx;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
}

/* Preconditioned CG (Hestenes-Stiefel):
 *   r = b - A x, z = M^{-1} r, p = z, rho = r.z
 *   repeat: q = A p; alpha = rho / p.q; x += alpha p; r -= alpha q;
 *           stop if ||r|| / ||b|| <= tol (Eq. 2);
 *           z = M^{-1} r; rho' = r.z; beta = rho'/rho; p = z + beta p.
 * At a stop on the recursive residual the true residual b - A x is formed;
 * if it is above tol, r is replaced by it and the recurrence restarts. */
static int pcg_core(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                    precond_fn apply, const void *ctx, const double *b, double *x, double tol,
                    int64_t maxit, int64_t *iters, double *relres) {
    *iters = 0;
    const double bn = sqrt(dot(n, b, b));
    if (bn == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        *relres = 0.0;
        return 0;
    }
    double *r = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    int status = 1;
    int64_t it = 0;
    int restarts = 0;
    orc_spmv(n, rp, ci, v, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double rel = sqrt(dot(n, r, r)) / bn;
    while (status == 1) {
        if (rel <= tol) { status = 0; break; }
        apply(n, ctx, r, z);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = z[i];
        double rho = dot(n, r, z);
        int restart = 0;
        while (it < maxit) {
            orc_spmv(n, rp, ci, v, p, q);
            const double pq = dot(n, p, q);
            if (!(pq > 0.0) || !isfinite(pq)) { status = 2; break; }
            const double alpha = rho / pq;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            ++it;
            rel = sqrt(dot(n, r, r)) / bn;
            if (rel <= tol) {
                orc_spmv(n, rp, ci, v, x, q);
#pragma omp parallel for schedule(static)
                for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
                const double tr = sqrt(dot(n, q, q)) / bn;
                if (tr <= tol) { rel = tr; status = 0; break; }
                for (int64_t i = 0; i < n; ++i) r[i] = q[i];
                rel = tr;
                restart = 1;
                break;
            }
            apply(n, ctx, r, z);
            const double rho1 = dot(n, r, z);
            const double beta = rho1 / rho;
            rho = rho1;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        if (status != 1) break;
        if (!restart || it >= maxit || ++restarts > 50) break;
    }
    *iters = it;
    *relres = rel;
    free(r); free(z); free(p); free(q);
    return status;
}

int orc_pcg(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
            const double *b, double *x, double tol, int64_t maxit,
            int64_t *iters, double *relres) {
    double *dinv = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) if (ci[k] == i) d = v[k];
        dinv[i] = 1.0 / d;
    }
    const int st = pcg_core(n, rp, ci, v, jacobi_apply, dinv, b, x, tol, maxit, iters, relres);
    free(dinv);
    return st;
}

/* Dense A = L L^T of an m x m row-major SPD matrix, the lower triangle
 * overwritten (textbook column-by-column form).  Returns 1 if not SPD. */
static int dense_cholesky(int64_t m, double *L) {
    for (int64_t j = 0; j < m; ++j) {
        double d = L[j * m + j];
        for (int64_t k = 0; k < j; ++k) d -= L[j * m + k] * L[j * m + k];
        if (!(d > 0.0)) return 1;
        d = sqrt(d);
        L[j * m + j] = d;
        for (int64_t i = j + 1; i < m; ++i) {
            double t = L[i * m + j];
            for (int64_t k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
            L[i * m + j] = t / d;
        }
    }
    return 0;
}

/* L y = b, then L^T x = y */
static void dense_cholesky_solve(int64_t m, const double *L, const double *b, double *x) {
    for (int64_t i = 0; i < m; ++i) {
        double t = b[i];
        for (int64_t k = 0; k < i; ++k) t -= L[i * m + k] * x[k];
        x[i] = t / L[i * m + i];
    }
    for (int64_t i = m - 1; i >= 0; --i) {
        double t = x[i];
        for (int64_t k = i + 1; k < m; ++k) t -= L[k * m + i] * x[k];
        x[i] = t / L[i * m + i];
    }
}

int orc_cholesky_solve(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                       const double *b, double *x) {
    double *L = (double *)calloc((size_t)(n * n), sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) L[i * n + ci[k]] = v[k];
    if (dense_cholesky(n, L)) { free(L); return 1; }
    dense_cholesky_solve(n, L, b, x);
    free(L);
    return 0;
}

/* ------------------------------------------------------- Block-Jacobi -- */
/* The block-Jacobi preconditioner named among the paper's preconditioners
 * (Sec. 3.2, with BiCGSTAB; Sec. 4.2 and its accuracy-vs-epsilon figure):
 * M = blockdiag(A_11, ..., A_mm),
 * A_jj the diagonal block of the rows [j bs, min(n, (j+1) bs)) -- bs
 * consecutive unknowns, the last block possibly shorter.  W holds each
 * block's inverse, dense row-major, nblk x bs x bs; a short last block fills
 * its leading m x m corner and leaves the rest 0.  Column c of A_jj^{-1} is
 * the Cholesky solution of A_jj w = e_c.  Returns 0, or 1 if a block is not
 * SPD. */
int orc_bjacobi(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int bs,
                double *W) {
    if (bs < 1) return 1;
    const int64_t nblk = (n + bs - 1) / bs;
    double *L = (double *)malloc(sizeof(double) * bs * bs);
    double *e = (double *)malloc(sizeof(double) * bs);
    double *w = (double *)malloc(sizeof(double) * bs);
    int rc = 0;
    for (int64_t j = 0; j < nblk && !rc; ++j) {
        const int64_t s = j * bs;
        const int64_t m = (n - s < bs) ? n - s : bs;
        for (int64_t a = 0; a < m * m; ++a) L[a] = 0.0;
        for (int64_t a = 0; a < m; ++a)
            for (int64_t k = rp[s + a]; k < rp[s + a + 1]; ++k)
                if (ci[k] >= s && ci[k] < s + m) L[a * m + (ci[k] - s)] = v[k];
        double *Wj = W + j * bs * bs;
        for (int64_t a = 0; a < (int64_t)bs * bs; ++a) Wj[a] = 0.0;
        if (dense_cholesky(m, L)) { rc = 1; break; }
        for (int64_t c = 0; c < m; ++c) {
            for (int64_t a = 0; a < m; ++a) e[a] = (a == c) ? 1.0 : 0.0;
            dense_cholesky_solve(m, L, e, w);
            for (int64_t a = 0; a < m; ++a) Wj[a * bs + c] = w[a];
        }
    }
    free(L); free(e); free(w);
    return rc;
}

/* z = M^{-1} r: z_B = W_j r_B for every block */
void orc_bjacobi_apply(int64_t n, int bs, const double *W, const double *r, double *z) {
    const int64_t nblk = (n + bs - 1) / bs;
    for (int64_t j = 0; j < nblk; ++j) {
        const int64_t s = j * bs;
        const int64_t m = (n - s < bs) ? n - s : bs;
        const double *Wj = W + j * bs * bs;
        for (int64_t a = 0; a < m; ++a) {
            double t = 0.0;
            for (int64_t c = 0; c < m; ++c) t += Wj[a * bs + c] * r[s + c];
            z[s + a] = t;
        }
    }
}

struct bj_ctx { int bs; const double *W; };
static void bjacobi_apply_cb(int64_t n, const void *ctx, const double *r, double *z) {
    const struct bj_ctx *c = (const struct bj_ctx *)ctx;
    orc_bjacobi_apply(n, c->bs, c->W, r, z);
}

int orc_pcg_bj(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int bs,
               const double *b, double *x, double tol, int64_t maxit, int64_t *iters,
               double *relres) {
    *iters = 0;
    *relres = 0.0;
    if (bs < 1) return 2;
    const int64_t nblk = (n + bs - 1) / bs;
    double *W = (double *)malloc(sizeof(double) * (nblk > 0 ? nblk : 1) * bs * bs);
    if (orc_bjacobi(n, rp, ci, v, bs, W)) { free(W); return 2; }
    struct bj_ctx c = {bs, W};
    const int st = pcg_core(n, rp, ci, v, bjacobi_apply_cb, &c, b, x, tol, maxit, iters, relres);
    free(W);
    return st;
}

/* ------------------------------------------------------------ BiCGSTAB -- */
/* BiCGSTAB (van der Vorst 1992), the Krylov method the paper runs (Sec. 3.2),
 * with the preconditioner applied on the right (x = M^{-1} y):
 *   r = b - A x, rh = r (shadow residual), rho0 = alpha = omega = 1, p = v = 0
 *   repeat: rho = rh.r; beta = (rho/rho0)(alpha/omega);
 *           p = r + beta (p - omega v); ph = M^{-1} p; v = A ph;
 *           alpha = rho / rh.v; s = r - alpha v;
 *           if ||s|| <= tol ||b||: x += alpha ph, stop;
 *           sh = M^{-1} s; t = A sh; omega = t.s / t.t;
 *           x += alpha ph + omega sh; r = s - omega t;
 *           stop if ||r|| <= tol ||b|| (Eq. 2); rho0 = rho.
 * A stop is confirmed on the true residual; above tol the recurrence restarts
 * from it (new shadow residual).  Breakdown (rh.v, t.t, rho or omega zero or
 * not finite) also restarts from the true residual, as long as that residual
 * is below 0.9 times the one the previous restart started from. */
static int bicgstab_core(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                         precond_fn apply, const void *ctx, const double *b, double *x, double tol,
                         int64_t maxit, int64_t *iters, double *relres) {
    *iters = 0;
    const double bn = sqrt(dot(n, b, b));
    if (bn == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        *relres = 0.0;
        return 0;
    }
    const size_t sz = sizeof(double) * (n > 0 ? n : 1);
    double *r = (double *)malloc(sz), *rh = (double *)malloc(sz), *p = (double *)malloc(sz);
    double *vv = (double *)malloc(sz), *ph = (double *)malloc(sz), *sv = (double *)malloc(sz);
    double *sh = (double *)malloc(sz), *t = (double *)malloc(sz);
    int status = 1, restarts = 0, broke = 0;
    int64_t it = 0;
    double rel = 0.0, rel_start = INFINITY;
    for (;;) {
        orc_spmv(n, rp, ci, v, x, t);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
        rel = sqrt(dot(n, r, r)) / bn;
        if (rel <= tol) { status = 0; break; }
        if (it >= maxit || restarts > 50) break;
        if (broke && !(rel < 0.9 * rel_start)) { status = 2; break; }
        broke = 0;
        rel_start = rel;
        if (it > 0) ++restarts;
        for (int64_t i = 0; i < n; ++i) { rh[i] = r[i]; p[i] = 0.0; vv[i] = 0.0; }
        double rho0 = 1.0, alpha = 1.0, omega = 1.0;
        int stop = 0;
        while (it < maxit) {
            const double rho = dot(n, rh, r);
            if (rho == 0.0 || !isfinite(rho)) { broke = 1; break; }
            const double beta = (rho / rho0) * (alpha / omega);
            for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * vv[i]);
            apply(n, ctx, p, ph);
            orc_spmv(n, rp, ci, v, ph, vv);
            const double rv = dot(n, rh, vv);
            if (rv == 0.0 || !isfinite(rv)) { broke = 1; break; }
            alpha = rho / rv;
            for (int64_t i = 0; i < n; ++i) sv[i] = r[i] - alpha * vv[i];
            ++it;
            if (sqrt(dot(n, sv, sv)) / bn <= tol) {
                for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i];
                stop = 1;
                break;
            }
            apply(n, ctx, sv, sh);
            orc_spmv(n, rp, ci, v, sh, t);
            const double tt = dot(n, t, t);
            if (tt == 0.0 || !isfinite(tt)) { broke = 1; break; }
            omega = dot(n, t, sv) / tt;
            for (int64_t i = 0; i < n; ++i) {
                x[i] += alpha * ph[i] + omega * sh[i];
                r[i] = sv[i] - omega * t[i];
            }
            if (sqrt(dot(n, r, r)) / bn <= tol) { stop = 1; break; }
            if (omega == 0.0 || !isfinite(omega)) { broke = 1; break; }
            rho0 = rho;
        }
        if (!stop && !broke) break; /* maxit */
    }
    if (status != 0) { /* report the true residual of the x returned */
        orc_spmv(n, rp, ci, v, x, t);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
        rel = sqrt(dot(n, r, r)) / bn;
    }
    *iters = it;
    *relres = rel;
    free(r); free(rh); free(p); free(vv); free(ph); free(sv); free(sh); free(t);
    return status;
}

int orc_bicgstab(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int bs,
                 const double *b, double *x, double tol, int64_t maxit, int64_t *iters,
                 double *relres) {
    *iters = 0;
    *relres = 0.0;
    if (bs <= 1) { /* Jacobi (bs 0 or 1: the same M) */
        double *dinv = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) {
            double d = 0.0;
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) if (ci[k] == i) d = v[k];
            dinv[i] = 1.0 / d;
        }
        const int st = bicgstab_core(n, rp, ci, v, jacobi_apply, dinv, b, x, tol, maxit, iters, relres);
        free(dinv);
        return st;
    }
    const int64_t nblk = (n + bs - 1) / bs;
    double *W = (double *)malloc(sizeof(double) * (nblk > 0 ? nblk : 1) * bs * bs);
    if (orc_bjacobi(n, rp, ci, v, bs, W)) { free(W); return 2; }
    struct bj_ctx c = {bs, W};
    const int st = bicgstab_core(n, rp, ci, v, bjacobi_apply_cb, &c, b, x, tol, maxit, iters, relres);
    free(W);
    return st;
}

/* ------------------------------------------------------------ block CG -- */
/* The multi-RHS system A X = B of Sec. 4.3 (B: the block of right-hand sides,
 * n x k, row-major here) solved by block conjugate gradients: one Krylov
 * space shared by all columns (O'Leary 1980), in the breakdown-free form of
 * Ji and Li (2017) -- the search block P is orthonormalised with a rank test
 * each step, so dependent directions (rank-deficient B, columns that converge
 * at different rates) are dropped instead of making P^T A P singular.
 * Preconditioner: Jacobi, M = diag(A).  Per step:
 *   Q = A P;  alpha = (P^T Q)^{-1} P^T R;  X += P alpha;  R -= Q alpha;
 *   stop when every column has ||R_j|| <= tol ||B_j|| (Eq. 2 per column);
 *   Z = M^{-1} R;  beta = -(P^T Q)^{-1} Q^T Z;  W = Z + P beta;  P = orth(W).
 * orth: the columns of W are first scaled by 1/||R_j|| (columns already below
 * tol are left out), so that the rank test sees directions, not residual
 * sizes; then with W^T W = V diag(lambda) V^T (cyclic Jacobi), the directions
 * with lambda_i > 1e-12 lambda_max are kept: P = W V_s diag(lambda_s)^{-1/2}.
 * At a stop on the recursive residuals the true residual B - A X is formed;
 * columns above tol restart the recurrence from it. */

/* eigen-decomposition of a symmetric m x m matrix (row-major, destroyed) by
 * cyclic Jacobi rotations: A = V diag(w) V^T, V's columns the eigenvectors */
static void sym_eig(int m, double *A, double *w, double *V) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) V[i * m + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                tot += A[i * m + j] * A[i * m + j];
                if (i != j) off += A[i * m + j] * A[i * m + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[p * m + q];
                if (apq == 0.0) continue;
                /* rotation angle zeroing A_pq: tan(2 t) = 2 A_pq / (A_qq - A_pp) */
                const double theta = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int r = 0; r < m; ++r) { /* A <- A J (columns p, q) */
                    const double arp = A[r * m + p], arq = A[r * m + q];
                    A[r * m + p] = c * arp - sn * arq;
                    A[r * m + q] = sn * arp + c * arq;
                }
                for (int r = 0; r < m; ++r) { /* A <- J^T A (rows p, q) */
                    const double apr = A[p * m + r], aqr = A[q * m + r];
                    A[p * m + r] = c * apr - sn * aqr;
                    A[q * m + r] = sn * apr + c * aqr;
                }
                for (int r = 0; r < m; ++r) { /* V <- V J */
                    const double vrp = V[r * m + p], vrq = V[r * m + q];
                    V[r * m + p] = c * vrp - sn * vrq;
                    V[r * m + q] = sn * vrp + c * vrq;
                }
            }
    }
    for (int i = 0; i < m; ++i) w[i] = A[i * m + i];
}

/* C (a x c) = U^T V for row-major U (n x a), V (n x c) */
static void gram(int64_t n, int a, int c, const double *U, int su, const double *V, int sv, double *C) {
    for (int i = 0; i < a * c; ++i) C[i] = 0.0;
    for (int64_t r = 0; r < n; ++r)
        for (int i = 0; i < a; ++i)
            for (int j = 0; j < c; ++j) C[i * c + j] += U[r * su + i] * V[r * sv + j];
}

/* Y (n x k) = A X column by column */
static void block_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int k,
                       const double *X, double *Y) {
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j) {
            double t = 0.0;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) t += v[e] * X[(int64_t)ci[e] * k + j];
            Y[i * k + j] = t;
        }
}

/* P (n x s, leading columns of n x k) = orth(W) with column weights cw (0 =
 * column left out); returns s */
static int orth_block(int64_t n, int k, const double *W, const double *cw, double *P) {
    double *G = (double *)malloc(sizeof(double) * k * k);
    double *V = (double *)malloc(sizeof(double) * k * k);
    double *w = (double *)malloc(sizeof(double) * k);
    double *T = (double *)malloc(sizeof(double) * k * k);
    int *ord = (int *)malloc(sizeof(int) * k);
    gram(n, k, k, W, k, W, k, G);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) G[i * k + j] *= cw[i] * cw[j];
    sym_eig(k, G, w, V);
    for (int i = 0; i < k; ++i) ord[i] = i;
    for (int i = 1; i < k; ++i) { /* descending eigenvalues, stable */
        int t = ord[i], j = i;
        while (j > 0 && w[ord[j - 1]] < w[t]) { ord[j] = ord[j - 1]; --j; }
        ord[j] = t;
    }
    const double lmax = k > 0 ? w[ord[0]] : 0.0;
    int s = 0;
    if (lmax > 0.0)
        while (s < k && w[ord[s]] > 1e-12 * lmax) ++s;
    /* T (k x s): column j = cw .* V[:, ord[j]] / sqrt(lambda) */
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < s; ++j) T[i * s + j] = cw[i] * V[i * k + ord[j]] / sqrt(w[ord[j]]);
    for (int64_t r = 0; r < n; ++r)
        for (int j = 0; j < k; ++j) {
            double t = 0.0;
            if (j < s)
                for (int i = 0; i < k; ++i) t += W[r * k + i] * T[i * s + j];
            P[r * k + j] = t;
        }
    free(G); free(V); free(w); free(T); free(ord);
    return s;
}

/* in-place Cholesky of an s x s SPD matrix (leading block, row stride ld) and
 * solve for nrhs columns of Y (s x nrhs, row stride ldy) */
static int chol_solve_small(int s, double *L, int ld, double *Y, int ldy, int nrhs) {
    for (int j = 0; j < s; ++j) {
        double d = L[j * ld + j];
        for (int q = 0; q < j; ++q) d -= L[j * ld + q] * L[j * ld + q];
        if (!(d > 0.0)) return 1;
        d = sqrt(d);
        L[j * ld + j] = d;
        for (int i = j + 1; i < s; ++i) {
            double t = L[i * ld + j];
            for (int q = 0; q < j; ++q) t -= L[i * ld + q] * L[j * ld + q];
            L[i * ld + j] = t / d;
        }
    }
    for (int c = 0; c < nrhs; ++c) {
        for (int i = 0; i < s; ++i) {
            double t = Y[i * ldy + c];
            for (int q = 0; q < i; ++q) t -= L[i * ld + q] * Y[q * ldy + c];
            Y[i * ldy + c] = t / L[i * ld + i];
        }
        for (int i = s - 1; i >= 0; --i) {
            double t = Y[i * ldy + c];
            for (int q = i + 1; q < s; ++q) t -= L[q * ld + i] * Y[q * ldy + c];
            Y[i * ldy + c] = t / L[i * ld + i];
        }
    }
    return 0;
}

int orc_block_cg(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int k,
                 const double *B, double *X, double tol, int64_t maxit, int64_t *iters,
                 double *relres) {
    *iters = 0;
    if (k < 1) return 2;
    const size_t nk = (size_t)(n > 0 ? n : 1) * k;
    double *dinv = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *R = (double *)malloc(sizeof(double) * nk), *Z = (double *)malloc(sizeof(double) * nk);
    double *W = (double *)malloc(sizeof(double) * nk), *P = (double *)malloc(sizeof(double) * nk);
    double *Q = (double *)malloc(sizeof(double) * nk);
    double *bn = (double *)malloc(sizeof(double) * k), *rn = (double *)malloc(sizeof(double) * k);
    double *cw = (double *)malloc(sizeof(double) * k);
    double *PtQ = (double *)malloc(sizeof(double) * k * k), *L = (double *)malloc(sizeof(double) * k * k);
    double *al = (double *)malloc(sizeof(double) * k * k);
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) if (ci[e] == i) d = v[e];
        dinv[i] = 1.0 / d;
    }
    for (int j = 0; j < k; ++j) {
        double t = 0.0;
        for (int64_t i = 0; i < n; ++i) t += B[i * k + j] * B[i * k + j];
        bn[j] = sqrt(t);
    }
    int status = 1, restarts = 0;
    int64_t it = 0;
#define COLREL(j) (bn[j] > 0.0 ? rn[j] / bn[j] : rn[j])
    for (;;) {
        /* true residual R = B - A X, column norms */
        block_spmv(n, rp, ci, v, k, X, Q);
        for (size_t e = 0; e < (size_t)n * k; ++e) R[e] = B[e] - Q[e];
        double worst = 0.0;
        for (int j = 0; j < k; ++j) {
            double t = 0.0;
            for (int64_t i = 0; i < n; ++i) t += R[i * k + j] * R[i * k + j];
            rn[j] = sqrt(t);
            if (COLREL(j) > worst) worst = COLREL(j);
        }
        if (worst <= tol) { status = 0; break; }
        if (it >= maxit || restarts > 50) break;
        if (it > 0) ++restarts;
        /* Z = M^-1 R, P = orth(Z) */
        for (int64_t i = 0; i < n; ++i)
            for (int j = 0; j < k; ++j) Z[i * k + j] = dinv[i] * R[i * k + j];
        for (int j = 0; j < k; ++j) cw[j] = COLREL(j) > tol ? 1.0 / rn[j] : 0.0;
        int s = orth_block(n, k, Z, cw, P);
        int restart = 0;
        while (it < maxit && !restart) {
            if (s == 0) { status = 2; break; }
            block_spmv(n, rp, ci, v, k, P, Q); /* columns >= s of P are 0 */
            gram(n, s, s, P, k, Q, k, PtQ);
            gram(n, s, k, P, k, R, k, al);
            for (int e = 0; e < s * s; ++e) L[e] = PtQ[e];
            if (chol_solve_small(s, L, s, al, k, k)) { status = 2; break; }
            for (int64_t i = 0; i < n; ++i)
                for (int j = 0; j < k; ++j) {
                    double dx = 0.0, dr = 0.0;
                    for (int q = 0; q < s; ++q) {
                        dx += P[i * k + q] * al[q * k + j];
                        dr += Q[i * k + q] * al[q * k + j];
                    }
                    X[i * k + j] += dx;
                    R[i * k + j] -= dr;
                }
            ++it;
            double worst2 = 0.0;
            for (int j = 0; j < k; ++j) {
                double t = 0.0;
                for (int64_t i = 0; i < n; ++i) t += R[i * k + j] * R[i * k + j];
                rn[j] = sqrt(t);
                if (COLREL(j) > worst2) worst2 = COLREL(j);
            }
            if (worst2 <= tol) { restart = 1; break; } /* confirm on the true residual */
            for (int64_t i = 0; i < n; ++i)
                for (int j = 0; j < k; ++j) Z[i * k + j] = dinv[i] * R[i * k + j];
            /* beta = -(P^T Q)^-1 Q^T Z (the factor of P^T Q is still in L) */
            gram(n, s, k, Q, k, Z, k, al);
            for (int e = 0; e < s * k; ++e) al[e] = -al[e];
            for (int c = 0; c < k; ++c) { /* reuse the factor: two triangular solves */
                for (int i = 0; i < s; ++i) {
                    double t = al[i * k + c];
                    for (int q = 0; q < i; ++q) t -= L[i * s + q] * al[q * k + c];
                    al[i * k + c] = t / L[i * s + i];
                }
                for (int i = s - 1; i >= 0; --i) {
                    double t = al[i * k + c];
                    for (int q = i + 1; q < s; ++q) t -= L[q * s + i] * al[q * k + c];
                    al[i * k + c] = t / L[i * s + i];
                }
            }
            for (int64_t i = 0; i < n; ++i)
                for (int j = 0; j < k; ++j) {
                    double t = Z[i * k + j];
                    for (int q = 0; q < s; ++q) t += P[i * k + q] * al[q * k + j];
                    W[i * k + j] = t;
                }
            for (int j = 0; j < k; ++j) cw[j] = COLREL(j) > tol ? 1.0 / rn[j] : 0.0;
            s = orth_block(n, k, W, cw, P);
        }
        if (status == 2) break;
        if (!restart) break; /* maxit */
    }
#undef COLREL
    for (int j = 0; j < k; ++j) relres[j] = bn[j] > 0.0 ? rn[j] / bn[j] : rn[j];
    *iters = it;
    free(dinv); free(R); free(Z); free(W); free(P); free(Q); free(bn); free(rn); free(cw);
    free(PtQ); free(L); free(al);
    return status;
}

/* ----------------------------------------------------------- SELL-C-sigma -- */
/* Rows are cut into windows of sigma consecutive rows; inside a window they are
 * ordered by descending row length, ties kept in original order (stable).  The
 * new order is cut into chunks of C rows; a chunk's width is its longest row. */
static void sell_perm(int64_t n, const int64_t *rp, int sigma, int32_t *perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    if (sigma <= 1) return;
    for (int64_t w0 = 0; w0 < n; w0 += sigma) {
        const int64_t w1 = w0 + sigma < n ? w0 + sigma : n;
        /* stable insertion sort of perm[w0..w1) by descending length */
        for (int64_t i = w0 + 1; i < w1; ++i) {
            const int32_t x = perm[i];
            const int64_t lx = rp[x + 1] - rp[x];
            int64_t j = i - 1;
            while (j >= w0 && (rp[perm[j] + 1] - rp[perm[j]]) < lx) { perm[j + 1] = perm[j]; --j; }
            perm[j + 1] = x;
        }
    }
}

void orc_sell_size(int64_t n, const int64_t *rp, int C, int sigma, int64_t *nchunks, int64_t *padded) {
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (n ? n : 1));
    sell_perm(n, rp, sigma, perm);
    const int64_t nc = (n + C - 1) / C;
    int64_t tot = 0;
    for (int64_t c = 0; c < nc; ++c) {
        int64_t w = 0;
        for (int64_t r = c * C; r < (c + 1) * C && r < n; ++r) {
            const int64_t l = rp[perm[r] + 1] - rp[perm[r]];
            if (l > w) w = l;
        }
        tot += w * C;
    }
    *nchunks = nc;
    *padded = tot;
    free(perm);
}

void orc_sell_fill(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                   int C, int sigma, int32_t *perm, int64_t *chunk_ptr,
                   int32_t *chunk_w, int32_t *row_len, int32_t *col, double *val) {
    sell_perm(n, rp, sigma, perm);
    int32_t *iperm = (int32_t *)malloc(sizeof(int32_t) * (n ? n : 1));
    for (int64_t r = 0; r < n; ++r) iperm[perm[r]] = (int32_t)r;
    const int64_t nc = (n + C - 1) / C;
    chunk_ptr[0] = 0;
    for (int64_t c = 0; c < nc; ++c) {
        int64_t w = 0;
        for (int64_t r = c * C; r < (c + 1) * C && r < n; ++r) {
            const int64_t l = rp[perm[r] + 1] - rp[perm[r]];
            if (l > w) w = l;
        }
        chunk_w[c] = (int32_t)w;
        chunk_ptr[c + 1] = chunk_ptr[c] + w * C;
        for (int64_t j = 0; j < w; ++j)
            for (int64_t t = 0; t < C; ++t) {
                const int64_t r = c * C + t;
                const int64_t slot = chunk_ptr[c] + j * C + t;
                if (r < n) {
                    const int32_t o = perm[r];
                    const int64_t l = rp[o + 1] - rp[o];
                    if (j < l) { col[slot] = iperm[ci[rp[o] + j]]; if (val) val[slot] = v[rp[o] + j]; }
                    else { col[slot] = (int32_t)r; if (val) val[slot] = 0.0; }
                } else {
                    col[slot] = 0;
                    if (val) val[slot] = 0.0;
                }
            }
    }
    for (int64_t r = 0; r < n; ++r) row_len[r] = (int32_t)(rp[perm[r] + 1] - rp[perm[r]]);
    free(iperm);
}
