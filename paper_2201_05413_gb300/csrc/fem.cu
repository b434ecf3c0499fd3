// fem.cu -- device mesh, dof numbering, stiffness assembly, Dirichlet data
// and lift (paper Sec. 2.2; P2-P4 as in the degree study of Sec. 4.2).
//
// The mesh is implicit: a vertex's coordinates and a cell's diagonal are pure
// functions of the lattice index and the counter-based generator, so nothing
// geometric is stored.  Assembly is a row gather: one thread owns one free dof,
// visits the elements of the (at most 2^dim) cells around it in increasing
// cell order, and accumulates its stiffness row into a dense stencil of
// (2*degree+1)^dim slots.  A count pass sizes the rows, a scan makes the row
// pointers and a fill pass writes columns (ascending) and values.  Element
// entries are evaluated for the ordered local pair (min, max), so K_ij and
// K_ji are the same sum of the same terms in the same order: K_II is
// bit-exactly symmetric and the assembly is deterministic without atomics.
#include <vector>

#include "common.cuh"

namespace gb {

// ------------------------------------------------------------------ RNG --
// SplitMix64 (Steele, Lea, Flood 2014) in counter form: output i of the
// sequential generator seeded with `key` is mix64(key + (i+1) * gamma).
__device__ __forceinline__ uint64_t sm_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sm_draw(uint64_t key, uint64_t i) {
    return sm_mix64(key + (i + 1) * 0x9E3779B97F4A7C15ULL);
}
static inline uint64_t stream_key(uint64_t seed, uint32_t stream) {
    return (seed << 40) ^ ((uint64_t)stream << 32);
}

struct MeshDev {
    int dim, deg, cells, S, V, jitter, diag_mode;
    uint64_t kx, ky, kz, kf;
    double q;  // jitter amplitude: h/4 in 2D, h/8 in 3D
    const double *ref;  // degree >= 3: reference gradient integrals [lo][hi][a][b] per unit volume
};

// 2D triangles of a cell as vertex offsets (dx, dy): [flip][tri][vertex].
// Unflipped: diagonal (0,0)-(1,1); flipped: diagonal (1,0)-(0,1).
__constant__ int8_t c_tri[2][2][3][2] = {
    {{{0, 0}, {1, 0}, {1, 1}}, {{0, 0}, {1, 1}, {0, 1}}},
    {{{0, 0}, {1, 0}, {0, 1}}, {{1, 0}, {1, 1}, {0, 1}}}};
// Kuhn: tetrahedron t walks from (0,0,0) along the axes in order c_kuhn[t].
__constant__ int8_t c_kuhn[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
// local edges (a,b), a<b, in lexicographic order
__constant__ int8_t c_edge2[3][2] = {{0, 1}, {0, 2}, {1, 2}};
__constant__ int8_t c_edge3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

__device__ __forceinline__ bool cell_flipped(const MeshDev &m, int64_t cell) {
    return m.diag_mode == 1 && (sm_draw(m.kf, (uint64_t)cell) >> 63) == 0;
}

// Coordinate of vertex v = (i,j[,k]) along `axis`: i/cells, moved by (2u-1)q
// on interior vertices of a jittered mesh (q = h/4 in 2D; h/8 in 3D, where a
// Kuhn tetrahedron could invert at h/4), u from stream 0, 1 or 3 for x, y, z.
// Correctly rounded basic operations with no contraction, so the value is
// reproducible exactly.
__device__ __forceinline__ double vertex_coord(const MeshDev &m, const int *vi, int axis) {
    double x = __ddiv_rn((double)vi[axis], (double)m.cells);
    if (m.jitter) {
        bool interior = true;
        for (int d = 0; d < m.dim; ++d) interior &= (vi[d] > 0 && vi[d] < m.cells);
        if (interior) {
            int64_t vid = vi[0] + (int64_t)m.V * (vi[1] + (m.dim == 3 ? (int64_t)m.V * vi[2] : 0));
            uint64_t r = sm_draw(axis == 0 ? m.kx : (axis == 1 ? m.ky : m.kz), (uint64_t)vid);
            double u = __dmul_rn((double)(r >> 11), 0x1p-53);
            double d = __dsub_rn(__dmul_rn(2.0, u), 1.0);
            x = __dadd_rn(x, __dmul_rn(d, m.q));
        }
    }
    return x;
}

// ------------------------------------------------------- dof numbering --
__device__ __forceinline__ bool on_boundary(const int *N, int dim, int S) {
    bool b = false;
    for (int d = 0; d < dim; ++d) b |= (N[d] == 0 || N[d] == S - 1);
    return b;
}
__device__ __forceinline__ int64_t full_id(const int *N, int dim, int S) {
    return dim == 2 ? N[0] + (int64_t)S * N[1] : N[0] + (int64_t)S * (N[1] + (int64_t)S * N[2]);
}
__device__ __forceinline__ int64_t free_id(const int *N, int dim, int S) {
    const int64_t m = S - 2;
    return dim == 2 ? (N[0] - 1) + m * (N[1] - 1) : (N[0] - 1) + m * ((N[1] - 1) + m * (N[2] - 1));
}
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
// number of interior points whose full id is below that of N
__device__ __forceinline__ int64_t free_before(const int *N, int dim, int S) {
    const int64_t m = S - 2;
    const int top = dim - 1;
    int64_t cnt = 0, plane = 1;
    for (int d = 0; d < top; ++d) plane *= m;
    // walk from the slowest axis: full slabs below, then recurse into the slab
    for (int d = top; d >= 0; --d) {
        cnt += (int64_t)clampi(N[d] - 1, 0, (int)m) * plane;
        if (N[d] < 1 || N[d] > S - 2) break;
        if (d > 0) plane /= m;
    }
    return cnt;
}
__device__ __forceinline__ int64_t bnd_id(const int *N, int dim, int S) {
    return full_id(N, dim, S) - free_before(N, dim, S);
}
__device__ __forceinline__ void free_to_lattice(int64_t f, int dim, int S, int *N) {
    const int64_t m = S - 2;
    for (int d = 0; d < dim; ++d) { N[d] = (int)(f % m) + 1; f /= m; }
}

// --------------------------------------------------------- element data --
template <int DIM>
struct Elem {
    int v[DIM + 1][DIM];  // vertex lattice indices
};

template <int DIM>
__device__ __forceinline__ void cell_element(const MeshDev &m, const int *cell, int t, Elem<DIM> &e) {
    if (DIM == 2) {
        const int64_t cid = cell[0] + (int64_t)m.cells * cell[1];
        const int fl = cell_flipped(m, cid) ? 1 : 0;
        for (int a = 0; a < 3; ++a) {
            e.v[a][0] = cell[0] + c_tri[fl][t][a][0];
            e.v[a][1] = cell[1] + c_tri[fl][t][a][1];
        }
    } else {
        int p[3] = {cell[0], cell[1], cell[2]};
        for (int d = 0; d < DIM; ++d) e.v[0][d] = p[d];
        for (int s = 0; s < 3; ++s) {
            p[c_kuhn[t][s]] += 1;
            for (int d = 0; d < DIM; ++d) e.v[s + 1][d] = p[d];
        }
    }
}

// Degree >= 3: local dof l is the Lagrange node with barycentric multi-index
// beta (|beta| = DEG), taken in the order beta_0 = DEG, DEG-1, ..., 0 (outer),
// then beta_1 likewise, ... (beta_DIM = the rest).
template <int DIM, int DEG>
__host__ __device__ __forceinline__ void node_beta(int l, int *beta) {
    int k = 0;
    for (int b0 = DEG; b0 >= 0; --b0) {
        if (DIM == 2) {
            for (int b1 = DEG - b0; b1 >= 0; --b1, ++k)
                if (k == l) { beta[0] = b0; beta[1] = b1; beta[2] = DEG - b0 - b1; return; }
        } else {
            for (int b1 = DEG - b0; b1 >= 0; --b1)
                for (int b2 = DEG - b0 - b1; b2 >= 0; --b2, ++k)
                    if (k == l) { beta[0] = b0; beta[1] = b1; beta[2] = b2; beta[3] = DEG - b0 - b1 - b2; return; }
        }
    }
}

// dof-lattice point of local dof `l` (P1/P2: vertices first, then edge
// midpoints; degree >= 3: the node sum_a beta_a v_a of the refined lattice)
template <int DIM, int DEG>
__device__ __forceinline__ void local_dof(const Elem<DIM> &e, int l, int *N) {
    if (DEG >= 3) {
        int beta[4] = {0, 0, 0, 0};
        node_beta<DIM, DEG>(l, beta);
        for (int d = 0; d < DIM; ++d) {
            int t = 0;
            for (int a = 0; a <= DIM; ++a) t += beta[a] * e.v[a][d];
            N[d] = t;
        }
        return;
    }
    if (l <= DIM) {
        for (int d = 0; d < DIM; ++d) N[d] = DEG * e.v[l][d];
    } else {
        const int k = l - DIM - 1;
        const int a = DIM == 2 ? c_edge2[k][0] : c_edge3[k][0];
        const int b = DIM == 2 ? c_edge2[k][1] : c_edge3[k][1];
        for (int d = 0; d < DIM; ++d) N[d] = e.v[a][d] + e.v[b][d];  // DEG == 2
    }
}

// Barycentric gradients g_a and |T|.  g_a is normal to the facet opposite
// vertex a, scaled so that g_a . (P_a - P_b) = 1 for a vertex b of that facet.
template <int DIM>
__device__ __forceinline__ double simplex_geometry(const MeshDev &m, const Elem<DIM> &e,
                                                   double G[DIM + 1][DIM + 1]) {
    double P[DIM + 1][DIM];
    for (int a = 0; a <= DIM; ++a)
        for (int d = 0; d < DIM; ++d) P[a][d] = vertex_coord(m, e.v[a], d);
    double g[DIM + 1][DIM];
    double vol;
    if (DIM == 2) {
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            const double ex = P[c][0] - P[b][0], ey = P[c][1] - P[b][1];
            const double nx = -ey, ny = ex;
            const double s = nx * (P[a][0] - P[b][0]) + ny * (P[a][1] - P[b][1]);
            g[a][0] = nx / s;
            g[a][1] = ny / s;
        }
        const double D = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]);
        vol = 0.5 * fabs(D);
    } else {
        vol = 0.0;
        for (int a = 0; a < 4; ++a) {
            const int b = (a + 1) & 3, c = (a + 2) & 3, dd = (a + 3) & 3;
            const double u[3] = {P[c][0] - P[b][0], P[c][1] - P[b][1], P[c][2] - P[b][2]};
            const double w[3] = {P[dd][0] - P[b][0], P[dd][1] - P[b][1], P[dd][2] - P[b][2]};
            const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
            const double s = n[0] * (P[a][0] - P[b][0]) + n[1] * (P[a][1] - P[b][1]) + n[2] * (P[a][2] - P[b][2]);
            for (int d = 0; d < 3; ++d) g[a][d] = n[d] / s;
            if (a == 0) vol = fabs(s) / 6.0;
        }
    }
    for (int a = 0; a <= DIM; ++a)
        for (int b = a; b <= DIM; ++b) {
            double t = 0.0;
            for (int d = 0; d < DIM; ++d) t += g[a][d] * g[b][d];
            G[a][b] = t;
            G[b][a] = t;
        }
    return vol;
}

// Stiffness entry K_{lo,hi} (lo <= hi) of one element.  P1: |T| g_a.g_b.
// P2 with phi_a = lambda_a(2 lambda_a - 1), phi_ab = 4 lambda_a lambda_b and
// int lambda_m lambda_n = |T| (1 + delta_mn) d!/(d+2)!, int lambda_m = |T|/(d+1):
//   vertex-vertex: |T| G_ab (16c(1+d_ab) - 8/(d+1) + 1)
//   vertex a - edge (b,e): 4|T| (mu_ab G_ae + mu_ae G_ab), mu_ab = 4c(1+d_ab) - 1/(d+1)
//   edge (a,b) - edge (c,e): 16c|T| ((1+d_ac) G_be + (1+d_ae) G_bc + (1+d_bc) G_ae + (1+d_be) G_ac)
// with c = d!/(d+2)! (1/12 in 2D, 1/20 in 3D).
template <int DIM, int DEG>
__device__ __forceinline__ double entry(int lo, int hi, double vol, const double G[DIM + 1][DIM + 1],
                                        const double *ref) {
    if (DEG == 1) return vol * G[lo][hi];
    if (DEG >= 3) {  // |T| sum_ab G_ab I[lo][hi][a][b], the table built on the host
        constexpr int NL = DIM == 2 ? (DEG + 1) * (DEG + 2) / 2 : (DEG + 1) * (DEG + 2) * (DEG + 3) / 6;
        const double *I = ref + ((size_t)lo * NL + hi) * (DIM + 1) * (DIM + 1);
        double t = 0.0;
        for (int a = 0; a <= DIM; ++a)
            for (int b = 0; b <= DIM; ++b) t += G[a][b] * __ldg(I + a * (DIM + 1) + b);
        return vol * t;
    }
    constexpr double c = DIM == 2 ? 1.0 / 12.0 : 1.0 / 20.0;
    constexpr double inv_d1 = 1.0 / (DIM + 1);
    if (hi <= DIM) {  // both vertices
        const double k = lo == hi ? 32.0 * c - 8.0 * inv_d1 + 1.0 : 16.0 * c - 8.0 * inv_d1 + 1.0;
        return vol * k * G[lo][hi];
    }
    const int kh = hi - DIM - 1;
    const int b = DIM == 2 ? c_edge2[kh][0] : c_edge3[kh][0];
    const int e = DIM == 2 ? c_edge2[kh][1] : c_edge3[kh][1];
    if (lo <= DIM) {  // vertex lo, edge (b,e)
        const int a = lo;
        const double mu_ab = 4.0 * c * (a == b ? 2.0 : 1.0) - inv_d1;
        const double mu_ae = 4.0 * c * (a == e ? 2.0 : 1.0) - inv_d1;
        return 4.0 * vol * (mu_ab * G[a][e] + mu_ae * G[a][b]);
    }
    const int kl = lo - DIM - 1;
    const int a = DIM == 2 ? c_edge2[kl][0] : c_edge3[kl][0];
    const int bb = DIM == 2 ? c_edge2[kl][1] : c_edge3[kl][1];
    // edge (a,bb) - edge (b,e)
    const double s = (a == b ? 2.0 : 1.0) * G[bb][e] + (a == e ? 2.0 : 1.0) * G[bb][b] +
                     (bb == b ? 2.0 : 1.0) * G[a][e] + (bb == e ? 2.0 : 1.0) * G[a][b];
    return 16.0 * c * vol * s;
}

// ------------------------------------------------------------ row gather --
template <int DIM, int DEG>
struct RowCfg {
    static constexpr int W = 2 * DEG + 1;
    static constexpr int NS = DIM == 2 ? W * W : W * W * W;
    static constexpr int NW = (NS + 31) / 32;
    static constexpr int NLOC = DEG == 1   ? DIM + 1
                                : DIM == 2 ? (DEG + 1) * (DEG + 2) / 2
                                           : (DEG + 1) * (DEG + 2) * (DEG + 3) / 6;
    static constexpr int NEL = DIM == 2 ? 2 : 6;
};

// Visits the elements around free dof f and accumulates its row.
// WANT_VAL=false: marks only (pattern).
template <int DIM, int DEG, bool WANT_VAL>
__device__ __forceinline__ void gather_row(const MeshDev &m, const int *I, double *acc, uint32_t *mark) {
    using R = RowCfg<DIM, DEG>;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int d = 0; d < DIM; ++d) {
        lo[d] = max(0, (I[d] + DEG - 1) / DEG - 1);
        hi[d] = min(m.cells - 1, I[d] / DEG);
    }
    int cell[3] = {0, 0, 0};
    for (cell[2] = (DIM == 3 ? lo[2] : 0); cell[2] <= (DIM == 3 ? hi[2] : 0); ++cell[2])
        for (cell[1] = lo[1]; cell[1] <= hi[1]; ++cell[1])
            for (cell[0] = lo[0]; cell[0] <= hi[0]; ++cell[0])
                for (int t = 0; t < R::NEL; ++t) {
                    Elem<DIM> e;
                    cell_element<DIM>(m, cell, t, e);
                    int li = -1;
                    int N[R::NLOC][DIM];
                    for (int l = 0; l < R::NLOC; ++l) {
                        local_dof<DIM, DEG>(e, l, N[l]);
                        bool same = true;
                        for (int d = 0; d < DIM; ++d) same &= (N[l][d] == I[d]);
                        if (same) li = l;
                    }
                    if (li < 0) continue;
                    double G[DIM + 1][DIM + 1];
                    double vol = 0.0;
                    if (WANT_VAL) vol = simplex_geometry<DIM>(m, e, G);
                    for (int l = 0; l < R::NLOC; ++l) {
                        int s = 0, mul = 1;
                        for (int d = 0; d < DIM; ++d) { s += (N[l][d] - I[d] + DEG) * mul; mul *= R::W; }
                        mark[s >> 5] |= 1u << (s & 31);
                        if (WANT_VAL) acc[s] += entry<DIM, DEG>(min(li, l), max(li, l), vol, G, m.ref);
                    }
                }
}

template <int DIM, int DEG>
__device__ __forceinline__ void slot_point(int s, const int *I, int *N) {
    using R = RowCfg<DIM, DEG>;
    for (int d = 0; d < DIM; ++d) { N[d] = I[d] + (s % R::W) - DEG; s /= R::W; }
}

template <int DIM, int DEG>
__global__ void __launch_bounds__(128) k_count_rows(MeshDev m, int64_t n_free, int32_t *len_ii,
                                                    int32_t *len_ib, int *max_row) {
    using R = RowCfg<DIM, DEG>;
    int local_max = 0;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_free;
         f += (int64_t)gridDim.x * blockDim.x) {
        int I[3] = {0, 0, 0};
        free_to_lattice(f, DIM, m.S, I);
        uint32_t mark[R::NW];
        for (int w = 0; w < R::NW; ++w) mark[w] = 0;
        gather_row<DIM, DEG, false>(m, I, nullptr, mark);
        int a = 0, b = 0;
        for (int s = 0; s < R::NS; ++s) {
            if (!((mark[s >> 5] >> (s & 31)) & 1u)) continue;
            int N[3] = {0, 0, 0};
            slot_point<DIM, DEG>(s, I, N);
            if (on_boundary(N, DIM, m.S)) ++b; else ++a;
        }
        len_ii[f] = a;
        len_ib[f] = b;
        local_max = max(local_max, a);
    }
    atomicMax(max_row, local_max);
}

template <int DIM, int DEG>
__global__ void __launch_bounds__(128) k_fill_rows(MeshDev m, int64_t n_free, const int32_t *rp_ii,
                                                   int32_t *col_ii, double *val_ii,
                                                   const int32_t *rp_ib, int32_t *col_ib,
                                                   double *val_ib, double *diag) {
    using R = RowCfg<DIM, DEG>;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_free;
         f += (int64_t)gridDim.x * blockDim.x) {
        int I[3] = {0, 0, 0};
        free_to_lattice(f, DIM, m.S, I);
        uint32_t mark[R::NW];
        double acc[R::NS];
        for (int w = 0; w < R::NW; ++w) mark[w] = 0;
        for (int s = 0; s < R::NS; ++s) acc[s] = 0.0;
        gather_row<DIM, DEG, true>(m, I, acc, mark);
        int32_t a = rp_ii[f], b = rp_ib[f];
        for (int s = 0; s < R::NS; ++s) {
            if (!((mark[s >> 5] >> (s & 31)) & 1u)) continue;
            int N[3] = {0, 0, 0};
            slot_point<DIM, DEG>(s, I, N);
            if (on_boundary(N, DIM, m.S)) {
                col_ib[b] = (int32_t)bnd_id(N, DIM, m.S);
                val_ib[b++] = acc[s];
            } else {
                col_ii[a] = (int32_t)free_id(N, DIM, m.S);
                val_ii[a++] = acc[s];
                if (s == (R::NS - 1) / 2) diag[f] = acc[s];
            }
        }
    }
}

// ------------------------------------------------------------ dof coords --
// Coordinates of dof-lattice point N: a vertex, or the midpoint of the edge
// whose endpoints round the odd coordinates down/up (in 2D, a cell-centre
// point lies on the cell's diagonal, whose direction depends on the flip).
// Degree >= 3: the node's smallest mesh face and its weights beta (|beta| =
// deg) come from the simplex holding the lattice point (2D: which side of the
// cell's diagonal; 3D: the Kuhn path of the sorted offsets -- ties put the
// point on a shared face, whose weights are the same from either side); the
// coordinate is (sum of beta_a P_a over that face, ascending vertex id) / deg
// with correctly rounded operations, a vertex node the vertex itself.
__device__ void node_coords(const MeshDev &m, const int *N, double *x) {
    const int dm = m.deg;
    int c[3] = {0, 0, 0}, f[3] = {0, 0, 0};
    for (int d = 0; d < m.dim; ++d) {
        c[d] = min(N[d] / dm, m.cells - 1);
        f[d] = N[d] - dm * c[d];
    }
    int vv[4][3], bb[4];
    int nv = m.dim + 1;
    for (int a = 0; a < 4; ++a) for (int d = 0; d < 3; ++d) vv[a][d] = c[d];
    if (m.dim == 2) {
        const bool fl = cell_flipped(m, c[0] + (int64_t)m.cells * c[1]);
        if (!fl) {  // diagonal (0,0)-(1,1)
            if (f[0] >= f[1]) {  // (0,0), (1,0), (1,1)
                vv[1][0] += 1; vv[2][0] += 1; vv[2][1] += 1;
                bb[0] = dm - f[0]; bb[1] = f[0] - f[1]; bb[2] = f[1];
            } else {             // (0,0), (1,1), (0,1)
                vv[1][0] += 1; vv[1][1] += 1; vv[2][1] += 1;
                bb[0] = dm - f[1]; bb[1] = f[0]; bb[2] = f[1] - f[0];
            }
        } else {    // diagonal (1,0)-(0,1)
            if (f[0] + f[1] <= dm) {  // (0,0), (1,0), (0,1)
                vv[1][0] += 1; vv[2][1] += 1;
                bb[0] = dm - f[0] - f[1]; bb[1] = f[0]; bb[2] = f[1];
            } else {                  // (1,0), (1,1), (0,1)
                vv[0][0] += 1; vv[1][0] += 1; vv[1][1] += 1; vv[2][1] += 1;
                bb[0] = dm - f[1]; bb[1] = f[0] + f[1] - dm; bb[2] = dm - f[0];
            }
        }
    } else {  // Kuhn: walk the axes in decreasing offset
        int p[3] = {0, 1, 2};
        for (int i = 1; i < 3; ++i)
            for (int j = i; j > 0 && f[p[j - 1]] < f[p[j]]; --j) { int t = p[j]; p[j] = p[j - 1]; p[j - 1] = t; }
        for (int s2 = 0; s2 < 3; ++s2) {
            for (int d = 0; d < 3; ++d) vv[s2 + 1][d] = vv[s2][d];
            vv[s2 + 1][p[s2]] += 1;
        }
        bb[0] = dm - f[p[0]]; bb[1] = f[p[0]] - f[p[1]]; bb[2] = f[p[1]] - f[p[2]]; bb[3] = f[p[2]];
    }
    // the face: vertices with beta > 0, ascending vertex id
    int64_t fid[4];
    int fi[4], nf = 0;
    for (int a = 0; a < nv; ++a) {
        if (bb[a] <= 0) continue;
        fid[nf] = vv[a][0] + (int64_t)m.V * (vv[a][1] + (m.dim == 3 ? (int64_t)m.V * vv[a][2] : 0));
        fi[nf++] = a;
    }
    for (int i = 1; i < nf; ++i)
        for (int j = i; j > 0 && fid[j - 1] > fid[j]; --j) {
            int64_t t = fid[j]; fid[j] = fid[j - 1]; fid[j - 1] = t;
            int u = fi[j]; fi[j] = fi[j - 1]; fi[j - 1] = u;
        }
    for (int d = 0; d < m.dim; ++d) {
        if (nf == 1) { x[d] = vertex_coord(m, vv[fi[0]], d); continue; }
        double t = 0.0;
        for (int i = 0; i < nf; ++i) t = __dadd_rn(t, __dmul_rn((double)bb[fi[i]], vertex_coord(m, vv[fi[i]], d)));
        x[d] = __ddiv_rn(t, (double)dm);
    }
}

__device__ void dof_coords(const MeshDev &m, const int *N, double *x) {
    if (m.deg >= 3) {
        node_coords(m, N, x);
        return;
    }
    if (m.deg == 1) {
        for (int d = 0; d < m.dim; ++d) x[d] = vertex_coord(m, N, d);
        return;
    }
    int a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    int nodd = 0;
    for (int d = 0; d < m.dim; ++d) {
        if (N[d] & 1) { a[d] = (N[d] - 1) / 2; b[d] = (N[d] + 1) / 2; ++nodd; }
        else { a[d] = b[d] = N[d] / 2; }
    }
    if (nodd == 0) {
        for (int d = 0; d < m.dim; ++d) x[d] = vertex_coord(m, a, d);
        return;
    }
    if (m.dim == 2 && nodd == 2) {
        const int64_t cid = a[0] + (int64_t)m.cells * a[1];
        if (cell_flipped(m, cid)) { int t = a[0]; a[0] = b[0]; b[0] = t; }  // (1,0)-(0,1) diagonal
    }
    for (int d = 0; d < m.dim; ++d)
        x[d] = __dmul_rn(__dadd_rn(vertex_coord(m, a, d), vertex_coord(m, b, d)), 0.5);
}

__device__ double gfun(int gid, const double *c, const double *p, int dim) {
    const double x = p[0], y = p[1], z = dim == 3 ? p[2] : 0.0;
    switch (gid) {
    case 0: {
        const double pi = 3.14159265358979323846;
        return sin(pi * x) * sinh(pi * y) / sinh(pi);
    }
    case 1: return x * x - y * y;
    case 2: return x * x + y * y - 2.0 * z * z;
    case 3: return c[0] + c[1] * x + c[2] * y + c[3] * z;
    default: {
        // Re/Im of w^k, w = x + iy, by repeated complex multiplication
        double re = 1.0, im = 0.0, t = c[0] * re + c[1] * im;
        for (int k = 1; k <= 4; ++k) {
            const double r2 = re * x - im * y, i2 = re * y + im * x;
            re = r2; im = i2;
            t += c[2 * k] * re + c[2 * k + 1] * im;
        }
        return t;
    }
    }
}

// lattice point of row r: free id (which=1) or boundary id via the stored map
__device__ __forceinline__ void row_point(const MeshDev &m, int which, int64_t r,
                                          const int32_t *full_of_bnd, int *N) {
    if (which == 1) { free_to_lattice(r, m.dim, m.S, N); return; }
    int64_t t = full_of_bnd[r];
    for (int d = 0; d < m.dim; ++d) { N[d] = (int)(t % m.S); t /= m.S; }
}

__global__ void k_coords(MeshDev m, int which, int64_t rows, const int32_t *fob, double *out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int N[3] = {0, 0, 0};
        row_point(m, which, r, fob, N);
        double x[3];
        dof_coords(m, N, x);
        for (int d = 0; d < m.dim; ++d) out[r * m.dim + d] = x[d];
    }
}

__global__ void k_dirichlet(MeshDev m, int which, int64_t rows, const int32_t *fob, int gid,
                            const double *coef, int ncoef, int k, double *out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int N[3] = {0, 0, 0};
        row_point(m, which, r, fob, N);
        double x[3] = {0, 0, 0};
        dof_coords(m, N, x);
        for (int c = 0; c < k; ++c) out[r * k + c] = gfun(gid, coef + (int64_t)c * ncoef, x, m.dim);
    }
}

__global__ void k_maps(MeshDev m, int64_t n_free, int64_t n_bnd, int64_t n_dof, int32_t *fof,
                       int32_t *fob, int32_t *free_of_full) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_dof; i += stride) {
        int N[3] = {0, 0, 0};
        int64_t t = i;
        for (int d = 0; d < m.dim; ++d) { N[d] = (int)(t % m.S); t /= m.S; }
        if (on_boundary(N, m.dim, m.S)) {
            if (fob) fob[bnd_id(N, m.dim, m.S)] = (int32_t)i;
            if (free_of_full) free_of_full[i] = -1;
        } else {
            if (fof) fof[free_id(N, m.dim, m.S)] = (int32_t)i;
            if (free_of_full) free_of_full[i] = (int32_t)free_id(N, m.dim, m.S);
        }
    }
    (void)n_free; (void)n_bnd;
}

// b[f][c] = -sum_q K_IB[f][q] gB[q][c]
__global__ void k_lift(int64_t n_free, int k, const int32_t *rp, const int32_t *ci, const double *v,
                       const double *gB, double *b) {
    const int64_t total = n_free * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / k;
        const int c = (int)(t - f * k);
        double s = 0.0;
        for (int32_t q = rp[f]; q < rp[f + 1]; ++q) s += v[q] * gB[(int64_t)ci[q] * k + c];
        b[t] = -s;
    }
}

}  // namespace gb

// ====================================================================== ABI ==
struct gb_fem_system {
    gb_fem_spec spec;
    gb::MeshDev m;
    gb::Mem mem;
    int64_t n_dof, n_free, n_bnd, nnz, nnz_ib;
    int max_row;
    int32_t *rp = nullptr, *col = nullptr, *rp_ib = nullptr, *col_ib = nullptr;
    double *val = nullptr, *val_ib = nullptr, *diag = nullptr;
    int32_t *full_of_bnd = nullptr;
    double *ref = nullptr;  // degree >= 3: reference integrals on the device
};

using namespace gb;

// Reference integrals of the degree-m (m >= 3) Lagrange basis on a d-simplex,
// per unit volume: I[l][k][a][b] = (1/|T|) int_T (d phi_l/d lambda_a)(d phi_k/d lambda_b),
// phi_beta = prod_c s_{beta_c}(lambda_c) with s_j(t) = prod_{i<j} (m t - i)/(i + 1).
// Each integrand is a product of one polynomial per lambda_c; with
// int_T prod lambda_c^e_c = |T| d! prod e_c! / (d + sum e_c)!, the integral is
// d! sum_E W[E] / (d + E)!, W the convolution over c of w_c[e] = coef_c[e] e!.
template <int DIM, int DEG>
static std::vector<double> reference_table() {
    constexpr int NL = RowCfg<DIM, DEG>::NLOC, NV = DIM + 1, PD = 2 * DEG;
    double sj[DEG + 1][DEG + 1] = {}, dsj[DEG + 1][DEG + 1] = {};  // coefficients by power
    for (int j = 0; j <= DEG; ++j) {
        double c[DEG + 1] = {};
        c[0] = 1.0;
        for (int i = 0; i < j; ++i) {  // times (m t - i)/(i + 1)
            double nc[DEG + 1] = {};
            for (int p = 0; p <= DEG; ++p) {
                if (p + 1 <= DEG) nc[p + 1] += c[p] * DEG / (i + 1.0);
                nc[p] -= c[p] * i / (i + 1.0);
            }
            for (int p = 0; p <= DEG; ++p) c[p] = nc[p];
        }
        for (int p = 0; p <= DEG; ++p) {
            sj[j][p] = c[p];
            dsj[j][p] = p + 1 <= DEG ? (p + 1) * c[p + 1] : 0.0;
        }
    }
    double fact[NV * PD + NV + 1];
    fact[0] = 1.0;
    for (int i = 1; i <= NV * PD + NV; ++i) fact[i] = fact[i - 1] * i;
    std::vector<double> I((size_t)NL * NL * NV * NV, 0.0);
    for (int l = 0; l < NL; ++l)
        for (int k = 0; k < NL; ++k) {
            int bl[4] = {0, 0, 0, 0}, bk[4] = {0, 0, 0, 0};
            node_beta<DIM, DEG>(l, bl);
            node_beta<DIM, DEG>(k, bk);
            for (int a = 0; a < NV; ++a)
                for (int b = 0; b < NV; ++b) {
                    std::vector<double> W(1, 1.0);  // running convolution
                    for (int c = 0; c < NV; ++c) {
                        const double *f = c == a ? dsj[bl[c]] : sj[bl[c]];
                        const double *h = c == b ? dsj[bk[c]] : sj[bk[c]];
                        double w[PD + 1] = {};
                        for (int p = 0; p <= DEG; ++p)
                            for (int q = 0; q <= DEG; ++q) w[p + q] += f[p] * h[q];
                        for (int e = 0; e <= PD; ++e) w[e] *= fact[e];
                        std::vector<double> nW(W.size() + PD, 0.0);
                        for (size_t x = 0; x < W.size(); ++x)
                            for (int e = 0; e <= PD; ++e) nW[x + e] += W[x] * w[e];
                        W.swap(nW);
                    }
                    double t = 0.0;
                    for (size_t E = 0; E < W.size(); ++E) t += W[E] * fact[DIM] / fact[DIM + E];
                    I[(((size_t)l * NL + k) * NV + a) * NV + b] = t;
                }
        }
    return I;
}

template <int DIM, int DEG>
static int assemble_impl(gb_fem_system *s, cudaStream_t st) {
    Mem &mem = s->mem;
    const int64_t n = s->n_free;
    if (DEG >= 3) {
        const std::vector<double> I = reference_table<DIM, DEG>();
        GB_TRY(mem.alloc_n(&s->ref, I.size()));
        GB_CHECK_CUDA(cudaMemcpyAsync(s->ref, I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));  // I is freed on return
        s->m.ref = s->ref;
    }
    int32_t *len = nullptr, *len_ib = nullptr;
    int *d_max = nullptr;
    struct Temps {  // the row-length temporaries go back on every return path
        Mem &m;
        int32_t *&a, *&b;
        int *&c;
        ~Temps() {
            m.release(a);
            m.release(b);
            m.release(c);
        }
    } temps{mem, len, len_ib, d_max};
    GB_TRY(mem.alloc_n(&len, (size_t)n + 1));
    GB_TRY(mem.alloc_n(&len_ib, (size_t)n + 1));
    GB_TRY(mem.alloc_n(&d_max, 1));
    GB_CHECK_CUDA(cudaMemsetAsync(d_max, 0, sizeof(int), st));
    const int grid = stride_grid(n, 128, 16);
    ::gb::count_launches(1); k_count_rows<DIM, DEG><<<grid, 128, 0, st>>>(s->m, n, len, len_ib, d_max);
    GB_CHECK_CUDA(cudaGetLastError());
    GB_TRY(mem.alloc_n(&s->rp, (size_t)n + 1));
    GB_TRY(mem.alloc_n(&s->rp_ib, (size_t)n + 1));
    int64_t nnz = 0, nnz_ib = 0;
    GB_TRY((scan_exclusive<int32_t, int32_t>(len, s->rp, n, &nnz, mem)));
    GB_TRY((scan_exclusive<int32_t, int32_t>(len_ib, s->rp_ib, n, &nnz_ib, mem)));
    if (nnz >= (int64_t)INT32_MAX || nnz_ib >= (int64_t)INT32_MAX) {
        set_error("system too large for int32 indices (nnz=%lld)", (long long)nnz);
        return GB_TOO_LARGE;
    }
    GB_CHECK_CUDA(cudaMemcpyAsync(&s->max_row, d_max, sizeof(int), cudaMemcpyDeviceToHost, st));
    s->nnz = nnz;
    s->nnz_ib = nnz_ib;
    GB_TRY(mem.alloc_n(&s->col, (size_t)nnz));
    GB_TRY(mem.alloc_n(&s->val, (size_t)nnz));
    GB_TRY(mem.alloc_n(&s->col_ib, (size_t)nnz_ib));
    GB_TRY(mem.alloc_n(&s->val_ib, (size_t)nnz_ib));
    GB_TRY(mem.alloc_n(&s->diag, (size_t)n));
    GB_TRY(mem.alloc_n(&s->full_of_bnd, (size_t)s->n_bnd));
    ::gb::count_launches(1); k_maps<<<stride_grid(s->n_dof, 256, 8), 256, 0, st>>>(s->m, n, s->n_bnd, s->n_dof, nullptr,
                                                         s->full_of_bnd, nullptr);
    ::gb::count_launches(1); k_fill_rows<DIM, DEG><<<grid, 128, 0, st>>>(s->m, n, s->rp, s->col, s->val, s->rp_ib, s->col_ib,
                                                 s->val_ib, s->diag);
    GB_CHECK_CUDA(cudaGetLastError());
    GB_CHECK_CUDA(cudaStreamSynchronize(st));
    return GB_OK;
}

extern "C" int fem_assemble(const gb_fem_spec *spec, const gb_allocator *alloc, void *stream,
                            gb_fem_system **out) {
    gb::Range range("gbpcg:fem_assemble");
    GB_REQUIRE(spec && out, "fem_assemble: NULL argument");
    *out = nullptr;
    GB_REQUIRE(spec->dim == 2 || spec->dim == 3, "fem_assemble: dim must be 2 or 3");
    GB_REQUIRE(spec->degree >= 1 && spec->degree <= 4, "fem_assemble: degree must be 1, 2, 3 or 4");
    GB_REQUIRE(spec->cells >= 2, "fem_assemble: cells must be >= 2");
    GB_REQUIRE(spec->jitter == 0 || spec->jitter == 1, "fem_assemble: jitter must be 0 or 1");
    GB_REQUIRE(spec->diag_mode == 0 || spec->diag_mode == 1, "fem_assemble: diag_mode must be 0 or 1");
    GB_REQUIRE(spec->dim == 2 || spec->diag_mode == 0,
               "fem_assemble: 3D meshes use the Kuhn split of every cube (diag_mode=0)");
    GB_REQUIRE(spec->reserved == 0, "fem_assemble: reserved must be 0");
    const int64_t S = (int64_t)spec->degree * spec->cells + 1;
    int64_t n_dof = 1, n_free = 1;
    for (int d = 0; d < spec->dim; ++d) { n_dof *= S; n_free *= (S - 2); }
    if (n_dof >= (int64_t)INT32_MAX / 2) {
        set_error("fem_assemble: %lld dofs exceed the int32 index range", (long long)n_dof);
        return GB_TOO_LARGE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    gb_fem_system *s = new gb_fem_system();
    s->spec = *spec;
    s->mem = Mem(alloc, st);
    MeshDev &m = s->m;
    m.dim = spec->dim; m.deg = spec->degree; m.cells = spec->cells; m.S = (int)S; m.V = spec->cells + 1;
    m.jitter = spec->jitter; m.diag_mode = spec->diag_mode;
    m.kx = stream_key(spec->seed, 0); m.ky = stream_key(spec->seed, 1); m.kf = stream_key(spec->seed, 2);
    m.kz = stream_key(spec->seed, 3);
    m.q = (spec->dim == 3 ? 0.125 : 0.25) / (double)spec->cells;
    s->n_dof = n_dof; s->n_free = n_free; s->n_bnd = n_dof - n_free;
    m.ref = nullptr;
    int rc;
    switch (m.dim * 10 + m.deg) {
    case 21: rc = assemble_impl<2, 1>(s, st); break;
    case 22: rc = assemble_impl<2, 2>(s, st); break;
    case 23: rc = assemble_impl<2, 3>(s, st); break;
    case 24: rc = assemble_impl<2, 4>(s, st); break;
    case 31: rc = assemble_impl<3, 1>(s, st); break;
    case 32: rc = assemble_impl<3, 2>(s, st); break;
    case 33: rc = assemble_impl<3, 3>(s, st); break;
    default: rc = assemble_impl<3, 4>(s, st); break;
    }
    if (rc != GB_OK) { fem_system_destroy(s); return rc; }
    *out = s;
    return GB_OK;
}

extern "C" int fem_system_info(const gb_fem_system *s, gb_fem_info *o) {
    GB_REQUIRE(s && o, "fem_system_info: NULL argument");
    o->n_dof = s->n_dof; o->n_free = s->n_free; o->n_bnd = s->n_bnd;
    o->nnz = s->nnz; o->nnz_ib = s->nnz_ib;
    o->dim = s->m.dim; o->degree = s->m.deg; o->cells = s->m.cells; o->side = s->m.S;
    o->max_row = s->max_row; o->reserved = 0;
    o->d_rowptr = s->rp; o->d_col = s->col; o->d_val = s->val;
    o->d_rowptr_ib = s->rp_ib; o->d_col_ib = s->col_ib; o->d_val_ib = s->val_ib;
    o->d_diag = s->diag;
    return GB_OK;
}

extern "C" int fem_dof_maps(const gb_fem_system *s, int32_t *d_full_of_free, int32_t *d_full_of_bnd,
                            int32_t *d_free_of_full, void *stream) {
    GB_REQUIRE(s, "fem_dof_maps: NULL system");
    cudaStream_t st = (cudaStream_t)stream;
    ::gb::count_launches(1); k_maps<<<stride_grid(s->n_dof, 256, 8), 256, 0, st>>>(s->m, s->n_free, s->n_bnd, s->n_dof,
                                                         d_full_of_free, d_full_of_bnd, d_free_of_full);
    GB_CHECK_CUDA(cudaGetLastError());
    return GB_OK;
}

extern "C" int fem_boundary_coords(const gb_fem_system *s, int which, double *d_xyz, void *stream) {
    GB_REQUIRE(s && d_xyz, "fem_boundary_coords: NULL argument");
    GB_REQUIRE(which == 0 || which == 1, "fem_boundary_coords: which must be 0 or 1");
    const int64_t rows = which == 0 ? s->n_bnd : s->n_free;
    cudaStream_t st = (cudaStream_t)stream;
    ::gb::count_launches(1); k_coords<<<stride_grid(rows, 256, 8), 256, 0, st>>>(s->m, which, rows, s->full_of_bnd, d_xyz);
    GB_CHECK_CUDA(cudaGetLastError());
    return GB_OK;
}

static int gid_ncoef(int gid) { return gid == 3 ? 4 : (gid == 4 ? 10 : 0); }

extern "C" int fem_dirichlet(const gb_fem_system *s, int gid, const double *h_coef, int k, int which,
                             double *d_out, void *stream) {
    GB_REQUIRE(s && d_out, "fem_dirichlet: NULL argument");
    GB_REQUIRE(gid >= 0 && gid <= 4, "fem_dirichlet: gid must be in 0..4");
    GB_REQUIRE(k >= 1, "fem_dirichlet: k must be >= 1");
    GB_REQUIRE(which == 0 || which == 1, "fem_dirichlet: which must be 0 or 1");
    GB_REQUIRE(s->m.dim == 2 || gid >= 2, "fem_dirichlet: gid %d is 2D only", gid);  // gid 4 (x + iy) is harmonic in 3D too
    const int nc = gid_ncoef(gid);
    GB_REQUIRE(nc == 0 || h_coef, "fem_dirichlet: gid %d needs coefficients", gid);
    cudaStream_t st = (cudaStream_t)stream;
    double *d_coef = nullptr;
    Mem mem(nullptr, st);
    if (nc) {
        GB_TRY(mem.alloc_n(&d_coef, (size_t)nc * k));
        GB_CHECK_CUDA(cudaMemcpyAsync(d_coef, h_coef, sizeof(double) * nc * k, cudaMemcpyHostToDevice, st));
    }
    const int64_t rows = which == 0 ? s->n_bnd : s->n_free;
    ::gb::count_launches(1); k_dirichlet<<<stride_grid(rows, 256, 8), 256, 0, st>>>(s->m, which, rows, s->full_of_bnd, gid, d_coef,
                                                          nc, k, d_out);
    cudaError_t e = cudaGetLastError();
    if (nc) {
        cudaStreamSynchronize(st);
        mem.release(d_coef);
    }
    GB_CHECK_CUDA(e);
    return GB_OK;
}

extern "C" int fem_lift_rhs(const gb_fem_system *s, const double *d_gB, int k, double *d_b, void *stream) {
    GB_REQUIRE(s && d_gB && d_b, "fem_lift_rhs: NULL argument");
    GB_REQUIRE(k >= 1, "fem_lift_rhs: k must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    ::gb::count_launches(1); k_lift<<<stride_grid(s->n_free * k, 256, 8), 256, 0, st>>>(s->n_free, k, s->rp_ib, s->col_ib,
                                                              s->val_ib, d_gB, d_b);
    GB_CHECK_CUDA(cudaGetLastError());
    return GB_OK;
}

extern "C" void fem_system_destroy(gb_fem_system *s) {
    if (!s) return;
    Mem &m = s->mem;
    m.release(s->rp); m.release(s->col); m.release(s->val);
    m.release(s->rp_ib); m.release(s->col_ib); m.release(s->val_ib);
    m.release(s->diag);
    m.release(s->full_of_bnd);
    m.release(s->ref);
    delete s;
}

// accessor for the SELL builder (same library)
namespace gb {
int fem_csr_view(const gb_fem_system *s, int64_t *n, const int32_t **rp, const int32_t **col,
                 const double **val, const double **diag, int *max_row) {
    *n = s->n_free; *rp = s->rp; *col = s->col; *val = s->val; *diag = s->diag; *max_row = s->max_row;
    return GB_OK;
}
}  // namespace gb
