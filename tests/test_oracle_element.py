"""Oracle pins: element stiffness matrices (CPU only).

Each pin reaches the stiffness by a route independent of the oracle's
barycentric-gradient formula: the cotangent weights of Sec. 2.2 (P1, 2D and
3D), and Lagrange bases built from a Vandermonde solve integrated with a
collapsed Gauss-Legendre rule (P1/P2, 2D and 3D)."""
import itertools

import numpy as np
import pytest

import oracle as O


def _elements(dim, degree, jitter, seed=4, cells=4):
    s = O.System(dim, degree, cells, jitter=jitter, diag_mode=1, seed=seed)
    return s, s.vertex_coords(), s.elements()


def _vertex_ids(s, e):
    """vertex ids of element e (its first dim+1 dofs are on vertices)"""
    X = s.dof_coords()
    E = s.elements()
    return X[E[e, : s.dim + 1]]


# ----------------------------------------------------------------- P1, 2D --
def test_p1_2d_cotangent_weights():
    """Sec. 2.2: w(i,j) = sum over the triangles at edge (i,j) of cot(opposite angle)/2;
    per triangle the stiffness off-diagonal is -cot(angle opposite the edge)/2."""
    s = O.System(2, 1, 6, jitter=1, diag_mode=1, seed=13)
    for e in range(0, s.n_elements, 7):
        P = _vertex_ids(s, e)
        K = s.element_matrix(e)
        for a, b in [(0, 1), (0, 2), (1, 2)]:
            c = 3 - a - b
            u, v = P[a] - P[c], P[b] - P[c]
            ang = np.arctan2(abs(u[0] * v[1] - u[1] * v[0]), u @ v)
            assert K[a, b] == pytest.approx(-0.5 / np.tan(ang), rel=1e-12, abs=1e-13)
        assert np.allclose(K.sum(1), 0.0, atol=1e-13)


# ----------------------------------------------------------------- P1, 3D --
@pytest.mark.parametrize("jitter", [0, 1])
def test_p1_3d_cotangent_weights(jitter):
    """Sec. 2.2: w(i,j) = (1/6) sum_k l_k cot(alpha_k), l_k the length of the edge
    opposite (i,j) in tet k and alpha_k the dihedral angle at that edge;
    the per-tet stiffness off-diagonal is -(1/6) l cot(alpha)."""
    s = O.System(3, 1, 3, jitter=jitter, seed=8)
    for e in range(s.n_elements):
        P = _vertex_ids(s, e)
        K = s.element_matrix(e)
        for a, b in itertools.combinations(range(4), 2):
            k, l = [m for m in range(4) if m not in (a, b)]
            edge = P[l] - P[k]
            L = np.linalg.norm(edge)
            t = edge / L
            # dihedral angle at edge (k,l) between faces (k,l,a) and (k,l,b)
            ua = P[a] - P[k]; ua = ua - (ua @ t) * t
            ub = P[b] - P[k]; ub = ub - (ub @ t) * t
            alpha = np.arctan2(np.linalg.norm(np.cross(ua, ub)), ua @ ub)
            want = -L / (6.0 * np.tan(alpha))
            assert K[a, b] == pytest.approx(want, rel=1e-12, abs=1e-14)


# ------------------------------------------------- Lagrange basis by Vandermonde
def _monomials(dim, deg):
    out = []
    for p in itertools.product(range(deg + 1), repeat=dim):
        if sum(p) <= deg:
            out.append(p)
    return out


def _lagrange_coeffs(nodes, mons):
    V = np.array([[np.prod([x[d] ** m[d] for d in range(len(m))]) for m in mons] for x in nodes])
    return np.linalg.solve(V, np.eye(len(nodes)))  # column i: basis i


def _grad_mono(m, x):
    g = np.zeros(len(m))
    for d in range(len(m)):
        if m[d] > 0:
            mm = list(m); mm[d] -= 1
            g[d] = m[d] * np.prod([x[q] ** mm[q] for q in range(len(m))])
    return g


def _quad_simplex(P, npts=5):
    """collapsed (Duffy) Gauss-Legendre rule on the simplex with vertices P"""
    dim = P.shape[1]
    t, w = np.polynomial.legendre.leggauss(npts)
    t = 0.5 * (t + 1.0); w = 0.5 * w
    J = np.stack([P[a] - P[0] for a in range(1, dim + 1)], 1)
    detJ = abs(np.linalg.det(J))
    pts, wts = [], []
    if dim == 2:
        for (u, wu), (v, wv) in itertools.product(zip(t, w), zip(t, w)):
            s_, t_ = u, v * (1 - u)
            pts.append(P[0] + J @ np.array([s_, t_])); wts.append(wu * wv * (1 - u) * detJ)
    else:
        for (u, wu), (v, wv), (z, wz) in itertools.product(zip(t, w), zip(t, w), zip(t, w)):
            a_, b_, c_ = u, v * (1 - u), z * (1 - u) * (1 - v)
            pts.append(P[0] + J @ np.array([a_, b_, c_]))
            wts.append(wu * wv * wz * (1 - u) ** 2 * (1 - v) * detJ)
    return np.array(pts), np.array(wts)


def _stiffness_by_quadrature(nodes, P, deg):
    dim = P.shape[1]
    mons = _monomials(dim, deg)
    Cf = _lagrange_coeffs(nodes, mons)
    pts, wts = _quad_simplex(P)
    n = len(nodes)
    K = np.zeros((n, n))
    for x, w in zip(pts, wts):
        G = np.array([_grad_mono(m, x) for m in mons])  # (nmon, dim)
        grads = Cf.T @ G  # (n, dim)
        K += w * grads @ grads.T
    return K


@pytest.mark.parametrize("dim,degree,jitter", [(2, 1, 1), (2, 2, 1), (2, 2, 0), (3, 1, 0), (3, 2, 0), (3, 1, 1),
                                               (3, 2, 1)])
def test_element_matrix_vs_lagrange_quadrature(dim, degree, jitter):
    s = O.System(dim, degree, 3, jitter=jitter, diag_mode=1, seed=21)
    X = s.dof_coords()
    E = s.elements()
    picks = range(0, s.n_elements, max(1, s.n_elements // 9))
    for e in picks:
        nodes = X[E[e]]
        P = nodes[: dim + 1]
        Kq = _stiffness_by_quadrature(nodes, P, degree)
        Ko = s.element_matrix(e)
        scale = np.abs(Kq).max()
        assert np.abs(Ko - Kq).max() <= 1e-11 * scale


def test_p2_2d_vertex_opposite_midpoint_zero():
    """P2 triangles: a vertex and the midpoint of the opposite edge do not couple."""
    s = O.System(2, 2, 4, jitter=1, diag_mode=1, seed=8)
    for e in range(s.n_elements):
        K = s.element_matrix(e)
        # local order: vertices 0,1,2 then midpoints of (0,1),(0,2),(1,2)
        for v, m in [(0, 5), (1, 4), (2, 3)]:
            assert abs(K[v, m]) < 1e-13 * np.abs(K).max()


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_element_rows_sum_to_zero_and_symmetric(dim, degree):
    s = O.System(dim, degree, 3, jitter=1 if dim == 2 else 0, diag_mode=1, seed=6)
    for e in range(s.n_elements):
        K = s.element_matrix(e)
        assert np.array_equal(K, K.T)
        assert np.abs(K.sum(1)).max() <= 1e-12 * np.abs(K).max()
        assert np.all(np.linalg.eigvalsh(K) > -1e-12 * np.abs(K).max())


def test_quadrature_pin_detects_planted_mistakes():
    """The quadrature pin separates the correct P2 matrix from a plausible error:
    the element's edge dofs numbered in transposed order."""
    s = O.System(2, 2, 2, jitter=1, diag_mode=1, seed=1)
    X = s.dof_coords(); E = s.elements()
    nodes = X[E[0]]
    Kq = _stiffness_by_quadrature(nodes, nodes[:3], 2)
    Ko = s.element_matrix(0)
    assert np.abs(Ko - Kq).max() < 1e-11
    wrong_nodes = nodes.copy()
    wrong_nodes[[3, 4]] = wrong_nodes[[4, 3]]  # transposed edge numbering
    Kw = _stiffness_by_quadrature(wrong_nodes, nodes[:3], 2)
    assert np.abs(Ko - Kw).max() > 1e-3
