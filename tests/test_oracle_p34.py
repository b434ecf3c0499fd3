"""Pins of the oracle's P3 and P4 elements (the degree study of Sec. 4.2,
Table 7), regular and jittered meshes, against routes independent of its
Silvester-basis table:

- element matrices = Lagrange bases from a Vandermonde solve at the nodes,
  integrated with a collapsed Gauss-Legendre rule;
- element and assembled matrices symmetric (bit-exact), zero row sums, PSD;
- exact reproduction: P3 reproduces the cubic harmonic polynomials, P4 the
  quartic ones (the discrete solution equals the nodal values), and P3 does
  not reproduce a quartic (control);
- convergence: for the smooth harmonic sin(pi x) sinh(pi y)/sinh(pi) the
  nodal error falls at least like h^m when h halves (order m+1 expected);
- pattern = brute-force set of pairs sharing an element; counts
  (m cells + 1)^d dofs, C(m+d, d) per element;
- node coordinates on jittered meshes follow their definition, (sum of
  beta_a P_a over the node's smallest face, ascending vertex id) / m, bit for
  bit from every element around the node.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O

from test_oracle_element import _quad_simplex, _monomials, _lagrange_coeffs, _grad_mono


def _elem_vertices(s, e, X, E):
    """the element's vertex nodes (dof-lattice coordinates multiples of m), in
    the element's vertex order"""
    S = s.n_dof ** (1.0 / s.dim)
    S = int(round(S))
    ids = E[e]
    lat = np.stack([(ids // S ** d) % S for d in range(s.dim)], 1)
    mask = np.all(lat % s.degree == 0, axis=1)
    assert mask.sum() == s.dim + 1
    return X[ids[mask]]


def _stiffness_by_quadrature(nodes, P, deg):
    dim = P.shape[1]
    mons = _monomials(dim, deg)
    Cf = _lagrange_coeffs(nodes, mons)
    pts, wts = _quad_simplex(P, npts=6)
    K = np.zeros((len(nodes), len(nodes)))
    for x, w in zip(pts, wts):
        G = np.array([_grad_mono(m, x) for m in mons])
        grads = Cf.T @ G
        K += w * grads @ grads.T
    return K


@pytest.mark.parametrize("dim,degree,cells,jitter", [(2, 3, 3, 0), (2, 4, 3, 0), (3, 3, 2, 0), (3, 4, 2, 0),
                                                     (2, 3, 4, 1), (2, 4, 4, 1), (3, 3, 3, 1), (3, 4, 3, 1)])
def test_element_matrix_vs_lagrange_quadrature(dim, degree, cells, jitter):
    s = O.System(dim, degree, cells, jitter=jitter, diag_mode=1 if dim == 2 else 0, seed=5)
    assert s.n_loc == math.comb(degree + dim, dim)
    assert s.n_dof == (degree * cells + 1) ** dim
    X = s.dof_coords()
    E = s.elements()
    for e in range(0, s.n_elements, max(1, s.n_elements // 7)):
        nodes = X[E[e]]
        P = _elem_vertices(s, e, X, E)
        Kq = _stiffness_by_quadrature(nodes, P, degree)
        Ko = s.element_matrix(e)
        assert np.abs(Ko - Kq).max() <= 1e-9 * np.abs(Kq).max()
        assert np.array_equal(Ko, Ko.T)
        assert np.abs(Ko.sum(1)).max() <= 1e-12 * np.abs(Ko).max()
        assert np.linalg.eigvalsh(Ko).min() > -1e-12 * np.abs(Ko).max()


def _solve_with_g(s, gfun):
    rp, ci, v = s.k_ii()
    fof, fob, foff, fofb = s.maps()
    X = s.dof_coords()
    gB = gfun(X[fofb])
    b = s.lift(gB[:, None])[:, 0]
    return O.cholesky_solve(rp, ci, v, b), gfun(X[foff])


CUBIC = [lambda X: X[:, 0] ** 3 - 3 * X[:, 0] * X[:, 1] ** 2, lambda X: 3 * X[:, 0] ** 2 * X[:, 1] - X[:, 1] ** 3]
QUARTIC = lambda X: X[:, 0] ** 4 - 6 * X[:, 0] ** 2 * X[:, 1] ** 2 + X[:, 1] ** 4


@pytest.mark.parametrize("dim,cells,jitter", [(2, 4, 0), (3, 2, 0), (2, 6, 1), (3, 3, 1)])
def test_exact_reproduction(dim, cells, jitter):
    s3 = O.System(dim, 3, cells, jitter, 1 if dim == 2 else 0, 2).assemble()
    for g in CUBIC:
        x, want = _solve_with_g(s3, g)
        assert np.abs(x - want).max() <= 1e-11 * np.abs(want).max()
    s4 = O.System(dim, 4, cells, jitter, 1 if dim == 2 else 0, 2).assemble()
    x, want = _solve_with_g(s4, QUARTIC)
    assert np.abs(x - want).max() <= 1e-11 * np.abs(want).max()
    x, want = _solve_with_g(s3, QUARTIC)  # a quartic is not in the P3 space
    assert np.abs(x - want).max() > 1e-6 * np.abs(want).max()


SMOOTH = lambda X: np.sin(np.pi * X[:, 0]) * np.sinh(np.pi * X[:, 1]) / np.sinh(np.pi)


@pytest.mark.parametrize("degree", [3, 4])
def test_convergence_order(degree):
    errs = []
    for cells in (4, 8):
        s = O.System(2, degree, cells, 0, 1, 3).assemble()
        x, want = _solve_with_g(s, SMOOTH)
        errs.append(np.abs(x - want).max())
    assert errs[0] / errs[1] >= 2.0 ** degree


def test_error_falls_with_degree():
    errs = []
    for degree in (1, 2, 3, 4):
        s = O.System(2, degree, 8, 0, 1, 3).assemble()
        x, want = _solve_with_g(s, SMOOTH)
        errs.append(np.abs(x - want).max())
    assert all(errs[i + 1] < 0.5 * errs[i] for i in range(3))


@pytest.mark.parametrize("dim,degree,cells", [(2, 3, 3), (2, 4, 2), (3, 3, 2), (3, 4, 1)])
def test_pattern_is_pairs_sharing_an_element(dim, degree, cells):
    s = O.System(dim, degree, cells, 0, 1, 7).assemble()
    rp, ci, v = s.full()
    E = s.elements()
    want = set()
    for row in E:
        for a, b in itertools.product(row, row):
            want.add((int(a), int(b)))
    got = set()
    for i in range(len(rp) - 1):
        for k in range(rp[i], rp[i + 1]):
            got.add((i, int(ci[k])))
    assert got == want
    assert np.all(np.diff(ci[rp[0]:rp[1]]) > 0)


def test_degree_above_4_rejected():
    with pytest.raises(ValueError):
        O.System(3, 5, 2)


@pytest.mark.parametrize("dim,degree,cells", [(2, 3, 5), (2, 4, 3), (3, 3, 3), (3, 4, 2)])
def test_jittered_node_coordinates_definition(dim, degree, cells):
    s = O.System(dim, degree, cells, 1, 1 if dim == 2 else 0, 8)
    X = s.dof_coords()
    V = s.vertex_coords()
    E = s.elements()
    S = degree * cells + 1
    Vn = cells + 1
    for e in range(s.n_elements):
        ids = E[e]
        lat = np.stack([(ids // S ** d) % S for d in range(dim)], 1)
        vmask = np.all(lat % degree == 0, axis=1)
        vlat = lat[vmask] // degree                       # the element's vertices (cell units)
        vid = sum(vlat[:, d] * Vn ** d for d in range(dim))
        # barycentric weights of each node: solve N = sum_a beta_a v_a (integers)
        M = np.vstack([vlat.T.astype(float), np.ones(dim + 1)])
        for l in range(len(ids)):
            beta = np.rint(np.linalg.solve(M, np.append(lat[l].astype(float), degree))).astype(int)
            face = sorted((int(vid[a]), int(beta[a])) for a in range(dim + 1) if beta[a] > 0)
            for d in range(dim):
                if len(face) == 1:
                    want = V[face[0][0], d]
                else:
                    t = 0.0
                    for v, b in face:
                        t = t + float(b) * float(V[v, d])
                    want = t / degree
                assert X[ids[l], d] == want
