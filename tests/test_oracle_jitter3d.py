"""Oracle pins for jittered 3D meshes (irregular tetrahedral meshes standing in
for the paper's Sphere meshes, Table 1): vertex i/cells moved by (2u-1)h/8 per
coordinate (streams 0, 1, 3), the Kuhn split kept.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle as O


def _base(s, cells):
    V = cells + 1
    v = np.arange(s.n_vertices)
    idx = np.stack([v % V, (v // V) % V, v // (V * V)], 1)
    return idx, idx / cells


def test_jitter3d_matches_definition_and_bounds():
    cells, seed = 8, 6
    s = O.System(3, 1, cells, jitter=1, seed=seed)
    X = s.vertex_coords()
    idx, base = _base(s, cells)
    h = 1.0 / cells
    onb = np.any((idx == 0) | (idx == cells), axis=1)
    d = X - base
    assert np.all(d[onb] == 0.0)
    assert np.all(np.abs(d[~onb]) <= 0.125 * h + 1e-17)
    assert d[~onb].std() > 0.05 * h
    for v in np.flatnonzero(~onb)[:25]:
        for axis, stream in enumerate((0, 1, 3)):
            u = (O.rng_u64(O.rng_key(seed, stream), int(v)) >> 11) * 2.0 ** -53
            want = idx[v, axis] / cells + (2.0 * u - 1.0) * (0.125 / cells)
            assert X[v, axis] == want


def test_jitter3d_tets_keep_positive_volume():
    """No Kuhn tetrahedron inverts at amplitude h/8: the determinant of its edge
    vectors is affine in each vertex's displacement, so over the jitter box it is
    smallest at box corners, where it is >= h^3/4 (volume >= h^3/24)."""
    cells = 6
    h = 1.0 / cells
    s = O.System(3, 1, cells, jitter=1, seed=2)
    X = s.vertex_coords()
    E = s.elements()
    P = X[E]
    D = np.linalg.det(np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], 1))
    # the unjittered edge vectors: jitter < h/2, so rounding to the lattice recovers them
    Dreg = np.linalg.det(np.stack([np.round((P[:, j] - P[:, 0]) * cells) / cells for j in (1, 2, 3)], 1))
    assert np.all(np.sign(D) == np.sign(Dreg))
    assert np.abs(D).min() >= h ** 3 / 4 * (1 - 1e-12)
    # the corner bound itself, by exhaustion for one Kuhn tetrahedron
    corners = np.array(list(itertools.product([-1, 1], repeat=3)), float) * 0.125
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]], float)
    worst = min(np.linalg.det(np.stack([W[1] - W[0], W[2] - W[0], W[3] - W[0]]))
                for W in (V + corners[list(c)] for c in itertools.product(range(8), repeat=4)))
    assert worst == pytest.approx(0.25)


@pytest.mark.parametrize("deg", [1, 2])
def test_jitter3d_pattern_and_matrix_properties(deg):
    cells = 3
    sj = O.System(3, deg, cells, jitter=1, seed=4).assemble()
    sr = O.System(3, deg, cells, jitter=0, seed=4).assemble()
    rpj, cij, vj = sj.full()
    rpr, cir, _ = sr.full()
    # topology unchanged: the structural pattern is the regular one, and it is
    # the set of dof pairs sharing an element
    assert np.array_equal(rpj, rpr) and np.array_equal(cij, cir)
    pairs = {(int(a), int(b)) for el in sj.elements() for a in el for b in el}
    got = {(i, int(j)) for i in range(sj.n_dof) for j in cij[rpj[i]:rpj[i + 1]]}
    assert got == pairs
    A = np.zeros((sj.n_dof, sj.n_dof))
    for i in range(sj.n_dof):
        A[i, cij[rpj[i]:rpj[i + 1]]] = vj[rpj[i]:rpj[i + 1]]
    assert np.array_equal(A, A.T)
    assert np.abs(A.sum(1)).max() < 1e-12 * np.abs(A).max()
    _, _, foff, _ = sj.maps()
    assert np.linalg.eigvalsh(A[np.ix_(foff, foff)]).min() > 0
    # and the values do change with the jitter
    _, _, vr = sr.full()
    assert np.abs(vj - vr).max() > 1e-3 * np.abs(vr).max()


def test_jitter3d_p1_not_exact_on_quadratics():
    """The regular Kuhn P1 matrix is the 7-point stencil, exact on quadratics; on a
    jittered mesh P1 is not (the exact-reproduction pins above are not vacuous)."""
    s, b, x, info = O.solve_system(3, 1, 6, jitter=1, seed=3, gid=O.G_X2_Y2_2Z2, tol=1e-14)
    u = s.eval_g(O.G_X2_Y2_2Z2, None, 1, "free")[:, 0]
    assert O.x_err(u, x[:, 0]) > 1e-6
