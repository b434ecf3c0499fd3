"""Oracle pins: counter-based RNG, mesh generation, dof numbering (CPU only)."""
import os

import numpy as np
import pytest

import oracle as O
from conftest import read_golden


def test_splitmix64_published_vector(golden_dir):
    want = [int(r[0]) for r in read_golden(os.path.join(golden_dir, "splitmix64_seed1234567.txt"))]
    got = [O.rng_u64(1234567, i) for i in range(len(want))]
    assert got == want


def test_rng_key_layout():
    assert O.rng_key(0, 0) == 0
    assert O.rng_key(1, 0) == 1 << 40
    assert O.rng_key(0, 2) == 2 << 32
    assert O.rng_key(3, 1) == (3 << 40) ^ (1 << 32)


@pytest.mark.parametrize("cells", [1, 3, 8])
def test_regular_2d_coordinates_exact(cells):
    s = O.System(2, 1, cells)
    X = s.vertex_coords()
    V = cells + 1
    i = np.arange(s.n_vertices) % V
    j = np.arange(s.n_vertices) // V
    assert np.array_equal(X[:, 0], i / cells)
    assert np.array_equal(X[:, 1], j / cells)


def test_jitter_bounds_and_boundary_fixed():
    cells = 32
    s = O.System(2, 1, cells, jitter=1, diag_mode=1, seed=7)
    X = s.vertex_coords()
    V = cells + 1
    i = np.arange(s.n_vertices) % V
    j = np.arange(s.n_vertices) // V
    base = np.stack([i / cells, j / cells], 1)
    d = X - base
    h = 1.0 / cells
    onb = (i == 0) | (i == cells) | (j == 0) | (j == cells)
    assert np.all(d[onb] == 0.0)
    assert np.all(np.abs(d[~onb]) <= 0.25 * h + 1e-17)
    # the jitter uses the whole range: not a constant shift
    assert d[~onb].std() > 0.1 * h


def test_jitter_matches_definition():
    """x = i/cells + (2u-1)*(0.25/cells), u = top 53 bits of stream 0 (x) / 1 (y)."""
    cells, seed = 16, 5
    s = O.System(2, 1, cells, jitter=1, diag_mode=0, seed=seed)
    X = s.vertex_coords()
    V = cells + 1
    for v in [V + 1, 5 * V + 7, (cells - 1) * V + cells - 1]:
        i, j = v % V, v // V
        for d, (idx, stream) in enumerate([(i, 0), (j, 1)]):
            u = (O.rng_u64(O.rng_key(seed, stream), v) >> 11) * 2.0 ** -53
            want = idx / cells + (2.0 * u - 1.0) * (0.25 / cells)
            assert X[v, d] == want


def test_triangles_positive_area_and_cover_square():
    s = O.System(2, 1, 24, jitter=1, diag_mode=1, seed=3)
    X = s.vertex_coords()
    E = s.elements()
    a = X[E[:, 1]] - X[E[:, 0]]
    b = X[E[:, 2]] - X[E[:, 0]]
    area = 0.5 * (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    assert np.all(area > 0)
    assert abs(area.sum() - 1.0) < 1e-13


def test_diagonal_flip_rate():
    cells = 64
    s = O.System(2, 1, cells, jitter=0, diag_mode=1, seed=11)
    E = s.elements()
    V = cells + 1
    # first triangle of cell c is (v00, v10, v11) unflipped, (v00, v10, v01) flipped
    flipped = E[0::2, 2] == E[0::2, 0] + V
    p = flipped.mean()
    assert 0.45 < p < 0.55
    # the rule: flip iff the stream-2 draw has its top bit clear (u < 1/2)
    k = O.rng_key(11, 2)
    want = np.array([(O.rng_u64(k, c) >> 63) == 0 for c in range(cells * cells)])
    assert np.array_equal(flipped, want)


def test_kuhn_tets_volume_and_count():
    n = 5
    s = O.System(3, 1, n)
    X = s.vertex_coords()
    E = s.elements()
    assert E.shape == (6 * n ** 3, 4)
    M = np.stack([X[E[:, k]] - X[E[:, 0]] for k in (1, 2, 3)], axis=2)
    vol = np.abs(np.linalg.det(M)) / 6.0
    assert np.allclose(vol, 1.0 / (6 * n ** 3), rtol=1e-12)
    assert abs(vol.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("dim,degree,cells", [(2, 1, 6), (2, 2, 6), (3, 1, 4), (3, 2, 3)])
def test_dof_counts_and_boundary(dim, degree, cells):
    s = O.System(dim, degree, cells, jitter=1 if dim == 2 else 0, diag_mode=1, seed=2)
    S = degree * cells + 1
    assert s.n_dof == S ** dim
    assert s.n_free == (S - 2) ** dim
    assert s.n_bnd == S ** dim - (S - 2) ** dim
    fof, bof, foff, fofb = s.maps()
    assert np.array_equal(np.sort(np.concatenate([foff, fofb])), np.arange(s.n_dof))
    assert np.all(np.diff(foff) > 0) and np.all(np.diff(fofb) > 0)
    X = s.dof_coords()
    on_b = np.any((X < 1e-14) | (X > 1 - 1e-14), axis=1)
    assert np.array_equal(np.where(on_b)[0], fofb)


def test_p2_midpoints_are_edge_means():
    s = O.System(2, 2, 8, jitter=1, diag_mode=1, seed=9)
    X = s.dof_coords()
    E = s.elements()
    for a, b, m in [(0, 1, 3), (0, 2, 4), (1, 2, 5)]:
        assert np.array_equal(X[E[:, m]], (X[E[:, a]] + X[E[:, b]]) * 0.5)
    # every dof of the doubled lattice belongs to some element
    assert np.array_equal(np.unique(E), np.arange(s.n_dof))


def test_bad_specs_rejected():
    with pytest.raises(ValueError):
        O.System(4, 1, 4)
    with pytest.raises(ValueError):
        O.System(2, 5, 4)  # degrees 1..4
