"""Pins of the oracle's block-Jacobi preconditioner (the paper's Block-Jacobi,
Sec. 3.2 and Sec. 4.2) against facts that do not depend on the oracle:

- each stored block times the matrix's diagonal block is the identity, and the
  blocks are symmetric;
- on the regular meshes the diagonal blocks are direct sums of tridiagonal
  Toeplitz matrices (the x-lines of the 5-point and 7-point stencils), whose
  inverses have the closed form
  (T^-1)_ij = sinh(i t) sinh((m+1-j) t) / (d sinh(t) sinh((m+1) t)), i <= j,
  for T = d tridiag(-1, 2 cosh t, -1), 1-based indices;
- bs = 1 is the Jacobi preconditioner; one block holding every row makes PCG
  a direct solver (one iteration, the Cholesky solution);
- (M^-1 K v)_B = v_B for v supported on one block B, short last block included.
"""
import numpy as np
import pytest

import oracle as O


def _K(case):
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    return s, rp, ci, v


def _dense_block(rp, ci, v, s0, m):
    B = np.zeros((m, m))
    for a in range(m):
        for k in range(rp[s0 + a], rp[s0 + a + 1]):
            if s0 <= ci[k] < s0 + m:
                B[a, ci[k] - s0] = v[k]
    return B


@pytest.mark.parametrize("case,bs", [
    ((2, 1, 10, 1, 1, 3), 4), ((2, 2, 7, 1, 1, 2), 8), ((3, 1, 6, 1, 0, 4), 16),
    ((3, 2, 3, 0, 0, 0), 32), ((2, 1, 12, 0, 0, 0), 2)])
def test_blocks_are_inverses(case, bs):
    _, rp, ci, v = _K(case)
    n = len(rp) - 1
    W = O.bjacobi(rp, ci, v, bs)
    assert W.shape == ((n + bs - 1) // bs, bs, bs)
    assert n % bs != 0  # the short last block is exercised
    for j in range(W.shape[0]):
        m = min(bs, n - j * bs)
        B = _dense_block(rp, ci, v, j * bs, m)
        Wj = W[j]
        assert np.all(Wj[m:, :] == 0) and np.all(Wj[:, m:] == 0)
        cond = np.linalg.cond(B)
        assert np.allclose(Wj[:m, :m] @ B, np.eye(m), atol=1e-14 * cond)
        assert np.allclose(Wj[:m, :m], Wj[:m, :m].T, rtol=0, atol=1e-14 * cond * np.abs(Wj).max())


def _tridiag_inverse(m, d, cosh_t):
    t = np.arccosh(cosh_t)
    T = np.zeros((m, m))
    for i in range(1, m + 1):
        for j in range(i, m + 1):
            T[i - 1, j - 1] = T[j - 1, i - 1] = (np.sinh(i * t) * np.sinh((m + 1 - j) * t)
                                                 / (d * np.sinh(t) * np.sinh((m + 1) * t)))
    return T


@pytest.mark.parametrize("dim,cells,bs", [(2, 10, 4), (2, 20, 16), (2, 33, 8), (3, 6, 4), (3, 18, 16)])
def test_regular_blocks_closed_form(dim, cells, bs):
    """Regular P1: 5-point (4, -1) in 2D, h (6, -1) in 3D.  Rows of one x-line
    (cells - 1 free unknowns per line) form tridiagonal segments; with bs at
    most the line length, unknowns of different lines inside one block are not
    coupled."""
    _, rp, ci, v = _K((dim, 1, cells, 0, 0, 0))
    n = len(rp) - 1
    line = cells - 1
    assert bs <= line
    h = 1.0 / cells
    d, cosh_t = (1.0, 2.0) if dim == 2 else (h, 3.0)
    W = O.bjacobi(rp, ci, v, bs)
    for j in range(W.shape[0]):
        s0 = j * bs
        m = min(bs, n - s0)
        want = np.zeros((m, m))
        a = 0
        while a < m:
            seg = min(m - a, line - (s0 + a) % line)  # to the end of the x-line
            want[a:a + seg, a:a + seg] = _tridiag_inverse(seg, d, cosh_t)
            a += seg
        assert np.allclose(W[j][:m, :m], want, rtol=1e-12, atol=1e-15 * np.abs(want).max())


@pytest.mark.parametrize("case", [(2, 1, 20, 1, 1, 5), (2, 2, 9, 1, 1, 1), (3, 1, 6, 1, 0, 2)])
def test_bs1_is_jacobi(case):
    s, rp, ci, v = _K(case)
    n = len(rp) - 1
    W = O.bjacobi(rp, ci, v, 1)
    diag = np.array([v[rp[i]:rp[i + 1]][ci[rp[i]:rp[i + 1]] == i][0] for i in range(n)])
    assert np.allclose(W[:, 0, 0], 1.0 / diag, rtol=4e-16, atol=0)
    gid = O.G_X2_Y2_2Z2 if case[0] == 3 else O.G_X2_Y2
    b = s.lift(s.eval_g(gid))[:, 0]
    x1, st1, it1, _ = O.pcg(rp, ci, v, b, tol=1e-12)
    x2, st2, it2, _ = O.pcg(rp, ci, v, b, tol=1e-12, bs=1)
    assert st1 == st2 == 0
    assert abs(it1 - it2) <= 1
    assert O.x_err(x1, x2) <= 1e-10


@pytest.mark.parametrize("case,bs", [((2, 1, 5, 1, 1, 7), 16), ((2, 1, 5, 1, 1, 7), 32),
                                     ((3, 1, 3, 0, 0, 0), 8), ((2, 2, 3, 1, 1, 2), 32)])
def test_one_block_is_a_direct_solve(case, bs):
    s, rp, ci, v = _K(case)
    n = len(rp) - 1
    assert n <= bs
    gid = O.G_X2_Y2_2Z2 if case[0] == 3 else O.G_LINEAR
    coef = None if gid != O.G_LINEAR else np.array([[0.3, -1.0, 2.0, 0.5]])
    b = s.lift(s.eval_g(gid, coef))[:, 0]
    x, st, it, rel = O.pcg(rp, ci, v, b, tol=1e-13, bs=bs)
    assert st == 0 and it == 1
    xc = O.cholesky_solve(rp, ci, v, b)
    assert O.x_err(xc, x) <= 1e-13


@pytest.mark.parametrize("case,bs", [((2, 2, 6, 1, 1, 3), 8), ((3, 1, 5, 1, 0, 1), 4), ((2, 1, 11, 0, 1, 2), 16)])
def test_apply_inverts_each_block(case, bs):
    _, rp, ci, v = _K(case)
    n = len(rp) - 1
    W = O.bjacobi(rp, ci, v, bs)
    rng = np.random.default_rng(0)
    for j in range(W.shape[0]):
        s0, m = j * bs, min(bs, n - j * bs)
        x = np.zeros(n)
        x[s0:s0 + m] = rng.standard_normal(m)
        z = O.bjacobi_apply(bs, W, O.spmv(rp, ci, v, x))
        assert np.allclose(z[s0:s0 + m], x[s0:s0 + m], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("case,bs", [((2, 2, 10, 1, 1, 4), 4), ((3, 2, 4, 1, 0, 3), 8), ((2, 1, 30, 1, 1, 8), 32)])
def test_bj_pcg_reaches_the_cholesky_solution(case, bs):
    s, rp, ci, v = _K(case)
    gid = O.G_X2_Y2_2Z2 if case[0] == 3 else O.G_X2_Y2
    b = s.lift(s.eval_g(gid))[:, 0]
    x, st, it, rel = O.pcg(rp, ci, v, b, tol=1e-13, bs=bs)
    assert st == 0 and rel <= 1e-13
    assert O.x_err(O.cholesky_solve(rp, ci, v, b), x) <= 1e-10


def test_bj_fewer_iterations_in_2d():
    s, rp, ci, v = _K((2, 2, 32, 1, 1, 1))
    b = s.lift(s.eval_g(O.G_X2_Y2))[:, 0]
    its = {bs: O.pcg(rp, ci, v, b, tol=1e-10, bs=bs)[2] for bs in (1, 4, 16)}
    assert its[4] < 0.9 * its[1] and its[16] <= its[4]
