"""Pins of the oracle's block CG (the block of right-hand sides of Sec. 4.3,
A X = B, solved in one shared Krylov space) against facts that do not depend
on the oracle:

- k = 1 is PCG (same iterates in exact arithmetic: iteration count within one,
  same solution);
- finite termination: the block Krylov space of k independent columns fills
  R^n after ceil(n/k) steps, so tiny systems converge to rounding in that many
  steps;
- every column equals the Cholesky solution;
- a rank-deficient block (repeated, combined and zero columns) still
  converges, to the same combinations of the solutions, with a zero column
  giving exactly zero;
- the shared space never needs more steps than the slowest column alone.
"""
import math

import numpy as np
import pytest

import oracle as O


def _K(case):
    s = O.System(*case).assemble()
    return s, *s.k_ii()


@pytest.mark.parametrize("case", [(2, 1, 24, 1, 1, 3), (2, 2, 10, 1, 1, 2), (3, 1, 8, 1, 0, 5)])
def test_k1_is_pcg(case):
    s, rp, ci, v = _K(case)
    gid = O.G_X2_Y2_2Z2 if case[0] == 3 else O.G_X2_Y2
    b = s.lift(s.eval_g(gid))[:, 0]
    X, st, it, rel = O.block_cg(rp, ci, v, b[:, None], tol=1e-12)
    x, stp, itp, _ = O.pcg(rp, ci, v, b, tol=1e-12)
    assert st == 0 and stp == 0 and rel[0] <= 1e-12
    assert abs(it - itp) <= 1
    assert O.x_err(x, X[:, 0]) <= 1e-10


@pytest.mark.parametrize("case,k", [((2, 1, 5, 1, 1, 7), 4), ((2, 1, 5, 1, 1, 7), 5), ((2, 2, 4, 1, 1, 1), 7),
                                    ((3, 1, 4, 0, 0, 0), 9), ((3, 1, 5, 1, 0, 2), 16)])
def test_finite_termination(case, k):
    s, rp, ci, v = _K(case)
    n = len(rp) - 1
    B = np.random.default_rng(k).standard_normal((n, k))
    X, st, it, rel = O.block_cg(rp, ci, v, B, tol=1e-11)
    assert st == 0 and rel.max() <= 1e-11
    assert it <= math.ceil(n / k) + 1


@pytest.mark.parametrize("case,k", [((2, 2, 8, 1, 1, 4), 3), ((3, 2, 3, 1, 0, 6), 6), ((2, 1, 20, 0, 1, 9), 8)])
def test_columns_are_cholesky_solutions(case, k):
    s, rp, ci, v = _K(case)
    n = len(rp) - 1
    B = np.random.default_rng(1).standard_normal((n, k))
    X, st, it, rel = O.block_cg(rp, ci, v, B, tol=1e-12)
    assert st == 0
    for j in range(k):
        assert O.x_err(O.cholesky_solve(rp, ci, v, B[:, j]), X[:, j]) <= 1e-9


def test_rank_deficient_block():
    s, rp, ci, v = _K((2, 2, 12, 1, 1, 5))
    n = len(rp) - 1
    rng = np.random.default_rng(3)
    b1, b2 = rng.standard_normal(n), rng.standard_normal(n)
    B = np.stack([b1, b2, b1, 2 * b1 - b2, np.zeros(n), 3 * b2], axis=1)
    X, st, it, rel = O.block_cg(rp, ci, v, B, tol=1e-11)
    assert st == 0 and rel.max() <= 1e-11
    x1, x2 = O.cholesky_solve(rp, ci, v, b1), O.cholesky_solve(rp, ci, v, b2)
    for j, want in enumerate([x1, x2, x1, 2 * x1 - x2, None, 3 * x2]):
        if want is None:
            assert np.all(X[:, j] == 0.0)
        else:
            assert O.x_err(want, X[:, j]) <= 1e-8
    # two independent columns: no more steps than a 2-column block
    X2, st2, it2, _ = O.block_cg(rp, ci, v, B[:, :2], tol=1e-11)
    assert it <= it2 + 2


def test_harmonic_block_not_slower_than_its_slowest_column():
    """Cfg4-like data: Dirichlet values from the harmonic basis (10
    coefficients per column, Im z^0 = 0), 12 columns of rank at most 9."""
    s, rp, ci, v = _K((2, 2, 16, 1, 1, 2))
    k = 12
    coef = np.random.default_rng(3).standard_normal((k, 10))
    B = s.lift(s.eval_g(O.G_HARMONIC, coef, k))
    X, st, it, rel = O.block_cg(rp, ci, v, B, tol=1e-10)
    assert st == 0 and rel.max() <= 1e-10
    its = [O.pcg(rp, ci, v, B[:, j], tol=1e-10)[2] for j in range(k)]
    assert it <= max(its)
    # P2 reproduces harmonic polynomials of degree <= 2 only: compare with Cholesky
    for j in (0, 5, 11):
        assert O.x_err(O.cholesky_solve(rp, ci, v, B[:, j]), X[:, j]) <= 1e-8
