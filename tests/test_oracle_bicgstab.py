"""Pins of the oracle's BiCGSTAB (the paper's Krylov method, Sec. 3.2; right
preconditioning with Jacobi or block-Jacobi) against facts that do not depend
on the oracle:

- on the SPD systems it reaches the Cholesky solution;
- with the exact preconditioner (one block-Jacobi block holding every row,
  M = A) the first step solves the system: one iteration;
- on tiny systems it terminates within n steps (each step contains a BiCG
  step, and BiCG terminates in at most n in exact arithmetic);
- it does not rely on symmetry: on a non-symmetric matrix (the SPD matrix plus
  an antisymmetric part on its pattern, a convection-like term) it reaches
  numpy's dense solution;
- b = 0 gives x = 0 without iterating.
"""
import numpy as np
import pytest

import oracle as O


def _K(case):
    s = O.System(*case).assemble()
    return s, *s.k_ii()


def _gid(dim):
    return O.G_X2_Y2_2Z2 if dim == 3 else O.G_X2_Y2


@pytest.mark.parametrize("case,bs", [((2, 1, 30, 1, 1, 3), 0), ((2, 2, 14, 1, 1, 2), 0), ((3, 1, 10, 1, 0, 5), 0),
                                     ((2, 2, 14, 1, 1, 2), 4), ((3, 2, 5, 1, 0, 1), 8)])
def test_spd_reaches_cholesky(case, bs):
    s, rp, ci, v = _K(case)
    b = s.lift(s.eval_g(_gid(case[0])))[:, 0]
    x, st, it, rel = O.bicgstab(rp, ci, v, b, tol=1e-12, bs=bs)
    assert st == 0 and rel <= 1e-12
    assert O.x_err(O.cholesky_solve(rp, ci, v, b), x) <= 1e-9


@pytest.mark.parametrize("case,bs", [((2, 1, 5, 1, 1, 7), 16), ((2, 2, 3, 1, 1, 2), 32), ((3, 1, 3, 0, 0, 0), 8)])
def test_exact_preconditioner_one_step(case, bs):
    s, rp, ci, v = _K(case)
    assert len(rp) - 1 <= bs
    b = s.lift(s.eval_g(_gid(case[0])))[:, 0]
    x, st, it, rel = O.bicgstab(rp, ci, v, b, tol=1e-13, bs=bs)
    assert st == 0 and it == 1
    assert O.x_err(O.cholesky_solve(rp, ci, v, b), x) <= 1e-13


@pytest.mark.parametrize("case", [(2, 1, 5, 1, 1, 7), (2, 1, 4, 0, 0, 0), (3, 1, 3, 1, 0, 2), (2, 2, 3, 1, 1, 1)])
def test_tiny_systems_terminate(case):
    s, rp, ci, v = _K(case)
    n = len(rp) - 1
    b = np.random.default_rng(n).standard_normal(n)
    x, st, it, rel = O.bicgstab(rp, ci, v, b, tol=1e-11)
    assert st == 0 and it <= n + 2


@pytest.mark.parametrize("case,c,bs", [((2, 1, 16, 1, 1, 4), 0.3, 0), ((2, 2, 8, 1, 1, 2), 0.5, 0),
                                       ((2, 2, 8, 1, 1, 2), 0.9, 0), ((3, 1, 6, 1, 0, 3), 0.2, 0)])
def test_nonsymmetric_matrix(case, c, bs):
    """K + c S with S antisymmetric on K's pattern (S_ij = -S_ji = |K_ij| for
    i < j): a non-symmetric matrix whose symmetric part is K, so it is
    nonsingular.  (Jacobi only: the block-Jacobi blocks are inverted by
    Cholesky, for the method's SPD matrices.)"""
    s, rp, ci, v = _K(case)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    sgn = np.sign(ci - rows)  # +1 above the diagonal, -1 below
    v2 = v + c * sgn * np.abs(v)
    A = np.zeros((n, n))
    A[rows, ci] = v2
    assert not np.allclose(A, A.T)
    b = np.random.default_rng(5).standard_normal(n)
    x, st, it, rel = O.bicgstab(rp, ci, v2, b, tol=1e-12, bs=bs)
    assert st == 0 and rel <= 1e-12
    xd = np.linalg.solve(A, b)
    assert O.x_err(xd, x) <= 1e-8


def test_zero_rhs():
    s, rp, ci, v = _K((2, 1, 10, 1, 1, 1))
    x, st, it, rel = O.bicgstab(rp, ci, v, np.zeros(len(rp) - 1), x0=np.ones(len(rp) - 1))
    assert st == 0 and it == 0 and np.all(x == 0)
