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
- b = 0 gives x = 0 without iterating;
- a breakdown (a zero shadow product) after the residual has fallen restarts
  the recurrence from the true residual with a new shadow vector and reaches
  the dense solution; a breakdown before the residual has fallen below 0.9 of
  the starting one is reported (status 2) instead of restarting forever.  Both
  cases are 3x3 / 2x2 matrices built so that the zero happens exactly, in
  every rounding order, at a known step.
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


def dense_csr(A):
    """CSR of a small dense matrix (its diagonal always stored)."""
    n = A.shape[0]
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0.0 or i == j:
                ci.append(j)
                v.append(A[i, j])
        rp.append(len(ci))
    return np.array(rp, np.int64), np.array(ci, np.int32), np.array(v)


# Breakdown after progress.  Row 0 of A is e0^T and b = e0, so the first step
# has alpha = (b.b)/(b.Ab) = 1 and s = b - Ab with s_0 = 0; then t_0 = (As)_0
# = s_0 = 0 and the new residual r = s - omega t has r_0 = 0, so the next
# shadow product rho = b.r = r_0 is exactly zero (rounding cannot change a
# sum of exact zeros).  omega = 0.8 and ||r|| = sqrt(0.1) < 0.9 ||b||: the
# residual has fallen, the recurrence restarts from x = (1, -0.4, -0.4) and,
# with r_0 = 0, runs on the 2x2 block [[1, 0.5], [-0.5, 1]] (BiCG there ends
# within two steps).  Solution: (1, -0.2, -0.6).
BREAK_AFTER_PROGRESS = np.array([[1.0, 0.0, 0.0], [0.5, 1.0, 0.5], [0.5, -0.5, 1.0]])
BREAK_AFTER_PROGRESS_B = np.array([1.0, 0.0, 0.0])
BREAK_AFTER_PROGRESS_X = np.array([1.0, -0.2, -0.6])

# Breakdown before progress.  A = [[1, 2], [0, -1]], Jacobi M^-1 = diag(1, -1),
# b = (1, 1): p = b, ph = (1, -1), v = A ph = (-1, 1) and rho_hat.v = b.v = 0
# exactly in the first step.  The true residual is still ||b||: nothing to
# restart from, so the solve reports a breakdown after 0 steps.
BREAK_AT_ONCE = np.array([[1.0, 2.0], [0.0, -1.0]])
BREAK_AT_ONCE_B = np.array([1.0, 1.0])


def test_breakdown_after_progress_restarts_to_the_solution():
    rp, ci, v = dense_csr(BREAK_AFTER_PROGRESS)
    assert np.allclose(np.linalg.solve(BREAK_AFTER_PROGRESS, BREAK_AFTER_PROGRESS_B), BREAK_AFTER_PROGRESS_X,
                       rtol=0, atol=1e-15)
    x, st, it, rel = O.bicgstab(rp, ci, v, BREAK_AFTER_PROGRESS_B, tol=1e-13)
    assert st == 0 and rel <= 1e-13
    # one step before the breakdown, at most two on the 2x2 block after it
    assert 2 <= it <= 3
    assert np.abs(x - BREAK_AFTER_PROGRESS_X).max() <= 1e-14


def test_breakdown_without_progress_is_reported():
    rp, ci, v = dense_csr(BREAK_AT_ONCE)
    x, st, it, rel = O.bicgstab(rp, ci, v, BREAK_AT_ONCE_B, tol=1e-12)
    assert st == 2 and it == 0
    assert np.all(x == 0.0) and rel == 1.0
