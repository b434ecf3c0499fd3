"""GPU parity: BiCGSTAB (the paper's Krylov method, Sec. 3.2), right-
preconditioned with Jacobi or block-Jacobi, against the oracle's BiCGSTAB and
the exact solutions.

Bar: Eq. (2) at 1e-10 (recomputed here in fp64 from the oracle's matrix),
Eq. (1) error <= 1e-8 against the oracle's solution at 1e-13, and the oracle's
step count up to rounding drift (BiCGSTAB's residual is not monotone and its
true-residual restarts depend on rounding, so the drift is allowed 15 %); one step with the exact preconditioner; tiny systems
within n steps; graph and direct launches give the same bits; the restart
after a breakdown (and the breakdown report when the residual has not fallen)
on matrices where the zero is exact, with the oracle's step and restart
counts; non-symmetric matrices against the oracle."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-10
XERR = 1e-8


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05413_gb300 as P
    P.load()
    return P


def _gid(dim):
    return O.G_X2_Y2_2Z2 if dim == 3 else O.G_X2_Y2


def _solve(P, case, bs, tol=TOL, **kw):
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256)
    opts = {"method": P.GB_BICGSTAB}
    if bs:
        A.block_jacobi(bs)
        opts["precond"] = P.GB_PC_BLOCK_JACOBI
    b = d.lift(d.dirichlet(_gid(case[0])))[:, 0]
    opts.update(kw)
    x, st = A.solve(b, tol=tol, max_iter=200000, **opts)
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    bo = s.lift(s.eval_g(_gid(case[0])))[:, 0]
    return d, A, b, x, st, (rp, ci, v), bo


@pytest.mark.parametrize("case,bs", [
    ((2, 1, 64, 0, 0, 0), 0), ((2, 1, 96, 1, 1, 1), 0), ((2, 2, 48, 1, 1, 1), 0), ((3, 1, 20, 1, 0, 2), 0),
    ((3, 2, 10, 0, 0, 0), 0), ((2, 2, 48, 1, 1, 1), 4), ((2, 1, 96, 1, 1, 1), 2), ((3, 2, 8, 1, 0, 3), 8)])
def test_matches_oracle(P, case, bs):
    d, A, b, x, st, K, bo = _solve(P, case, bs)
    rp, ci, v = K
    xd = x.cpu().numpy()
    assert st["status"] == 0 and st["relres"] <= TOL
    assert np.linalg.norm(bo - O.spmv(rp, ci, v, xd)) / np.linalg.norm(bo) <= 1.5 * TOL
    xe = O.pcg(rp, ci, v, bo, tol=1e-13)[0]
    assert O.x_err(xe, xd) <= XERR
    xo, sto, ito, _ = O.bicgstab(rp, ci, v, bo, tol=TOL, bs=bs)
    assert sto == 0
    assert abs(st["iterations"] - ito) <= max(5, 0.15 * ito), (st["iterations"], st["restarts"], ito)


@pytest.mark.parametrize("case,bs", [((2, 1, 5, 1, 1, 7), 16), ((2, 2, 3, 1, 1, 2), 32), ((3, 1, 3, 0, 0, 0), 8)])
def test_exact_preconditioner_one_step(P, case, bs):
    d, A, b, x, st, K, bo = _solve(P, case, bs, tol=1e-13)
    assert st["status"] == 0 and st["iterations"] == 1
    assert O.x_err(O.cholesky_solve(*K, bo), x.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("case", [(2, 1, 5, 1, 1, 7), (2, 1, 4, 0, 0, 0), (3, 1, 3, 1, 0, 2), (2, 2, 3, 1, 1, 1)])
def test_tiny_systems_terminate(P, case):
    d, A, b, x, st, K, bo = _solve(P, case, 0, tol=1e-11)
    assert st["status"] == 0 and st["iterations"] <= d.n_free + 2


def test_zero_rhs_and_graph_vs_direct(P):
    import torch
    d = P.FemSystem(2, 2, 40, 1, 1, 3)
    A = d.to_sell(32, 256)
    x, st = A.solve(torch.zeros(d.n_free, dtype=torch.float64, device="cuda"), method=P.GB_BICGSTAB)
    assert st["status"] == 0 and st["iterations"] == 0 and bool((x == 0).all())
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    x1, s1 = A.solve(b, tol=TOL, method=P.GB_BICGSTAB)
    x2, s2 = A.solve(b, tol=TOL, method=P.GB_BICGSTAB, use_graph=0)
    assert s1["iterations"] == s2["iterations"] and bool((x1 == x2).all())


def test_bad_arguments(P):
    d = P.FemSystem(2, 1, 20, 1, 1, 2)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    with pytest.raises(P.GbError):
        A.solve(b, method=P.GB_BICGSTAB, precision=P.GB_F32_IR)
    with pytest.raises(P.GbError):
        d.to_sell(64, 256).solve(b, method=P.GB_BICGSTAB)
    with pytest.raises(P.GbError):
        A.solve(b, method=5)
    with pytest.raises(P.GbError):
        P.pcg_solve_batched([A], [b], method=P.GB_BICGSTAB)


def _raw(P, rp, ci, v):
    import torch
    return P.Sell.from_csr(torch.tensor(rp, dtype=torch.int32, device="cuda"),
                           torch.tensor(ci, dtype=torch.int32, device="cuda"),
                           torch.tensor(v, dtype=torch.float64, device="cuda"), 32, 256)


def test_breakdown_after_progress_restarts_like_the_oracle(P):
    """The matrix whose second shadow product is exactly zero (after the
    residual fell to sqrt(0.1)): the device restarts once from the true
    residual, as the oracle does, and reaches the dense solution."""
    import torch
    from test_oracle_bicgstab import (BREAK_AFTER_PROGRESS, BREAK_AFTER_PROGRESS_B, BREAK_AFTER_PROGRESS_X,
                                      dense_csr)
    rp, ci, v = dense_csr(BREAK_AFTER_PROGRESS)
    A = _raw(P, rp, ci, v)
    b = torch.tensor(BREAK_AFTER_PROGRESS_B, device="cuda")
    x, st = A.solve(b, tol=1e-13, max_iter=100, method=P.GB_BICGSTAB)
    xo, sto, ito, _ = O.bicgstab(rp, ci, v, BREAK_AFTER_PROGRESS_B, tol=1e-13)
    assert st["status"] == 0 and sto == 0
    assert st["restarts"] == 1
    assert st["iterations"] == ito
    assert np.abs(x.cpu().numpy() - BREAK_AFTER_PROGRESS_X).max() <= 1e-14
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-14


def test_breakdown_without_progress_is_reported_like_the_oracle(P):
    """rho_hat.v exactly zero in the first step: GB_BREAKDOWN after 0 steps,
    x = x0 = 0, on both sides."""
    import torch
    from test_oracle_bicgstab import BREAK_AT_ONCE, BREAK_AT_ONCE_B, dense_csr
    rp, ci, v = dense_csr(BREAK_AT_ONCE)
    A = _raw(P, rp, ci, v)
    b = torch.tensor(BREAK_AT_ONCE_B, device="cuda")
    x, st = A.solve(b, tol=1e-12, max_iter=100, method=P.GB_BICGSTAB, raise_on_fail=False)
    xo, sto, ito, relo = O.bicgstab(rp, ci, v, BREAK_AT_ONCE_B, tol=1e-12)
    assert sto == 2 and ito == 0
    assert st["rc"] == P.gbpcg.GB_BREAKDOWN and st["status"] == P.gbpcg.GB_BREAKDOWN
    assert st["iterations"] == 0 and st["restarts"] == 0
    assert bool((x == 0).all()) and abs(st["relres"] - relo) <= 1e-15


@pytest.mark.parametrize("case,c", [((2, 1, 16, 1, 1, 4), 0.3), ((2, 2, 8, 1, 1, 2), 0.5),
                                    ((2, 2, 8, 1, 1, 2), 0.9), ((3, 1, 6, 1, 0, 3), 0.2),
                                    ((2, 1, 64, 1, 1, 5), 0.5), ((2, 2, 40, 1, 1, 6), 0.7)])
def test_nonsymmetric_matrix_matches_oracle(P, case, c):
    """K + c S with S antisymmetric on K's pattern (S_ij = -S_ji = |K_ij| for
    i < j), a convection-like non-symmetric matrix with K as its symmetric
    part: the device BiCGSTAB (Jacobi on the right) against the oracle's
    BiCGSTAB at 1e-13, itself checked against numpy's dense solve where n <= 2000."""
    import torch
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    v2 = v + c * np.sign(ci - rows) * np.abs(v)
    b = np.random.default_rng(5).standard_normal(n)
    A = _raw(P, rp, ci, v2)
    x, st = A.solve(torch.tensor(b, device="cuda"), tol=TOL, max_iter=20 * n + 100, method=P.GB_BICGSTAB)
    xd = x.cpu().numpy()
    assert st["status"] == 0
    assert np.linalg.norm(b - O.spmv(rp, ci, v2, xd)) / np.linalg.norm(b) <= 1.5 * TOL
    xo, sto, ito, _ = O.bicgstab(rp, ci, v2, b, tol=1e-13)
    assert sto == 0
    if n <= 2000:
        M = np.zeros((n, n))
        M[rows, ci] = v2
        assert O.x_err(np.linalg.solve(M, b), xo) <= 1e-11
    assert O.x_err(xo, xd) <= XERR
    xo10, sto10, ito10, _ = O.bicgstab(rp, ci, v2, b, tol=TOL)
    assert abs(st["iterations"] - ito10) <= max(5, 0.15 * ito10), (st["iterations"], ito10)
