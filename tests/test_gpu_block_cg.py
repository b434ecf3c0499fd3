"""GPU parity: block CG for A X = B (the block of right-hand sides of Sec. 4.3)
against the oracle's block CG and the exact solutions.

Bar: every column meets Eq. (2) at 1e-10 (recomputed here in fp64 from the
oracle's matrix) and has Eq. (1) error <= 1e-8 against the oracle's exact
solution; the fp64 recurrence takes the oracle's number of steps up to
rounding drift (the rank decisions compare rounded eigenvalues); finite
termination on tiny systems; rank-deficient and zero columns."""
import math

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


def _setup(P, case, k, kind="random", seed=1):
    import torch
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    n = len(rp) - 1
    if kind == "harmonic":
        coef = np.random.default_rng(seed).standard_normal((k, 10))
        Bo = s.lift(s.eval_g(O.G_HARMONIC, coef, k))
        Bd = d.lift(d.dirichlet(O.G_HARMONIC, coef, k))
    else:
        Bo = np.random.default_rng(seed).standard_normal((n, k))
        Bd = torch.tensor(Bo, device="cuda")
    return d, A, (rp, ci, v), np.ascontiguousarray(Bo), Bd


def _check_columns(K, Bo, X, tol=TOL, xerr=XERR):
    rp, ci, v = K
    for j in range(Bo.shape[1]):
        b = Bo[:, j]
        nb = np.linalg.norm(b)
        r = np.linalg.norm(b - O.spmv(rp, ci, v, X[:, j]))
        if nb == 0:
            assert np.all(X[:, j] == 0)
            continue
        assert r / nb <= 1.5 * tol, (j, r / nb)
        xe = O.pcg(rp, ci, v, b, tol=1e-13)[0]
        assert O.x_err(xe, X[:, j]) <= xerr, j


@pytest.mark.parametrize("case,k,kind", [
    ((2, 1, 24, 1, 1, 3), 4, "random"), ((2, 2, 16, 1, 1, 2), 8, "random"), ((3, 1, 10, 1, 0, 5), 16, "random"),
    ((2, 2, 20, 1, 1, 4), 32, "harmonic"), ((3, 2, 5, 0, 0, 0), 3, "random"), ((2, 1, 40, 1, 1, 6), 1, "random"),
    ((2, 2, 12, 1, 1, 7), 12, "harmonic")])
def test_f64_matches_oracle(P, case, k, kind):
    d, A, K, Bo, Bd = _setup(P, case, k, kind)
    X, st = A.solve_block(Bd, tol=TOL)
    Xd = X.cpu().numpy()
    assert st["status"] == 0 and st["relres"] <= TOL
    _check_columns(K, Bo, Xd)
    Xo, sto, ito, relo = O.block_cg(*K, Bo, tol=TOL)
    assert sto == 0
    assert abs(st["iterations"] - ito) <= max(2, 0.05 * ito), (st["iterations"], ito)


@pytest.mark.parametrize("case,k", [((2, 1, 5, 1, 1, 7), 4), ((2, 2, 4, 1, 1, 1), 7), ((3, 1, 4, 0, 0, 0), 9),
                                    ((3, 1, 5, 1, 0, 2), 16), ((2, 1, 8, 1, 1, 3), 32)])
def test_finite_termination(P, case, k):
    d, A, K, Bo, Bd = _setup(P, case, k, seed=k)
    X, st = A.solve_block(Bd, tol=1e-11)
    n = Bo.shape[0]
    assert st["status"] == 0
    assert st["iterations"] <= math.ceil(n / k) + 1
    _check_columns(K, Bo, X.cpu().numpy(), tol=1e-11)


def test_rank_deficient_and_zero_columns(P):
    import torch
    case = (2, 2, 12, 1, 1, 5)
    d, A, K, _, _ = _setup(P, case, 1)
    n = d.n_free
    rng = np.random.default_rng(3)
    b1, b2 = rng.standard_normal(n), rng.standard_normal(n)
    Bo = np.ascontiguousarray(np.stack([b1, b2, b1, 2 * b1 - b2, np.zeros(n), 3 * b2], axis=1))
    for prec in (P.GB_F64, P.GB_F32_IR):
        X, st = A.solve_block(torch.tensor(Bo, device="cuda"), tol=TOL, precision=prec)
        Xd = X.cpu().numpy()
        assert st["status"] == 0
        _check_columns(K, Bo, Xd)
        assert np.all(Xd[:, 4] == 0.0)


def test_k1_matches_pcg_solve(P):
    case = (2, 2, 32, 1, 1, 2)
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(O.G_X2_Y2))
    X, st = A.solve_block(b, tol=TOL)
    x, st1 = A.solve(b[:, 0], tol=TOL)
    assert abs(st["iterations"] - st1["iterations"]) <= 1
    assert float((X[:, 0] - x).norm() / x.norm()) <= 1e-9


@pytest.mark.parametrize("case,k,kind", [((2, 2, 64, 1, 1, 2), 32, "harmonic"), ((3, 1, 16, 1, 0, 3), 8, "random"),
                                         ((2, 1, 100, 1, 1, 4), 5, "random")])
def test_f32_inner_refinement(P, case, k, kind):
    d, A, K, Bo, Bd = _setup(P, case, k, kind)
    X, st = A.solve_block(Bd, tol=TOL, precision=P.GB_F32_IR)
    assert st["status"] == 0 and st["relres"] <= TOL and st["outer"] >= 1
    _check_columns(K, Bo, X.cpu().numpy())


def test_x0_and_agreement_with_batched(P):
    """A start near the solution takes fewer steps; the block solution equals
    the independent per-column recurrences' (pcg_solve_batched) to the
    tolerance."""
    import torch
    case, k = (2, 2, 24, 1, 1, 3), 6
    d, A, K, Bo, Bd = _setup(P, case, k, "harmonic")
    X, st = A.solve_block(Bd, tol=TOL)
    X0 = X + 1e-6 * torch.randn_like(X)
    X2, st2 = A.solve_block(Bd, X0=X0, tol=TOL)
    assert st2["status"] == 0 and st2["iterations"] < st["iterations"]
    Xb, sts = P.pcg_solve_batched([A], [Bd], tol=TOL)
    assert float((Xb[0] - X).norm() / X.norm()) <= 1e-8


def test_bad_arguments(P):
    import torch
    d = P.FemSystem(2, 1, 10, 1, 1, 1)
    A = d.to_sell(32, 256, P.GB_VAL_F64)
    B = torch.ones((d.n_free, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(P.GbError):
        A.solve_block(B)
    with pytest.raises(P.GbError):
        A.solve_block(B[:, :4], precision=P.GB_F32_RU)
    with pytest.raises(P.GbError):
        A.solve_block(B[:, :4], precision=P.GB_F32_IR)  # no fp32 values
    with pytest.raises(P.GbError):
        A.solve_block(B[:, :4], precond=P.GB_PC_BLOCK_JACOBI)
