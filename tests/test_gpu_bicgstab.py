"""GPU parity: BiCGSTAB (the paper's Krylov method, Sec. 3.2), right-
preconditioned with Jacobi or block-Jacobi, against the oracle's BiCGSTAB and
the exact solutions.

Bar: Eq. (2) at 1e-10 (recomputed here in fp64 from the oracle's matrix),
Eq. (1) error <= 1e-8 against the oracle's solution at 1e-13, and the oracle's
step count up to rounding drift (BiCGSTAB's residual is not monotone and its
true-residual restarts depend on rounding, so the drift is allowed 15 %); one step with the exact preconditioner; tiny systems
within n steps; graph and direct launches give the same bits."""
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
