"""GPU parity: Jacobi-PCG solves (fp64 and mixed-precision refinement)
against the oracle's solutions and the closed forms it is pinned to.

Bar: relative residual ||b - A x|| / ||b|| <= 1e-10 (Eq. 2, recomputed here in
fp64 on the host from the oracle's matrix) and relative error (Eq. 1) <= 1e-8
against the oracle's solution at 1e-13."""
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


def _solve_both(P, dim, deg, cells, jit, dm, seed, gid, coef=None, C=32, sigma=256, **kw):
    d = P.FemSystem(dim, deg, cells, jit, dm, seed)
    A = d.to_sell(C, sigma, P.GB_VAL_F64 | P.GB_VAL_F32 | P.GB_VAL_BF16)
    b = d.lift(d.dirichlet(gid, coef))[:, 0]
    kw.setdefault("max_iter", 200000)
    x, st = A.solve(b, tol=TOL, **kw)
    s = O.System(dim, deg, cells, jit, dm, seed).assemble()
    rp, ci, v = s.k_ii()
    bo = s.lift(s.eval_g(gid, coef))[:, 0]
    xo, sto, ito, rro = O.pcg(rp, ci, v, bo, tol=1e-13)
    xd = x.cpu().numpy()
    relres = np.linalg.norm(bo - O.spmv(rp, ci, v, xd)) / np.linalg.norm(bo)
    return d, s, xd, xo, st, ito, relres


@pytest.mark.parametrize("case", [
    (2, 1, 64, 0, 0, 0, O.G_SIN_SINH),      # 64x64 regular P1 (closed form below)
    (2, 1, 96, 1, 1, 1, O.G_X2_Y2),
    (2, 2, 48, 1, 1, 1, O.G_X2_Y2),
    (3, 1, 20, 0, 0, 0, O.G_X2_Y2_2Z2),
    (3, 2, 10, 0, 0, 0, O.G_X2_Y2_2Z2),
    (3, 1, 20, 1, 0, 2, O.G_X2_Y2_2Z2),     # jittered 3D P1: no closed form, oracle solve
])
@pytest.mark.parametrize("persist_off", [0, 1, 3])
def test_fp64_pcg_matches_oracle(P, case, persist_off):
    d, s, xd, xo, st, ito, relres = _solve_both(P, *case, persist_off=persist_off)
    assert st["status"] == 0
    assert st["relres"] <= TOL and relres <= 1.5 * TOL
    assert O.x_err(xo, xd) <= XERR
    # same recurrence as the oracle: iteration counts agree up to rounding drift
    assert abs(st["iterations"] - ito) <= max(3, 0.02 * ito) or st["iterations"] <= ito


def test_cfg1_closed_form(P):
    d, s, xd, xo, st, ito, relres = _solve_both(P, 2, 1, 64, 0, 0, 0, O.G_SIN_SINH)
    h = 1.0 / 64
    mu = np.arccosh(2.0 - np.cos(np.pi * h))
    X = d.coords("free").cpu().numpy()
    i, j = np.rint(X[:, 0] * 64), np.rint(X[:, 1] * 64)
    u = np.sin(np.pi * i * h) * np.sinh(mu * j) / np.sinh(64 * mu)
    assert O.x_err(u, xd) <= XERR


@pytest.mark.parametrize("case", [
    (2, 2, 40, 1, 1, 4, O.G_X2_Y2),         # P2 reproduces x^2 - y^2
    (3, 1, 16, 0, 0, 0, O.G_X2_Y2_2Z2),     # Kuhn 7-point reproduces quadratics
    (3, 2, 8, 0, 0, 0, O.G_X2_Y2_2Z2),
    (3, 2, 8, 1, 0, 3, O.G_X2_Y2_2Z2),      # jittered 3D: P2 reproduces quadratics
])
def test_exact_polynomial_reproduction(P, case):
    dim, deg, cells, jit, dm, seed, gid = case
    d = P.FemSystem(dim, deg, cells, jit, dm, seed)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(gid))[:, 0]
    x, st = A.solve(b, tol=TOL, max_iter=100000)
    u = d.dirichlet(gid, which="free")[:, 0]
    assert O.x_err(u.cpu().numpy(), x.cpu().numpy()) <= XERR


@pytest.mark.parametrize("prec", ["f32", "bf16", "f32ru", "bf16ru"])
@pytest.mark.parametrize("case", [
    (2, 1, 64, 1, 1, 2, O.G_X2_Y2),
    (2, 2, 32, 1, 1, 2, O.G_X2_Y2),
    (3, 1, 24, 0, 0, 0, O.G_X2_Y2_2Z2),
    (3, 2, 12, 0, 0, 0, O.G_X2_Y2_2Z2),
])
def test_mixed_refinement_matches_oracle(P, case, prec):
    p = {"f32": P.GB_F32_IR, "bf16": P.GB_BF16_IR, "f32ru": P.GB_F32_RU, "bf16ru": P.GB_BF16_RU}[prec]
    d, s, xd, xo, st, ito, relres = _solve_both(P, *case, precision=p)
    assert st["status"] == 0
    assert relres <= 1.5 * TOL
    assert O.x_err(xo, xd) <= XERR
    assert st["outer"] >= 1


def test_zero_rhs_gives_zero(P):
    import torch
    d = P.FemSystem(2, 1, 16)
    A = d.to_sell()
    x, st = A.solve(torch.zeros(d.n_free, dtype=torch.float64, device="cuda"))
    assert st["iterations"] == 0 and torch.count_nonzero(x).item() == 0


def test_max_iter_reports_not_converged(P):
    d = P.FemSystem(2, 2, 32, 1, 1, 1)
    A = d.to_sell()
    b = d.lift(d.dirichlet(1))[:, 0]
    x, st = A.solve(b, max_iter=5, raise_on_fail=False)
    assert st["rc"] == P.gbpcg.GB_NOT_CONVERGED and st["iterations"] == 5
    with pytest.raises(P.GbError):
        A.solve(b, max_iter=5)


def test_non_spd_reports_breakdown(P):
    d = P.FemSystem(2, 1, 16, 1, 1, 1)
    rp, ci, v = d.csr()
    A = P.Sell.from_csr(rp, ci, -v)
    b = d.lift(d.dirichlet(1))[:, 0]
    x, st = A.solve(b, raise_on_fail=False)
    assert st["rc"] == P.gbpcg.GB_BREAKDOWN


def test_graph_and_direct_launch_identical(P):
    d = P.FemSystem(2, 2, 30, 1, 1, 3)
    A = d.to_sell(32, 64)
    b = d.lift(d.dirichlet(1))[:, 0]
    x1, s1 = A.solve(b, use_graph=1, persist_off=1)
    x2, s2 = A.solve(b, use_graph=0, check_every=7, persist_off=1)
    x3, s3 = A.solve(b, use_graph=1, persist_off=1)
    assert s1["iterations"] == s2["iterations"] == s3["iterations"]
    assert bool((x1 == x2).all()) and bool((x1 == x3).all())


def test_warm_start_at_solution(P):
    d = P.FemSystem(2, 1, 32, 1, 1, 3)
    A = d.to_sell()
    b = d.lift(d.dirichlet(1))[:, 0]
    x, st = A.solve(b)
    x2, st2 = A.solve(b, x0=x)
    assert st2["iterations"] <= 2
    assert O.x_err(x.cpu().numpy(), x2.cpu().numpy()) < 1e-9


@pytest.mark.parametrize("C,sigma", [(32, 1), (64, 32), (128, 512)])
def test_layout_independent_solution(P, C, sigma):
    d = P.FemSystem(2, 2, 28, 1, 1, 6)
    b = d.lift(d.dirichlet(1))[:, 0]
    x, st = d.to_sell(C, sigma).solve(b)
    xr, _ = d.to_sell(32, 256).solve(b)
    assert O.x_err(xr.cpu().numpy(), x.cpu().numpy()) < 1e-8
