"""GPU parity of the single-launch persistent solves: one thread-block cluster
(pcg_solve's default for fp64 Jacobi-CG systems of up to 8192 rows) and a
group of CTAs of the grid tier (PcgOptions.persist_off = 3: pcg_solve up to
2^18 rows, pcg_solve_batched for 2^16 < n k2 <= 2^18), whose blocks exchange
their column sums through global memory with bounded waits.  Each solve forms
its residual, runs the CG rounds (Eq. 2 with true-residual confirmation) and
leaves x in one launch.

Each result is checked against the oracle's solution (1e-13) at the CG bar
(relative residual <= 1e-10 recomputed on the host, relative error <= 1e-8),
against the multi-kernel loop (persist_off = 1), and for determinism; grid
groups run from one block (n <= 2048) to 128 blocks."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05413_gb300 as P
    P.load()
    return P


def _oracle(spec, gid, coef=None, k=1):
    s = O.System(*spec).assemble()
    rp, ci, v = s.k_ii()
    bo = s.lift(s.eval_g(gid, coef, k))
    return rp, ci, v, bo


@pytest.mark.parametrize("spec,gid,po", [
    ((2, 2, 16, 1, 1, 1), O.G_X2_Y2, 0),          # n = 961: one cluster
    ((2, 1, 64, 0, 0, 0), O.G_SIN_SINH, 0),       # cfg1, n = 3969: one cluster
    ((2, 2, 16, 1, 1, 1), O.G_X2_Y2, 3),          # grid group of one block
    ((2, 1, 64, 0, 0, 0), O.G_SIN_SINH, 3),       # two blocks
    ((2, 2, 64, 1, 1, 3), O.G_X2_Y2, 3),          # n = 16129: 8 blocks
    ((3, 1, 24, 1, 0, 2), O.G_X2_Y2_2Z2, 3),      # jittered 3D P1, n = 12167
    ((3, 2, 12, 0, 0, 0), O.G_X2_Y2_2Z2, 3),      # 3D P2, n = 12167, 27 nnz per row
    ((2, 1, 256, 1, 1, 5), O.G_X2_Y2, 3),         # n = 65025: 32 blocks
])
def test_persistent_solve_matches_oracle_and_multikernel(P, spec, gid, po):
    d = P.FemSystem(*spec)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(gid))[:, 0]
    x, st = A.solve(b, tol=TOL, persist_off=po)      # one persistent launch
    xm, sm = A.solve(b, tol=TOL, persist_off=1)      # multi-kernel loop
    assert st["status"] == 0 and st["relres"] <= TOL
    assert st["kernel_launches"] <= 4                 # gathers, one persistent launch, scatter
    rp, ci, v, bo = _oracle(spec, gid)
    xo, _, ito, _ = O.pcg(rp, ci, v, bo[:, 0], tol=1e-13)
    xd = x.cpu().numpy()
    relres = np.linalg.norm(bo[:, 0] - O.spmv(rp, ci, v, xd)) / np.linalg.norm(bo[:, 0])
    assert relres <= 1.5 * TOL
    assert O.x_err(xo, xd) <= 1e-8
    # the same recurrence: iteration counts up to rounding drift, and the two
    # device paths agree far below the bar
    assert abs(st["iterations"] - sm["iterations"]) <= max(3, 0.02 * sm["iterations"])
    assert abs(st["iterations"] - ito) <= max(3, 0.02 * ito) or st["iterations"] <= ito
    assert O.x_err(xm.cpu().numpy(), xd) <= 1e-9
    # deterministic: the group's sums are added in a fixed order
    x2, st2 = A.solve(b, tol=TOL, persist_off=po)
    assert st2["iterations"] == st["iterations"] and bool((x2 == x).all())


@pytest.mark.parametrize("po", [0, 3])
def test_persistent_solve_warm_start_zero_rhs_and_cap(P, po):
    d = P.FemSystem(2, 1, 48, 1, 1, 7)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    x, st = A.solve(b, tol=TOL, persist_off=po)
    assert st["kernel_launches"] <= 4
    # warm start at the solution: at most a couple of iterations
    x2, st2 = A.solve(b, x0=x, tol=TOL, persist_off=po)
    assert st2["status"] == 0 and st2["iterations"] <= 2
    assert O.x_err(x.cpu().numpy(), x2.cpu().numpy()) < 1e-9
    # b = 0: x = 0 with no iteration, whatever x0 was
    z, sz = A.solve(b * 0.0, x0=x, tol=TOL, persist_off=po)
    assert sz["status"] == 0 and sz["iterations"] == 0 and float(z.abs().max()) == 0.0
    # the iteration cap: GB_NOT_CONVERGED, x and the stats still written
    x3, st3 = A.solve(b, tol=TOL, max_iter=10, raise_on_fail=False, persist_off=po)
    assert st3["rc"] == P.gbpcg.GB_NOT_CONVERGED and st3["iterations"] == 10
    assert 0.0 < st3["relres"] < 1.0


@pytest.mark.parametrize("po", [0, 3])
def test_persistent_solve_breakdown_on_negative_definite(P, po):
    d = P.FemSystem(2, 1, 40, 1, 1, 1)
    rp, ci, v = d.csr()
    A = P.Sell.from_csr(rp, ci, -v)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    x, st = A.solve(b, raise_on_fail=False, persist_off=po)
    assert st["rc"] == P.gbpcg.GB_BREAKDOWN


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_grid_tier_uneven_and_alone_equals_mix(P, prec):
    """Systems with 2^16 < n k2 <= 2^18 (grid tier) beside smaller and larger
    ones: every column against the oracle, and each system's result the same
    bits alone and in the batch (its group's arithmetic depends on its own
    size only)."""
    p = P.GB_F64 if prec == "f64" else P.GB_F32_RU
    specs = [((2, 1, 256, 1, 1, 11), 2), ((2, 2, 128, 1, 1, 12), 1), ((2, 1, 24, 1, 1, 13), 3),
             ((3, 1, 40, 0, 0, 0), 4), ((2, 1, 600, 1, 1, 14), 1)]
    mats, Bs, cols = [], [], []
    for spec, k in specs:
        d = P.FemSystem(*spec)
        mats.append(d.to_sell(32, 256))
        coef = np.random.default_rng(spec[-1]).standard_normal((k, 10))
        gid = 4 if spec[0] == 2 else 3
        c = coef if spec[0] == 2 else coef[:, :4]
        Bs.append(d.lift(d.dirichlet(gid, c, k)))
        cols.append((spec, gid, c, k))
    Xs, sts = P.pcg_solve_batched(mats, Bs, tol=TOL, precision=p, max_iter=400000, persist_off=3)
    for (spec, gid, c, k), X, st in zip(cols, Xs, sts):
        assert st["status"] == 0 and st["relres"] <= TOL
        if spec[2] <= 256 and spec[0] == 2 or spec[0] == 3:
            rp, ci, v, bo = _oracle(spec, gid, c, k)
            Xd = X.cpu().numpy()
            for j in range(k):
                xo, _, _, _ = O.pcg(rp, ci, v, bo[:, j], tol=1e-13)
                assert O.x_err(xo, Xd[:, j]) <= 1e-8, (spec, j)
    for i in (0, 1, 3):
        Xa, sa = P.pcg_solve_batched([mats[i]], [Bs[i]], tol=TOL, precision=p, max_iter=400000, persist_off=3)
        assert sa[0]["iterations"] == sts[i]["iterations"]
        assert bool((Xa[0] == Xs[i]).all()), specs[i]
