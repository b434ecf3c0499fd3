"""GPU: the RHS block width autotuner (pcg_batched_autotune_width) and the
grouped multi-RHS solve it feeds: the chosen width is one of the candidates,
every candidate is timed, and the solution through groups of that width
meets Eq. (2) per column and agrees with one batch of all k columns."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05413_gb300 as P
    P.load()
    return P


@pytest.mark.parametrize("k,prec", [(12, "GB_F64"), (32, "GB_F32_IR"), (3, "GB_F64")])
def test_autotune_width_and_grouped_solve(P, k, prec):
    d = P.FemSystem(2, 2, 64, 1, 1, 2)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
    coef = np.random.default_rng(k).standard_normal((k, 10))
    B = d.lift(d.dirichlet(O.G_HARMONIC, coef, k))
    precision = getattr(P, prec)
    w, ms = P.autotune_rhs_width(A, B, precision=precision)
    assert w in (1, 2, 4, 8, 16, 32) and w <= k
    assert set(ms) == {c for c in (1, 2, 4, 8, 16, 32) if c <= k} and all(t > 0 for t in ms.values())
    assert ms[w] == min(ms.values())
    X, sts = P.solve_multi(A, B, w, tol=1e-10, precision=precision)
    assert all(s["status"] == 0 and s["relres"] <= 1e-10 for s in sts)
    s = O.System(2, 2, 64, 1, 1, 2).assemble()
    rp, ci, v = s.k_ii()
    Bo = s.lift(s.eval_g(O.G_HARMONIC, coef, k))
    Xd = X.cpu().numpy()
    for j in range(k):
        assert np.linalg.norm(Bo[:, j] - O.spmv(rp, ci, v, Xd[:, j])) <= 1.5e-10 * np.linalg.norm(Bo[:, j])
    if k <= 32:
        X1, _ = P.pcg_solve_batched([A], [B], tol=1e-10, precision=precision)
        assert float((X1[0] - X).norm() / X.norm()) <= 1e-8
