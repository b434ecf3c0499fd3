"""GPU: the layout autotuner (sell_autotune, sell_set_variant).

Whatever layout it picks is a SELL-C-sigma layout of the same matrix, so the
tuned matrix must solve to the same tolerance, reproduce a solution the
element space holds exactly, and agree with the default layout's solve."""
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


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_autotuned_layout_solves_and_caches(P, prec):
    spec = (2, 2, 200, 1, 1, 11)
    d = P.FemSystem(*spec)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    tp = P.GB_F64 if prec == "f64" else P.GB_F32_IR
    A, cfg = P.autotune(d, b, precision=tp)
    assert not cfg["cached"] and cfg["candidates"] >= 5
    assert (A.C, A.sigma) == (cfg["C"], cfg["sigma"]) and cfg["C"] in (32, 64, 128)
    assert cfg["spmv_variant"] in (0, 1) and 0 < cfg["spmv_ms"] <= cfg["iter_ms"]
    sp = P.GB_F64 if prec == "f64" else P.GB_F32_RU
    x, st = A.solve(b, tol=TOL, precision=sp)
    assert st["status"] == 0 and st["relres"] <= TOL
    u = d.dirichlet(O.G_X2_Y2, which="free")[:, 0].cpu().numpy()
    assert O.x_err(u, x.cpu().numpy()) <= 1e-8
    x0, _ = d.to_sell(32, 256).solve(b, tol=TOL, precision=sp)
    assert O.x_err(x0.cpu().numpy(), x.cpu().numpy()) <= 1e-8
    # the same spec again comes from the cache with the same choice
    A2, cfg2 = P.autotune(d, b, precision=tp)
    assert cfg2["cached"] and (A2.C, A2.sigma, cfg2["spmv_variant"]) == (A.C, A.sigma, cfg["spmv_variant"])
    x2, st2 = A2.solve(b, tol=TOL, precision=sp)
    assert st2["iterations"] == st["iterations"] and bool((x2 == x).all())


def test_variant_hint_changes_only_the_kernel(P):
    """Variant 1 on a C = 32 layout runs the row-per-lane SpMV: same matrix,
    same iteration count within a few, same solution."""
    d = P.FemSystem(2, 1, 300, 1, 1, 4)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    A = d.to_sell(32, 256)
    x0, s0 = A.solve(b, tol=TOL)
    P.gbpcg.check(P.gbpcg.lib().sell_set_variant(A.handle, 1), "sell_set_variant")
    x1, s1 = A.solve(b, tol=TOL)
    assert s1["status"] == 0 and abs(s1["iterations"] - s0["iterations"]) <= 5
    assert O.x_err(x0.cpu().numpy(), x1.cpu().numpy()) <= 1e-8
    with pytest.raises(P.GbError):
        P.gbpcg.check(P.gbpcg.lib().sell_set_variant(A.handle, 7), "sell_set_variant")
