"""pcg_solve_noalloc: the fp64 solve for callers that cannot allocate device
memory (its scratch is a fixed file-scope device array).  Called through the
C ABI and compared with pcg_solve on the same system, twice in a row (the
second call reuses the array the first one left behind, and must leave the
library's allocation count and the device's free memory unchanged), and from
a nonzero starting iterate.  This file sorts last
so that a run stopping at the first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

XERR = 1e-8   # relative error bar of the solver tests
TOL = 1e-10   # Eq. (2) residual threshold


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05413_gb300 as P
    P.load()
    return P


def _noalloc(P, A, b, x0=None, **kw):
    import torch
    from paper_2201_05413_gb300 import gbpcg as G
    from paper_2201_05413_gb300.api import _opts
    x = x0.clone() if x0 is not None else torch.full_like(b, float("nan"))
    kw.setdefault("x0_zero", 0 if x0 is not None else 1)
    o = _opts(**kw)
    st = G.PcgStats()
    rc = G.lib().pcg_solve_noalloc(A.handle, G.ptr(b), G.ptr(x), C.byref(o), G.stream_ptr(), C.byref(st))
    return rc, x, st


def _xerr(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(a))


@pytest.mark.parametrize("spec", [(2, 2, 200, 1, 1, 3), (3, 1, 40, 0, 0, 0)])
def test_noalloc_matches_pcg_solve_twice(P, spec):
    d = P.FemSystem(*spec)
    assert d.n_free <= 262144
    A = d.to_sell(32, 256)
    gid = 1 if spec[0] == 2 else 2
    b = d.lift(d.dirichlet(gid))[:, 0].contiguous()
    x_ref, st_ref = A.solve(b, tol=TOL, max_iter=200000)
    import torch
    L = P.gbpcg.lib()
    x0 = torch.full_like(b, float("nan"))
    for call in range(2):
        # the second call must not allocate: the library's allocation count
        # and the device's free memory are the same after it as before
        torch.cuda.synchronize()
        n_alloc, free0 = L.gbpcg_device_allocations(), torch.cuda.mem_get_info()[0]
        rc, x, st = _noalloc(P, A, b, x0=x0, x0_zero=1, tol=TOL, max_iter=200000)
        torch.cuda.synchronize()
        if call == 1:
            assert L.gbpcg_device_allocations() == n_alloc
            assert torch.cuda.mem_get_info()[0] == free0
        assert rc == 0, L.gbpcg_last_error()
        assert st.status == 0 and st.relres <= TOL
        assert _xerr(x_ref, x) <= XERR
        assert abs(st.iterations - st_ref["iterations"]) <= 2


def test_noalloc_warm_start_matches_pcg_solve(P):
    """A nonzero x0 (a partly converged iterate) gathered into the static
    array: the same iterations and solution as pcg_solve from that x0."""
    d = P.FemSystem(2, 1, 150, 1, 1, 7)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(1))[:, 0].contiguous()
    x_part, _ = A.solve(b, tol=1e-4, max_iter=200000)
    x_ref, st_ref = A.solve(b, x0=x_part, tol=TOL, max_iter=200000)
    rc, x, st = _noalloc(P, A, b, x0=x_part, tol=TOL, max_iter=200000)
    assert rc == 0, P.gbpcg.lib().gbpcg_last_error()
    assert st.status == 0 and st.relres <= TOL
    assert abs(st.iterations - st_ref["iterations"]) <= 2
    assert _xerr(x_ref, x) <= XERR


def test_noalloc_second_system_after_first(P):
    """A smaller system after a larger one: nothing stale from the first call
    leaks in; the second result is also checked against the oracle."""
    import oracle as O
    d1 = P.FemSystem(2, 1, 400, 1, 1, 1)
    d2 = P.FemSystem(2, 2, 30, 1, 1, 2)
    for d in (d1, d2):
        A = d.to_sell()
        b = d.lift(d.dirichlet(1))[:, 0].contiguous()
        x_ref, _ = A.solve(b, tol=TOL)
        rc, x, st = _noalloc(P, A, b, tol=TOL)
        assert rc == 0 and _xerr(x_ref, x) <= XERR
    s = O.System(2, 2, 30, 1, 1, 2).assemble()
    rp, ci, v = s.k_ii()
    xo, _, _, _ = O.pcg(rp, ci, v, s.lift(s.eval_g(O.G_X2_Y2))[:, 0], tol=1e-13)
    assert O.x_err(xo, x.cpu().numpy()) <= XERR


def test_noalloc_rejects_oversized_and_other_precisions(P):
    from paper_2201_05413_gb300 import gbpcg as G
    d = P.FemSystem(2, 1, 600)  # 599^2 = 358801 rows > 262144
    A = d.to_sell()
    b = d.lift(d.dirichlet(1))[:, 0].contiguous()
    rc, x, st = _noalloc(P, A, b)
    assert rc == G.GB_TOO_LARGE
    assert b"262144" in G.lib().gbpcg_last_error()
    small = P.FemSystem(2, 1, 20)
    As = small.to_sell()
    bs = small.lift(small.dirichlet(1))[:, 0].contiguous()
    rc, x, st = _noalloc(P, As, bs, precision=G.GB_F32_IR)
    assert rc == G.GB_EINVAL
