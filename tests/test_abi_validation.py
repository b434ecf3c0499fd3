"""Host-side argument checks of the C ABI (no GPU needed: every check below
runs before the library touches the device).  Each call must fail with
GB_EINVAL and leave a message in gbpcg_last_error."""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def G():
    import paper_2201_05413_gb300 as P
    P.load()
    return P.gbpcg


def _spec(G, dim=2, degree=1, cells=8, jitter=0, diag_mode=0, reserved=0, seed=1):
    return G.gb_fem_spec(dim, degree, cells, jitter, diag_mode, reserved, seed)


def _einval(G, rc, needle):
    assert rc == G.GB_EINVAL
    msg = G.lib().gbpcg_last_error().decode()
    assert needle in msg, msg


@pytest.mark.parametrize("kw,needle", [
    ({"dim": 4}, "dim"), ({"degree": 5}, "degree"), ({"degree": 0}, "degree"), ({"cells": 1}, "cells"),
    ({"jitter": 2}, "jitter"), ({"dim": 3, "diag_mode": 1}, "Kuhn"), ({"reserved": 1}, "reserved")])
def test_fem_assemble_rejects_bad_specs(G, kw, needle):
    out = C.c_void_p()
    rc = G.lib().fem_assemble(C.byref(_spec(G, **kw)), None, None, C.byref(out))
    _einval(G, rc, needle)
    assert not out.value


def test_solver_entry_points_reject_null(G):
    L = G.lib()
    o = G.PcgOptions()
    st = G.PcgStats()
    _einval(G, L.pcg_solve(None, None, None, C.byref(o), None, C.byref(st)), "pcg_solve")
    _einval(G, L.pcg_solve_noalloc(None, None, None, C.byref(o), None, C.byref(st)), "pcg_solve_noalloc")
    _einval(G, L.pcg_solve_block(None, None, None, 4, C.byref(o), None, C.byref(st)), "pcg_solve_block")
    _einval(G, L.pcg_solve_batched(0, None, None, None, None, C.byref(o), None, C.byref(st)), "pcg_solve_batched")
    ms = (C.c_double * 3)()
    _einval(G, L.pcg_kernel_times(None, None, 0, 3, None, ms), "pcg_kernel_times")
    best = C.c_int(0)
    _einval(G, L.pcg_batched_autotune_width(None, None, 8, 0, None, C.byref(best), None),
            "pcg_batched_autotune_width")


def test_preconditioner_entry_points_reject_null(G):
    L = G.lib()
    _einval(G, L.sell_block_jacobi(None, 4, None), "sell_block_jacobi")
    info = G.gb_bjacobi_info()
    _einval(G, L.sell_block_jacobi_info(None, C.byref(info)), "sell_block_jacobi_info")
    _einval(G, L.sell_block_jacobi_apply(None, None, None, None), "sell_block_jacobi_apply")


def test_wait_selftest_rejects_bad_limits(G):
    waited = C.c_double(0)
    _einval(G, G.lib().gbpcg_wait_selftest(0.0, None, C.byref(waited)), "limit_ms")
    _einval(G, G.lib().gbpcg_wait_selftest(5000.0, None, C.byref(waited)), "limit_ms")


def test_grid_wait_selftest_rejects_bad_limits(G):
    waited = C.c_double(0)
    _einval(G, G.lib().gbpcg_grid_wait_selftest(0.0, None, C.byref(waited)), "limit_ms")
    _einval(G, G.lib().gbpcg_grid_wait_selftest(2500.0, None, C.byref(waited)), "limit_ms")
