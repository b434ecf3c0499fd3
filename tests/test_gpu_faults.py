"""Failure detection without a GPU fault: a bounded device wait that runs out
reports GB_TIMEOUT and leaves the device usable; allocation failures injected
on the host (an allocator that returns NULL) report GB_ENOMEM and release
every buffer taken before the failure."""
import ctypes as C

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


def test_bounded_wait_runs_out_and_device_stays_usable(P):
    rc, waited = P.wait_selftest(20.0)
    assert rc == P.gbpcg.GB_TIMEOUT
    assert 20.0 <= waited < 1000.0, waited
    # the context is intact: a solve right after succeeds
    d = P.FemSystem(2, 2, 12, 1, 1, 1)
    A = d.to_sell(32, 64)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    x, st = A.solve(b, tol=1e-10)
    assert st["status"] == 0 and st["relres"] <= 1e-10
    with pytest.raises(P.GbError):
        P.gbpcg.check(P.gbpcg.lib().gbpcg_wait_selftest(0.0, None, None), "bad limit")


def test_grid_barrier_wait_runs_out_and_device_stays_usable(P):
    """The grid tier's group barrier with one arrival that never comes: the
    wait gives up after its limit, the call reports GB_TIMEOUT, and a solve
    on the same tier right after succeeds."""
    rc, waited = P.grid_wait_selftest(20.0)
    assert rc == P.gbpcg.GB_TIMEOUT
    assert 20.0 <= waited < 1000.0, waited
    d = P.FemSystem(2, 1, 64, 0, 0, 0)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(O.G_SIN_SINH))[:, 0]
    x, st = A.solve(b, tol=1e-10, persist_off=3)  # one persistent grid-tier launch
    assert st["status"] == 0 and st["relres"] <= 1e-10 and st["kernel_launches"] <= 4
    with pytest.raises(P.GbError):
        P.gbpcg.check(P.gbpcg.lib().gbpcg_grid_wait_selftest(0.0, None, None), "bad limit")


class _FailingAllocator:
    """cudaMalloc-backed gb_allocator that returns NULL from its n-th call on."""

    def __init__(self, fail_at):
        import torch
        self.fail_at, self.calls, self.live = fail_at, 0, {}
        self._torch = torch
        G = __import__("paper_2201_05413_gb300.gbpcg", fromlist=["gbpcg"])
        self._a = G._ALLOC_TYPE(self._alloc)
        self._f = G._FREE_TYPE(self._free)
        self.struct = G.gb_allocator(None, self._a, self._f)

    def _alloc(self, ctx, nbytes, stream):
        self.calls += 1
        if self.calls >= self.fail_at:
            return None
        p = int(self._torch.cuda.caching_allocator_alloc(int(nbytes)))
        self.live[p] = nbytes
        return p

    def _free(self, ctx, ptr, stream):
        if ptr in self.live:
            del self.live[ptr]
            self._torch.cuda.caching_allocator_delete(ptr)


@pytest.mark.parametrize("fail_at", [1, 2, 3, 5, 8])
def test_allocation_failure_reports_enomem_and_releases(P, fail_at):
    G = P.gbpcg
    al = _FailingAllocator(fail_at)
    spec = G.gb_fem_spec(2, 2, 16, 1, 1, 0, 1)
    h = C.c_void_p()
    rc = G.lib().fem_assemble(C.byref(spec), C.byref(al.struct), G.stream_ptr(), C.byref(h))
    if rc == G.GB_OK:  # the system needed fewer allocations than fail_at
        assert al.calls < fail_at
        G.lib().fem_system_destroy(h)
    else:
        assert rc == G.GB_ENOMEM, G.lib().gbpcg_last_error()
        assert not h.value
    assert al.live == {}, f"{len(al.live)} buffers still held after the failure"


@pytest.mark.parametrize("fail_at", [1, 3, 6])
def test_sell_build_allocation_failure(P, fail_at):
    G = P.gbpcg
    d = P.FemSystem(2, 1, 24, 1, 1, 1)
    al = _FailingAllocator(fail_at)
    h = C.c_void_p()
    rc = G.lib().csr_to_sell(d.handle, 32, 64, G.GB_VAL_F64 | G.GB_VAL_F32, C.byref(al.struct), G.stream_ptr(),
                             C.byref(h))
    assert rc == G.GB_ENOMEM, G.lib().gbpcg_last_error()
    assert not h.value
    assert al.live == {}
