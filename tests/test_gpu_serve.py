"""GPU parity: the continuous-batching solve server (serve_*).

Each served result is checked against the oracle (Eq. 2 residual recomputed
on the host with the oracle's matrix, Eq. 1 error against the oracle solved to
1e-13), and against the same request served alone: a request's arithmetic
depends only on its own data, so it must not change in a mix."""
import time

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


MIX = [  # dim, degree, cells, jitter, diag, seed, k, gid
    (2, 1, 24, 1, 1, 1, 3, O.G_HARMONIC),
    (2, 2, 16, 1, 1, 2, 1, O.G_HARMONIC),
    (3, 1, 10, 0, 0, 0, 2, O.G_LINEAR),
    (2, 2, 31, 1, 1, 3, 5, O.G_HARMONIC),
    (3, 2, 6, 0, 0, 0, 4, O.G_LINEAR),
    (2, 1, 47, 1, 1, 4, 8, O.G_HARMONIC),
]


def _coef(i, k, gid):
    return np.random.default_rng(100 + i).standard_normal((k, O.NCOEF[gid]))


def _oracle(spec, k, gid, coef):
    dim, deg, cells, jit, dm, seed = spec
    s = O.System(dim, deg, cells, jit, dm, seed).assemble()
    rp, ci, v = s.k_ii()
    B = s.lift(s.eval_g(gid, coef, k, "bnd"))
    X = np.stack([O.pcg(rp, ci, v, B[:, j], tol=1e-13)[0] for j in range(k)], 1)
    return rp, ci, v, B, X


def _serve(P, reqs, **kw):
    srv = P.Server(**kw)
    try:
        ts = [srv.submit(*r[:6], k=r[6], gid=r[7], coef=_coef(i, r[6], r[7])) for i, r in enumerate(reqs)]
        res = srv.wait(ts, timeout_s=300)
        stats = srv.stats()
    finally:
        srv.close()
    return [res[t] for t in ts], stats


@pytest.mark.parametrize("prec", ["f32ru", "f64"])
def test_served_results_match_oracle(P, prec):
    p = P.GB_F32_RU if prec == "f32ru" else P.GB_F64
    out, stats = _serve(P, MIX, precision=p, max_slots=8, iters_per_step=50)
    assert stats["completed"] == len(MIX) and stats["max_resident"] >= 2
    for i, ((r, x), req) in enumerate(zip(out, MIX)):
        assert r["status"] == 0, r
        assert r["relres"] <= TOL
        rp, ci, v, B, X = _oracle(req[:6], req[6], req[7], _coef(i, req[6], req[7]))
        for j in range(req[6]):
            rel = np.linalg.norm(B[:, j] - O.spmv(rp, ci, v, x[:, j])) / np.linalg.norm(B[:, j])
            assert rel <= 1.5 * TOL
            assert O.x_err(X[:, j], x[:, j]) <= 1e-8


def test_same_result_alone_and_in_mix(P):
    mixed, _ = _serve(P, MIX, precision=P.GB_F32_RU, max_slots=8, iters_per_step=37)
    for i, req in enumerate(MIX):
        srv = P.Server(precision=P.GB_F32_RU, max_slots=1, iters_per_step=200)
        try:
            t = srv.submit(*req[:6], k=req[6], gid=req[7], coef=_coef(i, req[6], req[7]))
            (r, x), = srv.wait([t]).values()
        finally:
            srv.close()
        rm, xm = mixed[i]
        assert r["iterations"] == rm["iterations"] and r["updates"] == rm["updates"]
        assert np.array_equal(x, xm)  # bit for bit: nothing in the mix enters a request's arithmetic


def test_memory_budget_limits_residency(P):
    reqs = [(2, 2, 100, 1, 1, s, 2, O.G_HARMONIC) for s in range(5)]
    # each request is estimated at ~40 MB before assembly and holds less: a
    # 64 MB budget keeps at most a few resident, never all five
    budget = 64 << 20
    out, stats = _serve(P, reqs, precision=P.GB_F32_RU, mem_budget=budget, max_slots=16)
    assert all(r["status"] == 0 for r, _ in out), ([r for r, _ in out], stats)
    assert 1 <= stats["max_resident"] <= 3
    assert stats["mem_peak"] <= budget


def test_too_large_request_rejected(P):
    srv = P.Server(precision=P.GB_F32_RU, mem_budget=8 << 20)
    try:
        t_big = srv.submit(2, 2, 400, 1, 1, 0, k=1, gid=O.G_HARMONIC, coef=np.ones((1, 10)))
        t_ok = srv.submit(2, 1, 16, 1, 1, 0, k=1, gid=O.G_HARMONIC, coef=np.ones((1, 10)))
        res = srv.wait([t_big, t_ok])
    finally:
        srv.close()
    assert res[t_big][0]["status"] == P.gbpcg.GB_TOO_LARGE
    assert res[t_ok][0]["status"] == 0


def test_arrivals_while_running_are_admitted(P):
    srv = P.Server(precision=P.GB_F32_RU, max_slots=8, iters_per_step=20)
    try:
        t0 = srv.submit(2, 2, 120, 1, 1, 9, k=2, gid=O.G_HARMONIC, coef=np.ones((2, 10)))
        time.sleep(0.05)
        later = [srv.submit(2, 1, 20 + 4 * i, 1, 1, i, k=1, gid=O.G_HARMONIC, coef=np.ones((1, 10)))
                 for i in range(4)]
        res = srv.wait([t0] + later)
        stats = srv.stats()
    finally:
        srv.close()
    assert all(res[t][0]["status"] == 0 for t in [t0] + later)
    # the small late arrivals finished while the large request was resident
    assert max(res[t][0]["latency_ms"] for t in later) < res[t0][0]["latency_ms"] + 1e3
    assert stats["max_resident"] >= 2


def test_boundary_data_from_host(P):
    spec = (2, 2, 20, 1, 1, 5)
    s = O.System(*spec)
    gB = s.eval_g(O.G_X2_Y2, None, 1, "bnd")
    srv = P.Server(precision=P.GB_F64)
    try:
        t = srv.submit(*spec, k=1, gB=gB)
        (r, x), = srv.wait([t]).values()
    finally:
        srv.close()
    s.assemble()
    u = s.eval_g(O.G_X2_Y2, None, 1, "free")[:, 0]  # P2 reproduces x^2 - y^2 exactly
    assert r["status"] == 0 and O.x_err(u, x[:, 0]) <= 1e-8


MIX_TIERS = [  # one request per path: one block, the cluster lane (two), the lock-step loop
    (2, 1, 40, 1, 1, 11, 2, O.G_HARMONIC),   # n k2 = 3042: one block
    (2, 1, 200, 1, 1, 12, 1, O.G_HARMONIC),  # 39601: the cluster lane
    (3, 2, 20, 0, 0, 0, 1, O.G_LINEAR),      # 59319: the cluster lane
    (2, 1, 400, 1, 1, 13, 4, O.G_HARMONIC),  # 636804: lock-step loop
]


@pytest.mark.parametrize("lane", [1, 0])
@pytest.mark.parametrize("prec", ["f32ru", "f64"])
def test_requests_of_every_size_in_one_mix(P, prec, lane):
    """Requests of every size class in one served mix, with the cluster lane
    for the medium ones (lane=1) and without it (lane=0: lock-step loop):
    every column meets Eq. 2 against the oracle's matrix, the medium requests
    are within 1e-8 of the oracle's solution, and each request served alone
    gives the same bits."""
    p = P.GB_F32_RU if prec == "f32ru" else P.GB_F64
    mixed, stats = _serve(P, MIX_TIERS, precision=p, max_slots=8, cluster_lane=lane)
    assert stats["completed"] == len(MIX_TIERS)
    for i, ((r, x), req) in enumerate(zip(mixed, MIX_TIERS)):
        assert r["status"] == 0, r
        dim, deg, cells, jit, dm, seed = req[:6]
        s = O.System(dim, deg, cells, jit, dm, seed).assemble()
        rp, ci, v = s.k_ii()
        B = s.lift(s.eval_g(req[7], _coef(i, req[6], req[7]), req[6], "bnd"))
        for j in range(req[6]):
            rel = np.linalg.norm(B[:, j] - O.spmv(rp, ci, v, x[:, j])) / np.linalg.norm(B[:, j])
            assert rel <= 1.5 * TOL, (i, j, rel)
            if i in (1, 2):
                xo = O.pcg(rp, ci, v, B[:, j], tol=1e-13)[0]
                assert O.x_err(xo, x[:, j]) <= 1e-8
    for i, req in enumerate(MIX_TIERS):
        srv = P.Server(precision=p, max_slots=1, cluster_lane=lane)
        try:
            t = srv.submit(*req[:6], k=req[6], gid=req[7], coef=_coef(i, req[6], req[7]))
            (r, x), = srv.wait([t]).values()
        finally:
            srv.close()
        rm, xm = mixed[i]
        assert r["iterations"] == rm["iterations"], (i, r, rm)
        assert np.array_equal(x, xm), i
