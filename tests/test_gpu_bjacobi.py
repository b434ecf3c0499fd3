"""GPU parity: the block-Jacobi preconditioner (the paper's Block-Jacobi,
Sec. 3.2 and Sec. 4.2) against the oracle.

- the device's block inverses (Gauss-Jordan, symmetrised, packed) equal the
  oracle's (Cholesky solves against unit vectors) to 1e-12 of each block's
  largest entry; the fp32 copy is the fp64 value rounded to nearest; the row
  positions are bit-exact (they come from the SELL permutation, itself
  bit-exact against the oracle's); the eigenvalue bound is the oracle's
  largest absolute row sum and bounds every block's spectrum;
- z = M^-1 x agrees with the oracle's apply;
- PCG with M solves to Eq. (2)'s 1e-10 with the oracle's iteration count (up
  to rounding drift) and the oracle's solution (Eq. 1 error 1e-8); the
  fp32/bf16 inner refinement reaches the same tolerance; one block holding
  every row makes it a direct solve (one iteration)."""
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


def _unpack(w, bs):
    nblk = w.shape[0]
    W = np.zeros((nblk, bs, bs))
    k = 0
    for a in range(bs):
        for c in range(a, bs):
            W[:, a, c] = w[:, k]
            W[:, c, a] = w[:, k]
            k += 1
    return W


CASES = [  # dim, degree, cells, jitter, diag_mode, seed  (n: 1024, 289, 216, 343, 89401, 3969)
    (2, 1, 33, 1, 1, 5), (2, 2, 9, 1, 1, 3), (3, 1, 7, 0, 0, 0), (3, 2, 4, 1, 0, 10),
    (2, 1, 300, 1, 1, 3), (2, 1, 64, 0, 0, 0)]


def _gid(dim):
    return O.G_X2_Y2_2Z2 if dim == 3 else O.G_X2_Y2


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("bs", [1, 2, 4, 8, 16, 32])
def test_blocks_match_oracle(P, case, bs):
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256).block_jacobi(bs)
    info = A.block_jacobi_info()
    n = d.n_free
    nblk = (n + bs - 1) // bs
    assert info["bs"] == bs and info["nblk"] == nblk
    w = info["w"].cpu().numpy()
    Wd = _unpack(w, bs)
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    Wo = O.bjacobi(rp, ci, v, bs)
    scale = np.abs(Wo).reshape(nblk, -1).max(axis=1)[:, None, None]
    assert np.all(np.abs(Wd - Wo) <= 1e-12 * scale)
    assert np.array_equal(info["w32"].cpu().numpy(), w.astype(np.float32))
    # row positions from the oracle's SELL permutation (perm[new] = old)
    perm = O.sell(rp, ci, v, 32, 256)[0]
    iperm = np.empty(n, np.int64)
    iperm[perm] = np.arange(n)
    o = np.arange(n)
    loc = info["loc"].cpu().numpy()
    assert np.array_equal(loc[:n].astype(np.int64), iperm - 256 * (o // 256))
    assert np.all(loc[n:] == 0)
    rows = np.abs(Wo).sum(axis=2).max()
    assert abs(info["lam_bound"] - rows) <= 1e-12 * rows
    lmax = max(np.linalg.eigvalsh(Wo[j]).max() for j in range(0, nblk, max(1, nblk // 64)))
    assert info["lam_bound"] >= lmax * (1 - 1e-12)  # (the two sides round the inverses differently)


@pytest.mark.parametrize("case,bs", [(CASES[0], 4), (CASES[1], 8), (CASES[3], 32), (CASES[4], 16), (CASES[2], 1)])
def test_apply_matches_oracle(P, case, bs):
    import torch
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256).block_jacobi(bs)
    x = np.random.default_rng(7).standard_normal(d.n_free)
    y = A.block_jacobi_apply(torch.tensor(x, device="cuda")).cpu().numpy()
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    yo = O.bjacobi_apply(bs, O.bjacobi(rp, ci, v, bs), x)
    assert np.allclose(y, yo, rtol=1e-12, atol=1e-12 * np.abs(yo).max())


@pytest.mark.parametrize("case,bs", [
    ((2, 1, 96, 1, 1, 1), 4), ((2, 2, 48, 1, 1, 1), 8), ((3, 1, 20, 0, 0, 0), 4),
    ((3, 2, 10, 1, 0, 2), 16), ((2, 1, 64, 0, 0, 0), 32), ((2, 2, 30, 1, 1, 6), 1)])
def test_fp64_solve_matches_oracle(P, case, bs):
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256).block_jacobi(bs)
    gid = _gid(case[0])
    b = d.lift(d.dirichlet(gid))[:, 0]
    x, st = A.solve(b, tol=TOL, precond=P.GB_PC_BLOCK_JACOBI, max_iter=200000)
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    bo = s.lift(s.eval_g(gid))[:, 0]
    xo, sto, ito, _ = O.pcg(rp, ci, v, bo, tol=TOL, bs=bs)
    xe, _, _, _ = O.pcg(rp, ci, v, bo, tol=1e-13, bs=bs)
    xd = x.cpu().numpy()
    relres = np.linalg.norm(bo - O.spmv(rp, ci, v, xd)) / np.linalg.norm(bo)
    assert st["status"] == 0 and st["relres"] <= TOL and relres <= 1.5 * TOL
    assert O.x_err(xe, xd) <= XERR
    assert abs(st["iterations"] - ito) <= max(3, 0.02 * ito)


@pytest.mark.parametrize("prec", ["F32_IR", "BF16_IR"])
@pytest.mark.parametrize("case,bs", [((2, 2, 64, 1, 1, 2), 4), ((3, 1, 24, 1, 0, 1), 8)])
def test_inner_refinement_with_block_jacobi(P, prec, case, bs):
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32 | P.GB_VAL_BF16).block_jacobi(bs)
    b = d.lift(d.dirichlet(_gid(case[0])))[:, 0]
    precision = getattr(P, "GB_" + prec)
    x, st = A.solve(b, tol=TOL, precision=precision, precond=P.GB_PC_BLOCK_JACOBI, max_iter=200000)
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    bo = s.lift(s.eval_g(_gid(case[0])))[:, 0]
    xd = x.cpu().numpy()
    assert st["status"] == 0
    assert np.linalg.norm(bo - O.spmv(rp, ci, v, xd)) / np.linalg.norm(bo) <= 1.5 * TOL
    xe = O.pcg(rp, ci, v, bo, tol=1e-13)[0]
    assert O.x_err(xe, xd) <= XERR


@pytest.mark.parametrize("case,bs", [((2, 1, 5, 1, 1, 7), 16), ((2, 1, 5, 1, 1, 7), 32), ((3, 1, 3, 0, 0, 0), 8),
                                     ((2, 2, 3, 1, 1, 2), 32)])
def test_one_block_is_a_direct_solve(P, case, bs):
    d = P.FemSystem(*case)
    assert d.n_free <= bs
    A = d.to_sell(32, 256).block_jacobi(bs)
    b = d.lift(d.dirichlet(_gid(case[0])))[:, 0]
    x, st = A.solve(b, tol=1e-13, precond=P.GB_PC_BLOCK_JACOBI)
    assert st["status"] == 0 and st["iterations"] == 1
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    xc = O.cholesky_solve(rp, ci, v, s.lift(s.eval_g(_gid(case[0])))[:, 0])
    assert O.x_err(xc, x.cpu().numpy()) <= 1e-12


def test_fewer_iterations_than_jacobi_2d(P):
    d = P.FemSystem(2, 2, 128, 1, 1, 1)
    A = d.to_sell(32, 256).block_jacobi(4)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    _, s1 = A.solve(b, tol=TOL)
    _, s4 = A.solve(b, tol=TOL, precond=P.GB_PC_BLOCK_JACOBI)
    assert s1["status"] == 0 and s4["status"] == 0
    assert s4["iterations"] < 0.9 * s1["iterations"]


def test_sigma_one_and_reattach(P):
    """sigma = 1 (no permutation): positions are the identity; a second call
    replaces the blocks, bs = 0 detaches them."""
    d = P.FemSystem(2, 1, 40, 1, 1, 2)
    A = d.to_sell(32, 1).block_jacobi(8)
    info = A.block_jacobi_info()
    n = d.n_free
    assert np.array_equal(info["loc"].cpu().numpy()[:n].astype(np.int64), np.arange(n) % 256)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    _, s8 = A.solve(b, tol=TOL, precond=P.GB_PC_BLOCK_JACOBI)
    A.block_jacobi(2)
    assert A.block_jacobi_info()["bs"] == 2
    _, s2 = A.solve(b, tol=TOL, precond=P.GB_PC_BLOCK_JACOBI)
    assert s8["status"] == 0 and s2["status"] == 0
    A.block_jacobi(0)
    assert A.block_jacobi_info()["bs"] == 0
    with pytest.raises(P.GbError):
        A.solve(b, tol=TOL, precond=P.GB_PC_BLOCK_JACOBI)


def test_bad_arguments(P):
    d = P.FemSystem(2, 1, 20, 1, 1, 2)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    with pytest.raises(P.GbError):
        A.block_jacobi(3)
    with pytest.raises(P.GbError):
        A.block_jacobi(64)
    with pytest.raises(P.GbError):
        d.to_sell(32, 512).block_jacobi(4)  # sigma must divide 256
    with pytest.raises(P.GbError):
        A.solve(b, precond=P.GB_PC_BLOCK_JACOBI)  # nothing attached
    A.block_jacobi(4)
    with pytest.raises(P.GbError):
        A.solve(b, precond=P.GB_PC_BLOCK_JACOBI, precision=P.GB_F32_RU)
    with pytest.raises(P.GbError):
        A.solve(b, precond=7)
    with pytest.raises(P.GbError):
        P.pcg_solve_batched([A], [b], precond=P.GB_PC_BLOCK_JACOBI)


def test_kernel_times_block_jacobi(P):
    d = P.FemSystem(2, 2, 64, 1, 1, 1)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32).block_jacobi(4)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    for prec in (P.GB_F64, P.GB_F32_IR):
        ms = A.kernel_times(b, precision=prec | P.gbpcg.GB_KT_BLOCK_JACOBI, iters=5)
        assert all(t > 0 for t in ms)


def test_blocks_full_size_2d_p2(P):
    """2D jittered P2 512x512 cells (n = 1 046 529, 4089 windows): every block
    against the oracle, and a full solve to Eq. (2)."""
    case = (2, 2, 512, 1, 1, 1)
    bs = 4
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256).block_jacobi(bs)
    info = A.block_jacobi_info()
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    Wo = O.bjacobi(rp, ci, v, bs)
    Wd = _unpack(info["w"].cpu().numpy(), bs)
    scale = np.abs(Wo).reshape(Wo.shape[0], -1).max(axis=1)[:, None, None]
    assert np.all(np.abs(Wd - Wo) <= 1e-12 * scale)
    b = d.lift(d.dirichlet(O.G_X2_Y2))[:, 0]
    x, st = A.solve(b, tol=TOL, precond=P.GB_PC_BLOCK_JACOBI)
    xd = x.cpu().numpy()
    bo = s.lift(s.eval_g(O.G_X2_Y2))[:, 0]
    assert st["status"] == 0
    assert np.linalg.norm(bo - O.spmv(rp, ci, v, xd)) / np.linalg.norm(bo) <= 1.5 * TOL
    # P2 reproduces x^2 - y^2 at the nodes
    X = d.coords("free").cpu().numpy()
    assert O.x_err(X[:, 0] ** 2 - X[:, 1] ** 2, xd) <= XERR
