"""GPU parity: P3 and P4 Lagrange elements (the degree study of Sec. 4.2,
Table 7) on regular and jittered meshes, against the oracle.

Integer output (pattern, dof maps) and the node coordinates (both sides
evaluate (sum of beta_a P_a over the node's face, ascending vertex id) / m
with correctly rounded operations) bit-exact; stiffness values
within 1e-13 of the row's largest entry (the two sides tabulate the reference
integrals by different summations); solves reproduce the cubic (P3) and
quartic (P4) harmonic polynomials at the nodes and match the oracle's
solution."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

CASES = [(2, 3, 6, 0, 1, 3), (2, 4, 4, 0, 0, 0), (2, 4, 5, 0, 1, 2), (3, 3, 3, 0, 0, 0), (3, 4, 2, 0, 0, 0),
         (2, 3, 7, 1, 1, 4), (2, 4, 5, 1, 1, 6), (3, 3, 3, 1, 0, 2), (3, 4, 3, 1, 0, 5)]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05413_gb300 as P
    P.load()
    return P


@pytest.mark.parametrize("case", CASES)
def test_assembly_matches_oracle(P, case):
    dim, deg, cells, jit, dm, seed = case
    s = O.System(*case).assemble()
    d = P.FemSystem(*case)
    assert (d.n_free, d.n_bnd, d.nnz, d.nnz_ib) == (s.n_free, s.n_bnd, s.nnz_ii, s.nnz_ib)
    rp, ci, v = (t.cpu().numpy() for t in d.csr())
    orp, oci, ov = s.k_ii()
    assert np.array_equal(rp.astype(np.int64), orp) and np.array_equal(ci, oci)
    scale = np.repeat(np.maximum.reduceat(np.abs(ov), orp[:-1]), np.diff(orp))
    assert np.all(np.abs(v - ov) <= 1e-13 * scale)
    rpb, cib, vb = (t.cpu().numpy() for t in d.csr_ib())
    brp, bci, bv = s.k_ib()
    assert np.array_equal(rpb.astype(np.int64), brp) and np.array_equal(cib, bci)
    assert np.all(np.abs(vb - bv) <= 1e-13 * np.abs(ov).max())
    fof, fob, ff = (t.cpu().numpy() for t in d.dof_maps())
    ofof, obof, ofoff, ofofb = s.maps()
    assert np.array_equal(fof, ofoff) and np.array_equal(fob, ofofb)
    X = s.dof_coords()
    assert np.array_equal(d.coords("free").cpu().numpy(), X[ofoff])
    assert np.array_equal(d.coords("bnd").cpu().numpy(), X[ofofb])
    import scipy.sparse as sp
    K = sp.csr_matrix((v, ci, rp), shape=(d.n_free, d.n_free))
    assert (K != K.T).nnz == 0


def _harmonic(k):
    """coefficients of Re (x + iy)^k in the harmonic basis (gid 4)"""
    c = np.zeros((1, 10))
    c[0, 2 * k] = 1.0
    return c


@pytest.mark.parametrize("case,k", [((2, 3, 8, 0, 1, 4), 3), ((2, 4, 6, 0, 1, 5), 4), ((3, 3, 4, 0, 0, 0), 3),
                                    ((3, 4, 3, 0, 0, 0), 4), ((2, 3, 8, 1, 1, 4), 3), ((2, 4, 6, 1, 1, 5), 4),
                                    ((3, 3, 4, 1, 0, 1), 3), ((3, 4, 3, 1, 0, 2), 4)])
def test_exact_reproduction(P, case, k):
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256)
    coef = _harmonic(k)
    b = d.lift(d.dirichlet(O.G_HARMONIC, coef))[:, 0]
    x, st = A.solve(b, tol=1e-13, max_iter=200000)
    want = d.dirichlet(O.G_HARMONIC, coef, which="free")[:, 0]
    assert st["status"] == 0
    assert float((x - want).abs().max() / want.abs().max()) <= 1e-9


@pytest.mark.parametrize("case", [(2, 3, 24, 0, 1, 1), (2, 4, 16, 0, 1, 1), (3, 3, 6, 0, 0, 0), (2, 4, 16, 1, 1, 3),
                                  (3, 3, 6, 1, 0, 4)])
def test_solve_matches_oracle(P, case):
    d = P.FemSystem(*case)
    A = d.to_sell(32, 256)
    gid = O.G_X2_Y2_2Z2 if case[0] == 3 else O.G_SIN_SINH
    b = d.lift(d.dirichlet(gid))[:, 0]
    x, st = A.solve(b, tol=1e-10, max_iter=200000)
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    bo = s.lift(s.eval_g(gid))[:, 0]
    xo = O.pcg(rp, ci, v, bo, tol=1e-13)[0]
    xd = x.cpu().numpy()
    assert st["status"] == 0
    assert np.linalg.norm(bo - O.spmv(rp, ci, v, xd)) / np.linalg.norm(bo) <= 1.5e-10
    assert O.x_err(xo, xd) <= 1e-8


def test_degree_5_rejected(P):
    with pytest.raises(P.GbError):
        P.FemSystem(2, 5, 8)
