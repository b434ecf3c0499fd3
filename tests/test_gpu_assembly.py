"""GPU parity: device assembly and SELL conversion against the CPU oracle.

Integer output (pattern, dof maps, SELL permutation/chunks/columns) must be
bit-exact; coordinates too (both sides evaluate the same correctly rounded
expressions); stiffness values within 1e-13 of the row's largest entry (the
two sides sum the same element terms in a different order and with or without
fused multiply-adds: a few ulps of the row scale)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

CASES = [  # dim, degree, cells, jitter, diag_mode, seed
    (2, 1, 2, 0, 0, 0),       # smallest mesh: one interior dof
    (2, 1, 17, 0, 0, 0),
    (2, 1, 33, 1, 1, 5),
    (2, 2, 9, 1, 1, 3),
    (2, 2, 24, 0, 1, 7),
    (3, 1, 7, 0, 0, 0),
    (3, 2, 5, 0, 0, 0),
    (3, 1, 6, 1, 0, 9),       # jittered 3D (irregular tetrahedra)
    (3, 2, 4, 1, 0, 10),
]

VAL_RTOL = 1e-13


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05413_gb300 as P
    P.load()
    return P


def _oracle(case):
    dim, deg, cells, jit, dm, seed = case
    return O.System(dim, deg, cells, jit, dm, seed).assemble()


def _rowscale(rp, v):
    return np.maximum.reduceat(np.abs(v), rp[:-1]) if len(v) else np.zeros(0)


@pytest.mark.parametrize("case", CASES)
def test_pattern_maps_coords_bitexact(P, case):
    dim, deg, cells, jit, dm, seed = case
    s = _oracle(case)
    d = P.FemSystem(dim, deg, cells, jit, dm, seed)
    assert (d.n_free, d.n_bnd, d.n_dof, d.nnz, d.nnz_ib) == (s.n_free, s.n_bnd, s.n_dof, s.nnz_ii, s.nnz_ib)
    rp, ci, v = (t.cpu().numpy() for t in d.csr())
    orp, oci, ov = s.k_ii()
    assert np.array_equal(rp.astype(np.int64), orp)
    assert np.array_equal(ci, oci)
    rpb, cib, vb = (t.cpu().numpy() for t in d.csr_ib())
    brp, bci, bv = s.k_ib()
    assert np.array_equal(rpb.astype(np.int64), brp)
    assert np.array_equal(cib, bci)
    fof, fob, ff = (t.cpu().numpy() for t in d.dof_maps())
    ofof, obof, ofoff, ofofb = s.maps()
    assert np.array_equal(fof, ofoff) and np.array_equal(fob, ofofb) and np.array_equal(ff, ofof)
    X = s.dof_coords()
    assert np.array_equal(d.coords("bnd").cpu().numpy(), X[ofofb])
    assert np.array_equal(d.coords("free").cpu().numpy(), X[ofoff])


@pytest.mark.parametrize("case", CASES)
def test_values_and_lift(P, case):
    dim, deg, cells, jit, dm, seed = case
    s = _oracle(case)
    d = P.FemSystem(dim, deg, cells, jit, dm, seed)
    rp, ci, v = (t.cpu().numpy() for t in d.csr())
    orp, oci, ov = s.k_ii()
    scale = np.repeat(_rowscale(orp, ov), np.diff(orp))
    assert np.all(np.abs(v - ov) <= VAL_RTOL * scale)
    # diag view = the diagonal entries
    diag = d.diag().cpu().numpy()
    rows = np.repeat(np.arange(d.n_free), np.diff(orp))
    assert np.array_equal(diag, v[ci == rows])
    # K_IB
    _, _, vb = (t.cpu().numpy() for t in d.csr_ib())
    _, _, ovb = s.k_ib()
    assert np.all(np.abs(vb - ovb) <= VAL_RTOL * np.abs(ov).max())
    # device K_II is bit-exactly symmetric
    import scipy.sparse as sp
    K = sp.csr_matrix((v, ci, rp), shape=(d.n_free, d.n_free))
    assert (K != K.T).nnz == 0
    # Dirichlet data and lift
    gid = O.G_X2_Y2_2Z2 if dim == 3 else O.G_X2_Y2
    gB = d.dirichlet(gid)
    ogB = s.eval_g(gid)
    assert np.allclose(gB.cpu().numpy(), ogB, rtol=0, atol=1e-15)
    b = d.lift(gB).cpu().numpy()
    ob = s.lift(ogB)
    assert np.all(np.abs(b - ob) <= 1e-12 * max(1.0, np.abs(ob).max()))


def test_dirichlet_all_functions(P):
    s = _oracle((2, 2, 8, 1, 1, 2))
    d = P.FemSystem(2, 2, 8, 1, 1, 2)
    rng = np.random.default_rng(0)
    for gid in (O.G_SIN_SINH, O.G_X2_Y2, O.G_LINEAR, O.G_HARMONIC):
        k = 3 if O.NCOEF[gid] else 1
        coef = rng.standard_normal((k, O.NCOEF[gid])) if O.NCOEF[gid] else None
        for which in ("bnd", "free"):
            got = d.dirichlet(gid, coef, k, which).cpu().numpy()
            want = s.eval_g(gid, coef, k, which)
            assert np.allclose(got, want, rtol=1e-13, atol=1e-14), (gid, which)


@pytest.mark.parametrize("case", [CASES[2], CASES[3], CASES[6]])
@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 64), (64, 256), (128, 7)])
def test_sell_structure_bitexact(P, case, C, sigma):
    dim, deg, cells, jit, dm, seed = case
    s = _oracle(case)
    d = P.FemSystem(dim, deg, cells, jit, dm, seed)
    A = d.to_sell(C, sigma)
    st = {k: t.cpu().numpy() for k, t in A.structure().items() if t is not None}
    orp, oci, ov = s.k_ii()
    perm, cp, cw, rl, col, val = O.sell(orp, oci, ov, C, sigma)
    assert np.array_equal(st["perm"], perm)
    assert np.array_equal(st["chunk_ptr"], cp)
    assert np.array_equal(st["chunk_w"], cw)
    assert np.array_equal(st["row_len"], rl)
    assert np.array_equal(st["col"], col)
    scale = np.abs(ov).max()
    assert np.all(np.abs(st["val"] - val) <= VAL_RTOL * scale)
    assert np.allclose(st["dinv"], 1.0 / np.array([ov[orp[i]:orp[i + 1]][oci[orp[i]:orp[i + 1]] == i][0]
                                                    for i in range(len(orp) - 1)])[perm], rtol=1e-13)


@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[5], CASES[6]])
def test_sell_spmv_matches_oracle(P, case):
    import torch
    dim, deg, cells, jit, dm, seed = case
    s = _oracle(case)
    d = P.FemSystem(dim, deg, cells, jit, dm, seed)
    A = d.to_sell(32, 128)
    x = np.random.default_rng(1).standard_normal(d.n_free)
    y = A.spmv(torch.tensor(x, device="cuda")).cpu().numpy()
    orp, oci, ov = s.k_ii()
    yo = O.spmv(orp, oci, ov, x)
    assert np.allclose(y, yo, rtol=1e-12, atol=1e-12 * np.abs(yo).max())


def test_assembly_deterministic(P):
    a = P.FemSystem(2, 2, 40, 1, 1, 9).csr()[2].cpu().numpy()
    b = P.FemSystem(2, 2, 40, 1, 1, 9).csr()[2].cpu().numpy()
    assert np.array_equal(a, b)


def test_bad_specs_raise(P):
    with pytest.raises(P.GbError):
        P.FemSystem(4, 1, 8)
    with pytest.raises(P.GbError):
        P.FemSystem(3, 1, 8, jitter=1, diag_mode=1)  # 3D: the Kuhn split only
    with pytest.raises(P.GbError):
        P.FemSystem(2, 5, 8)
    with pytest.raises(P.GbError):
        P.FemSystem(2, 1, 1)


@pytest.mark.parametrize("case", [CASES[2], CASES[3], CASES[6]])
def test_sell_col16_deltas_reconstruct_columns(P, case):
    """16-bit deltas + min(row, n-1) give back every padded column index."""
    dim, deg, cells, jit, dm, seed = case
    d = P.FemSystem(dim, deg, cells, jit, dm, seed)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32 | P.gbpcg.GB_IDX16)
    st = {k: (t.cpu().numpy() if t is not None else None) for k, t in A.structure().items()}
    assert st["col16"] is not None
    n = d.n_free
    cp, cw = st["chunk_ptr"], st["chunk_w"]
    rows = np.zeros(len(st["col"]), np.int64)
    for c in range(len(cw)):
        w = cw[c]
        rr = np.arange(c * 32, c * 32 + 32)
        rows[cp[c]:cp[c + 1]] = np.tile(np.minimum(rr, n - 1), w)
    real = np.zeros(len(st["col"]), bool)
    for c in range(len(cw)):
        rr = np.arange(c * 32, c * 32 + 32)
        real[cp[c]:cp[c + 1]] = np.tile(rr < n, cw[c])
    rec = rows + st["col16"].astype(np.int64)
    assert np.array_equal(rec[real], st["col"][real].astype(np.int64))
    assert np.all((rec >= 0) & (rec < n))


def test_idx16_spmv_solve_matches_int32(P):
    """A solve streaming 16-bit deltas equals the 32-bit-index solve (same arithmetic)."""
    d = P.FemSystem(2, 2, 300, 1, 1, 3)
    b = d.lift(d.dirichlet(1))[:, 0]
    A32 = d.to_sell(32, 256)
    A16 = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32 | P.gbpcg.GB_IDX16)
    for prec in (P.GB_F64, P.GB_F32_RU):
        x1, s1 = A32.solve(b, precision=prec)
        x2, s2 = A16.solve(b, precision=prec)
        assert s1["iterations"] == s2["iterations"] and bool((x1 == x2).all())
