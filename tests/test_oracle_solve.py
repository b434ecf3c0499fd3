"""Oracle pins: solutions, PCG behaviour, Cholesky, SELL structure (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O


def test_cfg1_closed_form():
    """64x64 regular P1 = 5-point FD system with g = sin(pi x) sinh(pi y)/sinh(pi).
    Separation of variables gives its exact discrete solution
    u_ij = sin(pi i h) sinh(mu j) / sinh(64 mu), cosh(mu) = 2 - cos(pi h), h = 1/64."""
    s, b, x, info = O.solve_system(2, 1, 64, gid=O.G_SIN_SINH, tol=1e-13)
    assert info[0][0] == 0
    h = 1.0 / 64
    mu = np.arccosh(2.0 - np.cos(np.pi * h))
    _, _, foff, _ = s.maps()
    X = s.dof_coords()[foff]
    i = np.rint(X[:, 0] * 64)
    j = np.rint(X[:, 1] * 64)
    u = np.sin(np.pi * i * h) * np.sinh(mu * j) / np.sinh(64 * mu)
    assert O.x_err(u, x[:, 0]) < 1e-12
    # the discrete solution is O(h^2) from the analytic one (Eq. 1 error metric)
    ua = np.sin(np.pi * X[:, 0]) * np.sinh(np.pi * X[:, 1]) / np.sinh(np.pi)
    err = O.x_err(ua, x[:, 0])
    assert 1e-5 < err < 1e-3


@pytest.mark.parametrize("dim,deg,cells,jit,gid,coef", [
    (2, 1, 12, 1, O.G_LINEAR, [0.5, 1.0, -2.0, 0.0]),        # P1 exact on linear data
    (2, 2, 10, 1, O.G_X2_Y2, None),                          # P2 exact on x^2-y^2
    (2, 1, 12, 0, O.G_X2_Y2, None),                          # 5-point exact on quadratics
    (3, 1, 6, 0, O.G_X2_Y2_2Z2, None),                       # Kuhn 7-point exact on quadratics
    (3, 2, 4, 0, O.G_X2_Y2_2Z2, None),                       # P2 exact on quadratics
    (3, 1, 5, 0, O.G_LINEAR, [1.0, -0.5, 0.25, 2.0]),
    (3, 1, 6, 1, O.G_LINEAR, [1.0, -0.5, 0.25, 2.0]),       # jittered 3D: P1 exact on linear data
    (3, 2, 4, 1, O.G_X2_Y2_2Z2, None),                       # jittered 3D: P2 exact on quadratics
])
def test_exact_reproduction(dim, deg, cells, jit, gid, coef):
    s, b, x, info = O.solve_system(dim, deg, cells, jitter=jit, diag_mode=1, seed=3, gid=gid,
                                   coef=coef, tol=1e-14)
    u = s.eval_g(gid, coef, 1, "free")[:, 0]
    assert O.x_err(u, x[:, 0]) < 1e-11


def test_p1_jittered_not_exact_on_quadratics():
    """Sanity: a jittered P1 mesh does not reproduce x^2-y^2 (so the exactness pins
    above are informative)."""
    s, b, x, info = O.solve_system(2, 1, 12, jitter=1, diag_mode=1, seed=3, gid=O.G_X2_Y2, tol=1e-14)
    u = s.eval_g(O.G_X2_Y2, None, 1, "free")[:, 0]
    assert O.x_err(u, x[:, 0]) > 1e-5


@pytest.mark.parametrize("dim,deg,cells", [(2, 1, 10), (2, 2, 6), (3, 1, 4), (3, 2, 3)])
def test_pcg_matches_cholesky(dim, deg, cells):
    s = O.System(dim, deg, cells, jitter=1 if dim == 2 else 0, diag_mode=1, seed=17).assemble()
    rp, ci, v = s.k_ii()
    rng = np.random.default_rng(1)
    b = rng.standard_normal(s.n_free)
    xc = O.cholesky_solve(rp, ci, v, b)
    x, st, it, rr = O.pcg(rp, ci, v, b, tol=1e-13)
    assert st == 0 and rr <= 1e-13
    assert O.x_err(xc, x) < 1e-10
    # the Cholesky solve itself against numpy's dense solver
    A = sp.csr_matrix((v, ci, rp), shape=(s.n_free, s.n_free)).toarray()
    assert O.x_err(np.linalg.solve(A, b), xc) < 1e-12


def test_pcg_matches_scipy_spsolve_medium():
    s = O.System(2, 2, 48, jitter=1, diag_mode=1, seed=1).assemble()
    rp, ci, v = s.k_ii()
    b = s.lift(s.eval_g(O.G_HARMONIC, np.linspace(-1, 1, 10), 1, "bnd"))[:, 0]
    A = sp.csr_matrix((v, ci, rp), shape=(s.n_free, s.n_free))
    xs = spla.spsolve(A.tocsc(), b)
    x, st, it, rr = O.pcg(rp, ci, v, b, tol=1e-13)
    assert st == 0
    assert O.x_err(xs, x) < 1e-9
    # recursive-residual stop confirmed on the true residual (Eq. 2)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-13


def test_pcg_edge_cases():
    s = O.System(2, 1, 6).assemble()
    rp, ci, v = s.k_ii()
    n = s.n_free
    x, st, it, rr = O.pcg(rp, ci, v, np.zeros(n))
    assert st == 0 and it == 0 and np.all(x == 0)
    b = np.ones(n)
    x, st, it, rr = O.pcg(rp, ci, v, b, tol=1e-12, maxit=3)
    assert st == 1 and it == 3
    x, st, it, rr = O.pcg(rp, ci, v * -1.0, b)  # planted: negated K -> p.Ap < 0
    assert st == 2
    x, st, it, rr = O.pcg(rp, ci, v, b, tol=1e-10, x0=np.linalg.solve(
        sp.csr_matrix((v, ci, rp)).toarray(), b))
    assert st == 0 and it == 0  # warm start at the solution


def test_cholesky_rejects_indefinite():
    s = O.System(2, 1, 4).assemble()
    rp, ci, v = s.k_ii()
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky_solve(rp, ci, -v, np.ones(s.n_free))


def test_multi_rhs_lift_columns_independent():
    s = O.System(2, 2, 6, jitter=1, diag_mode=1, seed=2).assemble()
    coef = np.random.default_rng(3).standard_normal((3, 10))
    gB = s.eval_g(O.G_HARMONIC, coef, 3, "bnd")
    b = s.lift(gB)
    for c in range(3):
        g1 = s.eval_g(O.G_HARMONIC, coef[c], 1, "bnd")
        assert np.array_equal(g1[:, 0], gB[:, c])
        assert np.array_equal(s.lift(g1)[:, 0], b[:, c])


def test_harmonic_basis_is_harmonic_polynomials():
    """Re/Im (x+iy)^k evaluated by the oracle equal the complex powers."""
    s = O.System(2, 2, 5, jitter=1, diag_mode=1, seed=2)
    X = s.dof_coords()
    _, _, foff, _ = s.maps()
    z = X[foff, 0] + 1j * X[foff, 1]
    for k in range(5):
        for part in range(2):
            c = np.zeros(10); c[2 * k + part] = 1.0
            got = s.eval_g(O.G_HARMONIC, c, 1, "free")[:, 0]
            want = (z ** k).real if part == 0 else (z ** k).imag
            assert np.allclose(got, want, rtol=0, atol=1e-14)


def test_p2_exact_for_low_harmonics_cfg4_style():
    """Columns built only from k<=2 harmonics are reproduced exactly by P2."""
    s = O.System(2, 2, 16, jitter=1, diag_mode=1, seed=2).assemble()
    coef = np.zeros((2, 10))
    coef[0, :6] = [0.3, 0.0, -1.0, 0.5, 2.0, -0.7]
    coef[1, :6] = [1.0, 0.0, 0.0, 1.0, -1.0, 0.0]
    b = s.lift(s.eval_g(O.G_HARMONIC, coef, 2, "bnd"))
    rp, ci, v = s.k_ii()
    u = s.eval_g(O.G_HARMONIC, coef, 2, "free")
    for c in range(2):
        x, st, it, rr = O.pcg(rp, ci, v, b[:, c], tol=1e-14)
        assert O.x_err(u[:, c], x) < 1e-11


# ------------------------------------------------------------------- SELL --
@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 64), (8, 16), (32, 256), (4, 7)])
def test_sell_structure_brute_force(C, sigma):
    s = O.System(2, 2, 9, jitter=1, diag_mode=1, seed=8).assemble()
    rp, ci, v = s.k_ii()
    n = s.n_free
    perm, cp, cw, rl, col, val = O.sell(rp, ci, v, C, sigma)
    L = np.diff(rp)
    # permutation: stable descending-length sort inside each sigma window
    want = []
    for w0 in range(0, n, max(sigma, 1)):
        idx = list(range(w0, min(w0 + max(sigma, 1), n)))
        want += sorted(idx, key=lambda i: -L[i]) if sigma > 1 else idx
    assert np.array_equal(perm, np.array(want))
    iperm = np.empty(n, np.int64); iperm[perm] = np.arange(n)
    assert np.array_equal(rl, L[perm])
    nch = (n + C - 1) // C
    for c in range(nch):
        rows = perm[c * C:(c + 1) * C]
        assert cw[c] == L[rows].max()
        assert cp[c + 1] - cp[c] == cw[c] * C
    # SpMV through the padded layout equals CSR SpMV (in permuted numbering)
    x = np.random.default_rng(0).standard_normal(n)
    y_csr = O.spmv(rp, ci, v, x)
    xp = x[perm]
    y = np.zeros(n)
    for c in range(nch):
        for t in range(C):
            r = c * C + t
            if r >= n:
                continue
            for j in range(cw[c]):
                k = cp[c] + j * C + t
                y[r] += val[k] * xp[col[k]]
    assert np.allclose(y, y_csr[perm], rtol=1e-14, atol=1e-14)
    # padding points at the row itself with value 0
    for c in range(nch):
        for t in range(C):
            r = c * C + t
            if r < n:
                for j in range(rl[r], cw[c]):
                    k = cp[c] + j * C + t
                    assert col[k] == r and val[k] == 0.0
