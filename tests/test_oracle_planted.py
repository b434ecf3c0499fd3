"""The pins of the block-Jacobi, block CG, BiCGSTAB (its steps and its restart
after a breakdown) and P3/P4 oracle functions
catch plausible mistakes: each test builds a wrong variant (in numpy, on the
CPU) and shows that the pin that passes for the oracle rejects it."""
import math

import numpy as np

import oracle as O

from test_oracle_bicgstab import (BREAK_AFTER_PROGRESS, BREAK_AFTER_PROGRESS_B, BREAK_AFTER_PROGRESS_X,
                                   BREAK_AT_ONCE, BREAK_AT_ONCE_B)
from test_oracle_bjacobi import _tridiag_inverse, _dense_block
from test_oracle_p34 import _stiffness_by_quadrature, _elem_vertices


def _K(case):
    s = O.System(*case).assemble()
    rp, ci, v = s.k_ii()
    n = len(rp) - 1
    K = np.zeros((n, n))
    K[np.repeat(np.arange(n), np.diff(rp)), ci] = v
    return s, rp, ci, v, K


def test_bjacobi_closed_form_rejects_offset_blocks():
    """Blocks starting one row late (rows [j bs + 1, (j+1) bs + 1)) give other
    inverses than the x-line closed form; the oracle's blocks match it."""
    cells, bs = 20, 4
    _, rp, ci, v, K = _K((2, 1, cells, 0, 0, 0))
    n, line = len(rp) - 1, cells - 1
    W = O.bjacobi(rp, ci, v, bs)
    want0 = _tridiag_inverse(bs, 1.0, 2.0)  # block 0: rows 0..3 of the first x-line
    assert np.allclose(W[0], want0, rtol=1e-12)
    wrong0 = np.linalg.inv(K[1:1 + bs, 1:1 + bs])
    assert np.allclose(wrong0, _tridiag_inverse(bs, 1.0, 2.0), rtol=1e-12)  # same shape inside one line ...
    # ... but the offset blocks cross the line end at a different row: block 4 of the
    # correct partition (rows 16..19) holds rows 16-18 of line 0 and row 0 of line 1
    j = 4
    right = W[j][:bs, :bs]
    wrong = np.linalg.inv(K[j * bs + 1:(j + 1) * bs + 1, j * bs + 1:(j + 1) * bs + 1])
    seg = line - (j * bs) % line  # rows to the end of the line
    want = np.zeros((bs, bs))
    want[:seg, :seg] = _tridiag_inverse(seg, 1.0, 2.0)
    want[seg:, seg:] = _tridiag_inverse(bs - seg, 1.0, 2.0)
    assert np.allclose(right, want, rtol=1e-12, atol=1e-15)
    assert not np.allclose(wrong, want, rtol=1e-6, atol=1e-9)


def test_bjacobi_identity_rejects_dropped_short_block():
    """A short last block left at the identity (a dropped ragged block) fails
    the block-times-inverse pin; the oracle's passes."""
    _, rp, ci, v, K = _K((2, 1, 10, 1, 1, 3))
    n, bs = len(rp) - 1, 4
    W = O.bjacobi(rp, ci, v, bs)
    j = W.shape[0] - 1
    m = n - j * bs
    B = _dense_block(rp, ci, v, j * bs, m)
    assert np.allclose(W[j][:m, :m] @ B, np.eye(m), atol=1e-12)
    assert not np.allclose(np.eye(m) @ B, np.eye(m), atol=1e-3)


def _block_cg_numpy(K, B, tol, maxit, beta_sign=1.0):
    """breakdown-free block CG as in the oracle (Jacobi), with a switch that
    plants the mistake of a flipped beta"""
    d = 1.0 / np.diag(K)
    X = np.zeros_like(B)
    R = B.copy()
    bn = np.linalg.norm(B, axis=0)

    def orth(W, R):
        cw = 1.0 / np.linalg.norm(R, axis=0)
        G = (W * cw).T @ (W * cw)
        lam, V = np.linalg.eigh(G)
        keep = lam > 1e-12 * lam.max()
        return (W * cw) @ (V[:, keep] / np.sqrt(lam[keep]))

    P = orth(d[:, None] * R, R)
    for it in range(1, maxit + 1):
        Q = K @ P
        PtQ = P.T @ Q
        al = np.linalg.solve(PtQ, P.T @ R)
        X += P @ al
        R -= Q @ al
        if np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            return it
        Z = d[:, None] * R
        be = -np.linalg.solve(PtQ, Q.T @ Z)
        P = orth(Z + beta_sign * (P @ be), R)
    return maxit + 1


def test_block_cg_finite_termination_rejects_flipped_beta():
    _, rp, ci, v, K = _K((2, 1, 5, 1, 1, 7))
    n, k = K.shape[0], 4
    B = np.random.default_rng(4).standard_normal((n, k))
    bound = math.ceil(n / k) + 1
    _, st, it, _ = O.block_cg(rp, ci, v, B, tol=1e-11)
    assert st == 0 and it <= bound
    assert _block_cg_numpy(K, B, 1e-11, 50) <= bound
    assert _block_cg_numpy(K, B, 1e-11, 50, beta_sign=-1.0) > bound


def _bicgstab_numpy(K, b, tol, maxit, omega_inverted=False):
    d = 1.0 / np.diag(K)
    x = np.zeros_like(b)
    r = b.copy()
    rh = r.copy()
    p = np.zeros_like(b)
    vv = np.zeros_like(b)
    rho0 = alpha = omega = 1.0
    bn = np.linalg.norm(b)
    for it in range(1, maxit + 1):
        rho = rh @ r
        beta = (rho / rho0) * (alpha / omega)
        p = r + beta * (p - omega * vv)
        ph = d * p
        vv = K @ ph
        alpha = rho / (rh @ vv)
        s = r - alpha * vv
        if np.linalg.norm(s) <= tol * bn:
            return it
        sh = d * s
        t = K @ sh
        omega = (t @ t) / (t @ s) if omega_inverted else (t @ s) / (t @ t)
        x += alpha * ph + omega * sh
        r = s - omega * t
        if np.linalg.norm(r) <= tol * bn:
            return it
        rho0 = rho
    return maxit + 1


def test_bicgstab_pin_rejects_inverted_omega():
    """omega = t.t / t.s instead of t.s / t.t: the recurrence still terminates
    on tiny systems (its BiCG part does not depend on omega), but on the
    Cholesky pin's systems it no longer converges, while the oracle does -- in
    fewer steps than CG."""
    s, rp, ci, v, K = _K((2, 1, 30, 1, 1, 3))
    b = s.lift(s.eval_g(O.G_X2_Y2))[:, 0]
    _, st, it, rel = O.bicgstab(rp, ci, v, b, tol=1e-10)
    its_cg = O.pcg(rp, ci, v, b, tol=1e-10)[2]
    assert st == 0 and it <= its_cg
    assert _bicgstab_numpy(K, b, 1e-10, 2 * its_cg) <= its_cg
    with np.errstate(all="ignore"):
        assert _bicgstab_numpy(K, b, 1e-10, 2 * its_cg, omega_inverted=True) > 2 * its_cg


def test_p3_quadrature_pin_rejects_transposed_nodes():
    s = O.System(2, 3, 2, jitter=1, diag_mode=1, seed=3)
    X = s.dof_coords()
    E = s.elements()
    nodes = X[E[0]]
    P = _elem_vertices(s, 0, X, E)
    Ko = s.element_matrix(0)
    Kq = _stiffness_by_quadrature(nodes, P, 3)
    assert np.abs(Ko - Kq).max() <= 1e-9 * np.abs(Kq).max()
    wrong = nodes.copy()
    wrong[[1, 2]] = wrong[[2, 1]]  # two edge nodes swapped
    Kw = _stiffness_by_quadrature(wrong, P, 3)
    assert np.abs(Ko - Kw).max() > 1e-3 * np.abs(Kq).max()


def _bicgstab_restarting(A, b, tol, maxit=100, restart="oracle"):
    """Jacobi BiCGSTAB with the oracle's breakdown rule (restart from the true
    residual with a new shadow vector while the residual has fallen below 0.9
    of the one the recurrence started from; else report status 2), and three
    planted mistakes: restart="none" (a breakdown ends the solve), "keep_shadow"
    (the restart keeps the old shadow vector), "no_guard" (restart however
    little the residual fell).  Returns (x, status, steps)."""
    d = 1.0 / np.diag(A)
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    it, restarts, broke, rel_start = 0, 0, False, np.inf
    rh = None
    while True:
        r = b - A @ x
        rel = np.linalg.norm(r) / bn
        if rel <= tol:
            return x, 0, it
        if it >= maxit or restarts > 50:
            return x, 1, it
        if broke and (restart == "none" or (restart != "no_guard" and not rel < 0.9 * rel_start)):
            return x, 2, it
        broke, rel_start = False, rel
        if rh is not None:  # every start after the first is a restart
            restarts += 1
        if rh is None or restart != "keep_shadow":
            rh = r.copy()
        p = np.zeros_like(b)
        vv = np.zeros_like(b)
        rho0 = alpha = omega = 1.0
        while it < maxit:
            rho = rh @ r
            if rho == 0.0:
                broke = True
                break
            p = r + (rho / rho0) * (alpha / omega) * (p - omega * vv)
            ph = d * p
            vv = A @ ph
            rv = rh @ vv
            if rv == 0.0:
                broke = True
                break
            alpha = rho / rv
            s = r - alpha * vv
            it += 1
            if np.linalg.norm(s) <= tol * bn:
                x = x + alpha * ph
                break
            sh = d * s
            t = A @ sh
            omega = (t @ s) / (t @ t)
            x = x + alpha * ph + omega * sh
            r = s - omega * t
            if np.linalg.norm(r) <= tol * bn:
                break
            rho0 = rho
        else:
            return x, 1, it


def test_bicgstab_restart_pin_rejects_no_restart_and_stale_shadow():
    """After a breakdown that follows progress the oracle restarts and reaches
    the solution; ending the solve at the breakdown, or restarting with the
    old shadow vector (whose product with the new residual is zero again),
    report a breakdown instead."""
    A, b, xs = BREAK_AFTER_PROGRESS, BREAK_AFTER_PROGRESS_B, BREAK_AFTER_PROGRESS_X
    x, st, it = _bicgstab_restarting(A, b, 1e-13)
    assert st == 0 and np.abs(x - xs).max() <= 1e-14
    for wrong in ("none", "keep_shadow"):
        x, st, it = _bicgstab_restarting(A, b, 1e-13, restart=wrong)
        assert st == 2 and np.abs(x - xs).max() > 0.1, wrong


def test_bicgstab_breakdown_pin_rejects_unguarded_restart():
    """A breakdown before any progress is reported after 0 steps by the oracle;
    restarting without the 0.9 test repeats the same breakdown until the
    restart cap and returns 'not converged' (status 1) instead."""
    A, b = BREAK_AT_ONCE, BREAK_AT_ONCE_B
    x, st, it = _bicgstab_restarting(A, b, 1e-12)
    assert st == 2 and it == 0
    x, st, it = _bicgstab_restarting(A, b, 1e-12, restart="no_guard")
    assert st == 1
