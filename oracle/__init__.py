"""Plain CPU oracle for the FEM-Laplace Jacobi-PCG path (fp64, single thread).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product package never imports it.
The C source (``oracle.c``) shares no code with the CUDA library.

Each wrapper follows the passage named in ``oracle.c``: the Laplace/Dirichlet
problem and the P1 cotangent weights of Sec. 2.2, the P1-P4 degree study of
Sec. 4.2 (P1 and P2 here), the preconditioned Krylov solve of Sec. 2.1, the
stopping rule of Eq. (2) and the error metric of Eq. (1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def _compile(out, extra, force):
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off"] + extra +
                              ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, single thread): the
    pinned oracle.  Also compiles the same source with -fopenmp into
    liboracle_omp.so, a timing build for the all-core CPU baseline only."""
    _compile(_LIB_OMP, ["-fopenmp"], force)
    return _compile(_LIB, [], force)


_lib = None
_lib_omp = None


def lib_omp(threads):
    """The OpenMP timing build of the same source (the all-core CPU baseline;
    nothing is checked against it), set to `threads` threads."""
    global _lib_omp
    if _lib_omp is None:
        build()
        L = C.CDLL(_LIB_OMP)
        P = C.POINTER
        L.orc_pcg.restype = C.c_int
        L.orc_pcg.argtypes = [C.c_int64, P(C.c_int64), P(C.c_int32), P(C.c_double), P(C.c_double),
                              P(C.c_double), C.c_double, C.c_int64, P(C.c_int64), P(C.c_double)]
        L.omp_set_num_threads.argtypes = [C.c_int]
        _lib_omp = L
    _lib_omp.omp_set_num_threads(int(threads))
    return _lib_omp


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        i64p, i32p, f64p, u8p = P(C.c_int64), P(C.c_int32), P(C.c_double), P(C.c_uint8)
        L.orc_rng_u64.restype = C.c_uint64
        L.orc_rng_u64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_rng_key.restype = C.c_uint64
        L.orc_rng_key.argtypes = [C.c_uint64, C.c_uint32]
        L.orc_mesh.restype = C.c_void_p
        L.orc_mesh.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64]
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_sizes.argtypes = [C.c_void_p, i64p]
        L.orc_get_vertex_coords.argtypes = [C.c_void_p, f64p]
        L.orc_get_dof_coords.argtypes = [C.c_void_p, f64p]
        L.orc_get_elements.argtypes = [C.c_void_p, i32p]
        L.orc_get_maps.argtypes = [C.c_void_p, i32p, i32p, i32p, i32p]
        L.orc_element_matrix.argtypes = [C.c_void_p, C.c_int64, f64p]
        L.orc_assemble.restype = C.c_int
        L.orc_assemble.argtypes = [C.c_void_p, u8p]
        for f in (L.orc_get_full, L.orc_get_ii, L.orc_get_ib):
            f.argtypes = [C.c_void_p, i64p, i32p, f64p]
        L.orc_eval_g.restype = C.c_int
        L.orc_eval_g.argtypes = [C.c_void_p, C.c_int, f64p, C.c_int, C.c_int, f64p]
        L.orc_lift.argtypes = [C.c_void_p, f64p, C.c_int, f64p]
        L.orc_spmv.argtypes = [C.c_int64, i64p, i32p, f64p, f64p, f64p]
        L.orc_pcg.restype = C.c_int
        L.orc_pcg.argtypes = [C.c_int64, i64p, i32p, f64p, f64p, f64p, C.c_double, C.c_int64,
                              i64p, f64p]
        L.orc_pcg_bj.restype = C.c_int
        L.orc_pcg_bj.argtypes = [C.c_int64, i64p, i32p, f64p, C.c_int, f64p, f64p, C.c_double,
                                 C.c_int64, i64p, f64p]
        L.orc_bjacobi.restype = C.c_int
        L.orc_bjacobi.argtypes = [C.c_int64, i64p, i32p, f64p, C.c_int, f64p]
        L.orc_bjacobi_apply.argtypes = [C.c_int64, C.c_int, f64p, f64p, f64p]
        L.orc_bicgstab.restype = C.c_int
        L.orc_bicgstab.argtypes = [C.c_int64, i64p, i32p, f64p, C.c_int, f64p, f64p, C.c_double, C.c_int64,
                                   i64p, f64p]
        L.orc_block_cg.restype = C.c_int
        L.orc_block_cg.argtypes = [C.c_int64, i64p, i32p, f64p, C.c_int, f64p, f64p, C.c_double, C.c_int64,
                                   i64p, f64p]
        L.orc_cholesky_solve.restype = C.c_int
        L.orc_cholesky_solve.argtypes = [C.c_int64, i64p, i32p, f64p, f64p, f64p]
        L.orc_sell_size.argtypes = [C.c_int64, i64p, C.c_int, C.c_int, i64p, i64p]
        L.orc_sell_fill.argtypes = [C.c_int64, i64p, i32p, f64p, C.c_int, C.c_int, i32p, i64p,
                                    i32p, i32p, i32p, f64p]
        _lib = L
    return _lib


def _p(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


# Dirichlet data ids (same meaning on the device side)
G_SIN_SINH, G_X2_Y2, G_X2_Y2_2Z2, G_LINEAR, G_HARMONIC = 0, 1, 2, 3, 4
NCOEF = {G_SIN_SINH: 0, G_X2_Y2: 0, G_X2_Y2_2Z2: 0, G_LINEAR: 4, G_HARMONIC: 10}


def rng_u64(key: int, i: int) -> int:
    return int(lib().orc_rng_u64(key, i))


def rng_key(seed: int, stream: int) -> int:
    return int(lib().orc_rng_key(seed, stream))


class System:
    """Mesh, dofs, assembled stiffness and its Dirichlet split (Sec. 2.2)."""

    def __init__(self, dim, degree, cells, jitter=0, diag_mode=0, seed=0):
        self.dim, self.degree, self.cells = dim, degree, cells
        self._h = lib().orc_mesh(dim, degree, cells, jitter, diag_mode, seed)
        if not self._h:
            raise ValueError("invalid mesh spec")
        self._sizes()
        self.assembled = False

    def _sizes(self):
        s = np.zeros(9, np.int64)
        lib().orc_sizes(self._h, _p(s, C.c_int64))
        (self.n_vertices, self.n_dof, self.n_elements, self.n_loc, self.n_free,
         self.n_bnd, self.nnz_full, self.nnz_ii, self.nnz_ib) = (int(v) for v in s)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    # -- mesh ----------------------------------------------------------------
    def vertex_coords(self):
        a = np.empty((self.n_vertices, self.dim))
        lib().orc_get_vertex_coords(self._h, _p(a, C.c_double))
        return a

    def dof_coords(self):
        a = np.empty((self.n_dof, self.dim))
        lib().orc_get_dof_coords(self._h, _p(a, C.c_double))
        return a

    def elements(self):
        a = np.empty((self.n_elements, self.n_loc), np.int32)
        lib().orc_get_elements(self._h, _p(a, C.c_int32))
        return a

    def maps(self):
        fof = np.empty(self.n_dof, np.int32)
        bof = np.empty(self.n_dof, np.int32)
        foff = np.empty(max(self.n_free, 1), np.int32)[: self.n_free]
        fofb = np.empty(max(self.n_bnd, 1), np.int32)[: self.n_bnd]
        lib().orc_get_maps(self._h, _p(fof, C.c_int32), _p(bof, C.c_int32),
                           _p(foff, C.c_int32), _p(fofb, C.c_int32))
        return fof, bof, foff, fofb

    def element_matrix(self, e):
        a = np.empty((self.n_loc, self.n_loc))
        lib().orc_element_matrix(self._h, e, _p(a, C.c_double))
        return a

    # -- assembly ------------------------------------------------------------
    def assemble(self, row_mask=None):
        m = None if row_mask is None else np.ascontiguousarray(row_mask, dtype=np.uint8)
        rc = lib().orc_assemble(self._h, _p(m, C.c_uint8))
        if rc:
            raise RuntimeError("oracle assembly failed")
        self._sizes()
        self.assembled = True
        return self

    def _csr(self, fn, nrows, nnz):
        rp = np.empty(nrows + 1, np.int64)
        ci = np.empty(max(nnz, 1), np.int32)[:nnz]
        v = np.empty(max(nnz, 1))[:nnz]
        fn(self._h, _p(rp, C.c_int64), _p(ci, C.c_int32), _p(v, C.c_double))
        return rp, ci, v

    def full(self):
        return self._csr(lib().orc_get_full, self.n_dof, self.nnz_full)

    def k_ii(self):
        return self._csr(lib().orc_get_ii, self.n_free, self.nnz_ii)

    def k_ib(self):
        return self._csr(lib().orc_get_ib, self.n_free, self.nnz_ib)

    # -- Dirichlet data ------------------------------------------------------
    def eval_g(self, gid, coef=None, k=1, which="bnd"):
        rows = self.n_bnd if which == "bnd" else self.n_free
        out = np.empty((rows, k))
        c = None if coef is None else np.ascontiguousarray(coef, dtype=np.float64)
        rc = lib().orc_eval_g(self._h, gid, _p(c, C.c_double), k, 0 if which == "bnd" else 1,
                              _p(out, C.c_double))
        if rc:
            raise ValueError("bad Dirichlet id")
        return out

    def lift(self, gB):
        gB = np.ascontiguousarray(gB, dtype=np.float64)
        k = 1 if gB.ndim == 1 else gB.shape[1]
        b = np.empty((self.n_free, k))
        lib().orc_lift(self._h, _p(gB, C.c_double), k, _p(b, C.c_double))
        return b[:, 0] if gB.ndim == 1 else b


def spmv(rp, ci, v, x):
    n = len(rp) - 1
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n)
    lib().orc_spmv(n, _p(rp, C.c_int64), _p(ci, C.c_int32), _p(v, C.c_double),
                   _p(x, C.c_double), _p(y, C.c_double))
    return y


def pcg(rp, ci, v, b, tol=1e-10, maxit=None, x0=None, bs=None, threads=None):
    """PCG to ||b-Ax||/||b|| <= tol (Eq. 2) with the Jacobi preconditioner, or
    with block-Jacobi over blocks of bs consecutive rows when bs is given.
    threads (Jacobi only): run the OpenMP timing build on that many threads.
    Returns (x, status, iters, relres)."""
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    it = np.zeros(1, np.int64)
    rr = np.zeros(1)
    maxit = 20 * n + 100 if maxit is None else maxit
    args = (_p(b, C.c_double), _p(x, C.c_double), tol, maxit, _p(it, C.c_int64), _p(rr, C.c_double))
    A = (n, _p(rp, C.c_int64), _p(ci, C.c_int32), _p(v, C.c_double))
    if threads:
        st = lib_omp(threads).orc_pcg(*A, *args)
    else:
        st = lib().orc_pcg(*A, *args) if bs is None else lib().orc_pcg_bj(*A, int(bs), *args)
    return x, int(st), int(it[0]), float(rr[0])


def bicgstab(rp, ci, v, b, tol=1e-10, maxit=None, x0=None, bs=0):
    """Right-preconditioned BiCGSTAB (Jacobi for bs <= 1, block-Jacobi over bs
    rows otherwise).  Returns (x, status, iters, relres)."""
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    it = np.zeros(1, np.int64)
    rr = np.zeros(1)
    maxit = 20 * n + 100 if maxit is None else maxit
    st = lib().orc_bicgstab(n, _p(rp, C.c_int64), _p(ci, C.c_int32), _p(v, C.c_double), int(bs),
                            _p(b, C.c_double), _p(x, C.c_double), tol, maxit, _p(it, C.c_int64),
                            _p(rr, C.c_double))
    return x, int(st), int(it[0]), float(rr[0])


def block_cg(rp, ci, v, B, tol=1e-10, maxit=None, X0=None):
    """Block CG (breakdown-free, Jacobi-preconditioned) for A X = B, B (n, k).
    Returns (X, status, iters, relres per column)."""
    n = len(rp) - 1
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(n, -1))
    k = B.shape[1]
    X = np.zeros((n, k)) if X0 is None else np.array(X0, dtype=np.float64).reshape(n, k)
    it = np.zeros(1, np.int64)
    rel = np.zeros(k)
    maxit = 20 * n + 100 if maxit is None else maxit
    st = lib().orc_block_cg(n, _p(rp, C.c_int64), _p(ci, C.c_int32), _p(v, C.c_double), k,
                            _p(B.reshape(-1), C.c_double), _p(X.reshape(-1), C.c_double), tol, maxit,
                            _p(it, C.c_int64), _p(rel, C.c_double))
    return X, int(st), int(it[0]), rel


def bjacobi(rp, ci, v, bs):
    """Block-Jacobi inverses: array (ceil(n/bs), bs, bs), a short last block in
    its leading corner (zeros elsewhere)."""
    n = len(rp) - 1
    nblk = (n + bs - 1) // bs
    W = np.zeros(max(nblk, 1) * bs * bs)
    if lib().orc_bjacobi(n, _p(rp, C.c_int64), _p(ci, C.c_int32), _p(v, C.c_double), int(bs),
                         _p(W, C.c_double)):
        raise np.linalg.LinAlgError("a diagonal block is not SPD")
    return W[:nblk * bs * bs].reshape(nblk, bs, bs)


def bjacobi_apply(bs, W, r):
    """z = M^{-1} r for the block inverses W of bjacobi()."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    z = np.empty_like(r)
    lib().orc_bjacobi_apply(len(r), int(bs), _p(W.reshape(-1), C.c_double), _p(r, C.c_double),
                            _p(z, C.c_double))
    return z


def cholesky_solve(rp, ci, v, b):
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n)
    st = lib().orc_cholesky_solve(n, _p(rp, C.c_int64), _p(ci, C.c_int32), _p(v, C.c_double),
                                  _p(b, C.c_double), _p(x, C.c_double))
    if st:
        raise np.linalg.LinAlgError("matrix is not SPD")
    return x


def sell(rp, ci, v, C_, sigma):
    """SELL-C-sigma structure: (perm, chunk_ptr, chunk_w, row_len, col, val)."""
    n = len(rp) - 1
    nc = np.zeros(1, np.int64)
    pad = np.zeros(1, np.int64)
    lib().orc_sell_size(n, _p(rp, C.c_int64), C_, sigma, _p(nc, C.c_int64), _p(pad, C.c_int64))
    nc, pad = int(nc[0]), int(pad[0])
    perm = np.empty(max(n, 1), np.int32)[:n]
    cp = np.empty(nc + 1, np.int64)
    cw = np.empty(max(nc, 1), np.int32)[:nc]
    rl = np.empty(max(n, 1), np.int32)[:n]
    col = np.empty(max(pad, 1), np.int32)[:pad]
    val = np.empty(max(pad, 1))[:pad]
    lib().orc_sell_fill(n, _p(rp, C.c_int64), _p(ci, C.c_int32),
                        None if v is None else _p(v, C.c_double), C_, sigma,
                        _p(perm, C.c_int32), _p(cp, C.c_int64), _p(cw, C.c_int32),
                        _p(rl, C.c_int32), _p(col, C.c_int32),
                        None if v is None else _p(val, C.c_double))
    return perm, cp, cw, rl, col, val


def x_err(x_true, x):
    """Relative solution error of Eq. (1)."""
    x_true = np.asarray(x_true)
    return float(np.linalg.norm(x_true - x) / np.linalg.norm(x_true))


def solve_system(dim, degree, cells, jitter=0, diag_mode=0, seed=0, gid=G_X2_Y2, coef=None,
                 k=1, tol=1e-13, method="pcg"):
    """Whole oracle path: mesh, assembly, lift, solve.  Returns (System, b, x, info)."""
    s = System(dim, degree, cells, jitter, diag_mode, seed).assemble()
    gB = s.eval_g(gid, coef, k, "bnd")
    b = s.lift(gB)
    rp, ci, v = s.k_ii()
    xs, infos = [], []
    for c in range(k):
        if method == "chol":
            xs.append(cholesky_solve(rp, ci, v, b[:, c]))
            infos.append((0, 0, 0.0))
        else:
            x, st, it, rr = pcg(rp, ci, v, b[:, c], tol=tol)
            xs.append(x)
            infos.append((st, it, rr))
    return s, b, np.stack(xs, axis=1), infos
