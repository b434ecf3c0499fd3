"""Python objects over the C ABI: FemSystem (fem_assemble ...), Sell
(csr_to_sell ...), pcg_solve and pcg_solve_batched.  Marshalling only:
arguments become pointers and sizes, results come back as torch tensors that
share or copy device memory.  Nothing here computes the method."""
from __future__ import annotations

import ctypes as C
import sys

import torch

from . import gbpcg as G


class _DevArray:
    """Zero-copy view of library-owned device memory (``__cuda_array_interface__``)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3,
                                         "strides": None}


def _view(ptr, shape, dtype):
    typestr = {torch.int32: "<i4", torch.int64: "<i8", torch.float64: "<f8",
               torch.float32: "<f4", torch.int16: "<i2", torch.uint8: "|u1"}[dtype]
    if int(ptr or 0) == 0 or any(s == 0 for s in shape):
        return torch.empty(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


def _opts(tol=1e-10, max_iter=0, precision=G.GB_F64, max_outer=0, inner_tol=0.0, check_every=0,
          use_graph=1, x0_zero=1, spmv_variant=0, persist_off=0, precond=G.GB_PC_JACOBI, method=G.GB_CG):
    return G.PcgOptions(tol, max_iter, precision, max_outer, inner_tol, check_every, use_graph,
                        x0_zero, spmv_variant, persist_off, precond, method)


class FemSystem:
    """An assembled FEM-Laplace system: fem_assemble + fem_system_info."""

    def __init__(self, dim, degree, cells, jitter=0, diag_mode=0, seed=0, stream=None,
                 use_torch_allocator=True):
        self.spec = G.gb_fem_spec(dim, degree, cells, jitter, diag_mode, 0, seed)
        self._stream = stream
        h = C.c_void_p()
        alloc = G.torch_allocator() if use_torch_allocator else None
        G.check(G.lib().fem_assemble(C.byref(self.spec), alloc, G.stream_ptr(stream), C.byref(h)),
                "fem_assemble")
        self.handle = h
        info = G.gb_fem_info()
        G.check(G.lib().fem_system_info(h, C.byref(info)), "fem_system_info")
        self.info = info
        self.n_free, self.n_bnd, self.n_dof = info.n_free, info.n_bnd, info.n_dof
        self.nnz, self.nnz_ib, self.max_row = info.nnz, info.nnz_ib, info.max_row
        self.dim, self.degree = dim, degree

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and G._lib is not None and not sys.is_finalizing():
            torch.cuda.synchronize()
            G._lib.fem_system_destroy(h)
            self.handle = None

    # device views (copied, so they outlive the system)
    def csr(self):
        i = self.info
        return (_view(i.d_rowptr, (self.n_free + 1,), torch.int32).clone(),
                _view(i.d_col, (self.nnz,), torch.int32).clone(),
                _view(i.d_val, (self.nnz,), torch.float64).clone())

    def csr_ib(self):
        i = self.info
        return (_view(i.d_rowptr_ib, (self.n_free + 1,), torch.int32).clone(),
                _view(i.d_col_ib, (self.nnz_ib,), torch.int32).clone(),
                _view(i.d_val_ib, (self.nnz_ib,), torch.float64).clone())

    def diag(self):
        return _view(self.info.d_diag, (self.n_free,), torch.float64).clone()

    def dof_maps(self):
        fof = torch.empty(self.n_free, dtype=torch.int32, device="cuda")
        fob = torch.empty(self.n_bnd, dtype=torch.int32, device="cuda")
        ff = torch.empty(self.n_dof, dtype=torch.int32, device="cuda")
        G.check(G.lib().fem_dof_maps(self.handle, G.ptr(fof), G.ptr(fob), G.ptr(ff),
                                     G.stream_ptr(self._stream)), "fem_dof_maps")
        return fof, fob, ff

    def coords(self, which="bnd"):
        w = 0 if which == "bnd" else 1
        rows = self.n_bnd if w == 0 else self.n_free
        out = torch.empty((rows, self.dim), dtype=torch.float64, device="cuda")
        G.check(G.lib().fem_boundary_coords(self.handle, w, G.ptr(out), G.stream_ptr(self._stream)),
                "fem_boundary_coords")
        return out

    def dirichlet(self, gid, coef=None, k=1, which="bnd"):
        w = 0 if which == "bnd" else 1
        rows = self.n_bnd if w == 0 else self.n_free
        out = torch.empty((rows, k), dtype=torch.float64, device="cuda")
        cp = None
        if coef is not None:
            import numpy as np
            c = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
            cp = c.ctypes.data_as(C.POINTER(C.c_double))
        G.check(G.lib().fem_dirichlet(self.handle, gid, cp, k, w, G.ptr(out), G.stream_ptr(self._stream)),
                "fem_dirichlet")
        return out

    def lift(self, gB):
        gB = gB.contiguous()
        k = 1 if gB.dim() == 1 else gB.shape[1]
        b = torch.empty((self.n_free, k), dtype=torch.float64, device="cuda")
        G.check(G.lib().fem_lift_rhs(self.handle, G.ptr(gB), k, G.ptr(b), G.stream_ptr(self._stream)),
                "fem_lift_rhs")
        return b

    def to_sell(self, C_=32, sigma=256, val_types=G.GB_VAL_F64 | G.GB_VAL_F32, stream=None):
        h = C.c_void_p()
        G.check(G.lib().csr_to_sell(self.handle, C_, sigma, val_types, G.torch_allocator(),
                                    G.stream_ptr(stream if stream is not None else self._stream),
                                    C.byref(h)), "csr_to_sell")
        return Sell(h, stream if stream is not None else self._stream)


_TUNED = {}  # mesh spec + precision -> chosen (C, sigma, variant)


def autotune(system, b, precision=G.GB_F64, val_types=G.GB_VAL_F64 | G.GB_VAL_F32, stream=None):
    """sell_autotune: (Sell in the fastest layout, result dict).  The choice
    is cached per mesh spec and precision; a cached spec builds that layout
    directly."""
    spec = system.spec
    key = (spec.dim, spec.degree, spec.cells, spec.jitter, spec.diag_mode, spec.seed, precision, val_types)
    if key in _TUNED:
        cfg = _TUNED[key]
        A = system.to_sell(cfg["C"], cfg["sigma"], val_types, stream=stream)
        G.check(G.lib().sell_set_variant(A.handle, cfg["spmv_variant"]), "sell_set_variant")
        return A, dict(cfg, cached=True)
    res = G.SellTuneResult()
    h = C.c_void_p()
    G.check(G.lib().sell_autotune(system.handle, G.ptr(b.contiguous().reshape(-1)), precision, val_types,
                                  G.torch_allocator(), G.stream_ptr(stream), C.byref(res), C.byref(h)),
            "sell_autotune")
    cfg = res.as_dict()
    _TUNED[key] = cfg
    return Sell(h, stream), dict(cfg, cached=False)


class Sell:
    """A SELL-C-sigma matrix (csr_to_sell / csr_to_sell_raw)."""

    def __init__(self, handle, stream=None):
        self.handle = handle
        self._stream = stream
        info = G.gb_sell_info()
        G.check(G.lib().sell_info(handle, C.byref(info)), "sell_info")
        self.info = info
        self.n, self.nnz, self.padded, self.nchunks = info.n, info.nnz, info.padded, info.nchunks
        self.C, self.sigma = info.C, info.sigma

    @staticmethod
    def from_csr(rowptr, col, val, C_=32, sigma=256, val_types=G.GB_VAL_F64 | G.GB_VAL_F32, stream=None):
        h = C.c_void_p()
        n = rowptr.numel() - 1
        G.check(G.lib().csr_to_sell_raw(n, G.ptr(rowptr), G.ptr(col), G.ptr(val), C_, sigma, val_types,
                                        G.torch_allocator(), G.stream_ptr(stream), C.byref(h)),
                "csr_to_sell_raw")
        return Sell(h, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and G._lib is not None and not sys.is_finalizing():
            torch.cuda.synchronize()
            G._lib.sell_destroy(h)
            self.handle = None

    def structure(self):
        i = self.info
        return {"perm": _view(i.d_perm, (self.n,), torch.int32).clone(),
                "chunk_ptr": _view(i.d_chunk_ptr, (self.nchunks + 1,), torch.int64).clone(),
                "chunk_w": _view(i.d_chunk_w, (self.nchunks,), torch.int32).clone(),
                "row_len": _view(i.d_row_len, (self.n,), torch.int32).clone(),
                "col": _view(i.d_col, (self.padded,), torch.int32).clone(),
                "val": _view(i.d_val, (self.padded,), torch.float64).clone(),
                "dinv": _view(i.d_dinv, (self.n,), torch.float64).clone(),
                "col16": (None if not i.d_col16 else
                          _view(i.d_col16, (self.padded,), torch.int16).clone())}

    def spmv(self, x):
        y = torch.empty_like(x)
        G.check(G.lib().sell_spmv(self.handle, G.ptr(x.contiguous()), G.ptr(y), G.stream_ptr(self._stream)),
                "sell_spmv")
        return y

    def solve_block(self, B, X0=None, raise_on_fail=True, stream=None, **kw):
        """pcg_solve_block: block CG for the n x k block B (k <= 32); returns (X, stats dict)."""
        B = (B if B.dim() == 2 else B.reshape(-1, 1)).contiguous()
        X = X0.clone().contiguous() if X0 is not None else torch.empty_like(B)
        o = _opts(x0_zero=0 if X0 is not None else 1, **kw)
        st = G.PcgStats()
        rc = G.lib().pcg_solve_block(self.handle, G.ptr(B), G.ptr(X), B.shape[1], C.byref(o),
                                     G.stream_ptr(stream if stream is not None else self._stream), C.byref(st))
        if raise_on_fail:
            G.check(rc, "pcg_solve_block")
        d = st.as_dict()
        d["rc"] = rc
        return X, d

    def block_jacobi(self, bs, stream=None):
        """sell_block_jacobi: attaches the block-Jacobi inverses (bs = 0 detaches them)."""
        G.check(G.lib().sell_block_jacobi(self.handle, int(bs),
                                          G.stream_ptr(stream if stream is not None else self._stream)),
                "sell_block_jacobi")
        return self

    def block_jacobi_info(self):
        """The attached block-Jacobi data: bs, nblk, lam_bound and copies of the packed
        inverses (nblk, bs(bs+1)/2) in fp64 and fp32 and the row positions (nblk*bs)."""
        i = G.gb_bjacobi_info()
        G.check(G.lib().sell_block_jacobi_info(self.handle, C.byref(i)), "sell_block_jacobi_info")
        if i.bs == 0:
            return {"bs": 0}
        T = i.bs * (i.bs + 1) // 2
        return {"bs": i.bs, "nblk": i.nblk, "lam_bound": i.lam_bound,
                "w": _view(i.d_w, (i.nblk, T), torch.float64).clone(),
                "w32": _view(i.d_w32, (i.nblk, T), torch.float32).clone(),
                "loc": _view(i.d_loc, (i.nblk * i.bs,), torch.uint8).clone()}

    def block_jacobi_apply(self, x, stream=None):
        """sell_block_jacobi_apply: y = M^-1 x (free-dof order)."""
        x = x.contiguous()
        y = torch.empty_like(x)
        G.check(G.lib().sell_block_jacobi_apply(self.handle, G.ptr(x), G.ptr(y),
                                                G.stream_ptr(stream if stream is not None else self._stream)),
                "sell_block_jacobi_apply")
        return y

    def kernel_times(self, b, precision=G.GB_F64, iters=50, stream=None):
        """pcg_kernel_times: mean ms of (SpMV + p.Ap, x/r update, p update)."""
        ms = (C.c_double * 3)()
        G.check(G.lib().pcg_kernel_times(self.handle, G.ptr(b.contiguous().reshape(-1)), precision, iters,
                                         G.stream_ptr(stream if stream is not None else self._stream), ms),
                "pcg_kernel_times")
        return list(ms)

    def solve(self, b, x0=None, raise_on_fail=True, stream=None, **kw):
        """pcg_solve: returns (x, stats dict)."""
        b = b.contiguous().reshape(-1)
        x = x0.clone().reshape(-1) if x0 is not None else torch.empty_like(b)
        o = _opts(x0_zero=0 if x0 is not None else 1, **kw)
        st = G.PcgStats()
        rc = G.lib().pcg_solve(self.handle, G.ptr(b), G.ptr(x), C.byref(o),
                               G.stream_ptr(stream if stream is not None else self._stream), C.byref(st))
        if raise_on_fail:
            G.check(rc, "pcg_solve")
        d = st.as_dict()
        d["rc"] = rc
        return x, d


def pcg_solve_batched(mats, Bs, Xs=None, raise_on_fail=True, stream=None, **kw):
    """pcg_solve_batched over Sell matrices with row-major (n, k) blocks."""
    ns = len(mats)
    Bs = [b.contiguous() if b.dim() == 2 else b.contiguous().reshape(-1, 1) for b in Bs]
    if Xs is None:
        Xs = [torch.empty_like(b) for b in Bs]
        kw.setdefault("x0_zero", 1)
    else:
        Xs = [x.contiguous() if x.dim() == 2 else x.contiguous().reshape(-1, 1) for x in Xs]
        kw.setdefault("x0_zero", 0)
    A_arr = (C.c_void_p * ns)(*[m.handle.value for m in mats])
    B_arr = (C.c_void_p * ns)(*[b.data_ptr() for b in Bs])
    X_arr = (C.c_void_p * ns)(*[x.data_ptr() for x in Xs])
    k_arr = (C.c_int * ns)(*[b.shape[1] for b in Bs])
    o = _opts(**kw)
    stats = (G.PcgStats * ns)()
    rc = G.lib().pcg_solve_batched(ns, A_arr, B_arr, X_arr, k_arr, C.byref(o), G.stream_ptr(stream), stats)
    if raise_on_fail:
        G.check(rc, "pcg_solve_batched")
    return Xs, [dict(s.as_dict(), rc=rc) for s in stats]


def batched_kernel_times(mats, Bs, precision=G.GB_F64, iters=20, stream=None):
    """pcg_batched_kernel_times: mean ms of (SpMM + p.Ap, X/R update, P update)
    of the blocked multi-RHS iteration over the given systems."""
    ns = len(mats)
    Bs = [b.contiguous() if b.dim() == 2 else b.contiguous().reshape(-1, 1) for b in Bs]
    A_arr = (C.c_void_p * ns)(*[m.handle.value for m in mats])
    B_arr = (C.c_void_p * ns)(*[b.data_ptr() for b in Bs])
    k_arr = (C.c_int * ns)(*[b.shape[1] for b in Bs])
    ms = (C.c_double * 3)()
    G.check(G.lib().pcg_batched_kernel_times(ns, A_arr, B_arr, k_arr, precision, iters, G.stream_ptr(stream), ms),
            "pcg_batched_kernel_times")
    return list(ms)


def autotune_rhs_width(A, B, precision=G.GB_F64, stream=None):
    """pcg_batched_autotune_width: the RHS block width (columns per system of
    the batch) with the fastest blocked iteration for the n x k block B;
    returns (width, {width: iteration ms})."""
    B = B.contiguous()
    k = B.shape[1]
    best = C.c_int(0)
    ms = (C.c_double * 6)()
    G.check(G.lib().pcg_batched_autotune_width(A.handle, G.ptr(B), k, precision, G.stream_ptr(stream),
                                               C.byref(best), ms), "pcg_batched_autotune_width")
    return best.value, {w: ms[i] for i, w in enumerate((1, 2, 4, 8, 16, 32)) if w <= k}


def solve_multi(A, B, width, stream=None, **kw):
    """pcg_solve_batched over groups of `width` columns of the n x k block B
    (the blocked multi-RHS solve of Eq. MRH); returns (X, per-group stats)."""
    B = B.contiguous()
    groups = [B[:, j:j + width].contiguous() for j in range(0, B.shape[1], width)]
    Xs, sts = pcg_solve_batched([A] * len(groups), groups, stream=stream, **kw)
    return torch.cat(Xs, dim=1), sts


def wait_selftest(limit_ms=20.0, stream=None):
    """gbpcg_wait_selftest: (status code, milliseconds the bounded wait waited)."""
    waited = C.c_double(0.0)
    rc = G.lib().gbpcg_wait_selftest(float(limit_ms), G.stream_ptr(stream), C.byref(waited))
    return rc, waited.value


def grid_wait_selftest(limit_ms=20.0, stream=None):
    """gbpcg_grid_wait_selftest: (status code, milliseconds the grid kernel ran)."""
    waited = C.c_double(0.0)
    rc = G.lib().gbpcg_grid_wait_selftest(float(limit_ms), G.stream_ptr(stream), C.byref(waited))
    return rc, waited.value


class Server:
    """serve_create / serve_submit / serve_poll: a continuous-batching solve
    server.  Host result buffers (numpy, n_free x k) are kept here until the
    request completes."""

    def __init__(self, mem_budget=40 << 30, max_slots=64, precision=G.GB_F32_RU, tol=1e-10,
                 max_iter=0, iters_per_step=0, device=-1, cluster_lane=0):
        import numpy as np  # noqa: F401
        o = G.ServeOptions(int(mem_budget), max_slots, precision, tol, max_iter, iters_per_step, device,
                           cluster_lane)
        h = C.c_void_p()
        # no caller allocator: the server allocates from its own stream-ordered
        # pool (its thread would otherwise call back into Python)
        G.check(G.lib().serve_create(C.byref(o), None, C.byref(h)), "serve_create")
        self.handle = h
        self._live = {}

    @staticmethod
    def sizes(dim, degree, cells):
        S = degree * cells + 1
        return (S - 2) ** dim, S ** dim - (S - 2) ** dim  # n_free, n_bnd

    def submit(self, dim, degree, cells, jitter=0, diag_mode=0, seed=0, k=1, gid=1, coef=None, gB=None):
        import numpy as np
        n_free, n_bnd = self.sizes(dim, degree, cells)
        x = np.zeros((n_free, k))
        keep = [x]
        req = G.ServeRequest()
        req.spec = G.gb_fem_spec(dim, degree, cells, jitter, diag_mode, 0, seed)
        req.k, req.gid = k, gid
        req.h_x = x.ctypes.data_as(C.POINTER(C.c_double))
        if coef is not None:
            c = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
            keep.append(c)
            req.h_coef = c.ctypes.data_as(C.POINTER(C.c_double))
        if gB is not None:
            g = np.ascontiguousarray(gB, dtype=np.float64).reshape(n_bnd, k)
            keep.append(g)
            req.h_gB = g.ctypes.data_as(C.POINTER(C.c_double))
        t = C.c_uint64()
        G.check(G.lib().serve_submit(self.handle, C.byref(req), C.byref(t)), "serve_submit")
        self._live[t.value] = keep
        return t.value

    def poll(self, ticket):
        """None while pending, else (result dict, x)."""
        r = G.ServeResult()
        rc = G.lib().serve_poll(self.handle, ticket, C.byref(r))
        if rc == G.GB_PENDING:
            return None
        if rc == G.GB_EINVAL and ticket not in self._live:
            G.check(rc, "serve_poll")
        keep = self._live.pop(ticket)
        return r.as_dict(), keep[0]

    def wait(self, tickets, timeout_s=600.0, sleep_s=0.001):
        import time
        out, left = {}, set(tickets)
        t0 = time.time()
        while left:
            for t in list(left):
                r = self.poll(t)
                if r is not None:
                    out[t] = r
                    left.discard(t)
            if left:
                if time.time() - t0 > timeout_s:
                    raise TimeoutError(f"{len(left)} requests still pending")
                time.sleep(sleep_s)
        return out

    def stats(self):
        st = G.ServeStats()
        G.check(G.lib().serve_stats(self.handle, C.byref(st)), "serve_stats")
        return st.as_dict()

    def close(self):
        h = getattr(self, "handle", None)
        if h and G._lib is not None:
            G._lib.serve_destroy(h)
            self.handle = None

    def __del__(self):
        if not sys.is_finalizing():
            self.close()
