"""Thin ctypes binding of libgbpcg.so (the C ABI declared in include/gbpcg.h).

Argument marshalling only: every step of assembly, format conversion and the
solves runs in the library's CUDA kernels.  PyTorch supplies device memory
(``torch.cuda.caching_allocator_alloc``) and streams.  There is no fallback:
if the library cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbpcg.so")

GB_OK, GB_EINVAL, GB_ENOMEM, GB_ECUDA = 0, -1, -2, -3
GB_NOT_CONVERGED, GB_BREAKDOWN, GB_TIMEOUT, GB_TOO_LARGE, GB_PENDING = -4, -5, -6, -7, 1
GB_VAL_F64, GB_VAL_F32, GB_VAL_BF16, GB_IDX16 = 1, 2, 4, 8
GB_F64, GB_F32_IR, GB_BF16_IR, GB_F32_RU, GB_BF16_RU = 0, 1, 2, 3, 4
GB_PC_JACOBI, GB_PC_BLOCK_JACOBI = 0, 1
GB_KT_BLOCK_JACOBI = 256
GB_CG, GB_BICGSTAB = 0, 1
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "NOT_CONVERGED",
                -5: "BREAKDOWN", -6: "TIMEOUT", -7: "TOO_LARGE", 1: "PENDING"}


class GbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class gb_allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p),
                ("alloc", C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p))]


class gb_fem_spec(C.Structure):
    _fields_ = [("dim", C.c_int32), ("degree", C.c_int32), ("cells", C.c_int32),
                ("jitter", C.c_int32), ("diag_mode", C.c_int32), ("reserved", C.c_int32),
                ("seed", C.c_uint64)]


class gb_fem_info(C.Structure):
    _fields_ = [("n_dof", C.c_int64), ("n_free", C.c_int64), ("n_bnd", C.c_int64),
                ("nnz", C.c_int64), ("nnz_ib", C.c_int64),
                ("dim", C.c_int32), ("degree", C.c_int32), ("cells", C.c_int32), ("side", C.c_int32),
                ("max_row", C.c_int32), ("reserved", C.c_int32),
                ("d_rowptr", C.c_void_p), ("d_col", C.c_void_p), ("d_val", C.c_void_p),
                ("d_rowptr_ib", C.c_void_p), ("d_col_ib", C.c_void_p), ("d_val_ib", C.c_void_p),
                ("d_diag", C.c_void_p)]


class gb_sell_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("padded", C.c_int64), ("nchunks", C.c_int64),
                ("C", C.c_int32), ("sigma", C.c_int32), ("max_row", C.c_int32), ("reserved", C.c_int32),
                ("d_perm", C.c_void_p), ("d_chunk_ptr", C.c_void_p), ("d_chunk_w", C.c_void_p),
                ("d_row_len", C.c_void_p), ("d_col", C.c_void_p), ("d_val", C.c_void_p),
                ("d_dinv", C.c_void_p), ("d_col16", C.c_void_p)]


class PcgOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int64), ("precision", C.c_int32),
                ("max_outer", C.c_int32), ("inner_tol", C.c_double), ("check_every", C.c_int32),
                ("use_graph", C.c_int32), ("x0_zero", C.c_int32), ("spmv_variant", C.c_int32),
                ("persist_off", C.c_int32), ("precond", C.c_int32), ("method", C.c_int32)]


class PcgStats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("restarts", C.c_int64), ("outer", C.c_int32),
                ("status", C.c_int32), ("relres", C.c_double), ("bnorm", C.c_double),
                ("solve_ms", C.c_double), ("kernel_launches", C.c_int64), ("bytes_moved", C.c_double),
                ("fallback_iterations", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class gb_bjacobi_info(C.Structure):
    _fields_ = [("bs", C.c_int32), ("reserved", C.c_int32), ("nblk", C.c_int64), ("d_w", C.c_void_p),
                ("d_w32", C.c_void_p), ("d_loc", C.c_void_p), ("lam_bound", C.c_double)]


class SellTuneResult(C.Structure):
    _fields_ = [("C", C.c_int32), ("sigma", C.c_int32), ("spmv_variant", C.c_int32),
                ("candidates", C.c_int32), ("iter_ms", C.c_double), ("spmv_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServeOptions(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("max_slots", C.c_int32), ("precision", C.c_int32),
                ("tol", C.c_double), ("max_iter", C.c_int64), ("iters_per_step", C.c_int32),
                ("device", C.c_int32), ("cluster_lane", C.c_int32)]


class ServeRequest(C.Structure):
    _fields_ = [("spec", gb_fem_spec), ("k", C.c_int32), ("gid", C.c_int32),
                ("h_coef", C.POINTER(C.c_double)), ("h_gB", C.POINTER(C.c_double)),
                ("h_x", C.POINTER(C.c_double))]


class ServeResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("k", C.c_int32), ("n", C.c_int64), ("iterations", C.c_int64),
                ("updates", C.c_int32), ("reserved", C.c_int32), ("relres", C.c_double),
                ("queue_ms", C.c_double), ("latency_ms", C.c_double), ("bytes", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64),
                ("pending", C.c_int64), ("resident", C.c_int64), ("steps", C.c_int64),
                ("mem_in_use", C.c_double), ("mem_peak", C.c_double), ("max_resident", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_P = C.c_void_p
_SIGS = {
    "gbpcg_last_error": (C.c_char_p, []),
    "gbpcg_version": (C.c_char_p, []),
    "gbpcg_kernel_launches": (C.c_int64, []),
    "gbpcg_device_allocations": (C.c_int64, []),
    "fem_assemble": (C.c_int, [C.POINTER(gb_fem_spec), C.POINTER(gb_allocator), _P, C.POINTER(_P)]),
    "fem_system_info": (C.c_int, [_P, C.POINTER(gb_fem_info)]),
    "fem_dof_maps": (C.c_int, [_P, _P, _P, _P, _P]),
    "fem_boundary_coords": (C.c_int, [_P, C.c_int, _P, _P]),
    "fem_dirichlet": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double), C.c_int, C.c_int, _P, _P]),
    "fem_lift_rhs": (C.c_int, [_P, _P, C.c_int, _P, _P]),
    "fem_system_destroy": (None, [_P]),
    "csr_to_sell": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(gb_allocator), _P, C.POINTER(_P)]),
    "csr_to_sell_raw": (C.c_int, [C.c_int64, _P, _P, _P, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(gb_allocator), _P, C.POINTER(_P)]),
    "sell_info": (C.c_int, [_P, C.POINTER(gb_sell_info)]),
    "sell_autotune": (C.c_int, [_P, _P, C.c_int, C.c_int, C.POINTER(gb_allocator), _P,
                                C.POINTER(SellTuneResult), C.POINTER(_P)]),
    "sell_set_variant": (C.c_int, [_P, C.c_int]),
    "sell_spmv": (C.c_int, [_P, _P, _P, _P]),
    "sell_block_jacobi": (C.c_int, [_P, C.c_int, _P]),
    "sell_block_jacobi_info": (C.c_int, [_P, C.POINTER(gb_bjacobi_info)]),
    "sell_block_jacobi_apply": (C.c_int, [_P, _P, _P, _P]),
    "sell_destroy": (None, [_P]),
    "pcg_solve": (C.c_int, [_P, _P, _P, C.POINTER(PcgOptions), _P, C.POINTER(PcgStats)]),
    "pcg_solve_noalloc": (C.c_int, [_P, _P, _P, C.POINTER(PcgOptions), _P, C.POINTER(PcgStats)]),
    "pcg_kernel_times": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, C.POINTER(C.c_double)]),
    "serve_create": (C.c_int, [C.POINTER(ServeOptions), _P, C.POINTER(_P)]),
    "serve_submit": (C.c_int, [_P, C.POINTER(ServeRequest), C.POINTER(C.c_uint64)]),
    "serve_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(ServeResult)]),
    "serve_stats": (C.c_int, [_P, C.POINTER(ServeStats)]),
    "serve_destroy": (None, [_P]),
    "pcg_solve_block": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(PcgOptions), _P, C.POINTER(PcgStats)]),
    "pcg_solve_batched": (C.c_int, [C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                    C.POINTER(C.c_int), C.POINTER(PcgOptions), _P, C.POINTER(PcgStats)]),
    "gbpcg_wait_selftest": (C.c_int, [C.c_double, _P, C.POINTER(C.c_double)]),
    "gbpcg_grid_wait_selftest": (C.c_int, [C.c_double, _P, C.POINTER(C.c_double)]),
    "pcg_batched_autotune_width": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "pcg_batched_kernel_times": (C.c_int, [C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(C.c_int), C.c_int,
                                           C.c_int, _P, C.POINTER(C.c_double)]),
}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Loads libgbpcg.so (builds it first if it is missing); raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            from . import build as _b
            _b.build()
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def lib():
    return _lib if _lib is not None else load()


def check(rc, what=""):
    if rc != GB_OK:
        msg = lib().gbpcg_last_error().decode(errors="replace")
        raise GbError(rc, f"{what}: {msg}" if what else msg)
    return rc


# --------------------------------------------------------------- memory --
_ALLOC_TYPE = gb_allocator._fields_[1][1]
_FREE_TYPE = gb_allocator._fields_[2][1]


_torch = None


def _torch_mod():
    global _torch
    if _torch is None:
        import torch
        _torch = torch
    return _torch


def _torch_alloc(ctx, nbytes, stream):
    torch = _torch_mod()
    try:
        dev = torch.cuda.current_device()
        s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream(dev)
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, s))
    except Exception:  # the library reports ENOMEM
        return None


def _torch_free(ctx, ptr, stream):
    torch = _torch
    if ptr and torch is not None:
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:  # interpreter shutdown: the process frees everything
            pass


_alloc_cb = _ALLOC_TYPE(_torch_alloc)
_free_cb = _FREE_TYPE(_torch_free)
TORCH_ALLOCATOR = gb_allocator(None, _alloc_cb, _free_cb)


def torch_allocator():
    """gb_allocator backed by PyTorch's caching allocator."""
    return C.byref(TORCH_ALLOCATOR)


def stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None
