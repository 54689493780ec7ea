"""ctypes binding of libdichotomy.so: one Python function per C entry point, same names.

Argument marshalling only -- every step of the solve runs in the library's CUDA kernels.
Device buffers are torch CUDA tensors (float64, contiguous); streams default to torch's
current stream.  There is no CPU fallback: without the built library or a CUDA device
these functions raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int32, c_int64, c_double, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                  ctypes.c_void_p, ctypes.c_size_t)

DICH_OK = 0
STATUS_NAMES = {
    0: "DICH_OK", 1: "DICH_ERR_ARG", 2: "DICH_ERR_NOT_DOMINANT", 3: "DICH_ERR_SINGULAR", 4: "DICH_ERR_TIMEOUT",
    5: "DICH_ERR_NONFINITE", 6: "DICH_ERR_CUDA", 7: "DICH_ERR_ALIAS", 8: "DICH_ERR_UNBOUND",
    9: "DICH_ERR_WORKSPACE", 10: "DICH_ERR_SCHEDULE", 11: "DICH_ERR_UNSUPPORTED",
}
PREC_F64, PREC_MIXED, PREC_AUTO = 0, 1, 2
FLAG_FORCE_GENERAL, FLAG_CHECK_FINITE, FLAG_HOST_PRELIM, FLAG_DEVICE_PRELIM, FLAG_ALLOW_NOT_DOMINANT = 1, 2, 4, 8, 16
FLAG_REG_PATH, FLAG_SMEM_PATH = 32, 64

EXPORTS = [
    "dichotomy_plan", "dichotomy_plan_ex", "dichotomy_plan_quasi", "dichotomy_plan_info", "dichotomy_plan_workspace_bytes",
    "dichotomy_plan_bind", "dichotomy_solve", "dichotomy_solve_series", "dichotomy_solve_host", "dichotomy_adjoint", "dichotomy_residual", "dichotomy_status", "dichotomy_destroy",
    "dichotomy_solve_noalloc",
    "dichotomy_batch_prepare", "dichotomy_batch_prepare_quasi", "dichotomy_batch_workspace_bytes", "dichotomy_batch_bind",
    "dichotomy_solve_batched", "dichotomy_adjoint_batched", "dichotomy_batch_status", "dichotomy_batch_info",
    "dichotomy_batch_destroy", "dichotomy_strerror", "dichotomy_last_cuda_error", "dichotomy_version",
    "dichotomy_gen_plan", "dichotomy_gen_info", "dichotomy_gen_workspace_bytes", "dichotomy_gen_bind",
    "dichotomy_gen_solve", "dichotomy_gen_solve_series", "dichotomy_gen_residual", "dichotomy_gen_status", "dichotomy_gen_destroy",
    "dichotomy_shard_info", "dichotomy_shard_reduce", "dichotomy_shard_bounds", "dichotomy_shard_finish",
]


class DichotomyError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        name = STATUS_NAMES.get(code, str(code))
        msg = f"{where}: {name}"
        if _lib_obj is not None:
            msg += " (" + _lib_obj.dichotomy_strerror(code).decode() + ")"
            if code == 6:
                msg += ": " + _lib_obj.dichotomy_last_cuda_error().decode()
        super().__init__(msg)


class dich_opts(ctypes.Structure):
    _fields_ = [("block_size", c_int32), ("precision", c_int32), ("threads", c_int32), ("flags", c_int32),
                ("trunc_eps", c_double)]


class dich_plan_info(ctypes.Structure):
    _fields_ = [("N", c_int64), ("P", c_int64), ("n", c_int32), ("n_last", c_int32), ("threads", c_int32),
                ("halo_l", c_int32), ("halo_r", c_int32), ("path", c_int32), ("precision", c_int32),
                ("tiles", c_int64), ("Lv", c_int32), ("Lw", c_int32), ("kl", c_int32), ("kr", c_int32),
                ("rs", c_double), ("ib", c_double), ("z", c_double), ("workspace_bytes", c_size_t),
                ("beta_offset", c_size_t), ("iface_offset", c_size_t), ("growth", c_double)]


class dich_shard_info(ctypes.Structure):
    _fields_ = [("row_lo", c_int64), ("row_hi", c_int64), ("block_lo", c_int64), ("block_hi", c_int64),
                ("workspace_bytes", c_size_t)]


_lib_obj = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdichotomy.so (building it with nvcc if it is missing or stale)."""
    global _lib_obj
    with _lock:
        if _lib_obj is not None:
            return _lib_obj
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError("libdichotomy.so is not built; run paper_1002_2469_gb300/build.py")
        L = ctypes.CDLL(_build.LIB)
        P = c_void_p
        I = ctypes.c_int
        sig = {
            "dichotomy_plan": ([c_double, c_double, c_double, c_int64, ctypes.POINTER(P)], I),
            "dichotomy_plan_ex": ([c_double, c_double, c_double, c_int64, ctypes.POINTER(dich_opts),
                                   ctypes.POINTER(P)], I),
            "dichotomy_plan_quasi": ([c_double, c_double, c_double, c_double, c_double, c_int64,
                                      ctypes.POINTER(dich_opts), ctypes.POINTER(P)], I),
            "dichotomy_plan_info": ([P, ctypes.POINTER(dich_plan_info)], I),
            "dichotomy_plan_workspace_bytes": ([P, ctypes.POINTER(c_size_t)], I),
            "dichotomy_plan_bind": ([P, P, c_size_t, P], I),
            "dichotomy_solve": ([P, P, P, P], I),
            "dichotomy_solve_series": ([P, c_int64, P, c_int64, P, c_int64, P], I),
            "dichotomy_solve_host": ([P, P, P, P, P, c_int32, P], I),
            "dichotomy_adjoint": ([P, P, P, P, P, P], I),
            "dichotomy_residual": ([P, P, P, ctypes.POINTER(c_double), P], I),
            "dichotomy_status": ([P, P, ctypes.POINTER(I)], I),
            "dichotomy_destroy": ([P], None),
            "dichotomy_solve_noalloc": ([c_double, c_double, c_double, c_int64, P, P, P], I),
            "dichotomy_batch_prepare": ([c_int64, P, P, P, P, P, ctypes.POINTER(dich_opts), ctypes.POINTER(P)], I),
            "dichotomy_batch_prepare_quasi": ([c_int64, P, P, P, P, P, P, P, ctypes.POINTER(dich_opts),
                                               ctypes.POINTER(P)], I),
            "dichotomy_batch_workspace_bytes": ([P, ctypes.POINTER(c_size_t)], I),
            "dichotomy_batch_bind": ([P, P, c_size_t, P], I),
            "dichotomy_solve_batched": ([P, P, P, P], I),
            "dichotomy_adjoint_batched": ([P, P, P, P, P, P], I),
            "dichotomy_batch_status": ([P, P, ctypes.POINTER(I)], I),
            "dichotomy_batch_info": ([P, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64), P], I),
            "dichotomy_batch_destroy": ([P], None),
            "dichotomy_strerror": ([I], ctypes.c_char_p),
            "dichotomy_last_cuda_error": ([], ctypes.c_char_p),
            "dichotomy_version": ([], ctypes.c_char_p),
            "dichotomy_gen_plan": ([c_int64, P, P, P, ctypes.POINTER(dich_opts), ctypes.POINTER(P)], I),
            "dichotomy_gen_info": ([P, ctypes.POINTER(dich_plan_info)], I),
            "dichotomy_gen_workspace_bytes": ([P, ctypes.POINTER(c_size_t)], I),
            "dichotomy_gen_bind": ([P, P, c_size_t, P], I),
            "dichotomy_gen_solve": ([P, P, P, P], I),
            "dichotomy_gen_solve_series": ([P, c_int64, P, c_int64, P, c_int64, P], I),
            "dichotomy_gen_residual": ([P, P, P, ctypes.POINTER(c_double), P], I),
            "dichotomy_gen_status": ([P, P, ctypes.POINTER(I)], I),
            "dichotomy_gen_destroy": ([P], None),
            "dichotomy_shard_info": ([P, c_int32, c_int32, ctypes.POINTER(dich_shard_info)], I),
            "dichotomy_shard_reduce": ([P, c_int32, c_int32, P, P, P, c_size_t, ctypes.POINTER(c_double), P], I),
            "dichotomy_shard_bounds": ([P, c_int32, c_int32, ctypes.POINTER(c_double), P, c_size_t,
                                        ctypes.POINTER(c_double), P], I),
            "dichotomy_shard_finish": ([P, c_int32, c_int32, P, P, ctypes.POINTER(c_double), P, c_size_t, P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib_obj = L
        return L


def check(rc: int, where: str) -> None:
    if rc != DICH_OK:
        raise DichotomyError(rc, where)


def make_opts(block_size=0, precision=PREC_F64, threads=0, flags=0, trunc_eps=0.0) -> dich_opts:
    return dich_opts(int(block_size), int(precision), int(threads), int(flags), float(trunc_eps))
