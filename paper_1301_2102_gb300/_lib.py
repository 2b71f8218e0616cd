"""ctypes binding to the C ABI in ``include/bminres.h`` (argument marshalling only).

Every numerical step runs in the CUDA library; if the library is missing this module raises
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbminres.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bminres.h")

STATUS = {0: "BMINRES_OK", 1: "BMINRES_NOT_CONVERGED", 2: "BMINRES_RESIDUAL_GAP", -1: "BMINRES_ERR_INVALID",
          -2: "BMINRES_ERR_CUDA",
          -3: "BMINRES_ERR_OOM", -4: "BMINRES_ERR_BREAKDOWN", -5: "BMINRES_ERR_BENCH_EXHAUSTED",
          -6: "BMINRES_ERR_NONFINITE", -7: "BMINRES_ERR_TIMEOUT"}
OK, NOT_CONVERGED, RESIDUAL_GAP = 0, 1, 2
FP64, MIXED, MIXED_DW, FP64_REFINED = 0, 1, 2, 3


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("gamma", ctypes.c_double), ("bench", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("ghost", ctypes.c_int), ("tol_inner", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("max_blocks", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("cycles", ctypes.c_int),
                ("outer", ctypes.c_int), ("deflations", ctypes.c_int), ("setup_deflations", ctypes.c_int),
                ("bench_used", ctypes.c_int), ("grid_blocks", ctypes.c_int), ("relres_est_max", ctypes.c_double),
                ("relres_true_max", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("stream_ms", ctypes.c_double), ("reduce_ms", ctypes.c_double),
                ("scalar_ms", ctypes.c_double), ("timeline_ms", ctypes.c_double), ("qr_ms", ctypes.c_double),
                ("launches", ctypes.c_int), ("spmm_ms", ctypes.c_double), ("dir_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BminresError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


_lib = None


def exported_symbols() -> list[str]:
    """Function names declared in include/bminres.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(bminres_[a-z_]+)\s*\(", txt)))


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.bminres_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.bminres_default_opts.restype = None
    lib.bminres_create.argtypes = [ctypes.POINTER(P), I64, I64, P, P, P, ctypes.POINTER(Opts)]
    lib.bminres_create.restype = I
    lib.bminres_set_values.argtypes = [P, P, P]
    lib.bminres_set_values.restype = I
    lib.bminres_solve.argtypes = [P, I, P, P, D, I, P, P, ctypes.POINTER(Info)]
    lib.bminres_solve.restype = I
    lib.bminres_backward.argtypes = [P, I, P, P, P, P, D, I, P, ctypes.POINTER(Info)]
    lib.bminres_backward.restype = I
    lib.bminres_spmm.argtypes = [P, I, P, P, P]
    lib.bminres_spmm.restype = I
    lib.bminres_set_history.argtypes = [P, I]
    lib.bminres_set_history.restype = I
    lib.bminres_get_history.argtypes = [P, P, ctypes.POINTER(I)]
    lib.bminres_get_history.restype = I
    lib.bminres_destroy.argtypes = [P]
    lib.bminres_destroy.restype = None
    lib.bminres_fp64_peak.argtypes = [I, P, ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.bminres_fp64_peak.restype = I
    lib.bminres_status_string.argtypes = [I]
    lib.bminres_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def default_opts() -> Opts:
    o = Opts()
    load().bminres_default_opts(ctypes.byref(o))
    return o


def fp64_peak_gflops(iters: int = 200000, stream=None) -> tuple[float, float]:
    """Measured FP64 FMA throughput of the current GPU (GFLOP/s) and the timed launch's ms."""
    g, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().bminres_fp64_peak(int(iters), ctypes.c_void_p(stream or 0), ctypes.byref(g), ctypes.byref(ms))
    if st != OK:
        raise BminresError(st, "bminres_fp64_peak")
    return g.value, ms.value
