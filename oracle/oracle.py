"""ctypes wrapper around the plain-C FP64 block MINRES oracle (``bminres_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``.  The library's product path never imports this module.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bminres_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
# build variants of the one source: the parity oracle (plain FP64), the same arithmetic with
# inner products and matvec sums accumulated in long double (a second reference that differs only in
# summation rounding), and the all-core OpenMP build used only to time the oracle on the host
_VARIANTS = {
    "fp64": ("liboracle.so", []),
    "ext": ("liboracle_ext.so", ["-DORACLE_ACC=long double"]),
    "extfma": ("liboracle_extfma.so", ["-DORACLE_ACC=long double", "-DORACLE_FMA"]),
    "omp": ("liboracle_omp.so", ["-fopenmp", "-DORACLE_OMP"]),
}
_SO = os.path.join(_BUILD, "liboracle.so")

STATUS = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_INVALID", -3: "ERR_OOM", -4: "ERR_BREAKDOWN",
          -5: "ERR_BENCH_EXHAUSTED", -6: "ERR_NONFINITE"}


def build(force: bool = False, variant: str = "fp64") -> str:
    """Compile the oracle with plain IEEE arithmetic (no FMA contraction, no fast-math)."""
    name, extra = _VARIANTS[variant]
    so = os.path.join(_BUILD, name)
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               *extra, "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


def build_all(force: bool = False) -> None:
    for v in _VARIANTS:
        build(force, v)


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("deflations", ctypes.c_int),
                ("setup_deflations", ctypes.c_int), ("bench_used", ctypes.c_int)]


_libs = {}


def _load(variant: str = "fp64"):
    if variant not in _libs:
        lib = ctypes.CDLL(build(variant=variant))
        P = ctypes.c_void_p
        lib.oracle_bminres.restype = ctypes.c_int
        lib.oracle_bminres.argtypes = [
            ctypes.c_int64, P, P, P, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int,
            ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, P, P, P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P, P,
            ctypes.POINTER(_Info)]
        lib.oracle_bench_value.restype = ctypes.c_double
        lib.oracle_bench_value.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_csr_spmm.restype = None
        lib.oracle_csr_spmm.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int, P, P]
        _libs[variant] = lib
    return _libs[variant]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass
class Result:
    X: np.ndarray
    status: int
    iters: int
    deflations: int
    setup_deflations: int
    bench_used: int
    f0norm: np.ndarray
    rho: np.ndarray | None = None  # (iters, p) recursive residual norms
    H: np.ndarray | None = None  # (iters, 2p+1) column j of H, rows j-p..j+p
    R: np.ndarray | None = None  # (iters, 2p+1) column j of R, rows j-2p..j
    Xhist: np.ndarray | None = None  # (k, n, p) iterates X_1..X_k
    U: np.ndarray | None = None  # (m, n) Lanczos vectors u_1..u_m in creation order
    defl_iters: list | None = None

    @property
    def status_name(self) -> str:
        return STATUS.get(self.status, str(self.status))


def bminres(A, B, X0=None, tol=1e-10, maxit=1000, gamma=1e-8, bench=4, seed=0, ghost=False,
            qr="householder", hist=0, xhist=0, uhist=0, variant="fp64") -> Result:
    """Run the oracle on CSR ``A`` (a ``workloads.CSR``) and row-major ``B`` (n, p).

    ``variant``: "fp64" (the parity oracle), "ext" (long-double accumulation of the sums) or
    "omp" (all host cores; for timing)."""
    lib = _load(variant)
    n = A.n
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    p = B.shape[1]
    X = np.zeros((n, p)) if X0 is None else np.array(X0, dtype=np.float64, order="C", copy=True)
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
    vals = np.ascontiguousarray(A.vals, dtype=np.float64)
    hist = int(min(hist, maxit))
    xhist = int(min(xhist, maxit))
    rho = np.zeros((hist, p)) if hist else None
    H = np.zeros((hist, 2 * p + 1)) if hist else None
    R = np.zeros((hist, 2 * p + 1)) if hist else None
    Xh = np.zeros((xhist, n, p)) if xhist else None
    U = np.zeros((uhist, n)) if uhist else None
    dcap = bench + p + 8
    defl = np.zeros(dcap, dtype=np.int32)
    f0 = np.zeros(p)
    info = _Info()
    lib.oracle_bminres(n, _ptr(rowptr), _ptr(colidx), _ptr(vals), p, _ptr(B), _ptr(X), float(tol),
                       int(maxit), float(gamma), int(bench), int(seed) & ((1 << 64) - 1),
                       int(bool(ghost)), 0 if qr == "householder" else 1, hist, _ptr(rho), _ptr(H),
                       _ptr(R), xhist, _ptr(Xh), int(uhist), _ptr(U), dcap, _ptr(defl), _ptr(f0),
                       ctypes.byref(info))
    k = info.iters
    return Result(X=X, status=info.status, iters=k, deflations=info.deflations,
                  setup_deflations=info.setup_deflations, bench_used=info.bench_used, f0norm=f0,
                  rho=None if rho is None else rho[: min(k, hist)],
                  H=None if H is None else H[: min(k, hist)],
                  R=None if R is None else R[: min(k, hist)],
                  Xhist=None if Xh is None else Xh[: min(k, xhist)],
                  U=None if U is None else U[: min(uhist, p + k)],
                  defl_iters=[int(v) for v in defl[: min(info.deflations, dcap)]])


def bench_values(seed: int, k: int, n: int, rows) -> np.ndarray:
    lib = _load()
    return np.array([lib.oracle_bench_value(seed & ((1 << 64) - 1), k, n, int(r)) for r in rows])


def spmm(A, X: np.ndarray) -> np.ndarray:
    """``A @ X`` for row-major ``X`` (n, p), summed in CSR order."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    Y = np.empty_like(X)
    lib.oracle_csr_spmm(A.n, _ptr(np.ascontiguousarray(A.rowptr, dtype=np.int32)),
                        _ptr(np.ascontiguousarray(A.colidx, dtype=np.int32)),
                        _ptr(np.ascontiguousarray(A.vals, dtype=np.float64)), X.shape[1], _ptr(X), _ptr(Y))
    return Y


def relres(A, B, X) -> np.ndarray:
    """Per-column true relative residual ``||b_i - A x_i|| / ||b_i||`` (0 where b_i = 0)."""
    R = np.asarray(B).reshape(A.n, -1) - spmm(A, X)
    nb = np.linalg.norm(np.asarray(B).reshape(A.n, -1), axis=0)
    return np.where(nb > 0, np.linalg.norm(R, axis=0) / np.where(nb > 0, nb, 1.0), 0.0)
