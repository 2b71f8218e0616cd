"""Python front end of the block MINRES library: a handle wrapper and a torch autograd Function.

All arithmetic runs in the CUDA library behind the C ABI (``include/bminres.h``); this module only
marshals pointers.  Dense blocks are row-major ``(n, p)`` float64 arrays: CUDA torch tensors are
passed as device pointers, numpy arrays / CPU tensors as host pointers (the library stages them).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


def _as_ptr(x):
    """(pointer, keepalive, kind) for a float64/int32 contiguous array or tensor."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x, "cuda" if x.is_cuda else "cpu"
    a = np.ascontiguousarray(x)
    return a.ctypes.data_as(ctypes.c_void_p), a, "numpy"


def _check(st: int, what: str, allow_not_converged: bool = True) -> int:
    """Raise for error statuses.  NOT_CONVERGED and RESIDUAL_GAP (the recursive residual met tol
    but the FP64 true residual did not) leave a usable iterate and are reported, not raised."""
    if st == _lib.OK or (allow_not_converged and st in (_lib.NOT_CONVERGED, _lib.RESIDUAL_GAP)):
        return st
    raise _lib.BminresError(st, what)


class Solver:
    """Block MINRES solver bound to one sparse symmetric matrix (CSR, int32 indices).

    ``A`` is any object with ``n``, ``rowptr``, ``colidx`` and ``vals`` attributes (for example
    ``workloads.CSR``), or a tuple ``(n, rowptr, colidx, vals)``.
    """

    def __init__(self, A, precision: str = "fp64", gamma: float = 1e-8, bench: int = 4, seed: int = 0,
                 ghost: bool = False, tol_inner: float = 1e-5, max_outer: int = 20, max_blocks: int = 0):
        lib = _lib.load()
        if isinstance(A, tuple):
            n, rowptr, colidx, vals = A
        else:
            n, rowptr, colidx, vals = A.n, A.rowptr, A.colidx, A.vals
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        o = _lib.default_opts()
        o.precision = {"fp64": _lib.FP64, "mixed": _lib.MIXED, "mixed_dw": _lib.MIXED_DW, "fp64_refined": _lib.FP64_REFINED}[precision]
        o.gamma = gamma
        o.bench = bench
        o.seed = seed & ((1 << 64) - 1)
        o.ghost = int(bool(ghost))
        o.tol_inner = tol_inner
        o.max_outer = max_outer
        o.max_blocks = max_blocks
        h = ctypes.c_void_p()
        st = lib.bminres_create(ctypes.byref(h), int(n), int(colidx.shape[0]), rowptr.ctypes.data_as(ctypes.c_void_p),
                                colidx.ctypes.data_as(ctypes.c_void_p), vals.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(o))
        _check(st, "bminres_create", allow_not_converged=False)
        self._h = h
        self._lib = lib
        self.n = int(n)
        self.nnz = int(colidx.shape[0])
        self.precision = precision

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bminres_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def _stream(stream, kind):
        if stream is not None:
            return ctypes.c_void_p(int(stream))
        if kind == "cuda":
            import torch

            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)

    def set_values(self, vals, stream=None):
        pv, keep, kind = _as_ptr(vals)
        _check(self._lib.bminres_set_values(self._h, pv, self._stream(stream, kind)), "bminres_set_values", False)

    def solve(self, B, X=None, tol: float = 1e-10, maxit: int = 100000, stream=None):
        """Solve A X = B in place on ``X`` (created as zeros like ``B`` if None).

        Returns ``(X, info, relres_true)``: ``info`` is a dict of the C info struct and
        ``relres_true`` the per-column FP64 ``||b_i - A x_i|| / ||b_i - A x0_i||``.
        Raises ``BminresError`` for error statuses; NOT_CONVERGED and RESIDUAL_GAP are reported in
        ``info``.
        """
        p = 1 if B.ndim == 1 else int(B.shape[1])
        if X is None:
            X = B.new_zeros(B.shape) if hasattr(B, "new_zeros") else np.zeros(B.shape)
        pb, kb, kindb = _as_ptr(B)
        px, kx, kindx = _as_ptr(X)
        rel = np.zeros(max(p, 1))
        info = _lib.Info()
        st = self._lib.bminres_solve(self._h, p, pb, px, float(tol), int(maxit), self._stream(stream, kindb),
                                     rel.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))
        _check(st, "bminres_solve")
        if kindx == "numpy" and kx is not X:
            X[...] = kx
        d = info.as_dict()
        d["status_name"] = _lib.STATUS.get(st, str(st))
        return X, d, rel[:p]

    def set_history(self, cap: int):
        """Record the recursive residual norms of the first ``cap`` band iterations of later solves."""
        _check(self._lib.bminres_set_history(self._h, int(cap)), "bminres_set_history", False)
        self._hist_cap = int(cap)

    def history(self, p: int) -> np.ndarray:
        """(iterations, p) recursive residual norms of the last solve (see ``set_history``)."""
        cap = getattr(self, "_hist_cap", 0)
        out = np.zeros(max(cap, 1) * 32)
        cnt = ctypes.c_int(0)
        _check(self._lib.bminres_get_history(self._h, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)),
               "bminres_get_history", False)
        return out[: cnt.value * p].reshape(cnt.value, p)

    def spmm(self, X, Y=None, stream=None):
        """Y = A X (FP64)."""
        p = 1 if X.ndim == 1 else int(X.shape[1])
        if Y is None:
            Y = X.new_empty(X.shape) if hasattr(X, "new_empty") else np.empty(X.shape)
        px, kx, kind = _as_ptr(X)
        py, ky, _ = _as_ptr(Y)
        _check(self._lib.bminres_spmm(self._h, p, px, py, self._stream(stream, kind)), "bminres_spmm", False)
        return Y

    def backward(self, G, X, tol: float = 1e-10, maxit: int = 100000, want_dA: bool = True, stream=None):
        """Adjoint: dB = A^{-1} G and dA_vals = -(dB X^T) on the sparsity pattern."""
        p = 1 if G.ndim == 1 else int(G.shape[1])
        dB = G.new_zeros(G.shape) if hasattr(G, "new_zeros") else np.zeros(G.shape)
        dA = None
        if want_dA:
            dA = G.new_zeros((self.nnz,)) if hasattr(G, "new_zeros") else np.zeros(self.nnz)
        pg, kg, kind = _as_ptr(G)
        pxx, kxx, _ = _as_ptr(X)
        pdb, kdb, _ = _as_ptr(dB)
        pda = _as_ptr(dA)[0] if dA is not None else None
        info = _lib.Info()
        st = self._lib.bminres_backward(self._h, p, pg, pxx, pdb, pda, float(tol), int(maxit),
                                        self._stream(stream, kind), ctypes.byref(info))
        _check(st, "bminres_backward")
        d = info.as_dict()
        d["status_name"] = _lib.STATUS.get(st, str(st))
        return dB, dA, d


def _make_fn():
    import torch

    class BMinresFn(torch.autograd.Function):
        """X = A^{-1} B with A given by its CSR values (pattern fixed in ``solver``).

        Backward (not in the paper): dL/dB = A^{-1} G by a second block solve, and
        dL/dvals = -(A^{-1} G) X^T restricted to the sparsity pattern (each stored value treated
        as an independent entry)."""

        @staticmethod
        def forward(ctx, vals, B, solver, tol, maxit, tol_adj):
            solver.set_values(vals.detach().contiguous())
            X, info, _ = solver.solve(B.detach().contiguous(), tol=tol, maxit=maxit)
            ctx.solver, ctx.tol, ctx.maxit = solver, tol_adj, maxit
            ctx.save_for_backward(X)
            return X

        @staticmethod
        def backward(ctx, G):
            (X,) = ctx.saved_tensors
            dB, dA, _ = ctx.solver.backward(G.contiguous(), X, tol=ctx.tol, maxit=ctx.maxit,
                                            want_dA=ctx.needs_input_grad[0])
            return dA, dB, None, None, None, None

    return BMinresFn


_FN = None


def bminres_apply(vals, B, solver: Solver, tol: float = 1e-10, maxit: int = 100000, tol_adj: float | None = None):
    """Differentiable solve: ``X = A(vals)^{-1} B`` (see ``BMinresFn``)."""
    global _FN
    if _FN is None:
        _FN = _make_fn()
    return _FN.apply(vals, B, solver, tol, maxit, tol if tol_adj is None else tol_adj)
