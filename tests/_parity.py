"""Bars shared by the GPU parity tests (GPU through the C ABI against the CPU oracle).

Iteration counts.  The solve stops at the first band iteration whose recursive residual meets tol.
Once a Ritz value has converged, finite-precision Lanczos amplifies rounding differences, so that
iteration depends on how the inner products are rounded.  Two oracle builds that differ ONLY in
the accumulation type of their sums (FP64, and long double: 80-bit on x86, IEEE binary128 on Arm)
measure that spread on each case; the GPU (tree-summed inner products) must lie within +-2 of the
interval the two span.  Where the two oracles agree this is the plain +-2 bar.

Residuals.  FP64 mode returns BMINRES_OK only if the FP64 true residual of every column is <= tol,
and BMINRES_RESIDUAL_GAP if the recursive residual met tol but the true one did not; the latter is
accepted only where the oracle's own result misses tol too (a property of the method on that case,
e.g. a dropped dependent direction), with the GPU's true residual within 10 % of the oracle's.
"""
from __future__ import annotations

import numpy as np

SLACK = 2


def oracle_pair(oracle_mod, A, B, **kw):
    """The parity oracle and its extended-accumulation build on the same inputs."""
    ref = oracle_mod.bminres(A, B, **kw)
    ext = oracle_mod.bminres(A, B, variant="ext", **kw)
    return ref, ext


def iter_bracket(ref, ext, slack: int = SLACK) -> tuple[int, int]:
    return min(ref.iters, ext.iters) - slack, max(ref.iters, ext.iters) + slack


def iters_ok(gpu_iters: int, ref, ext, slack: int = SLACK) -> bool:
    lo, hi = iter_bracket(ref, ext, slack)
    return lo <= gpu_iters <= hi


def true_relres(oracle_mod, A, B, X, X0=None) -> np.ndarray:
    """||b_i - A x_i|| / ||b_i - A x0_i|| per column (0 for a zero initial residual)."""
    B = np.asarray(B).reshape(A.n, -1)
    F0 = B if X0 is None else B - oracle_mod.spmm(A, np.asarray(X0).reshape(A.n, -1))
    R = B - oracle_mod.spmm(A, np.asarray(X).reshape(A.n, -1))
    f = np.linalg.norm(F0, axis=0)
    return np.where(f > 0, np.linalg.norm(R, axis=0) / np.where(f > 0, f, 1.0), 0.0)


def check_fp64_result(info, rel, ref_rel_max: float, tol: float):
    """Status and true residual of an FP64-mode GPU solve that ended on the stopping test."""
    r = float(np.max(rel))
    if r <= tol:
        assert info["status"] == 0, (info["status_name"], r)
    else:
        assert info["status"] == 2, (info["status_name"], r)
        assert ref_rel_max > tol, ("only the GPU missed tol", r, ref_rel_max)
        assert r <= 1.1 * ref_rel_max, (r, ref_rel_max)


def rel_err(X, Xref) -> float:
    return float(np.linalg.norm(X - Xref) / np.linalg.norm(Xref))
