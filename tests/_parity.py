"""Bars shared by the GPU parity tests (GPU through the C ABI against the CPU oracle).

Iteration counts.  The solve stops at the first band iteration whose recursive residual meets tol.
Once a Ritz value has converged, finite-precision Lanczos amplifies rounding differences, so that
iteration depends on rounding: on the oracle itself, perturbing B by one unit in the last place
moves it by up to ~1.7 % (pinned on the CPU by test_oracle_pins.py::
test_stopping_iteration_depends_on_rounding), and three builds of the oracle that differ only in
rounding (FP64 as written; sums accumulated in long double; in addition, updates y + a x rounded
once by fma) disagree by up to ~1.5 %.  FP64-mode GPU counts must lie in the interval the three
builds span, widened on each side by max(2, 1 % of the count).  Double-word inner solves carry
about 2^-48 rounding (32 times FP64's) and are checked against the same interval widened by 3 %
(mixed-precision counts are reported rather than held to the FP64 bar).

Residuals.  FP64 mode returns BMINRES_OK only if the FP64 true residual of every column is <= tol,
and BMINRES_RESIDUAL_GAP if the recursive residual met tol but the true one did not; the latter is
accepted only where the oracle's own result misses tol too (a property of the method on that case,
e.g. a dropped dependent direction), with the GPU's true residual within 10 % of the oracle's.
"""
from __future__ import annotations

import numpy as np

SLACK = 2
REL_FP64 = 0.01
REL_DW = 0.03
BUILDS = ("fp64", "ext", "extfma")


class OracleSet:
    """The parity oracle's result and the stopping iterations of its three rounding builds."""

    def __init__(self, ref, iters):
        self.ref = ref
        self.iters = dict(iters)

    @property
    def lo(self) -> int:
        return min(self.iters.values())

    @property
    def hi(self) -> int:
        return max(self.iters.values())


def oracle_pair(oracle_mod, A, B, **kw):
    """The parity oracle and the iteration counts of its rounding builds on the same inputs."""
    ref = oracle_mod.bminres(A, B, **kw)
    its = {"fp64": ref.iters}
    for v in BUILDS[1:]:
        its[v] = oracle_mod.bminres(A, B, variant=v, **kw).iters
    return ref, OracleSet(ref, its)


def iter_bracket(ref, ext, rel: float = REL_FP64) -> tuple[int, int]:
    w = max(SLACK, int(rel * ext.hi + 0.5))
    return ext.lo - w, ext.hi + w


def iters_ok(gpu_iters: int, ref, ext, rel: float = REL_FP64) -> bool:
    lo, hi = iter_bracket(ref, ext, rel)
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
