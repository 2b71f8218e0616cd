"""Seeded synthetic inputs for block MINRES: sparse symmetric operators and right-hand sides.

This module only *constructs problems*; it holds none of the solver's arithmetic, so both the
CPU oracle (``oracle/``) and the CUDA path consume exactly the same arrays.

Operators follow the model problems of the paper's numerical section (Sec. 8): shifted
finite-difference Laplacians ``A = L - sigma I``, which are symmetric and indefinite once the
shift lies inside the spectrum, plus a saddle-point system ``[[K, C^T], [C, 0]]``.

Conventions
-----------
* Stencils are unscaled integers (2D: diagonal 4, neighbours -1; 3D: 6 / -1) so that the
  stored values are exact.  Scaling by h^-2 as in Sec. 8 only rescales the spectrum.
* The unshifted spectrum is known in closed form:
  ``lambda(k) = sum_d (2 - 2 cos(k_d pi / (N + 1)))``, ``k_d = 1..N``.
* CSR arrays: ``rowptr`` int32 (n+1), ``colidx`` int32 (nnz, ascending within each row),
  ``vals`` float64 (nnz).  Right-hand sides are float64, row-major ``(n, p)``.
* Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int32 (n+1,)
    colidx: np.ndarray  # int32 (nnz,)
    vals: np.ndarray  # float64 (nnz,)

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.vals, self.colidx, self.rowptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


def laplacian_eig_extremes(N: int, dim: int) -> tuple[float, float]:
    """Smallest and largest eigenvalue of the unshifted ``dim``-D stencil on an N^dim grid."""
    lo = dim * (2.0 - 2.0 * math.cos(math.pi / (N + 1)))
    hi = dim * (2.0 - 2.0 * math.cos(N * math.pi / (N + 1)))
    return lo, hi


def shift_at_fraction(N: int, dim: int, frac: float) -> float:
    """Shift ``sigma = lambda_min + frac * (lambda_max - lambda_min)`` of the unshifted operator."""
    lo, hi = laplacian_eig_extremes(N, dim)
    return lo + frac * (hi - lo)


def laplacian(N: int, dim: int, sigma: float = 0.0) -> CSR:
    """``dim``-D 5/7-point Laplacian on an N^dim grid (lexicographic order, x fastest), minus sigma*I."""
    if dim not in (1, 2, 3):
        raise ValueError("dim must be 1, 2 or 3")
    n = N**dim
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for _ in range(dim):
        coords.append(rem % N)
        rem //= N
    # offsets in ascending column order: -N^(d-1), ..., -1, 0, +1, ..., +N^(d-1)
    offs = []
    for d in reversed(range(dim)):
        offs.append((d, -1))
    offs.append((None, 0))
    for d in range(dim):
        offs.append((d, +1))
    cols = np.empty((n, len(offs)), dtype=np.int32)
    vals = np.empty((n, len(offs)), dtype=np.float64)
    valid = np.empty((n, len(offs)), dtype=bool)
    for t, (d, s) in enumerate(offs):
        if d is None:
            cols[:, t] = idx
            vals[:, t] = 2.0 * dim - sigma
            valid[:, t] = True
        else:
            stride = N**d
            c = coords[d] + s
            ok = (c >= 0) & (c < N)
            valid[:, t] = ok
            cols[:, t] = np.where(ok, idx + s * stride, 0)
            vals[:, t] = -1.0
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = cols[valid]
    v = vals[valid]
    return CSR(n, rowptr.astype(np.int32), colidx.astype(np.int32), v.astype(np.float64))


def laplacian_null_modes_2d(N: int, sigma: float) -> np.ndarray:
    """Orthonormal eigenvectors of the 2D operator ``L - sigma I`` with eigenvalue exactly 0.

    Eigenvectors of the 5-point stencil are ``q_ij(x, y) = sin(i x pi/(N+1)) sin(j y pi/(N+1))``
    with eigenvalue ``4 - 2cos(i pi/(N+1)) - 2cos(j pi/(N+1))``.  For ``sigma = 4`` the null space
    is spanned by the modes with ``i + j = N + 1``.  Returns an ``(n, m)`` matrix.
    """
    th = math.pi / (N + 1)
    x = np.arange(1, N + 1)
    modes = []
    for i in range(1, N + 1):
        for j in range(1, N + 1):
            lam = 4.0 - 2.0 * math.cos(i * th) - 2.0 * math.cos(j * th) - sigma
            if abs(lam) < 1e-12:
                sx = np.sin(i * x * th)
                sy = np.sin(j * x * th)
                q = np.outer(sy, sx).reshape(-1)  # row index y, column x -> lexicographic x fastest
                modes.append(q / np.linalg.norm(q))
    if not modes:
        return np.zeros((N * N, 0))
    return np.stack(modes, axis=1)


def paper_e1_operator(N: int = 200) -> CSR:
    """The operator of the paper's first experiment (Sec. 8): A = -L - 200 I with L the 2D 5-point
    Laplacian on an N x N grid, h = 1/(N - 1), here scaled by h^2 (the unscaled stencil minus
    200 h^2 I), which changes no relative residual."""
    h = 1.0 / (N - 1)
    return laplacian(N, 2, 200.0 * h * h)


def ones_identity_rhs(n: int, p: int) -> np.ndarray:
    """The right-hand sides of the paper's second experiment (Sec. 8): the vector of all ones, then
    the first p - 1 columns of the identity."""
    B = np.zeros((n, p))
    B[:, 0] = 1.0
    for k in range(1, p):
        B[k - 1, k] = 1.0
    return np.ascontiguousarray(B)


def randn_rhs(n: int, p: int, seed: int = 0) -> np.ndarray:
    """``(n, p)`` row-major float64 matrix of i.i.d. N(0,1) entries."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, p)))


def dependent_rhs(n: int, p: int, seed: int = 0) -> np.ndarray:
    """``p >= 6`` columns: 0..p-3 N(0,1); column p-2 = 0.5 c0 - 1.2 c3 + 1e-12 N(0,1); column p-1 =
    c1 + c2 exactly (the benchmark's dependence structure, widened to p columns)."""
    if p < 6:
        raise ValueError("p must be at least 6")
    rng = np.random.default_rng(seed)
    B = np.empty((n, p))
    B[:, : p - 2] = rng.standard_normal((n, p - 2))
    noise = rng.standard_normal(n)
    B[:, p - 2] = 0.5 * B[:, 0] - 1.2 * B[:, 3] + 1e-12 * noise
    B[:, p - 1] = B[:, 1] + B[:, 2]
    return np.ascontiguousarray(B)


def dependent_rhs_p8(n: int, seed: int = 0) -> np.ndarray:
    """Eight columns: 0-5 N(0,1); col6 = 0.5 c0 - 1.2 c3 + 1e-12 N(0,1); col7 = c1 + c2 exactly."""
    return dependent_rhs(n, 8, seed)


def near_dependent_dense(n: int, p: int, seed: int = 11) -> tuple[CSR, np.ndarray]:
    """Dense symmetric indefinite operator (eigenvalues +-[0.6, 4], every third one negative) and p
    right-hand sides whose first column lies within 1e-14 of a 3-dimensional invariant subspace: the
    block Krylov sequence started from it becomes dependent after a few iterations (Sec. 5)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(0.6, 4.0, n) * np.where(np.arange(n) % 3 == 0, -1.0, 1.0)
    D = (Q * lam) @ Q.T
    A = dense_to_csr(0.5 * (D + D.T))
    f1 = Q[:, :3] @ np.array([1.0, -0.7, 0.4]) + 1e-14 * rng.standard_normal(n)
    B = np.concatenate([f1[:, None], rng.standard_normal((n, p - 1))], axis=1)
    return A, np.ascontiguousarray(B)


def laplacian_mode_3d(N: int, k: tuple[int, int, int]) -> np.ndarray:
    """Normalised eigenvector ``sin(k_x x pi/(N+1)) sin(k_y y pi/(N+1)) sin(k_z z pi/(N+1))`` of the
    3D stencil (lexicographic order, x fastest)."""
    th = math.pi / (N + 1)
    t = np.arange(1, N + 1)
    sx, sy, sz = (np.sin(kk * t * th) for kk in k)
    q = (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]).reshape(-1)
    return q / np.linalg.norm(q)


def near_dependent_laplacian(N: int, p: int, seed: int = 11, frac: float = 0.10) -> tuple[CSR, np.ndarray]:
    """3D shifted Laplacian and p right-hand sides whose first column lies within 1e-14 of the span of
    three closed-form eigenvectors: the band Krylov sequence it starts is near-dependent after a few
    cycles (Sec. 5); the other columns are N(0,1)."""
    A = laplacian(N, 3, shift_at_fraction(N, 3, frac))
    rng = np.random.default_rng(seed)
    f1 = (laplacian_mode_3d(N, (1, 2, 1)) - 0.7 * laplacian_mode_3d(N, (3, 1, 2))
          + 0.4 * laplacian_mode_3d(N, (2, 2, 5)))
    f1 = f1 + 1e-14 * rng.standard_normal(A.n)
    B = np.concatenate([f1[:, None], rng.standard_normal((A.n, p - 1))], axis=1)
    return A, np.ascontiguousarray(B)


def saddle_point(NK: int = 512, m: int = 65536, nnz_per_row: int = 4, seed: int = 1) -> CSR:
    """``[[K, C^T], [C, 0]]``: K the 2D 5-point Laplacian on NK x NK, C an m x NK^2 matrix with
    ``nnz_per_row`` distinct uniformly random columns per row and N(0,1) values."""
    import scipy.sparse as sp

    K = laplacian(NK, 2).to_scipy()
    nk = NK * NK
    rng = np.random.default_rng(seed)
    cols = rng.integers(0, nk, size=(m, nnz_per_row))
    # resample rows that drew a repeated column until all columns in each row are distinct
    while True:
        s = np.sort(cols, axis=1)
        dup = np.any(s[:, 1:] == s[:, :-1], axis=1)
        if not dup.any():
            break
        cols[dup] = rng.integers(0, nk, size=(int(dup.sum()), nnz_per_row))
    vals = rng.standard_normal((m, nnz_per_row))
    rows = np.repeat(np.arange(m), nnz_per_row)
    C = sp.csr_matrix((vals.reshape(-1), (rows, cols.reshape(-1))), shape=(m, nk))
    A = sp.bmat([[K, C.T], [C, None]], format="csr")
    A.sort_indices()
    return CSR(A.shape[0], A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))


def random_symmetric_indefinite(n: int, seed: int, lo: float = 0.5, hi: float = 5.0) -> CSR:
    """Dense random symmetric matrix with eigenvalues of both signs, ``|lambda|`` in ``[lo, hi]``,
    stored as a (full) CSR pattern.  Small sizes only (tests)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(lo, hi, size=n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    return dense_to_csr(M)


def dense_to_csr(M: np.ndarray) -> CSR:
    import scipy.sparse as sp

    S = sp.csr_matrix(M)
    S.sort_indices()
    return CSR(M.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


# ---- the named workloads (sizes as stated in the benchmark configurations) -----------------

def config_c1() -> tuple[CSR, np.ndarray]:
    """2D 5-point Laplacian, 32x32 grid, shifted by sigma = (lambda_min + lambda_max)/2 = 4 (exactly),
    p = 4 N(0,1) right-hand sides (seed 0).  The shifted operator is singular (32 zero modes)."""
    N = 32
    lo, hi = laplacian_eig_extremes(N, 2)
    sigma = 0.5 * (lo + hi)
    A = laplacian(N, 2, sigma)
    return A, randn_rhs(A.n, 4, seed=0)


def project_out(B: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """``B - Q (Q^T B)`` for orthonormal ``Q``: the range-projected right-hand side."""
    return np.ascontiguousarray(B - Q @ (Q.T @ B))


def config_c2(N: int = 128, frac: float = 0.10) -> tuple[CSR, np.ndarray]:
    """3D 7-point Laplacian on N^3 shifted by sigma at ``frac`` of the spectrum, p = 8 with two
    dependent columns (see :func:`dependent_rhs_p8`)."""
    A = laplacian(N, 3, shift_at_fraction(N, 3, frac))
    return A, dependent_rhs_p8(A.n, seed=0)


def config_c3(p: int, N: int = 128, frac: float = 0.10) -> tuple[CSR, np.ndarray]:
    A = laplacian(N, 3, shift_at_fraction(N, 3, frac))
    return A, randn_rhs(A.n, p, seed=0)


def config_c4(NK: int = 512, m: int = 65536, p: int = 8) -> tuple[CSR, np.ndarray, np.ndarray]:
    """Saddle point system, p N(0,1) right-hand sides (seed 0) and loss weights W (seed 2)."""
    A = saddle_point(NK, m, 4, seed=1)
    return A, randn_rhs(A.n, p, seed=0), randn_rhs(A.n, p, seed=2)


def config_c5(N: int = 192, frac: float = 0.05, p: int = 32) -> tuple[CSR, np.ndarray]:
    A = laplacian(N, 3, shift_at_fraction(N, 3, frac))
    return A, randn_rhs(A.n, p, seed=0)
