"""GPU parity: the CUDA block MINRES (through the C ABI) against the FP64 CPU oracle on the same
seeded inputs.  Bars (tests/_parity.py): FP64 true relative residual <= tol with status OK (or the
residual-gap status where the oracle's own result misses tol too); ||X_gpu - X_oracle|| /
||X_oracle|| <= 1e-7 in FP64; recursive-residual histories equal to 1e-10 relative before rounding
is amplified; iteration counts within the interval spanned by three rounding builds of the oracle,
widened by max(2, 1 %) (the spread that rounding alone causes on each case).
"""
import numpy as np
import pytest

from _parity import REL_DW, check_fp64_result, iter_bracket, iters_ok, oracle_pair, rel_err, true_relres

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_2102_gb300 import build

    build.build()
    return torch


def _solve(torch, A, B, tol=1e-10, maxit=20000, X0=None, **kw):
    from paper_1301_2102_gb300 import Solver

    with Solver(A, **kw) as s:
        Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        Xd = torch.zeros_like(Bd) if X0 is None else torch.from_numpy(np.ascontiguousarray(X0)).cuda()
        X, info, rel = s.solve(Bd, Xd, tol=tol, maxit=maxit)
        torch.cuda.synchronize()
        return X.cpu().numpy(), info, rel


def test_spmm_matches_csr_order(torch_cuda, oracle_mod, workloads):
    from paper_1301_2102_gb300 import Solver

    for A in [workloads.laplacian(9, 3, 0.7), workloads.saddle_point(16, 40, 4, seed=1),
              workloads.random_symmetric_indefinite(37, 2)]:
        for p in (1, 3, 8, 17):
            X = workloads.randn_rhs(A.n, p, 5)
            with Solver(A) as s:
                Y = s.spmm(torch_cuda.from_numpy(X).cuda()).cpu().numpy()
            ref = oracle_mod.spmm(A, X)
            assert np.abs(Y - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 8])
def test_parity_2d_small(torch_cuda, oracle_mod, workloads, p):
    A = workloads.laplacian(20, 2, workloads.shift_at_fraction(20, 2, 0.2))
    B = workloads.randn_rhs(A.n, p, 1)
    ref, ext = oracle_pair(oracle_mod, A, B, tol=1e-10, maxit=20000)
    X, info, rel = _solve(torch_cuda, A, B)
    check_fp64_result(info, rel, true_relres(oracle_mod, A, B, ref.X).max(), 1e-10)
    assert iters_ok(info["iters"], ref, ext), (info["iters"], iter_bracket(ref, ext))
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) <= 1e-7


def test_parity_config1_projected(torch_cuda, oracle_mod, workloads):
    A, B = workloads.config_c1()
    Q = workloads.laplacian_null_modes_2d(32, 4.0)
    Bp = workloads.project_out(B, Q)
    ref, ext = oracle_pair(oracle_mod, A, Bp, tol=1e-10, maxit=4000)
    X, info, rel = _solve(torch_cuda, A, Bp, maxit=4000)
    check_fp64_result(info, rel, true_relres(oracle_mod, A, Bp, ref.X).max(), 1e-10)
    assert iters_ok(info["iters"], ref, ext), (info["iters"], iter_bracket(ref, ext))
    Xr = X - Q @ (Q.T @ X)
    Rr = ref.X - Q @ (Q.T @ ref.X)
    assert np.linalg.norm(Xr - Rr) / np.linalg.norm(Rr) <= 1e-7


@pytest.mark.parametrize("p", [4, 8])
def test_parity_3d_ragged(torch_cuda, oracle_mod, workloads, p):
    A = workloads.laplacian(13, 3, workloads.shift_at_fraction(13, 3, 0.1))  # n = 2197, not a tile multiple
    B = workloads.randn_rhs(A.n, p, 2)
    ref, ext = oracle_pair(oracle_mod, A, B, tol=1e-10, maxit=40000)
    X, info, rel = _solve(torch_cuda, A, B, maxit=40000)
    check_fp64_result(info, rel, true_relres(oracle_mod, A, B, ref.X).max(), 1e-10)
    assert iters_ok(info["iters"], ref, ext), (info["iters"], iter_bracket(ref, ext))
    kappa_tol = 1e-7
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) <= kappa_tol


def test_parity_setup_deflation(torch_cuda, oracle_mod, workloads):
    """Config-2 right-hand-side structure on a 12^3 grid: two columns dependent at set-up."""
    A = workloads.laplacian(12, 3, workloads.shift_at_fraction(12, 3, 0.10))
    B = workloads.dependent_rhs_p8(A.n, seed=0)
    ref, ext = oracle_pair(oracle_mod, A, B, tol=1e-10, maxit=40000, bench=4)
    X, info, rel = _solve(torch_cuda, A, B, maxit=40000, bench=4)
    assert ref.setup_deflations == 2 and info["setup_deflations"] == 2
    check_fp64_result(info, rel, true_relres(oracle_mod, A, B, ref.X).max(), 1e-10)
    assert iters_ok(info["iters"], ref, ext), (info["iters"], iter_bracket(ref, ext))
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) <= 1e-7


def test_parity_dependence_demo(torch_cuda, oracle_mod, workloads):
    """B = [e_1, A e_1]: dependence at iteration 1, bench substitution, column 2 solved by e_1."""
    A = workloads.laplacian(20, 2, workloads.shift_at_fraction(20, 2, 0.3))
    e1 = np.zeros(A.n)
    e1[0] = 1.0
    B = np.stack([e1, oracle_mod.spmm(A, e1[:, None])[:, 0]], axis=1)
    ref, ext = oracle_pair(oracle_mod, A, B, tol=1e-10, maxit=4000)
    X, info, rel = _solve(torch_cuda, A, B, maxit=4000)
    assert ref.defl_iters[0] == 1 and info["deflations"] >= 1
    check_fp64_result(info, rel, true_relres(oracle_mod, A, B, ref.X).max(), 1e-10)
    assert np.linalg.norm(X[:, 1] - e1) <= 1e-12
    assert iters_ok(info["iters"], ref, ext), (info["iters"], iter_bracket(ref, ext))
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) <= 1e-7


def test_parity_nonzero_x0_and_zero_column(torch_cuda, oracle_mod, workloads):
    # (15 x 15 at 25% would be singular: sigma equals the eigenvalue of mode (1, 8))
    A = workloads.laplacian(15, 2, workloads.shift_at_fraction(15, 2, 0.23))
    B = workloads.randn_rhs(A.n, 3, 4)
    B[:, 1] = 0.0
    X0 = 0.1 * workloads.randn_rhs(A.n, 3, 5)
    X0[:, 1] = 0.0
    ref, ext = oracle_pair(oracle_mod, A, B, X0=X0, tol=1e-10, maxit=4000)
    X, info, rel = _solve(torch_cuda, A, B, X0=X0, maxit=4000)
    assert info["setup_deflations"] == 1
    check_fp64_result(info, rel, true_relres(oracle_mod, A, B, ref.X, X0).max(), 1e-10)
    assert np.all(X[:, 1] == 0.0)
    assert iters_ok(info["iters"], ref, ext), (info["iters"], iter_bracket(ref, ext))
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) <= 1e-7


def test_maxit_and_degenerate(torch_cuda, oracle_mod, workloads):
    A = workloads.laplacian(10, 2, workloads.shift_at_fraction(10, 2, 0.3))
    B = workloads.randn_rhs(A.n, 2, 3)
    ref = oracle_mod.bminres(A, B, tol=1e-12, maxit=7, xhist=7)
    X, info, rel = _solve(torch_cuda, A, B, tol=1e-12, maxit=7)
    assert info["status"] == 1 and info["iters"] == 7
    assert np.linalg.norm(X - ref.X) <= 1e-12 * np.linalg.norm(ref.X)
    X, info, rel = _solve(torch_cuda, A, np.zeros((A.n, 2)), maxit=10)
    assert info["status"] == 0 and info["iters"] == 0 and np.all(X == 0)


def test_mixed_precision_reaches_tol(torch_cuda, oracle_mod, workloads):
    A = workloads.laplacian(16, 3, workloads.shift_at_fraction(16, 3, 0.1))
    B = workloads.randn_rhs(A.n, 4, 1)
    ref = oracle_mod.bminres(A, B, tol=1e-10, maxit=40000)
    X, info, rel = _solve(torch_cuda, A, B, maxit=200000, precision="mixed")
    assert info["status"] == 0, info
    assert rel.max() < 1e-10
    # error against the FP64 oracle is bounded by the conditioning times the residual gap
    err = np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X)
    assert err < 1e-6, err


@pytest.mark.parametrize("p", [1, 4, 8])
def test_double_word_inner_solve_matches_oracle(torch_cuda, oracle_mod, workloads, p):
    """One double-word inner solve (no refinement step) to a recursive 1e-10: the iterate agrees
    with the FP64 oracle to the FP64 bar (1e-7 relative) and the band iteration count meets the
    double-word bar, because ~48-bit vectors keep the recurrence close to FP64's."""
    A = workloads.laplacian(24, 2, workloads.shift_at_fraction(24, 2, 0.15))
    B = workloads.randn_rhs(A.n, p, 11)
    ref, ext = oracle_pair(oracle_mod, A, B, tol=1e-10, maxit=20000)
    X, info, rel = _solve(torch_cuda, A, B, maxit=20000, precision="mixed_dw", tol_inner=1e-10, max_outer=1)
    assert info["outer"] == 1
    assert iters_ok(info["iters"], ref, ext, REL_DW), (info["iters"], iter_bracket(ref, ext, REL_DW))
    assert np.linalg.norm(X - ref.X) <= 1e-7 * np.linalg.norm(ref.X)


def test_double_word_refinement_reaches_tol(torch_cuda, oracle_mod, workloads):
    A = workloads.laplacian(16, 3, workloads.shift_at_fraction(16, 3, 0.1))
    B = workloads.dependent_rhs_p8(A.n, seed=2)
    ref = oracle_mod.bminres(A, B, tol=1e-10, maxit=40000)
    X, info, rel = _solve(torch_cuda, A, B, maxit=200000, precision="mixed_dw")
    assert info["status"] == 0, info
    assert rel.max() < 1e-10 and info["setup_deflations"] == ref.setup_deflations
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) < 1e-7


def test_fp64_refined_reaches_true_tol(torch_cuda, oracle_mod, workloads):
    """FP64 inner solves inside the refinement loop: the FP64 true residual meets tol (one restart
    at most here) and the result agrees with the oracle."""
    A = workloads.laplacian(16, 3, workloads.shift_at_fraction(16, 3, 0.1))
    B = workloads.randn_rhs(A.n, 4, 3)
    ref = oracle_mod.bminres(A, B, tol=1e-10, maxit=40000)
    X, info, rel = _solve(torch_cuda, A, B, maxit=200000, precision="fp64_refined", tol_inner=1e-6)
    assert info["status"] == 0 and 1 <= info["outer"] <= 3, info
    assert rel.max() < 1e-10
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) < 1e-7


def test_double_word_rejects_p_above_16(torch_cuda, workloads):
    from paper_1301_2102_gb300 import Solver
    from paper_1301_2102_gb300._lib import BminresError

    A = workloads.laplacian(12, 2, 0.3)
    with Solver(A, precision="mixed_dw") as s, pytest.raises(BminresError):
        s.solve(torch_cuda.from_numpy(workloads.randn_rhs(A.n, 17, 0)).cuda(), tol=1e-8, maxit=100)


@pytest.mark.parametrize("p", [1, 3, 8])
def test_residual_history_matches_before_amplification(torch_cuda, oracle_mod, workloads, p):
    """Iterate-by-iterate parity: the recursive residual norms of every band iteration agree with
    the oracle's to 1e-10 (relative to ||f0_i||) over the first 60 iterations."""
    from paper_1301_2102_gb300 import Solver

    A = workloads.laplacian(24, 2, workloads.shift_at_fraction(24, 2, 0.15))
    B = workloads.randn_rhs(A.n, p, 6)
    ref = oracle_mod.bminres(A, B, tol=1e-14, maxit=60, hist=60)
    with Solver(A) as s:
        s.set_history(60)
        X, info, rel = s.solve(torch_cuda.from_numpy(B).cuda(), tol=1e-14, maxit=60)
        H = s.history(p)
    assert info["iters"] == 60 and H.shape == (60, p)
    assert np.abs(H - ref.rho).max() <= 1e-10 * ref.f0norm.max()
    Xr = ref.X
    assert np.linalg.norm(X.cpu().numpy() - Xr) <= 1e-10 * np.linalg.norm(Xr)


def test_parity_near_dependence(torch_cuda, oracle_mod, workloads):
    """f_1 lies within 1e-14 of a 3-dimensional invariant subspace: with p = 2 the vector built at
    iteration 5 is near-dependent (||w|| <= gamma ||A u_5||) and is replaced by a bench vector."""
    n = 300
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(0.6, 4.0, n) * np.where(np.arange(n) % 3 == 0, -1.0, 1.0)
    D = (Q * lam) @ Q.T
    A = workloads.dense_to_csr(0.5 * (D + D.T))
    f1 = Q[:, :3] @ np.array([1.0, -0.7, 0.4]) + 1e-14 * rng.standard_normal(n)
    B = np.stack([f1, rng.standard_normal(n)], axis=1)
    ref, ext = oracle_pair(oracle_mod, A, B, tol=1e-10, maxit=3000)
    X, info, rel = _solve(torch_cuda, A, B, maxit=3000)
    assert ref.defl_iters[:1] == [5] and info["deflations"] >= 1
    check_fp64_result(info, rel, true_relres(oracle_mod, A, B, ref.X).max(), 1e-10)
    assert iters_ok(info["iters"], ref, ext), (info["iters"], iter_bracket(ref, ext))
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) <= 1e-7


def test_removed_vector_retention_same_process(torch_cuda, oracle_mod, workloads):
    """With retention switched on (ghost=True) the GPU keeps the same removed vector: the recursive
    residuals agree with the oracle's before the dependence to rounding and after it (iterations
    5..12) to 1e-4: the kept direction is w / ||w|| with ||w|| ~ 1e-8 ||A u_5||, which magnifies
    rounding differences of w by ~1e8."""
    from paper_1301_2102_gb300 import Solver

    n = 300
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(0.6, 4.0, n) * np.where(np.arange(n) % 3 == 0, -1.0, 1.0)
    D = (Q * lam) @ Q.T
    A = workloads.dense_to_csr(0.5 * (D + D.T))
    f1 = Q[:, :3] @ np.array([1.0, -0.7, 0.4]) + 1e-14 * rng.standard_normal(n)
    B = np.stack([f1, rng.standard_normal(n)], axis=1)
    ref = oracle_mod.bminres(A, B, tol=1e-14, maxit=12, hist=12, ghost=True)
    with Solver(A, ghost=True) as s:
        s.set_history(12)
        X, info, rel = s.solve(torch_cuda.from_numpy(B).cuda(), tol=1e-14, maxit=12)
        H = s.history(2)
    assert info["deflations"] == 1 and ref.defl_iters == [5]
    assert np.abs(H[:4] - ref.rho[:4]).max() <= 1e-12 * ref.f0norm.max()
    assert np.abs(H - ref.rho).max() <= 1e-4 * ref.f0norm.max()
