"""GPU parity for every shipped kernel instantiation beyond p = 8: FP64 <double,16> (p = 9..16) and
<double,32> (p = 17..32), double-word <dw,16>, and the FP32 inner solves <float,8>/<float,16> of
the mixed form, against the CPU oracle on small 3D shifted Laplacians (12^3 = 1728 rows, a ragged
tail for every tile shape).  Each block size runs three structures: N(0,1) right-hand sides, the
benchmark's dependence structure widened to p columns (two set-up substitutions, Sec. 5.1), and a
first column inside a 3-dimensional invariant subspace (a dependence in the middle of the iteration,
at band iteration 2p + 1, Sec. 5).  Bars as in tests/_parity.py."""
import numpy as np
import pytest

from _parity import REL_DW, check_fp64_result, iter_bracket, iters_ok, oracle_pair, rel_err, true_relres

pytestmark = pytest.mark.gpu

N = 12
TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_2102_gb300 import build

    build.build()
    return torch


def _problem(workloads, kind, p):
    if kind == "randn":
        A = workloads.laplacian(N, 3, workloads.shift_at_fraction(N, 3, 0.1))
        return A, workloads.randn_rhs(A.n, p, 2)
    if kind == "setup_dependence":
        A = workloads.laplacian(N, 3, workloads.shift_at_fraction(N, 3, 0.1))
        return A, workloads.dependent_rhs(A.n, p, 0)
    return workloads.near_dependent_laplacian(N, p)


def _solve(torch, A, B, maxit, **kw):
    from paper_1301_2102_gb300 import Solver

    with Solver(A, **kw) as s:
        Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        X, info, rel = s.solve(Bd, tol=TOL, maxit=maxit)
        torch.cuda.synchronize()
        return X.cpu().numpy(), info, rel


@pytest.mark.parametrize("p", [12, 16, 20, 32])
@pytest.mark.parametrize("kind", ["randn", "setup_dependence", "mid_dependence"])
def test_fp64_large_blocks(torch_cuda, oracle_mod, workloads, p, kind):
    A, B = _problem(workloads, kind, p)
    ref, ext = oracle_pair(oracle_mod, A, B, tol=TOL, maxit=40000)
    X, info, rel = _solve(torch_cuda, A, B, 40000)
    assert info["setup_deflations"] == ref.setup_deflations
    assert info["deflations"] == ref.deflations
    if kind == "setup_dependence":
        assert ref.setup_deflations == 2
    if kind == "mid_dependence":
        assert ref.defl_iters == [2 * p + 1]
    check_fp64_result(info, rel, true_relres(oracle_mod, A, B, ref.X).max(), TOL)
    assert iters_ok(info["iters"], ref, ext), (info["iters"], iter_bracket(ref, ext))
    assert rel_err(X, ref.X) <= 1e-7


@pytest.mark.parametrize("p", [12, 16, 20, 32])
def test_fp64_large_blocks_history(torch_cuda, oracle_mod, workloads, p):
    """Iterate-by-iterate: recursive residuals of the first 3p band iterations to 1e-10 of ||f0||,
    and the iterate after them to 1e-10."""
    from paper_1301_2102_gb300 import Solver

    A, B = _problem(workloads, "setup_dependence", p)
    K = 3 * p
    ref = oracle_mod.bminres(A, B, tol=1e-14, maxit=K, hist=K)
    with Solver(A) as s:
        s.set_history(K)
        X, info, rel = s.solve(torch_cuda.from_numpy(B).cuda(), tol=1e-14, maxit=K)
        H = s.history(p)
    assert info["iters"] == K == ref.iters and info["status"] == 1
    assert np.abs(H - ref.rho).max() <= 1e-10 * ref.f0norm.max()
    assert rel_err(X.cpu().numpy(), ref.X) <= 1e-10


@pytest.mark.parametrize("p", [12, 16])
@pytest.mark.parametrize("kind", ["randn", "setup_dependence", "mid_dependence"])
def test_double_word_p16_inner_solve(torch_cuda, oracle_mod, workloads, p, kind):
    """One double-word inner solve (no refinement) to a recursive 1e-10 on the <dw,16> kernel: the
    iterate agrees with the FP64 oracle to 1e-7 and the iteration count meets the double-word bar."""
    A, B = _problem(workloads, kind, p)
    ref, ext = oracle_pair(oracle_mod, A, B, tol=TOL, maxit=40000)
    X, info, rel = _solve(torch_cuda, A, B, 40000, precision="mixed_dw", tol_inner=TOL, max_outer=1)
    assert info["outer"] == 1 and info["setup_deflations"] == ref.setup_deflations
    assert iters_ok(info["iters"], ref, ext, REL_DW), (info["iters"], iter_bracket(ref, ext, REL_DW))
    assert rel_err(X, ref.X) <= 1e-7


@pytest.mark.parametrize("p", [16])
def test_double_word_p16_refined_reaches_tol(torch_cuda, oracle_mod, workloads, p):
    A, B = _problem(workloads, "setup_dependence", p)
    ref = oracle_mod.bminres(A, B, tol=TOL, maxit=40000)
    X, info, rel = _solve(torch_cuda, A, B, 400000, precision="mixed_dw", tol_inner=1e-6)
    assert info["status"] == 0 and rel.max() <= TOL
    assert rel_err(X, ref.X) <= 1e-7


@pytest.mark.parametrize("p", [8, 16])
@pytest.mark.parametrize("kind", ["randn", "setup_dependence"])
def test_fp32_inner_solves_refined(torch_cuda, oracle_mod, workloads, p, kind):
    """The FP32-inner mixed form on the <float,8> and <float,16> kernels (the ones the mixed
    benchmark mode times): FP32 vectors, block product and orthogonalisation inside FP64 iterative
    refinement reach an FP64 true residual <= tol; the error against the FP64 oracle is stated
    (bounded by the conditioning times tol: 1e-6 here)."""
    A, B = _problem(workloads, kind, p)
    ref = oracle_mod.bminres(A, B, tol=TOL, maxit=40000)
    X, info, rel = _solve(torch_cuda, A, B, 400000, precision="mixed", tol_inner=1e-4)
    assert info["status"] == 0, info
    assert rel.max() <= TOL
    assert info["setup_deflations"] >= ref.setup_deflations
    assert rel_err(X, ref.X) <= 1e-6


def test_fp32_single_inner_solve_tracks_oracle(torch_cuda, oracle_mod, workloads):
    """One FP32 inner solve of the <float,8> kernel, 40 band iterations: recursive residuals within
    FP32 rounding (1e-5 of ||f0||) of the FP64 oracle's; the iterate to 1e-5."""
    from paper_1301_2102_gb300 import Solver

    A, B = _problem(workloads, "randn", 8)
    K = 40
    ref = oracle_mod.bminres(A, B, tol=1e-14, maxit=K, hist=K)
    with Solver(A, precision="mixed", tol_inner=1e-14, max_outer=1) as s:
        s.set_history(K)
        X, info, rel = s.solve(torch_cuda.from_numpy(B).cuda(), tol=1e-14, maxit=K)
        H = s.history(8)
    assert info["iters"] == K
    assert np.abs(H - ref.rho).max() <= 1e-5 * ref.f0norm.max()
    assert rel_err(X.cpu().numpy(), ref.X) <= 1e-5
