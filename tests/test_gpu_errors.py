"""Error statuses of the solve, produced without any GPU fault: NaN input, an exhausted bench, the
iteration limit, and the bounded grid-barrier wait running out (host-side fault injection:
BMINRES_DEBUG_BARRIER_TIMEOUT_MS makes every barrier wait for one block more than the grid has).
After each error the handle and the CUDA context stay usable."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_2102_gb300 import build

    build.build()
    return torch


def _ok_after(s, torch, A):
    B = torch.from_numpy(np.random.default_rng(1).standard_normal((A.n, 2))).cuda()
    X, info, rel = s.solve(B, tol=1e-8, maxit=50000)
    assert info["status"] == 0 and rel.max() < 1e-8


def test_nan_in_rhs_is_nonfinite(torch_cuda, workloads):
    from paper_1301_2102_gb300 import Solver
    from paper_1301_2102_gb300._lib import BminresError

    A = workloads.laplacian(12, 2, workloads.shift_at_fraction(12, 2, 0.2))
    B = workloads.randn_rhs(A.n, 3, 0)
    B[5, 1] = np.nan
    with Solver(A) as s:
        with pytest.raises(BminresError) as e:
            s.solve(torch_cuda.from_numpy(B).cuda(), tol=1e-8, maxit=1000)
        assert e.value.status == -6
        _ok_after(s, torch_cuda, A)


def test_exhausted_bench(torch_cuda, workloads):
    from paper_1301_2102_gb300 import Solver
    from paper_1301_2102_gb300._lib import BminresError

    A = workloads.laplacian(10, 3, workloads.shift_at_fraction(10, 3, 0.1))
    B = workloads.dependent_rhs_p8(A.n, seed=1)  # two dependent columns, one bench vector
    with Solver(A, bench=1) as s:
        with pytest.raises(BminresError) as e:
            s.solve(torch_cuda.from_numpy(B).cuda(), tol=1e-8, maxit=1000)
        assert e.value.status == -5
        _ok_after(s, torch_cuda, A)


def test_iteration_limit_keeps_the_iterate(torch_cuda, workloads):
    from paper_1301_2102_gb300 import Solver

    A = workloads.laplacian(16, 3, workloads.shift_at_fraction(16, 3, 0.1))
    B = workloads.randn_rhs(A.n, 4, 2)
    with Solver(A) as s:
        X, info, rel = s.solve(torch_cuda.from_numpy(B).cuda(), tol=1e-12, maxit=60)
    assert info["status"] == 1 and info["iters"] == 60 and 0 < rel.max() < 1.0


def test_barrier_wait_runs_out(torch_cuda, workloads, monkeypatch):
    from paper_1301_2102_gb300 import Solver
    from paper_1301_2102_gb300._lib import BminresError

    A = workloads.laplacian(64, 2, workloads.shift_at_fraction(64, 2, 0.2))  # 8 blocks
    B = torch_cuda.from_numpy(workloads.randn_rhs(A.n, 2, 0)).cuda()
    with Solver(A) as s:
        monkeypatch.setenv("BMINRES_DEBUG_BARRIER_TIMEOUT_MS", "50")
        with pytest.raises(BminresError) as e:
            s.solve(B, tol=1e-8, maxit=1000)
        assert e.value.status == -7
        monkeypatch.delenv("BMINRES_DEBUG_BARRIER_TIMEOUT_MS")
        _ok_after(s, torch_cuda, A)
