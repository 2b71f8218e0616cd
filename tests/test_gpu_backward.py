"""The adjoint of the block solve on the GPU (bminres_backward and the autograd Function):
parity with the oracle-based adjoint, and central finite differences of GPU forward solves
(bar: 1e-5 relative), on a small saddle-point system of the config-4 family."""
import numpy as np
import pytest

from test_oracle_pins import _symmetric_pairs, adjoint_from_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_2102_gb300 import build

    build.build()
    return torch


def test_backward_matches_oracle_adjoint(torch_cuda, oracle_mod, workloads):
    from paper_1301_2102_gb300 import Solver

    torch = torch_cuda
    A = workloads.saddle_point(12, 40, 4, seed=2)
    rng = np.random.default_rng(5)
    B = rng.standard_normal((A.n, 4))
    G = rng.standard_normal((A.n, 4))
    Xo = oracle_mod.bminres(A, B, tol=1e-13, maxit=20 * A.n).X
    dBo, dAo = adjoint_from_oracle(oracle_mod, A, Xo, G)
    with Solver(A) as s:
        Xd, info, rel = s.solve(torch.from_numpy(B).cuda(), tol=1e-13, maxit=20 * A.n)
        dB, dA, binfo = s.backward(torch.from_numpy(G).cuda(), Xd, tol=1e-13, maxit=20 * A.n)
    assert binfo["status"] == 0
    dB, dA = dB.cpu().numpy(), dA.cpu().numpy()
    assert np.linalg.norm(dB - dBo) <= 1e-7 * np.linalg.norm(dBo)
    assert np.linalg.norm(dA - dAo) <= 1e-7 * np.linalg.norm(dAo)


def test_autograd_matches_finite_differences(torch_cuda, workloads):
    """L = sum(W * X), X = A(vals)^{-1} B: autograd gradients against central differences
    (h = 1e-6) of GPU forward solves, on B entries and on symmetric pairs of A."""
    from paper_1301_2102_gb300 import Solver, bminres_apply

    torch = torch_cuda
    A = workloads.saddle_point(10, 30, 4, seed=3)
    rng = np.random.default_rng(8)
    B0 = rng.standard_normal((A.n, 3))
    W = torch.from_numpy(rng.standard_normal((A.n, 3))).cuda()
    tol = 1e-13
    with Solver(A) as s:
        vals = torch.from_numpy(A.vals.copy()).cuda().requires_grad_(True)
        B = torch.from_numpy(B0).cuda().requires_grad_(True)
        X = bminres_apply(vals, B, s, tol=tol, maxit=20 * A.n)
        (W * X).sum().backward()
        gB, gV = B.grad.cpu().numpy(), vals.grad.cpu().numpy()

        def loss(v, b):
            s.set_values(torch.from_numpy(v).cuda())
            Xf, info, _ = s.solve(torch.from_numpy(b).cuda(), tol=tol, maxit=20 * A.n)
            assert info["status"] == 0
            return float((W * Xf).sum())

        h = 1e-6
        for (i, c) in [(0, 0), (A.n // 3, 1), (A.n - 1, 2), (A.n // 2, 0)]:
            Bp, Bm = B0.copy(), B0.copy()
            Bp[i, c] += h
            Bm[i, c] -= h
            fd = (loss(A.vals, Bp) - loss(A.vals, Bm)) / (2 * h)
            assert abs(fd - gB[i, c]) <= 1e-5 * max(1.0, abs(fd)), (i, c, fd, gB[i, c])
        pairs = _symmetric_pairs(A)
        for k, kt in [pairs[i] for i in (1, len(pairs) // 4, len(pairs) // 2, len(pairs) - 2)]:
            vp, vm = A.vals.copy(), A.vals.copy()
            for q in {k, kt}:
                vp[q] += h
                vm[q] -= h
            fd = (loss(vp, B0) - loss(vm, B0)) / (2 * h)
            an = gV[k] + (gV[kt] if kt != k else 0.0)
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (k, kt, fd, an)
        s.set_values(torch.from_numpy(A.vals).cuda())
