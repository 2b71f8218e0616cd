"""The allocation-free entry point bminres_solve_noalloc, called through the C ABI.

It serves callers that must not call cudaMalloc (device memory owned by another framework's pool,
or loops that cannot take cudaMalloc's implicit device-wide synchronisation): all of its
workspace lives in one static device array.  Its result must equal that of the regular entry
point (bminres_create + bminres_solve) and of the CPU oracle within the tolerance of the other
parity tests, on two calls in a row (the array keeps the previous call's contents); the second
call must leave the device's free memory unchanged; sizes that do not fit the array must be
rejected.  This file is collected last so that a stop-at-first-failure run has
already run every other test; it also passes when run alone.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_2102_gb300 import _lib, build

    build.build()
    lib = _lib.load()
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.bminres_solve_noalloc.argtypes = [I64, I64, P, P, P, I, P, P, D, I, P, P, P, ctypes.POINTER(_lib.Info)]
    lib.bminres_solve_noalloc.restype = I
    return torch, lib, _lib


def _prepare(torch, A, B, X0=None):
    dev = torch.device("cuda")
    t = {"rowptr": torch.from_numpy(A.rowptr.astype(np.int32)).to(dev),
         "colidx": torch.from_numpy(A.colidx.astype(np.int32)).to(dev),
         "vals": torch.from_numpy(A.vals.astype(np.float64)).to(dev),
         "B": torch.from_numpy(np.ascontiguousarray(B)).to(dev)}
    t["X"] = torch.zeros_like(t["B"]) if X0 is None else torch.from_numpy(np.ascontiguousarray(X0)).to(dev)
    return t


def _raw_call(torch, lib, _lib, A, p, t, tol, maxit, rel, info):
    """Only the C call: no tensor is created here, so the caching allocator stays out of the way."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.bminres_solve_noalloc(A.n, A.nnz, ctypes.c_void_p(t["rowptr"].data_ptr()),
                                     ctypes.c_void_p(t["colidx"].data_ptr()), ctypes.c_void_p(t["vals"].data_ptr()),
                                     p, ctypes.c_void_p(t["B"].data_ptr()), ctypes.c_void_p(t["X"].data_ptr()), tol,
                                     maxit, None, stream, rel.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))


def _call_noalloc(torch, lib, _lib, A, B, tol, maxit, X0=None):
    t = _prepare(torch, A, B, X0)
    rel = np.zeros(B.shape[1])
    info = _lib.Info()
    st = _raw_call(torch, lib, _lib, A, B.shape[1], t, tol, maxit, rel, info)
    torch.cuda.synchronize()
    return st, t["X"].cpu().numpy(), info, rel


def test_noalloc_matches_regular_entry_point_twice(env, workloads, oracle_mod):
    torch, lib, _lib = env
    from paper_1301_2102_gb300 import Solver

    tol, maxit = 1e-10, 40000
    A = workloads.laplacian(14, 3, workloads.shift_at_fraction(14, 3, 0.1))  # n = 2744
    B = workloads.dependent_rhs_p8(A.n, seed=3)  # two dependent columns: bench substitution at set-up
    with Solver(A) as s:
        Xr, info_r, rel_r = s.solve(torch.from_numpy(B).cuda(), tol=tol, maxit=maxit)
        Xr = Xr.cpu().numpy()
    assert info_r["status"] == 0
    ref = oracle_mod.bminres(A, B, tol=tol, maxit=maxit)  # second reference: the CPU oracle
    for call in range(2):  # the second call starts from the first call's leftovers in the array
        t = _prepare(torch, A, B)
        rel = np.zeros(B.shape[1])
        info = _lib.Info()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _raw_call(torch, lib, _lib, A, B.shape[1], t, tol, maxit, rel, info)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        X = t["X"].cpu().numpy()
        assert st == 0, _lib.STATUS.get(st)
        if call == 1:  # the first call on a device may load the module; later calls allocate nothing
            assert free1 == free0, (free0, free1)
        assert info.iters == info_r["iters"] and info.setup_deflations == info_r["setup_deflations"]
        assert rel.max() <= tol
        assert np.linalg.norm(X - Xr) <= 1e-7 * np.linalg.norm(Xr), call
        assert np.linalg.norm(X - ref.X) <= 1e-7 * np.linalg.norm(ref.X), call


def test_noalloc_other_shape_then_original(env, workloads):
    """A smaller p between two calls of the original shape: stale contents must not leak in."""
    torch, lib, _lib = env
    from paper_1301_2102_gb300 import Solver

    A = workloads.laplacian(20, 2, workloads.shift_at_fraction(20, 2, 0.2))
    B = workloads.randn_rhs(A.n, 5, 7)
    with Solver(A) as s:
        Xr, info_r, _ = s.solve(torch.from_numpy(B).cuda(), tol=1e-10, maxit=4000)
        Xr = Xr.cpu().numpy()
    st, X1, _, _ = _call_noalloc(torch, lib, _lib, A, B, 1e-10, 4000)
    st2, _, _, _ = _call_noalloc(torch, lib, _lib, A, B[:, :2].copy(), 1e-10, 4000)
    st3, X3, info3, _ = _call_noalloc(torch, lib, _lib, A, B, 1e-10, 4000)
    assert st == 0 and st2 == 0 and st3 == 0
    for X in (X1, X3):
        assert np.linalg.norm(X - Xr) <= 1e-7 * np.linalg.norm(Xr)
    assert info3.iters == info_r["iters"]


def test_noalloc_rejects_sizes_beyond_the_array(env, workloads):
    torch, lib, _lib = env
    A = workloads.laplacian(40, 3, 0.5)  # n = 64000: (6*32 + 8) * 8 * n bytes > 64 MiB at p = 32
    B = workloads.randn_rhs(A.n, 32, 1)
    st, X, info, rel = _call_noalloc(torch, lib, _lib, A, B, 1e-10, 10)
    assert st == -1 and np.all(X == 0.0)
