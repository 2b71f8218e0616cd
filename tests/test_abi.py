"""CPU-side checks of the C ABI boundary: the library loads and exports every declared symbol."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1301_2102_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    from paper_1301_2102_gb300 import _lib

    syms = _lib.exported_symbols()
    for s in ["bminres_create", "bminres_solve", "bminres_backward", "bminres_set_values", "bminres_spmm",
              "bminres_destroy", "bminres_status_string", "bminres_default_opts"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib_path):
    from paper_1301_2102_gb300 import _lib

    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for s in _lib.exported_symbols():
        assert s in exported, s
    lib = ctypes.CDLL(lib_path)
    for s in _lib.exported_symbols():
        assert hasattr(lib, s)


def test_host_only_entry_points(lib_path):
    """Entry points that need no GPU: defaults, status strings, argument validation."""
    from paper_1301_2102_gb300 import _lib

    lib = _lib.load()
    o = _lib.default_opts()
    assert o.precision == _lib.FP64 and o.gamma == 1e-8 and o.bench == 4 and o.ghost == 0
    for code, name in _lib.STATUS.items():
        assert lib.bminres_status_string(code).decode() == name
    h = ctypes.c_void_p()
    # invalid sizes are rejected before any device call
    assert lib.bminres_create(ctypes.byref(h), -1, 0, None, None, None, None) == -1
    assert lib.bminres_create(None, 1, 0, None, None, None, None) == -1
    info = _lib.Info()
    assert lib.bminres_solve(None, 1, None, None, 1e-10, 10, None, None, ctypes.byref(info)) == -1
    lib.bminres_destroy(None)


def test_sources_target_sm103a_only():
    from paper_1301_2102_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
