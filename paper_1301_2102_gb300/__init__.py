"""GB300 (sm_103a) block MINRES for symmetric indefinite systems with several right-hand sides.

The method is the band-Lanczos block MINRES of Soodhalter ("A block MINRES algorithm based on the
band Lanczos method"); the numerical work runs in hand-written CUDA kernels behind the C ABI in
``include/bminres.h``.  ``workloads`` builds the synthetic test operators and right-hand sides.
"""
import importlib

__all__ = ["Solver", "bminres_apply", "workloads"]


def __getattr__(name):
    if name in ("Solver", "bminres_apply"):
        return getattr(importlib.import_module(__name__ + ".solver"), name)
    if name == "workloads":
        return importlib.import_module(__name__ + ".workloads")
    raise AttributeError(name)
