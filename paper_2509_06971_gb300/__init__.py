"""GB300-native hot path of PeTTO (pseudo-transient topology optimisation, arXiv 2509.06971).

The numerics live in libpetto.so (hand-written CUDA for sm_103a behind the C ABI of
include/petto.h).  ``capi`` is the ctypes binding with the C names, ``problem.Problem``
a thin owner of one context, ``problem.Batch`` of a batch of 2D contexts advanced by one
launch per sweep, ``workloads`` the seeded synthetic problem instances.
Nothing is loaded at import time; the first use loads (and if needed builds) the
library and raises if that fails -- there is no CPU fallback.
"""
from . import workloads  # noqa: F401  (inputs only: numpy, no GPU)

__all__ = ["workloads", "capi", "problem"]


def __getattr__(name):
    if name in ("capi", "problem", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
