"""B300-native two-component TDSLDA step (arXiv:2009.00745, LISE).

The hot path lives in the CUDA library ``liblise.so`` behind a C ABI
(include/lise.h); ``paper_2009_00745_b300.lise`` is its thin ctypes binding and
``paper_2009_00745_b300.workloads`` builds seeded synthetic inputs.
"""
import importlib

__all__ = ["lise", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
