"""GB300 (sm_103a) local nucleus decomposition: incidence construction and
the iterated h-index update (SND, AND with notification) behind a C ABI.

Submodules:
    nd      -- ctypes binding of libnd (the CUDA library); loads it on use
    graphs  -- seeded synthetic graph generators and CSR normalisation
"""
import importlib

__all__ = ["nd", "graphs"]


def __getattr__(name):
    # import submodules lazily so that graph generation needs no CUDA library
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
