"""GB300-native (sm_103a) right-hand side of entropy-stable flux-differencing LGL-DGSEM for the
compressible Euler equations (Ranocha et al., arXiv:2112.10517).

The compute path is the C-ABI library ``libdg.so`` (hand-written CUDA, declared in ``include/dg.h``);
``paper_2112_10517_gb300.dg`` is its thin ctypes binding. Importing this package does not load the
library; ``inputs`` (seeded initial conditions) needs neither CUDA nor the library.
"""
import importlib

__all__ = ["dg", "inputs"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
