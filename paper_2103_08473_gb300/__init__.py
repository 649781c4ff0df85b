"""GB300-native engine for the Kramers-unrestricted complex CCSD iteration.

The compute path lives in ``libccsd.so`` (CUDA kernels for sm_103a behind a
C ABI, declared in ``include/ccsd.h``); :mod:`paper_2103_08473_gb300.ccsd` is the
thin ctypes binding. :mod:`.inputs` holds the seeded synthetic input
generators and :mod:`.flops` the operation counts used for reporting.
Submodules are imported lazily so that importing the generators never loads
the CUDA library.
"""
import importlib

__all__ = ["ccsd", "inputs", "flops", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
