"""RANLUX++ random number streams on one GB300 (sm_103a), after Hahnfeld & Moneta,
"A Portable Implementation of RANLUX++" (arXiv 2106.02504).

The compute path is the CUDA library ``librlxpp.so`` (C ABI in ``include/rlxpp.h``);
``paper_2106_02504_gb300._rlxpp`` is its ctypes binding.  Importing the binding fails
when the library has not been built: there is no CPU fallback.
"""
import importlib

__all__ = ["build", "workloads", "native"]


def __getattr__(name):
    if name == "native":
        return importlib.import_module("._rlxpp", __name__)
    if name in ("build", "workloads"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
