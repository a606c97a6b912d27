"""GB300-native gelpad IPC step (TacEx's GIPC physics layer, arXiv 2411.04776).

The CUDA library (libtxgel.so, C ABI in include/tx_gel.h) does all the work; `binding` is its
ctypes front end and `workloads` builds the seeded synthetic GelSight-style inputs.  The binding
is imported lazily so that building inputs never needs a GPU.
"""
import importlib

from . import workloads  # noqa: F401


def __getattr__(name):
    if name in ("binding", "serving"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
