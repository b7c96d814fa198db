"""GB300-native fluid-solute step of RW-MI-DELBM (arXiv 2308.05007).

`Simulation` (the ctypes binding of librwmi.so) loads the CUDA library on first use and raises if
it is not built; `inputs` holds the seeded synthetic workloads.
"""
import importlib

from . import inputs  # noqa: F401  (numpy only)

__all__ = ["Simulation", "RwmiError", "inputs"]


def __getattr__(name):
    if name in ("Simulation", "RwmiError", "RwmiWarning", "load"):
        return getattr(importlib.import_module(__name__ + ".rwmi"), name)
    raise AttributeError(name)
