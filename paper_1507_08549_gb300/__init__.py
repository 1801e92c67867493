"""GB300-native WENO5 / Lax-Friedrichs / SSP-RK3 hydrodynamics of the 2D Euler equations with a
level-set flame scalar (Leung, Chu & Lin 2015, Sec. 2.1-2.2), as hand-written sm_103a CUDA kernels
behind a C ABI.

Submodules load lazily: ``workloads`` (seeded inputs) needs only numpy; ``hydro`` (the ctypes binding
of the CUDA library) needs the built shared library and raises if it is missing.
"""
import importlib

__all__ = ["workloads", "hydro", "build"]


def __getattr__(name):
    if name in ("workloads", "hydro", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
