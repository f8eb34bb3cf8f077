"""GB300 (sm_103a) D1Q3 Monte Carlo Lattice Gas.

The hot path (stream + C exact random sub-collisions per node and step) runs in
the CUDA library ``_build/libmclg.so`` behind the C ABI of ``include/mclg.h``;
``mclg`` is its ctypes binding and ``workloads`` generates seeded synthetic
inputs.  Importing this package does not load the library; the first call that
needs it does, and raises if it has not been built.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "mclg", "build"]


def __getattr__(name):
    if name in ("mclg", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
