"""GB300-native implicit ADI solver for the 2D acoustic wave equation.

The compute path is the C-ABI library ``libadiwave.so`` (hand-written sm_103a
CUDA kernels, declared in ``include/adiwave.h``).  This package is its thin
Python binding: argument marshalling onto the library, with PyTorch used only
for device memory and streams.  Importing the package does not load the
library; the first call that needs it does, and fails loudly if it is missing.
"""
import importlib

_SUBMODULES = {"api": ".api", "lib": "._lib", "inputs": ".inputs", "autotune": ".autotune",
               "build": ".build", "shard": ".shard"}


def __getattr__(name):
    if name in _SUBMODULES:
        mod = importlib.import_module(_SUBMODULES[name], __name__)
        globals()[name] = mod
        return mod
    raise AttributeError(name)
