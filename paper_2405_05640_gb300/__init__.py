"""GB300-native (sm_103a) spectral-element pressure-Poisson hot path.

The compute lives in the CUDA shared library built from ``csrc/`` and
declared in ``include/sem.h``; ``binding`` marshals arguments to it through
ctypes.  Importing this package does not load the library; ``binding.lib()``
does, and raises if it has not been built.
"""
__all__ = ["inputs", "binding"]
