"""GB300-native hot path of the Lagrangian particle (LP) method.

The compute path is the CUDA library ``liblp.so`` (sources in ``csrc/``,
C-ABI declared in ``include/lp.h``); ``lp`` is its thin ctypes binding and
``inputs`` holds the seeded synthetic workloads.  Importing the package loads
nothing; the library is loaded on first use and a missing library is an error.
"""
__all__ = ["lp", "inputs"]
