"""GB300-native p-bit simulated annealing (pSA) with device variability.

The compute path is the C-ABI library ``libpbit.so`` (hand-written sm_103a
CUDA behind ``include/pbit.h``); :mod:`.pbit` is its thin ctypes binding and
:mod:`.inputs` draws seeded synthetic workloads.  Importing the package loads
nothing; the library is loaded on first use and the binding raises if it is
missing.
"""
__all__ = ["inputs", "pbit"]
