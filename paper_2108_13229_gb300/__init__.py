"""GB300-native monolithic Stokes-Darcy solver (arXiv 2108.13229, Secs. 2 and 4).

The solver is the CUDA library ``libsd.so`` behind the C ABI declared in
``include/sd.h``; ``paper_2108_13229_gb300.sd`` is its thin ctypes binding.
Importing this package loads nothing: the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["inputs", "sd"]
