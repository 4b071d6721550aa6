"""GB300-native turbulent gas-kinetic scheme (Righi 2013, after Xu 2001).

The compute path is the CUDA library ``libgks.so`` (sources in ``csrc/``, C ABI in
``include/gks.h``); ``gks`` is its thin ctypes binding and ``inputs`` draws the seeded synthetic
workloads.  Import ``paper_1302_2132_gb300.gks`` to load the library.
"""
__all__ = ["gks", "inputs"]
