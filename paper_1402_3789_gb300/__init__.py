"""GB300-native nearest-neighbour-method (NNM) single-linkage clustering.

The compute path is the CUDA library ``libnnm.so`` (sm_103a kernels behind a C ABI,
declared in ``include/nnm.h``); :mod:`paper_1402_3789_gb300.nnm` is the thin ctypes
binding over it.  Importing the package does not load the library: the binding loads
it on first use and raises if it is missing, so nothing here falls back to the CPU.
"""
