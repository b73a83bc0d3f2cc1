"""GB300-native partial Fourier transform (PFT) and PIE hot path.

The compute lives in a CUDA shared library with a C ABI (``include/pft.h``);
``paper_2408_03532_gb300.pft`` is the thin ctypes binding over it. Importing
this package does not load the library; the binding loads it on first use and
raises if it has not been built.
"""
