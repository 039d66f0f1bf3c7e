"""GB300-native B-spline x-ray transform (SplineSplat, arXiv 2511.11078).

The compute path is the C-ABI library ``libspl.so`` (hand-written sm_103a
CUDA kernels) built from ``csrc/``; ``spl`` is its thin ctypes binding.
Importing this package does not load the library: ``spl.lib()`` does, and
raises if it is missing -- there is no CPU fallback.
"""
