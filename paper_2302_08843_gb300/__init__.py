"""GB300-native finite-difference micromagnetic hot path (arXiv 2302.08843).

The compute path lives in the C-ABI library ``libmm.so`` (CUDA for sm_103a,
sources in ``csrc/``, declarations in ``include/mm.h``); ``binding`` is the
thin ctypes layer above it.  Importing this package does not load the
library; ``binding.lib()`` does, and raises if it is missing.
"""
