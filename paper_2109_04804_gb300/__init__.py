"""GB300-native HBPC two-derivative deferred-correction DGSEM hot path.

The compute path is the CUDA library ``libhbpc`` (sources in ``csrc/``,
C-ABI in ``include/hbpc.h``); ``hbpc`` is its thin ctypes binding.  Importing
the package loads nothing; ``from paper_2109_04804_gb300 import hbpc`` loads
the library and raises if it has not been built.
"""
