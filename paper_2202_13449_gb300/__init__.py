"""GB300 (sm_103a) solver for 2D RTLBFS (arXiv 2202.13449).

The solver is the CUDA library built from ``csrc/`` (``build.py``) behind
the C ABI of ``include/rtlbfs.h``; ``capi`` is its ctypes binding and
``inputs`` the seeded synthetic inputs of the tests and the benchmark.
"""
