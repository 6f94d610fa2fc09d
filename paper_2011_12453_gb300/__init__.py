"""GB300-native graph-neural-ansatz variational Monte Carlo (arXiv:2011.12453).

The compute path lives in the CUDA library ``libgna.so`` built from ``csrc/``; the
Python module ``gna`` is a thin ctypes binding over its C ABI (``include/gna.h``).
Importing this package does not load the library; ``gna`` loads it on first use and
raises if it is missing.
"""
__all__ = ["gna", "workloads"]
