"""GB300-native Monte Carlo KS cutoffs for the discrete power law (Rappos & Robert, 2013).

The compute path lives in the CUDA shared library built from ``csrc/`` and
declared in ``include/pl.h``; ``paper_1305_6738_gb300.pl`` is the thin ctypes
binding over it (argument marshalling only).  Importing this package does not
load the library; ``paper_1305_6738_gb300.pl`` does, and raises if it is
missing.
"""
__all__ = ["inputs"]
