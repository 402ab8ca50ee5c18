"""GB300-native exact Gaussian process with compactly supported nonstationary kernels (arXiv 2411.05869).

The compute path lives in the CUDA library ``libgp.so`` (csrc/, C-ABI declared in include/gp.h); ``gp`` is
its thin ctypes binding. ``synth`` draws seeded synthetic inputs. Importing the package loads nothing; the
library is opened on first use of ``gp``.
"""
__all__ = ["gp", "synth"]
