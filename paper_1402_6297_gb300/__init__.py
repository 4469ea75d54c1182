"""GB300-native null-space-free (NSF) Maxwell eigensolver.

The compute path lives in ``libnfs.so`` (hand-written sm_103a CUDA behind a C
ABI, ``include/nfs.h``); :mod:`paper_1402_6297_gb300.nfs` is its thin ctypes
binding.  Importing this package loads nothing; the binding loads the library
on first use and raises if it has not been built.
"""

__all__ = ["nfs"]
