"""GB300-native recursive Hermite-regularized lattice Boltzmann (arXiv:1710.02065).

The compute path is the CUDA library ``liblbm.so`` (sources in ``csrc/``,
C ABI in ``include/lbm.h``); ``lbm`` is its thin ctypes binding.  Importing
this package does not load the library; ``paper_1710_02065_gb300.lbm`` does.
"""
__all__ = ["lbm", "inputs"]
