"""GB300-native hot path of the hybrid pseudopotential phase-change lattice
Boltzmann method with conjugate heat transfer (arXiv:1911.10747).

The compute path lives in the CUDA library ``csrc/`` (C ABI in
``include/lbm.h``); :mod:`.lbm` is its ctypes binding and :mod:`.workloads`
holds the run configurations.  Importing the package loads nothing native.
"""
__all__ = ["lbm", "workloads"]
