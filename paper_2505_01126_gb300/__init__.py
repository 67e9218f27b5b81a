"""GB300-native fused two-phase lattice Boltzmann step (accLB, arXiv 2505.01126).

The compute path is the CUDA library ``csrc/liblbgb.so`` (C ABI declared in
``include/lbgb.h``); ``lbgb`` is its thin ctypes binding.  Nothing is loaded at
import time: ``from paper_2505_01126_gb300 import lbgb`` loads the library and
fails loudly if it has not been built.
"""
__all__ = ["lbgb", "inputs", "build"]
