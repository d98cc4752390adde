"""GB300-native coupled power-law / Cahn-Hilliard lattice Boltzmann step.

The compute path is the CUDA library built from ``csrc/`` for sm_103a and
reached through ``paper_2207_09431_gb300.lbm`` (ctypes over the C ABI in
``include/lbm.h``).  Importing this package does not load the library.
"""
__all__ = ["inputs"]
