"""GB300-native conservative sharp-interface solver with multi-time-step
sub-cycling (Long, Cai & Pan, arXiv 1905.03917).

The compute path is ``libsif`` (hand-written CUDA for sm_103a behind a
C-ABI, ``include/sif.h``); ``paper_1905_03917_gb300.sif`` is its thin
ctypes binding.  Importing the package loads nothing; the binding loads
the library on first use and fails loudly if it is missing.
"""
__all__ = ["inputs", "sif"]
