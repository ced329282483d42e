"""GB300-native (sm_103a) hierarchical (r,s) nucleus decomposition.

The compute path lives in the CUDA library ``libnucleus.so`` (sources in ``csrc/``, C-ABI in
``include/nucleus.h``); ``nucleus`` is the thin Python binding over it and ``graphgen`` holds the
seeded synthetic input generators.  Importing the package does not load the library.
"""
__all__ = ["graphgen", "nucleus"]
