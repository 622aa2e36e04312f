"""GB300-native FAS multigrid solver for the ISIS scalar-field equations
(Llinares, Mota & Winther 2013, arXiv:1307.6748).

The compute path is the CUDA library ``libisis_gb300.so`` (C ABI in
``include/isis.h``); ``paper_1307_6748_gb300.isis`` binds it for PyTorch
tensors.  ``synth`` holds the seeded synthetic inputs.
"""
__all__ = ["build", "isis", "synth"]
