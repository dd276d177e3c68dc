"""GB300-native row-wise PairHMM forward algorithm (Endeavor's row reformulation).

The compute path is the CUDA library built from ``csrc/`` (C ABI declared in
``include/phmm.h``); ``phmm`` is its thin ctypes binding.  ``workloads`` draws seeded
synthetic inputs.  Importing the package does not load the CUDA library; the first use
of ``phmm`` does, and fails loudly if it is missing.
"""
__all__ = ["phmm", "workloads"]
