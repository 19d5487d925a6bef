"""GB300-native heterogeneous-DSA S_N transport (arXiv 2001.09196 hot path).

The compute path lives in the CUDA library libsn (csrc/, declared in include/sn.h);
this package is its thin Python binding.  Importing the package does not load the
library: `paper_2001_09196_gb300.sn` does, and fails loudly when it is missing.
"""
__all__ = ["inputs", "sn"]
