"""GB300-native multi-scale shape-filter bank for blob detection.

Kennedy, "Digital filters with vanishing moments for shape analysis"
(arXiv:1912.07133).  The compute path is the C-ABI library built from
``csrc/`` (hand-written sm_103a CUDA kernels); ``kf`` is its thin Python
binding.  Importing this package does not load the library: ``kf`` does, and
it fails loudly when the library or a CUDA device is missing.
"""
__all__ = ["kf", "synthetic"]
