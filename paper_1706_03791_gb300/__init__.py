"""GB300 (sm_103a) error-bounded lossy compressor for FP32 arrays.

Multilayer prediction from preceding decompressed values, error-controlled
quantization with truncated-binary fallback, and Huffman coding
(arXiv:1706.03791), with every step of the path in hand-written CUDA behind
the C ABI of include/szgb.h.  ``szgb`` is the Python binding.
"""
from . import szgb  # noqa: F401
