"""GB300-native generalized concurrent heap (arXiv 1906.06504).

The heap runs in hand-written CUDA kernels for sm_103a behind the C ABI of
include/gheap.h; ``heap.GHeap`` is the thin Python binding of that ABI.
"""
from . import build  # noqa: F401
