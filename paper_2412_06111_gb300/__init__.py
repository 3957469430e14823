"""GB300-native tree tensor network Nystrom (TTNN / STTNN) sketching.

The compute path is libttnn.so (hand-written sm_103a CUDA behind the C ABI in
include/ttnn.h); ``api`` is its thin Python binding with the same names.
"""
from . import api  # noqa: F401
from ._native import build, load  # noqa: F401
