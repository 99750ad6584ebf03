"""GB300-native U(1)-sector matrix-free H x (divide-and-conquer basis ranking).

The compute path is the C-ABI library ``libdq.so`` (CUDA for sm_103a plus a C++ host sector
builder); ``binding`` wraps it with ctypes. Importing this package does not load the library;
``binding`` does, and fails loudly if it has not been built.
"""

__all__ = ["workloads", "binding"]
