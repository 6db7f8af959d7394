"""GB300-native 3-path and centred 3-path sampling (Jha, Seshadhri & Pinar)
for estimating the six connected induced 4-vertex subgraph counts.

The compute path is the CUDA library ``libpathsample.so`` (C interface in
include/pathsample.h); ``pathsample`` is its ctypes binding.
"""
from . import pathsample  # noqa: F401
from .pathsample import Graph, PathSampleError, load_library  # noqa: F401
