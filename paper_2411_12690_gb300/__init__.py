"""GB300-native implementation of the MORE-Stress online stage (arXiv 2411.12690).

The compute lives in ``libmstress.so`` (CUDA C++ for sm_103a behind the C ABI
in ``include/mstress.h``); this package only builds, loads and calls it.
Importing the package does not load the library; ``api.Context`` does, and
fails loudly when it has not been built.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "api", "build"]
