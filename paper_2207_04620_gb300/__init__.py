"""GB300-native RNS-CKKS evaluation for the Hercules packed matrix product and
composite-polynomial sign/ReLU (arXiv 2207.04620).

The compute path is libhx.so (hand-written CUDA for sm_103a behind the C ABI
in include/hx.h); `hx` is its ctypes binding, `workloads` the seeded input
generators shared with the tests.
"""
from . import hx  # noqa: F401
