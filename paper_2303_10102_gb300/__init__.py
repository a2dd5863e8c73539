"""GB300-native HODLR Gaussian-process maximum likelihood (arXiv 2303.10102 hot path).

The computation lives in the CUDA library built from ``csrc/`` (C ABI: include/hodlr.h);
``lib.Hodlr`` is its thin Python binding.  There is no CPU fallback.
"""
from .lib import Hodlr, HodlrError, from_workload, load  # noqa: F401
