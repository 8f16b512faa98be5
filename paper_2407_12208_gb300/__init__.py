"""Mixed-precision Lloyd's k-means on GB300 (sm_103a).

Carson, Chen & Liu, "Computing k-means in Mixed Precision" (arXiv 2407.12208):
expanded-formula distances with a low-precision tensor-core cross term, the
rounding-error reliability test of Section 4.3, direct-formula recomputation
from the original data, certified argmin, and the centre update of
Section 4.4.  The compute runs in libmpkm.so (CUDA kernels behind the C-ABI in
include/mpkm.h); this package is its Python binding.
"""
from ._binding import (BF16, E4M3, EMPTY_FARTHEST, EMPTY_KEEP, EXPORTS, FP16, FP32_DIRECT, FP64_DIRECT,
                       TEST_OFF, TEST_PAPER, TEST_TC, Context, KmError, Params, device_array, load, params)

__all__ = ["Context", "KmError", "Params", "params", "load", "device_array", "EXPORTS", "FP64_DIRECT",
           "FP32_DIRECT", "FP16", "BF16", "E4M3", "TEST_TC", "TEST_PAPER", "TEST_OFF", "EMPTY_KEEP",
           "EMPTY_FARTHEST"]
