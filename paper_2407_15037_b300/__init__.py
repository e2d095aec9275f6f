"""B300-native guaranteed-error-bound lossy quantizers (arXiv 2407.15037).

The compute path is the CUDA library liblcq.so (sources in csrc/, C ABI in
include/lcq.h); this package is its Python binding.  Importing the package
does not load the library; the first call does, and raises if it is missing.
"""
from .lcq import (ABS, F32, F64, NOA, REL, Batch, BatchInfo, BatchItem, Header, LcqError, Quantized, alloc_outputs,  # noqa: F401
                  debug_set_scan, dequantize, dequantize_into, finite_range, lib, new_workspace, quantize,
                  quantize_into, quantize_noa_range_into, quantize_host, host_stage_size, sync_status, workspace_size)
