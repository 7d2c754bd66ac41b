"""GB300-native CSR SpGEMM (C = A*B, FP64, and FP32) after Liu & Vinter's four-stage framework.

The compute path is the CUDA library libspgemm.so (libspgemm_f32.so for float values;
C ABI in include/spgemm.h);
this package only marshals arguments.  Importing it does not touch the GPU; the
library is loaded on first use and the call fails loudly if it is missing."""
from ._lib import SpgemmError, load as load_library, lib_path  # noqa: F401
from .spgemm import (CSR, BatchPlan, DeviceGraph, DevicePlan, Plan, ReplayGraph, galerkin, galerkin_device,  # noqa: F401
                     make_opts, merge_micro, pool_trim, spgemm, spgemm_batched)

__all__ = ["CSR", "Plan", "BatchPlan", "ReplayGraph", "DevicePlan", "DeviceGraph", "spgemm", "spgemm_batched",
           "galerkin", "galerkin_device", "make_opts", "merge_micro", "pool_trim", "SpgemmError", "load_library",
           "lib_path"]
