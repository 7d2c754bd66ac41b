"""ctypes mirror of include/spgemm.h (argument marshalling only).

Loads paper_1504_05022_gb300/_build/libspgemm.so (double values) or libspgemm_f32.so
(float values, the same entry points).  If a library is missing the call fails loudly:
there is no CPU fallback."""
from __future__ import annotations

import ctypes
import os

from . import _build

c_i32, c_i64, c_ptr, c_f64, c_f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_float

STATUS = {
    0: "SPGEMM_OK", 1: "SPGEMM_ERR_INVALID_ARG", 2: "SPGEMM_ERR_SHAPE", 3: "SPGEMM_ERR_UNSORTED",
    4: "SPGEMM_ERR_OOM", 5: "SPGEMM_ERR_CUDA", 6: "SPGEMM_ERR_TIMEOUT", 7: "SPGEMM_ERR_INTERNAL",
}
POLICY = {"hybrid": 0, "upper_bound": 1, "learned": 2, "precise": 3}
LONG_ROWS = {"split": 0, "level1": 1}
KERNELS = ["bound", "bin", "heap", "esc", "merge", "scan", "arrange", "other"]
NUM_BINS = 38


class CsrIn(ctypes.Structure):
    _fields_ = [("nrows", c_i64), ("ncols", c_i64), ("nnz", c_i64), ("row_ptr", c_ptr),
                ("rowptr_bits", c_i32), ("col_idx", c_ptr), ("val", c_ptr)]


class CsrOut(ctypes.Structure):
    _fields_ = [("nrows", c_i64), ("ncols", c_i64), ("nnz", c_i64), ("row_ptr", c_ptr),
                ("col_idx", c_ptr), ("val", c_ptr)]


class Opts(ctypes.Structure):
    _fields_ = [("alloc_policy", c_i32), ("initial_cap", c_i32), ("check_inputs", c_i32),
                ("record_timing", c_i32), ("merge_batch", c_i32), ("smem_cap_max", c_i32),
                ("heap_block", c_i32), ("long_rows", c_i32), ("wave_mproducts", c_i32), ("heap_max_u", c_i32),
                ("merge_wide_above", c_i32), ("merge_kernel", c_i32), ("merge_miss", c_i32),
                ("dense_min_u", c_i32), ("dense_span", c_i32), ("dense_span_div", c_i32),
                ("predictor", c_ptr),
                ("predictor_margin", c_f64), ("dense_pred_min", c_i32), ("dense_keep", c_i32),
                ("max_bytes", c_i64)]


class Stats(ctypes.Structure):
    _fields_ = [("bin_count", c_i64 * NUM_BINS), ("sum_u", c_i64), ("nnz_ctilde", c_i64), ("nnz_c", c_i64),
                ("merge_rounds", c_i64), ("rows_relaunched", c_i64), ("rows_level1", c_i64), ("rows_split", c_i64),
                ("rows_fallback", c_i64), ("bytes_ctilde", c_i64), ("peak_bytes", c_i64),
                ("launches", c_i32 * 8), ("kernel_ms", c_f32 * 8), ("held_bytes", c_i64), ("rows_dense", c_i64),
                ("dense_slices", c_i64), ("item_rounds", c_i64), ("alloc_host_ms", c_f64), ("allocs", c_i64)]


class PlanArrays(ctypes.Structure):
    _fields_ = [("nrows", c_i64), ("u", c_ptr), ("bin", c_ptr), ("bin_rows", c_ptr), ("bin_start", c_ptr),
                ("ctilde_row_ptr", c_ptr), ("row_nnz", c_ptr)]


# Every function declared in include/spgemm.h, with its ctypes signature.
SIGNATURES = {
    "spgemm_opts_init": ([ctypes.POINTER(Opts)], c_i32),
    "spgemm_symbolic": ([ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(Opts), c_ptr,
                         ctypes.POINTER(c_ptr), ctypes.POINTER(c_i64)], c_i32),
    "spgemm_numeric": ([c_ptr, ctypes.POINTER(CsrOut)], c_i32),
    "spgemm_free": ([c_ptr], c_i32),
    "spgemm_pool_trim": ([c_i32, c_i64], c_i32),
    "spgemm_check_status": ([ctypes.POINTER(c_i64), c_i32], c_i32),
    "spgemm_status_string": ([c_i32], ctypes.c_char_p),
    "spgemm_plan_stats": ([c_ptr, ctypes.POINTER(Stats)], c_i32),
    "spgemm_plan_arrays_get": ([c_ptr, ctypes.POINTER(PlanArrays)], c_i32),
    "spgemm_rowptr_scan_noalloc": ([c_ptr, c_i64, c_ptr, c_ptr], c_i32),
    "spgemm_rowptr_scan_noalloc_max_rows": ([], c_i64),
    "spgemm_batched_waves": ([c_ptr, ctypes.POINTER(c_i64)], c_i32),
    "spgemm_batched_wave": ([c_ptr, c_i64, ctypes.POINTER(c_ptr), ctypes.POINTER(c_i64)], c_i32),
    "spgemm_batched_wave_pairs": ([c_ptr, ctypes.POINTER(c_i64)], c_i32),
    "spgemm_batched_symbolic": ([c_i64, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(Opts), c_ptr,
                                 ctypes.POINTER(c_ptr), ctypes.POINTER(c_i64)], c_i32),
    "spgemm_batched_numeric": ([c_ptr, ctypes.POINTER(CsrOut)], c_i32),
    "spgemm_numeric_replay": ([c_ptr], c_i32),
    "spgemm_plan_check": ([c_ptr], c_i32),
    "spgemm_graph_create": ([ctypes.POINTER(c_ptr), c_i64, ctypes.POINTER(c_ptr)], c_i32),
    "spgemm_graph_launch": ([c_ptr], c_i32),
    "spgemm_graph_free": ([c_ptr], c_i32),
    "spgemm_galerkin": ([ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(Opts),
                         c_ptr, ctypes.POINTER(c_ptr), ctypes.POINTER(c_ptr), ctypes.POINTER(CsrOut)], c_i32),
    "spgemm_dplan_create": ([ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), c_i64, ctypes.POINTER(Opts), c_ptr,
                             ctypes.POINTER(c_ptr), ctypes.POINTER(CsrOut)], c_i32),
    "spgemm_dplan_batched_create": ([c_i64, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), c_i64, ctypes.POINTER(Opts),
                                     c_ptr, ctypes.POINTER(c_ptr), ctypes.POINTER(CsrOut)], c_i32),
    "spgemm_dplan_run": ([c_ptr], c_i32),
    "spgemm_dplan_result": ([c_ptr, ctypes.POINTER(CsrOut)], c_i32),
    "spgemm_dplan_graph_create": ([ctypes.POINTER(c_ptr), c_i64, ctypes.POINTER(c_ptr)], c_i32),
    "spgemm_dplan_free": ([c_ptr], c_i32),
    "spgemm_dplan_bytes": ([c_ptr, ctypes.POINTER(c_i64)], c_i32),
    "spgemm_merge_micro": ([c_i32, c_i32, c_i32, c_ptr, c_ptr, c_i64, c_i32, c_ptr, c_ptr, c_ptr], c_i32),
    "spgemm_predictor_create": ([c_ptr, c_i64, ctypes.POINTER(c_ptr)], c_i32),
    "spgemm_predictor_free": ([c_ptr], c_i32),
    "spgemm_row_features": ([ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), c_ptr, c_ptr], c_i32),
    "spgemm_mlp_forward": ([c_ptr, c_ptr, c_i64, c_ptr, c_ptr], c_i32),
    "spgemm_mlp_work_floats": ([c_i64], c_i64),
    "spgemm_mlp_loss_grad": ([c_ptr, c_ptr, c_ptr, c_ptr, c_i64, c_ptr, c_ptr, c_ptr, c_ptr], c_i32),
    "spgemm_mlp_adam": ([c_ptr, c_ptr, c_ptr, c_ptr, c_i64, ctypes.c_float, ctypes.c_float, c_ptr], c_i32),
}

MLP_FEATURES, MLP_HIDDEN, MLP_CLASSES, MLP_NUM_PARAMS, MLP_NUM_TOTAL = 8, 32, 16, 1905, 1921

_lib = None          # the double-precision library, once loaded
_libs = {}           # value type ("f64", "f32") -> loaded library
VALUE_TYPES = ("f64", "f32")


def checked() -> bool:
    """SPGEMM_CHECKED=1 selects the bounds-checked build for double precision."""
    return os.environ.get("SPGEMM_CHECKED") == "1"


def lib_path(dtype: str = "f64") -> str:
    if dtype == "f32":
        return _build.LIB_F32
    return _build.LIB_CHECK if checked() else _build.LIB


def load(build_if_missing: bool = True, dtype: str = "f64"):
    """Returns the loaded library for the value type ("f64": libspgemm.so, "f32":
    libspgemm_f32.so).  Builds the libraries first when missing and a compiler exists."""
    global _lib
    if dtype not in VALUE_TYPES:
        raise ValueError(f"value type must be one of {VALUE_TYPES}")
    if dtype == "f64" and _lib is not None:
        return _lib
    if dtype in _libs:
        return _libs[dtype]
    path = lib_path(dtype)
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{os.path.basename(path)} not built ({path}); run __graft_entry__.build()")
        if dtype == "f64" and checked():
            _build.build_check()
        else:
            _build.build()
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _libs[dtype] = lib
    if dtype == "f64":
        _lib = lib
    return lib


class SpgemmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().spgemm_status_string(code).decode()
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")


def check(code: int, where: str) -> None:
    if code != 0:
        raise SpgemmError(code, where)
