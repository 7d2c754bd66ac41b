"""CPU oracle for CSR SpGEMM (test infrastructure only).

This package is the independent reference the CUDA library is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does, and the two share no
code.  The C source ``spgemm_oracle.c`` is compiled with gcc (``-O2
-ffp-contract=off -fopenmp``) into ``oracle/_build/liboracle.so`` and loaded with
ctypes.

Functions (each follows a passage of Liu & Vinter's paper):

* :func:`spgemm`         C = A*B by Gustavson's row-wise algorithm (Algorithm 1) with a
                         dense sparse accumulator (Section 2.2); structural zeros kept
                         (Section 3.1); returns also den_ij = sum_k |a_ik b_kj|.
* :func:`spgemm_rows`    the same for a subset of rows (sampled parity at full size).
* :func:`row_counts`     nnz per row only (row pointers checked at full size).
* :func:`upper_bound`    u_i of Algorithm 2.
* :func:`binning`        bins and temporary-row sizes of Algorithm 3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_libs = {}

NUM_BINS = 38


def _path(variant: int) -> str:
    return _LIB_PATH if variant == 0 else os.path.join(_BUILD, f"liboracle_mutant{variant}.so")


def build(force: bool = False, variant: int = 0) -> str:
    """Compile the oracle with gcc (no CUDA involved).  ``variant`` != 0 builds one of the
    deliberately wrong mutants that the oracle's own tests use to show the pins are sensitive."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _path(variant)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", f"-DORACLE_MUTANT={int(variant)}", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


def _load(variant: int = 0):
    with _lock:
        if variant not in _libs:
            lib = ctypes.CDLL(build(variant=variant))
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.oracle_rows_count.argtypes = [I64, P, P, P, P, P, I64, P, ctypes.c_int]
            lib.oracle_rows_count.restype = ctypes.c_int
            lib.oracle_rows_fill.argtypes = [I64, P, P, P, P, P, P, P, I64, P, P, P, P, ctypes.c_int]
            lib.oracle_rows_fill.restype = ctypes.c_int
            lib.oracle_upper_bound.argtypes = [I64, P, P, P, P]
            lib.oracle_upper_bound.restype = None
            lib.oracle_binning.argtypes = [I64, P, P, P, P, P]
            lib.oracle_binning.restype = I64
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _libs[variant] = lib
    return _libs[variant]


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr_arrays(M):
    rp = np.ascontiguousarray(M.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(M.col, dtype=np.int32)
    val = np.ascontiguousarray(M.val, dtype=np.float64)
    return rp, col, val


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def row_counts(A, B, rows: np.ndarray | None = None, nthreads: int = 0, variant: int = 0) -> np.ndarray:
    """nnz of the selected rows of C = A*B (all rows for rows=None): the size pass of
    spgemm_rows alone (Gustavson's structure, Alg. 1), for checking row pointers at full size."""
    lib = _load(variant)
    if A.ncols != B.nrows:
        raise ValueError("shape mismatch")
    arp, acol, _ = _csr_arrays(A)
    brp, bcol, _ = _csr_arrays(B)
    rows_arr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nsel = A.nrows if rows_arr is None else rows_arr.shape[0]
    counts = np.zeros(max(nsel, 1), dtype=np.int64)
    if lib.oracle_rows_count(B.ncols, _p(arp), _p(acol), _p(brp), _p(bcol),
                             _p(rows_arr) if rows_arr is not None else None, nsel, _p(counts), nthreads) != 0:
        raise MemoryError("oracle accumulator allocation failed")
    return counts[:nsel]


def spgemm_rows(A, B, rows: np.ndarray | None, nthreads: int = 0, variant: int = 0):
    """Rows of C = A*B.  ``rows=None`` means all rows.  Returns (offsets, col, val, den):
    offsets has len(rows)+1 entries and delimits each selected row in col/val/den."""
    lib = _load(variant)
    if A.ncols != B.nrows:
        raise ValueError("shape mismatch")
    arp, acol, aval = _csr_arrays(A)
    brp, bcol, bval = _csr_arrays(B)
    if rows is None:
        nsel = A.nrows
        rows_arr = None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nsel = rows_arr.shape[0]
        if nsel and (rows_arr.min() < 0 or rows_arr.max() >= A.nrows):
            raise ValueError("row index out of range")
    counts = np.zeros(max(nsel, 1), dtype=np.int64)
    rptr = _p(rows_arr) if rows_arr is not None else None
    if lib.oracle_rows_count(B.ncols, _p(arp), _p(acol), _p(brp), _p(bcol), rptr, nsel,
                             _p(counts), nthreads) != 0:
        raise MemoryError("oracle accumulator allocation failed")
    off = np.zeros(nsel + 1, dtype=np.int64)
    np.cumsum(counts[:nsel], out=off[1:])
    total = int(off[-1])
    col = np.zeros(max(total, 1), dtype=np.int32)
    val = np.zeros(max(total, 1), dtype=np.float64)
    den = np.zeros(max(total, 1), dtype=np.float64)
    if lib.oracle_rows_fill(B.ncols, _p(arp), _p(acol), _p(aval), _p(brp), _p(bcol), _p(bval),
                            rptr, nsel, _p(off), _p(col), _p(val), _p(den), nthreads) != 0:
        raise MemoryError("oracle accumulator allocation failed")
    return off, col[:total], val[:total], den[:total]


class OracleResult:
    """C = A*B from the oracle: CSR arrays plus the tolerance denominators den_ij."""

    def __init__(self, nrows, ncols, row_ptr, col, val, den):
        self.nrows, self.ncols = nrows, ncols
        self.row_ptr, self.col, self.val, self.den = row_ptr, col, val, den

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def spgemm(A, B, nthreads: int = 0, variant: int = 0) -> OracleResult:
    off, col, val, den = spgemm_rows(A, B, None, nthreads, variant)
    return OracleResult(A.nrows, B.ncols, off, col, val, den)


def upper_bound(A, B) -> np.ndarray:
    """u_i of Algorithm 2 (int64)."""
    lib = _load()
    arp, acol, _ = _csr_arrays(A)
    brp, _, _ = _csr_arrays(B)
    u = np.zeros(max(A.nrows, 1), dtype=np.int64)
    lib.oracle_upper_bound(A.nrows, _p(arp), _p(acol), _p(brp), _p(u))
    return u[:A.nrows]


def binning(u: np.ndarray):
    """Algorithm 3: returns (bin[m] int32, size[m] int64, bin_count[38] int64,
    bin_rows[m] int32, nnz_Ctilde)."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.int64)
    m = u.shape[0]
    b = np.zeros(max(m, 1), dtype=np.int32)
    sz = np.zeros(max(m, 1), dtype=np.int64)
    cnt = np.zeros(NUM_BINS, dtype=np.int64)
    rows = np.zeros(max(m, 1), dtype=np.int32)
    total = lib.oracle_binning(m, _p(u), _p(b), _p(sz), _p(cnt), _p(rows))
    return b[:m], sz[:m], cnt, rows[:m], int(total)
