"""Python binding of the C ABI: device CSR matrices as torch tensors, and
C = A*B through spgemm_symbolic / spgemm_numeric / spgemm_free.

torch is used only for device memory, streams and as the tensor container; every
step of the product runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


@dataclass
class CSR:
    """A CSR matrix whose arrays are torch tensors on one CUDA device.

    row_ptr: int32 or int64 (nrows+1), col: int32 (nnz), val: float64 or float32 (nnz; the
    product runs in the values' precision); columns of a row strictly ascending."""

    row_ptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor
    shape: tuple

    @property
    def nrows(self) -> int:
        return int(self.shape[0])

    @property
    def ncols(self) -> int:
        return int(self.shape[1])

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def value_type(self) -> str:
        """"f64" or "f32": which library (double or single precision) computes with it."""
        return {torch.float64: "f64", torch.float32: "f32"}[self.val.dtype]

    @classmethod
    def from_host(cls, M, device="cuda", rowptr_dtype=torch.int64, pin: bool = False,
                  dtype: torch.dtype = torch.float64) -> "CSR":
        """Copies a host CSR (anything with row_ptr/col/val numpy arrays and nrows/ncols);
        values are stored as `dtype` (float64 or float32)."""
        rp = torch.from_numpy(np.ascontiguousarray(M.row_ptr)).to(rowptr_dtype)
        col = torch.from_numpy(np.ascontiguousarray(M.col, dtype=np.int32))
        npdt = {torch.float64: np.float64, torch.float32: np.float32}[dtype]
        val = torch.from_numpy(np.ascontiguousarray(M.val, dtype=npdt))
        if pin:
            rp, col, val = rp.pin_memory(), col.pin_memory(), val.pin_memory()
        return cls(rp.to(device, non_blocking=pin), col.to(device, non_blocking=pin),
                   val.to(device, non_blocking=pin), (int(M.nrows), int(M.ncols)))

    def to_host(self):
        """(row_ptr int64, col int32, val float64 or float32) numpy arrays."""
        return (self.row_ptr.to("cpu", torch.int64).numpy(), self.col.cpu().numpy(), self.val.cpu().numpy())

    def _c_in(self) -> _lib.CsrIn:
        for t in (self.row_ptr, self.col, self.val):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("CSR arrays must be contiguous CUDA tensors")
        if self.col.dtype != torch.int32 or self.val.dtype not in (torch.float64, torch.float32):
            raise TypeError("col must be int32 and val float64 or float32")
        if self.row_ptr.dtype not in (torch.int32, torch.int64):
            raise TypeError("row_ptr must be int32 or int64")
        if self.row_ptr.numel() != self.nrows + 1 or self.val.numel() != self.col.numel():
            raise ValueError("inconsistent CSR array sizes")
        return _lib.CsrIn(self.nrows, self.ncols, self.nnz, self.row_ptr.data_ptr(),
                          32 if self.row_ptr.dtype == torch.int32 else 64,
                          self.col.data_ptr() if self.nnz else None,
                          self.val.data_ptr() if self.nnz else None)


class _PlanHandle:
    """Owns an spgemm_plan*; freed (stream-ordered) when the last reference goes."""

    def __init__(self, ptr: int, stream: torch.cuda.Stream, L):
        self.ptr = ptr
        self.stream = stream
        self.L = L  # the library (value type) that made the plan

    def free(self):
        if self.ptr:
            self.L.spgemm_free(ctypes.c_void_p(self.ptr))
            self.ptr = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _PlanArray:
    """Exposes one plan-owned device array through __cuda_array_interface__ and keeps the
    plan alive while a tensor views it."""

    def __init__(self, ptr: int, n: int, typestr: str, owner: _PlanHandle, device: int):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": None}
        self._device = device


def _wrap(ptr: int, n: int, dtype: torch.dtype, owner: _PlanHandle, device: int) -> torch.Tensor:
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.float64: "<f8", torch.float32: "<f4"}[dtype]
    if n == 0:
        return torch.empty(0, dtype=dtype, device=f"cuda:{device}")
    return torch.as_tensor(_PlanArray(ptr, n, typestr, owner, device), device=f"cuda:{device}")


def _wrap_u8(ptr: int, n: int, owner: _PlanHandle, device: int) -> torch.Tensor:
    if n == 0:
        return torch.empty(0, dtype=torch.uint8, device=f"cuda:{device}")
    return torch.as_tensor(_PlanArray(ptr, n, "|u1", owner, device), device=f"cuda:{device}")


def make_opts(alloc_policy: str = "hybrid", initial_cap: int = 256, check_inputs: bool = False,
              record_timing: bool = False, merge_batch: int = 0, smem_cap_max: int = 0,
              heap_block: int = 0, long_rows: str = "split", predictor=None,
              predictor_margin: float = 1.0, wave_mproducts: int = 0, heap_max_u: int = 0,
              merge_wide_above: int = 0, merge_kernel: str = "auto", merge_miss: int = 0,
              dense_min_u: int = 0, dense_span: int = 0, dense_span_div: int = 0,
              dense_pred_min: int = 0, dense_keep: int = 0, max_bytes: int = 0) -> _lib.Opts:
    L = _lib.load()
    o = _lib.Opts()
    _lib.check(L.spgemm_opts_init(ctypes.byref(o)), "spgemm_opts_init")
    o.alloc_policy = _lib.POLICY[alloc_policy]
    o.initial_cap = int(initial_cap)
    o.check_inputs = int(bool(check_inputs))
    o.record_timing = int(bool(record_timing))
    o.merge_batch = int(merge_batch)
    o.smem_cap_max = int(smem_cap_max)
    o.heap_block = int(heap_block)
    o.long_rows = _lib.LONG_ROWS[long_rows]
    o.wave_mproducts = int(wave_mproducts)
    o.heap_max_u = int(heap_max_u)
    o.merge_wide_above = int(merge_wide_above)
    o.merge_kernel = {"auto": 0, "merge_path": 1, "bitmap": 2}[merge_kernel]
    o.merge_miss = int(merge_miss)
    o.dense_min_u = int(dense_min_u)
    o.dense_span = int(dense_span)
    o.dense_span_div = int(dense_span_div)
    o.dense_pred_min = int(dense_pred_min)
    o.dense_keep = int(dense_keep)
    o.max_bytes = int(max_bytes)
    # a Predictor object (whose device weights the caller keeps alive) or a raw handle
    o.predictor = getattr(predictor, "handle", predictor)
    o.predictor_margin = float(predictor_margin)
    return o


def _value_type(mats, opts) -> str:
    """The value type shared by the matrices (and the predictor, if any)."""
    vts = {m.value_type for m in mats}
    if len(vts) != 1:
        raise TypeError("A and B must have the same value type (float64 or float32)")
    vt = vts.pop()
    pred = opts.get("predictor")
    if pred is not None and getattr(pred, "dtype", vt) != vt:
        raise TypeError(f"the predictor was made for {pred.dtype} values, the matrices hold {vt}")
    return vt


class Plan:
    """C = A*B split into the symbolic part (stages 1-2) and the numeric part (stages 3-4).
    The precision of the matrices' values (float64 or float32) selects the library."""

    def __init__(self, A: CSR, B: CSR, stream: torch.cuda.Stream | None = None, **opts):
        vt = _value_type([A, B], opts)
        L = self.L = _lib.load(dtype=vt)
        self.A, self.B = A, B  # keep inputs alive until numeric work completes
        self.device = A.val.device.index if A.val.is_cuda else torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.opts = make_opts(**opts)
        self._predictor = opts.get("predictor")  # the weights are read on the stream during symbolic
        a_in, b_in = A._c_in(), B._c_in()
        plan = ctypes.c_void_p()
        ub = ctypes.c_int64()
        with torch.cuda.device(self.device):
            _lib.check(L.spgemm_symbolic(ctypes.byref(a_in), ctypes.byref(b_in), ctypes.byref(self.opts),
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(plan),
                                         ctypes.byref(ub)), "spgemm_symbolic")
        self.handle = _PlanHandle(plan.value, self.stream, L)
        self.upper_bound_nnz = int(ub.value)
        self._C = None

    def numeric(self) -> CSR:
        if self._C is not None:
            return self._C
        L = self.L
        out = _lib.CsrOut()
        with torch.cuda.device(self.device):
            _lib.check(L.spgemm_numeric(ctypes.c_void_p(self.handle.ptr), ctypes.byref(out)), "spgemm_numeric")
        h = self.handle
        rp = _wrap(out.row_ptr, out.nrows + 1, torch.int64, h, self.device)
        col = _wrap(out.col_idx, out.nnz, torch.int32, h, self.device)
        val = _wrap(out.val, out.nnz, self.A.val.dtype, h, self.device)
        self._C = CSR(rp, col, val, (int(out.nrows), int(out.ncols)))
        return self._C

    def stats(self) -> dict:
        L = self.L
        s = _lib.Stats()
        _lib.check(L.spgemm_plan_stats(ctypes.c_void_p(self.handle.ptr), ctypes.byref(s)), "spgemm_plan_stats")
        return {
            "bin_count": list(s.bin_count), "sum_u": s.sum_u, "nnz_ctilde": s.nnz_ctilde, "nnz_c": s.nnz_c,
            "merge_rounds": s.merge_rounds, "rows_relaunched": s.rows_relaunched, "rows_level1": s.rows_level1,
            "rows_split": s.rows_split,
            "rows_fallback": s.rows_fallback, "bytes_ctilde": s.bytes_ctilde, "peak_bytes": s.peak_bytes, "held_bytes": s.held_bytes,
            "rows_dense": s.rows_dense, "dense_slices": s.dense_slices, "item_rounds": s.item_rounds,
            "alloc_host_ms": s.alloc_host_ms, "allocs": s.allocs,
            "launches": dict(zip(_lib.KERNELS, list(s.launches))),
            "kernel_ms": dict(zip(_lib.KERNELS, [float(x) for x in s.kernel_ms])),
        }

    def arrays(self) -> dict:
        """Copies of the plan's intermediate arrays to host numpy (for inspection and tests):
        u, bin, bin_rows, bin_start, ctilde_row_ptr, row_nnz."""
        return self._arrays_of(self.handle.ptr)

    def _arrays_of(self, ptr: int) -> dict:
        L = self.L
        a = _lib.PlanArrays()
        _lib.check(L.spgemm_plan_arrays_get(ctypes.c_void_p(ptr), ctypes.byref(a)), "spgemm_plan_arrays_get")
        self.stream.synchronize()
        m = int(a.nrows)
        h = self.handle
        out = {
            "u": _wrap(a.u, m, torch.int64, h, self.device).cpu().numpy(),
            "bin": _wrap_u8(a.bin, m, h, self.device).cpu().numpy(),
            "bin_rows": _wrap(a.bin_rows, m, torch.int32, h, self.device).cpu().numpy(),
            "bin_start": np.ctypeslib.as_array(ctypes.cast(a.bin_start, ctypes.POINTER(ctypes.c_int64)),
                                               shape=(39,)).copy(),
            "ctilde_row_ptr": _wrap(a.ctilde_row_ptr, m + 1, torch.int64, h, self.device).cpu().numpy(),
            "row_nnz": _wrap(a.row_nnz, m, torch.int32, h, self.device).cpu().numpy(),
        }
        return out

    def replay(self) -> None:
        """Recomputes C's values in place for new values of A and B with the same structure
        (no allocation, no host synchronisation after the first call)."""
        with torch.cuda.device(self.device):
            _lib.check(self.L.spgemm_numeric_replay(ctypes.c_void_p(self.handle.ptr)), "spgemm_numeric_replay")

    def check(self) -> None:
        """Raises if a device-side consistency check failed (e.g. a replay with changed structure)."""
        _lib.check(self.L.spgemm_plan_check(ctypes.c_void_p(self.handle.ptr)), "spgemm_plan_check")

    def free(self) -> None:
        """Releases the plan now; tensors of C obtained from numeric() become invalid."""
        self._C = None
        self.handle.free()


def spgemm(A: CSR, B: CSR, stream: torch.cuda.Stream | None = None, **opts) -> CSR:
    """C = A*B on the GPU (four-stage framework).  The returned tensors keep the plan alive."""
    if A.ncols != B.nrows:
        raise ValueError(f"shape mismatch: {A.shape} x {B.shape}")
    return Plan(A, B, stream=stream, **opts).numeric()


class BatchPlan(Plan):
    """Many independent C_i = A_i * B_i in one pipeline (block-diagonal concatenation)."""

    def __init__(self, As, Bs, stream: torch.cuda.Stream | None = None, **opts):  # noqa: D401
        if len(As) != len(Bs) or not As:
            raise ValueError("need as many A as B matrices, at least one")
        L = self.L = _lib.load(dtype=_value_type(list(As) + list(Bs), opts))
        self.As, self.Bs = list(As), list(Bs)
        self.A, self.B = self.As[0], self.Bs[0]
        self.device = As[0].val.device.index
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.opts = make_opts(**opts)
        self._predictor = opts.get("predictor")
        n = len(As)
        ain = (_lib.CsrIn * n)(*[a._c_in() for a in As])
        bin_ = (_lib.CsrIn * n)(*[b._c_in() for b in Bs])
        plan = ctypes.c_void_p()
        ub = ctypes.c_int64()
        with torch.cuda.device(self.device):
            _lib.check(L.spgemm_batched_symbolic(n, ain, bin_, ctypes.byref(self.opts),
                                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(plan),
                                                 ctypes.byref(ub)), "spgemm_batched_symbolic")
        self.handle = _PlanHandle(plan.value, self.stream, L)
        self.upper_bound_nnz = int(ub.value)
        self._C = None
        self._Cs = None

    def numeric(self):
        if self._Cs is not None:
            return self._Cs
        L = self.L
        n = len(self.As)
        outs = (_lib.CsrOut * n)()
        with torch.cuda.device(self.device):
            _lib.check(L.spgemm_batched_numeric(ctypes.c_void_p(self.handle.ptr), outs), "spgemm_batched_numeric")
        h = self.handle
        self._Cs = [CSR(_wrap(o.row_ptr, o.nrows + 1, torch.int64, h, self.device),
                        _wrap(o.col_idx, o.nnz, torch.int32, h, self.device),
                        _wrap(o.val, o.nnz, self.A.val.dtype, h, self.device), (int(o.nrows), int(o.ncols)))
                    for o in outs]
        return self._Cs


    @property
    def n_waves(self) -> int:
        n = ctypes.c_int64()
        _lib.check(self.L.spgemm_batched_waves(ctypes.c_void_p(self.handle.ptr), ctypes.byref(n)),
                   "spgemm_batched_waves")
        return int(n.value)

    def pair_order(self) -> np.ndarray:
        """Pairs in the order the waves compute them (largest product count first)."""
        order = np.zeros(len(self.As), dtype=np.int64)
        _lib.check(self.L.spgemm_batched_wave_pairs(ctypes.c_void_p(self.handle.ptr),
                                                         order.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
                   "spgemm_batched_wave_pairs")
        return order

    def arrays(self) -> dict:
        """As Plan.arrays, for the rows of all pairs concatenated in pair_order(); with several
        waves only u, bin and row_nnz (the per-wave bin_rows, bin_start and ctilde_row_ptr are
        not merged)."""
        nw = self.n_waves
        if nw == 1:
            return super().arrays()
        L = self.L
        parts = []
        for i in range(nw):
            sub = ctypes.c_void_p()
            first = ctypes.c_int64()
            _lib.check(L.spgemm_batched_wave(ctypes.c_void_p(self.handle.ptr), i, ctypes.byref(sub),
                                             ctypes.byref(first)), "spgemm_batched_wave")
            parts.append(self._arrays_of(sub.value))
        return {k: np.concatenate([p[k] for p in parts]) for k in ("u", "bin", "row_nnz")}


def pool_trim(device: int = 0, keep_bytes: int = 0) -> None:
    """Returns the device memory that the libraries' pools (double and single precision) keep
    for reuse on `device` to the system, down to keep_bytes each (synchronises the device
    first)."""
    torch.cuda.synchronize(device)
    for dt in ("f64", "f32"):
        _lib.check(_lib.load(dtype=dt).spgemm_pool_trim(int(device), int(keep_bytes)), "spgemm_pool_trim")


def spgemm_batched(As, Bs, stream=None, **opts):
    """[A_i * B_i] for all pairs, computed as one block-diagonal product."""
    return BatchPlan(As, Bs, stream=stream, **opts).numeric()


class ReplayGraph:
    """CUDA graph of values-only replays of several plans sharing one stream (for instance both
    products of a Galerkin chain); launch() recomputes all their results for new input values."""

    def __init__(self, plans):
        self.plans = list(plans)
        if len({p.L._name for p in self.plans}) != 1:
            raise ValueError("the plans of one graph must share a value type")
        L = self.L = self.plans[0].L
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.ptr for p in self.plans])
        g = ctypes.c_void_p()
        with torch.cuda.device(self.plans[0].device):
            _lib.check(L.spgemm_graph_create(arr, len(self.plans), ctypes.byref(g)), "spgemm_graph_create")
        self.handle = g.value

    def launch(self) -> None:
        _lib.check(self.L.spgemm_graph_launch(ctypes.c_void_p(self.handle)), "spgemm_graph_launch")

    def __del__(self):
        try:
            if self.handle:
                self.L.spgemm_graph_free(ctypes.c_void_p(self.handle))
                self.handle = None
        except Exception:
            pass


def galerkin(R: CSR, A: CSR, P: CSR, stream: torch.cuda.Stream | None = None, **opts):
    """Ac = R * (A * P) with two plans on one stream; returns (Ac, plan_ap, plan_rap)."""
    stream = stream if stream is not None else torch.cuda.current_stream()
    p1 = Plan(A, P, stream=stream, **opts)
    AP = p1.numeric()
    p2 = Plan(R, AP, stream=stream, **opts)
    Ac = p2.numeric()
    p2._keep = p1
    return Ac, p1, p2


class _DPlanHandle(_PlanHandle):
    """Owns an spgemm_dplan*."""

    def free(self):
        if self.ptr:
            self.L.spgemm_dplan_free(ctypes.c_void_p(self.ptr))
            self.ptr = 0


class DevicePlan:
    """C = A*B (or a batch of C_i = A_i*B_i) with every size kept on the device: the precise
    method (count, then compute every row straight into C) with persistent per-bin kernels.
    run() enqueues the whole product -- stages 1-4 -- without allocating or synchronising, so
    it can run again on new contents of the same input arrays (structure included) and be
    captured in a CUDA graph (DeviceGraph).  C has room for `capacity` entries; result()
    synchronises, reads nnz(C) and returns C (a list of C_i for a batch), raising
    SpgemmError(SPGEMM_ERR_OOM) if the product outgrew the capacity."""

    def __init__(self, A, B, capacity: int, stream: torch.cuda.Stream | None = None, **opts):
        batched = isinstance(A, (list, tuple))
        mats = (list(A) + list(B)) if batched else [A, B]
        L = self.L = _lib.load(dtype=_value_type(mats, opts))
        self.inputs = mats  # borrowed by every run
        first = mats[0]
        self.device = first.val.device.index
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.opts = make_opts(**{k: v for k, v in opts.items() if k != "alloc_policy"})
        self.capacity = int(capacity)
        self.dtype = first.val.dtype
        plan = ctypes.c_void_p()
        c = _lib.CsrOut()
        with torch.cuda.device(self.device):
            if batched:
                n = len(A)
                ain = (_lib.CsrIn * n)(*[a._c_in() for a in A])
                bin_ = (_lib.CsrIn * n)(*[b._c_in() for b in B])
                rc = L.spgemm_dplan_batched_create(n, ain, bin_, self.capacity, ctypes.byref(self.opts),
                                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(plan),
                                                   ctypes.byref(c))
            else:
                a_in, b_in = A._c_in(), B._c_in()
                rc = L.spgemm_dplan_create(ctypes.byref(a_in), ctypes.byref(b_in), self.capacity,
                                           ctypes.byref(self.opts), ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.byref(plan), ctypes.byref(c))
            _lib.check(rc, "spgemm_dplan_create")
        self.handle = _DPlanHandle(plan.value, self.stream, L)
        self.npairs = len(A) if batched else 0
        self.shape = (int(c.nrows), int(c.ncols))
        h = self.handle
        self._rp = _wrap(c.row_ptr, c.nrows + 1, torch.int64, h, self.device)
        self._col = _wrap(c.col_idx, self.capacity, torch.int32, h, self.device)
        self._val = _wrap(c.val, self.capacity, self.dtype, h, self.device)

    def run(self) -> None:
        with torch.cuda.device(self.device):
            _lib.check(self.L.spgemm_dplan_run(ctypes.c_void_p(self.handle.ptr)), "spgemm_dplan_run")

    def as_input(self) -> CSR:
        """C's arrays as the input of a later plan on the same stream (its entries beyond nnz(C)
        are never read): chains two products on the device."""
        return CSR(self._rp, self._col, self._val, self.shape)

    def result(self):
        n = max(1, self.npairs)
        outs = (_lib.CsrOut * n)()
        _lib.check(self.L.spgemm_dplan_result(ctypes.c_void_p(self.handle.ptr), outs), "spgemm_dplan_result")
        h = self.handle
        cs = [CSR(_wrap(o.row_ptr, o.nrows + 1, torch.int64, h, self.device),
                  _wrap(o.col_idx, o.nnz, torch.int32, h, self.device),
                  _wrap(o.val, o.nnz, self.dtype, h, self.device), (int(o.nrows), int(o.ncols))) for o in outs]
        return cs if self.npairs else cs[0]

    @property
    def held_bytes(self) -> int:
        b = ctypes.c_int64()
        _lib.check(self.L.spgemm_dplan_bytes(ctypes.c_void_p(self.handle.ptr), ctypes.byref(b)), "spgemm_dplan_bytes")
        return int(b.value)


class DeviceGraph:
    """One CUDA graph holding a full run (stages 1-4, every size on the device) of each of
    several DevicePlans sharing one created stream, in order -- a whole batch, or both products
    of a Galerkin chain R*(A*P).  launch() recomputes everything from the inputs' current
    contents."""

    def __init__(self, plans):
        self.plans = list(plans)
        L = self.L = self.plans[0].L
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.ptr for p in self.plans])
        g = ctypes.c_void_p()
        with torch.cuda.device(self.plans[0].device):
            _lib.check(L.spgemm_dplan_graph_create(arr, len(self.plans), ctypes.byref(g)), "spgemm_dplan_graph_create")
        self.handle = g.value

    def launch(self) -> None:
        _lib.check(self.L.spgemm_graph_launch(ctypes.c_void_p(self.handle)), "spgemm_graph_launch")

    def __del__(self):
        try:
            if self.handle:
                self.L.spgemm_graph_free(ctypes.c_void_p(self.handle))
                self.handle = None
        except Exception:
            pass


def galerkin_device(R: CSR, A: CSR, P: CSR, cap_ap: int, cap_ac: int, stream: torch.cuda.Stream, **opts):
    """Ac = R*(A*P) as two DevicePlans chained on `stream` and one CUDA graph of both:
    returns (plan_ap, plan_rap, graph); graph.launch() recomputes the chain from the current
    contents of R, A and P, and plan_rap.result() is Ac."""
    p1 = DevicePlan(A, P, cap_ap, stream=stream, **opts)
    p2 = DevicePlan(R, p1.as_input(), cap_ac, stream=stream, **opts)
    p2._keep = p1
    return p1, p2, DeviceGraph([p1, p2])


MERGE_METHODS = {"ranking": 0, "merge_path": 1, "bitonic": 2}


def merge_micro(keys: torch.Tensor, l: int, method: str = "merge_path", threads: int = 256,
                vals: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None):
    """The merge evaluation of Section 4.2: every group of 2l int32 keys holds two ascending
    runs of length l, and is merged into one ascending sequence by one CTA of `threads`
    threads with the ranking merge, merge path or bitonic merge.  vals (4- or 8-byte
    elements, optional) move with their keys.  Returns (keys, vals or None)."""
    if keys.dtype != torch.int32 or not keys.is_cuda or not keys.is_contiguous():
        raise TypeError("keys must be a contiguous int32 CUDA tensor")
    vb = 0 if vals is None else vals.element_size()
    if vals is not None and (not vals.is_cuda or not vals.is_contiguous() or vals.numel() != keys.numel()):
        raise ValueError("vals must be a contiguous CUDA tensor of keys' length")
    out_k = torch.empty_like(keys)
    out_v = None if vals is None else torch.empty_like(vals)
    stream = stream if stream is not None else torch.cuda.current_stream(keys.device)
    with torch.cuda.device(keys.device):
        _lib.check(_lib.load().spgemm_merge_micro(
            MERGE_METHODS[method], int(threads), vb, ctypes.c_void_p(keys.data_ptr()),
            ctypes.c_void_p(vals.data_ptr() if vals is not None else 0), keys.numel(), int(l),
            ctypes.c_void_p(out_k.data_ptr()), ctypes.c_void_p(out_v.data_ptr() if out_v is not None else 0),
            ctypes.c_void_p(stream.cuda_stream)), "spgemm_merge_micro")
    return out_k, out_v
