"""The Python binding's argument marshalling, on the CPU: its tables agree with the
header's enumerations and constants, every plan option reaches its field of spgemm_opts,
and mixed value types are refused before any call into the library."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header():
    src = open(os.path.join(ROOT, "include", "spgemm.h")).read()
    return re.sub(r"/\*.*?\*/", "", src, flags=re.S)


def _enum(prefix):
    return {m.group(1): int(m.group(2)) for m in re.finditer(rf"\b({prefix}[A-Z0-9_]*)\s*=\s*(\d+)", _header())}


def test_tables_match_the_header():
    from paper_1504_05022_gb300 import _lib
    status = _enum("SPGEMM_(?:OK|ERR_)")
    assert {v: k for k, v in status.items()} == _lib.STATUS
    pol = _enum("SPGEMM_ALLOC_")
    assert {k[len("SPGEMM_ALLOC_"):].lower(): v for k, v in pol.items()} == _lib.POLICY
    lr = _enum("SPGEMM_LONG_ROWS_")
    assert {k[len("SPGEMM_LONG_ROWS_"):].lower(): v for k, v in lr.items()} == _lib.LONG_ROWS
    kinds = _enum("SPGEMM_K_")
    count = kinds.pop("SPGEMM_K_COUNT")
    assert count == len(_lib.KERNELS) == _lib.Stats.launches.size // 4 == _lib.Stats.kernel_ms.size // 4
    assert [k[len("SPGEMM_K_"):].lower() for k, _ in sorted(kinds.items(), key=lambda kv: kv[1])] == _lib.KERNELS
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(SPGEMM_MLP_[A-Z_]+)\s+(\d+)", _header())}
    assert (defs["SPGEMM_MLP_FEATURES"], defs["SPGEMM_MLP_HIDDEN"], defs["SPGEMM_MLP_CLASSES"],
            defs["SPGEMM_MLP_NUM_PARAMS"], defs["SPGEMM_MLP_NUM_TOTAL"]) == (
        _lib.MLP_FEATURES, _lib.MLP_HIDDEN, _lib.MLP_CLASSES, _lib.MLP_NUM_PARAMS, _lib.MLP_NUM_TOTAL)
    mk = _enum("SPGEMM_MERGE_")
    assert mk == {"SPGEMM_MERGE_AUTO": 0, "SPGEMM_MERGE_PATH": 1, "SPGEMM_MERGE_BITMAP": 2}


def test_make_opts_sets_every_field():
    pytest.importorskip("torch")
    from paper_1504_05022_gb300 import _build, _lib
    from paper_1504_05022_gb300.spgemm import make_opts
    _build.build()
    d = make_opts()
    ref = _lib.Opts()
    assert _lib.load().spgemm_opts_init(ctypes.byref(ref)) == 0
    for name, _ in _lib.Opts._fields_:
        if name != "predictor_margin":
            assert getattr(d, name) == getattr(ref, name), name
    o = make_opts(alloc_policy="upper_bound", initial_cap=512, check_inputs=True, record_timing=True,
                  merge_batch=1024, smem_cap_max=4096, heap_block=64, long_rows="level1", predictor=12345,
                  predictor_margin=1.5, wave_mproducts=7, heap_max_u=16, merge_wide_above=2048,
                  merge_kernel="bitmap", merge_miss=8192, dense_min_u=-1, dense_span=10912, dense_span_div=16,
                  dense_pred_min=4096, dense_keep=-1, max_bytes=1 << 40)
    got = {name: getattr(o, name) for name, _ in _lib.Opts._fields_}
    assert got == {"alloc_policy": 1, "initial_cap": 512, "check_inputs": 1, "record_timing": 1,
                   "merge_batch": 1024, "smem_cap_max": 4096, "heap_block": 64, "long_rows": 1,
                   "wave_mproducts": 7, "heap_max_u": 16, "merge_wide_above": 2048, "merge_kernel": 2,
                   "merge_miss": 8192, "dense_min_u": -1, "dense_span": 10912, "dense_span_div": 16,
                   "predictor": 12345, "predictor_margin": 1.5, "dense_pred_min": 4096,
                   "dense_keep": -1, "max_bytes": 1 << 40}

    class _Pred:
        handle = 777
    assert make_opts(alloc_policy="learned", predictor=_Pred()).predictor == 777
    assert make_opts(merge_kernel="merge_path").merge_kernel == 1
    assert make_opts(alloc_policy="precise").alloc_policy == 3
    with pytest.raises(KeyError):
        make_opts(alloc_policy="exact")
    with pytest.raises(KeyError):
        make_opts(long_rows="level2")


def test_value_types_are_checked_before_any_call():
    pytest.importorskip("torch")
    from paper_1504_05022_gb300.spgemm import _value_type

    class _M:
        def __init__(self, vt):
            self.value_type = vt

    class _P:
        def __init__(self, dt):
            self.dtype = dt
    assert _value_type([_M("f64"), _M("f64")], {}) == "f64"
    assert _value_type([_M("f32")], {"predictor": _P("f32")}) == "f32"
    with pytest.raises(TypeError):
        _value_type([_M("f64"), _M("f32")], {})
    with pytest.raises(TypeError):
        _value_type([_M("f32"), _M("f32")], {"predictor": _P("f64")})


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built library the binding raises instead of computing
    anything itself; a nonzero status becomes an exception naming it."""
    from paper_1504_05022_gb300 import _build, _lib
    _build.build()
    with pytest.raises(_lib.SpgemmError, match="SPGEMM_ERR_UNSORTED"):
        _lib.check(3, "probe")
    _lib.check(0, "probe")
    with pytest.raises(ValueError):
        _lib.load(dtype="f16")
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "_libs", {})
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libspgemm.so"))
    monkeypatch.setattr(_build, "LIB_F32", str(tmp_path / "libspgemm_f32.so"))
    with pytest.raises(ImportError, match="not built"):
        _lib.load(build_if_missing=False)
    with pytest.raises(ImportError, match="not built"):
        _lib.load(build_if_missing=False, dtype="f32")
