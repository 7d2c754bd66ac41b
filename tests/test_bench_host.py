"""Host-side logic of bench.py and the autotuner that needs no GPU: the memory comparison
against the precise method, the choice of tuned parameters per value type, and the
algorithmic-byte model of the roofline."""
import json
import os
import sys

import numpy as np

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_memory_comparison_against_the_precise_method():
    A = gen.rmat(8, 4, seed=1)
    inputs = A.nnz * 12 + (A.nrows + 1) * 4          # A*A: the input counted once
    c_bytes = 1000
    mem = bench.memory_comparison([(A, A)], c_bytes, "learned", {"peak_bytes": 5000},
                                  {"hybrid": {"peak_bytes": 9000}})
    assert mem["precise"] == inputs + c_bytes
    assert mem["learned"] == inputs + 5000 and mem["hybrid"] == inputs + 9000
    assert mem["ratio_to_precise"]["hybrid"] == (inputs + 9000) / (inputs + c_bytes)
    B = gen.erdos_renyi(A.ncols, 3, seed=2, ncols=50)
    mem2 = bench.memory_comparison([(A, B)], c_bytes, "learned", {"peak_bytes": 0}, {})
    assert mem2["precise"] == inputs + B.nnz * 12 + (B.nrows + 1) * 4 + c_bytes


def test_algorithmic_bytes_model():
    """A entries 28 B (col + value + the B row_ptr pair), products 12 B, outputs 12 B."""
    A = gen.lap2d(8)
    blen = np.diff(A.row_ptr)
    u = np.array([blen[A.col[A.row_ptr[i]:A.row_ptr[i + 1]]].sum() for i in range(A.nrows)])
    rows = np.array([0, 5, 9])
    rn = np.arange(A.nrows) % 7
    got = bench.algorithmic_bytes(A, A, u, rows, rn)
    want = sum(int(blen[i]) * 28 + int(u[i]) * 12 + int(rn[i]) * 12 for i in rows)
    assert got == want


def test_single_precision_tuned_entries(tmp_path, monkeypatch):
    from paper_1504_05022_gb300 import autotune
    f = tmp_path / "tuned.json"
    f.write_text(json.dumps({"w": {"learned": {"params": {"heap_max_u": 16}}},
                             "w:f32": {"learned": {"params": {"dense_span": 16384}}}}))
    monkeypatch.setattr(autotune, "TUNED", str(f))
    assert autotune.load("w", "learned") == {"heap_max_u": 16}
    assert autotune.load("w:f32", "learned") == {"dense_span": 16384}
    assert autotune.load("x:f32", "learned") is None
    opts = autotune.apply({"alloc_policy": "learned"}, {"dense_span": 16384, "dense_span_div": 0})
    assert opts == {"alloc_policy": "learned", "dense_span": 16384, "dense_span_div": 0}
