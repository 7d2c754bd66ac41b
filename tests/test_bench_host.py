"""Host-side logic of bench.py and the autotuner that needs no GPU: the memory comparison
against the precise method, the choice of tuned parameters per value type, the
algorithmic-byte model and the roofline object built from a measurement, the rule that
profiled DRAM traffic is dropped once its kernels' sources change, and the tuner's
coordinate descent with its memory slack."""
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
    assert mem["inputs_plus_C"] == inputs + c_bytes and "precise" not in mem
    assert mem["learned"] == inputs + 5000 and mem["hybrid"] == inputs + 9000
    assert mem["ratio_to_precise"]["hybrid"] == (inputs + 9000) / (inputs + c_bytes)
    # the measured precise policy, when it ran, is the denominator
    mem1 = bench.memory_comparison([(A, A)], c_bytes, "learned", {"peak_bytes": 5000},
                                   {"hybrid": {"peak_bytes": 9000}, "precise": {"peak_bytes": 1500}})
    assert mem1["precise"] == inputs + 1500 and mem1["precise_source"].startswith("measured")
    assert mem1["ratio_to_precise"]["hybrid"] == (inputs + 9000) / (inputs + 1500)
    assert mem1["ratio_to_precise"]["inputs_plus_C"] == (inputs + c_bytes) / (inputs + 1500)
    B = gen.erdos_renyi(A.ncols, 3, seed=2, ncols=50)
    mem2 = bench.memory_comparison([(A, B)], c_bytes, "learned", {"peak_bytes": 0}, {})
    assert mem2["inputs_plus_C"] == inputs + B.nnz * 12 + (B.nrows + 1) * 4 + c_bytes


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


class _Args:
    workload = "w"


def _fake_measurement(A, kms, clocks=None):
    """A bench measurement record of one product C = A*A: per-row products u, output
    counts and bins, the per-class kernel times (ms per step) and the launch counts."""
    blen = np.diff(A.row_ptr)
    u = np.array([blen[A.col[A.row_ptr[i]:A.row_ptr[i + 1]]].sum() for i in range(A.nrows)], dtype=np.int64)
    rn = (u + 1) // 2
    bins = np.where(u > 256, 37, np.where(u > 32, 34, np.where(u > 1, 8, 1)))
    return {"kms": kms, "st_all": [{"launches": {"merge": 4, "arrange": 1}}],
            "arrays": [{"u": u, "row_nnz": rn, "bin": bins}], "policy": "learned", "ms_per_step": 5.0,
            "clocks": clocks}, u, rn, bins


def test_roofline_of_the_dominant_class(tmp_path, monkeypatch):
    """The class with the largest time is reported; its algorithmic bytes count only its own
    rows (bin 37 for the merge class); the FP64 ceiling follows the sampled SM clock."""
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 5000.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    A = gen.rmat(9, 16, seed=4)
    m, u, rn, bins = _fake_measurement(A, {"merge": 2.0, "arrange": 1.0, "esc": 0.5}, {"sm_mhz": 1000.0})
    r = bench.roofline(_Args, [(A, A)], m)
    long_rows = np.nonzero(bins == 37)[0]
    assert long_rows.size > 0 and long_rows.size < A.nrows
    want = bench.algorithmic_bytes(A, A, u, long_rows, rn)
    assert r["kernel"] == "merge" and r["bound"] == "hbm" and r["peak_source"] == "measured"
    assert r["algorithmic_bytes_per_step"] == want
    assert abs(r["achieved"] - want / 2e-3 / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 5000.0) < 1e-12
    assert r["launches_per_step"] == 4 and r["traffic"] is None
    f = r["fp64"]
    assert f["flops_per_step"] == 2 * int(u[long_rows].sum())
    assert abs(f["peak"] - 608.0) < 1e-9  # 2 FMA x 2 flop x 152 SMs x 1 GHz
    comp = A.nnz * 12 + (A.nrows + 1) * 4 + int(rn.sum()) * 12 + (A.nrows + 1) * 8
    assert r["compulsory_bytes_per_step"] == comp
    # the arrange class: C written and read once (24 B an entry) plus its row pointer
    m2, _, _, _ = _fake_measurement(A, {"merge": 1.0, "arrange": 3.0})
    r2 = bench.roofline(_Args, [(A, A)], m2)
    assert r2["kernel"] == "arrange" and r2["fp64"] is None
    assert r2["algorithmic_bytes_per_step"] == int(rn.sum()) * 24 + 8 * (A.nrows + 1)


def test_roofline_without_measured_peaks_uses_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    A = gen.rmat(8, 16, seed=5)
    m, _, _, _ = _fake_measurement(A, {"merge": 1.0})
    r = bench.roofline(_Args, [(A, A)], m)
    assert r["peak"] == 6800.0 and r["peak_source"] == "fallback"
    assert abs(r["fp64"]["peak"] - 2 * 2 * 152 * 2070e6 / 1e9) < 1e-9  # no clock samples: the maximum clock


def test_traffic_only_while_the_kernel_sources_match(tmp_path, monkeypatch):
    """DRAM traffic from a profile is reported only while the digest of the sources it was
    taken from matches the sources as they are; after a change it is null."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    for f in bench.KERNEL_SOURCES["merge"]:
        p = tmp_path / f
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_text(f"// {f}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"w": {"learned": {"merge": {"bytes_per_step": 12345,
                                       "source_digest": bench.src_digest(bench.KERNEL_SOURCES["merge"])}}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    A = gen.rmat(8, 16, seed=6)
    m, _, _, _ = _fake_measurement(A, {"merge": 1.0})
    assert bench.roofline(_Args, [(A, A)], m)["traffic"] == 12345
    (tmp_path / bench.KERNEL_SOURCES["merge"][1]).write_text("// changed\n")
    assert bench.roofline(_Args, [(A, A)], m)["traffic"] is None


class _FakeRunner:
    """Device time and peak memory of a configuration from a table, for the tuner's logic."""

    def __init__(self, cost):
        self.cost, self.calls = cost, []

    def time(self, opts, reps=3):
        self.calls.append(dict(opts))
        return self.cost(opts)


def test_tuner_keeps_faster_configurations_within_the_memory_slack():
    from paper_1504_05022_gb300 import autotune

    def cost(o):
        ms, peak = 10.0, 1000
        if o.get("heap_max_u") == 16:
            ms -= 2.0                    # faster, same memory: kept
        if o.get("merge_batch") == 512:
            ms -= 5.0
            peak += 1000                 # much faster but twice the memory: refused
        if o.get("smem_cap_max") == 4096:
            ms -= 1.0
            peak += 40                   # faster, within 5% more memory: kept
        if o.get("merge_miss") == 8192:
            ms -= 0.05                   # under the 1% threshold: not worth a change
        return ms, peak

    runner = _FakeRunner(cost)
    rec = autotune.tune(runner, "upper_bound", rounds=3, reps=1, log=lambda *_: None)
    best = rec["params"]
    assert best["heap_max_u"] == 16 and best["smem_cap_max"] == 4096
    assert best["merge_batch"] == autotune.SPACE["merge_batch"][0]
    assert rec["default_ms"] == 10.0 and rec["ms"] == 7.0 and rec["default_peak_bytes"] == 1000
    assert set(best) == set(autotune.POLICY_PARAMS["upper_bound"])
    # the second round changes nothing, so the search stops there: default + 2 rounds of trials
    per_round = sum(len(autotune.SPACE[k]) - 1 for k in autotune.POLICY_PARAMS["upper_bound"])
    assert len(runner.calls) == 1 + 2 * per_round == rec["trials"]
    assert all(c["alloc_policy"] == "upper_bound" for c in runner.calls)


class _RefArgs:
    def __init__(self, workload, steps, warmup):
        self.workload, self.steps, self.warmup = workload, steps, warmup


def test_oracle_sample_is_bounded(oracle_mod):
    """A pass covers the whole workload when it fits the product cap, otherwise a seeded row
    sample whose products stay within the cap plus one row."""
    args = _RefArgs("rmat14x16", 1, 0)
    pairs = bench.make_workload("rmat14x16")
    A = pairs[0][0]
    blen = np.diff(A.row_ptr)
    u = np.array([blen[A.col[A.row_ptr[i]:A.row_ptr[i + 1]]].sum() for i in range(A.nrows)])
    _, prods, _, sample = bench.oracle_sample(args, pairs, 10 ** 12)
    assert prods == int(u.sum()) and sample == "full workload"
    cap = int(u.sum()) // 10
    step, prods, _, sample = bench.oracle_sample(args, pairs, cap)
    assert cap <= prods <= cap + int(u.max()) and "rows (random, seed 0)" in sample
    step()


def test_reference_arm_times_exactly_k_steps_after_w(oracle_mod, monkeypatch):
    calls = []
    real = bench.oracle_sample

    def counted(args, pairs, cap):
        step, prods, n, sample = real(args, pairs, cap)

        def wrapped():
            calls.append(1)
            step()
        return wrapped, prods, n, sample
    monkeypatch.setattr(bench, "oracle_sample", counted)
    r = bench.run_reference(_RefArgs("lap2d64", 3, 2))
    assert len(calls) == 5 and "3 timed steps after 2 untimed" in r["sample"]
    assert r["value"] > 0 and r["ms_per_step"] > 0 and r["kind"] == "oracle" and r["cores"] >= 1


def test_row_blocks_cover_every_row_and_balance_the_products():
    """The end-to-end figure's row blocks: consecutive, covering all rows, none empty, at most
    the block limit, and about equal in products."""
    import gen
    A = gen.rmat(12, 16, seed=3)
    blen = np.diff(A.row_ptr)
    u = np.array([blen[A.col[A.row_ptr[i]:A.row_ptr[i + 1]]].sum() for i in range(A.nrows)])
    for max_blocks, block_bytes in ((8, 1 << 20), (3, 1 << 20), (8, 1 << 40)):
        bl = bench.row_blocks(A, A, max_blocks=max_blocks, block_bytes=block_bytes)
        assert bl[0][0] == 0 and bl[-1][1] == A.nrows
        assert all(r1 > r0 for r0, r1 in bl) and all(bl[k][1] == bl[k + 1][0] for k in range(len(bl) - 1))
        assert 1 <= len(bl) <= max_blocks
        if block_bytes == 1 << 40:
            assert len(bl) == 1
        else:
            parts = [int(u[r0:r1].sum()) for r0, r1 in bl]
            assert max(parts) <= u.sum() / len(bl) + u.max()  # a cut falls within one row of the target
