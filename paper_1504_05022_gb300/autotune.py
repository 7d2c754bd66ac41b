"""Autotuner for the library's launch parameters on a given workload.

The paper notes that the bin boundaries and the kernel chosen for each bin depend
on the architecture (Section 4.1).  This tuner searches, by coordinate descent on
measured device time, over the parameters the library exposes for that choice:

* heap_max_u   - the longest rows (u_i) given to the heap kernel; the rest of
                 bins 2..32 go to the bitonic ESC kernel with 32 slots;
* heap_block   - threads per block of the heap kernel;
* merge_batch  - products absorbed per batch by the bin-37 merge kernel;
* smem_cap_max - the largest result held in shared memory by the merge kernel
                 (smaller values leave room for more CTAs per SM, and split
                 long rows earlier);
* merge_wide_above - result capacities above this run 512-thread merge CTAs,
                 smaller ones 256-thread CTAs (two can share an SM);
* merge_miss   - entries of the bitmap merge kernel's miss buffer (how often new
                 columns are merged into the result);
* initial_cap  - the first bin-37 row size of the plain (hybrid) policy;
* predictor_margin - the safety factor of the learned policy;
* dense_min_u, dense_span_div - which bin-37 rows the dense column slices take;
* dense_span   - the slices' width (and with it their form: one sum per column of a
                 narrow slice, or a bitmap with compact sums for a wide one);
* dense_pred_min - the learned policy's choice of kernel: rows predicted at least this
                 long go to the dense column slices;
* dense_keep   - whether the slices' counting pass leaves its column bitmaps for the
                 fill (device memory for a pass over the products).

A configuration is kept only if it is faster and its peak device memory stays
within 5% of the default configuration's, so tuning never buys time with memory.
Results are exact for every configuration (the tests check that), so the tuner
only ever trades time.  Each trial times the whole product (symbolic + numeric)
with CUDA events after a warm-up, median of `reps`.

    python -m paper_1504_05022_gb300.autotune --workload rmat16x16 [--policy learned]

writes the best parameters to paper_1504_05022_gb300/tuned.json, which
bench.py applies to the policy it reports.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

TUNED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")

SPACE = {
    "heap_max_u": [32, 24, 16, 8],
    "heap_block": [128, 64, 256],
    "merge_batch": [2048, 1024, 512],
    "smem_cap_max": [0, 8192, 6144, 4096],
    "merge_wide_above": [2048, 4096, 6144, 1 << 20],
    "merge_miss": [4096, 2048, 8192],
    "initial_cap": [256, 512, 1024],
    "predictor_margin": [None, 1.15, 1.5, 2.0],  # None = the margin stored with the weights
    "dense_min_u": [0, 16384, 8192, 4096, 2048, 1024, -1],  # 0 = the rule of dense_span_div, -1 = no slice rows
    "dense_span": [0, 65536, 32768, 21856, 16384, 10912],  # 0 = 131,072-column slices (bitmap, compact
                                                           # sums); narrow enough for a sum per column
                                                           # (21,856 and below in double): single-pass
    "dense_span_div": [0, 16, 4, 64],     # 0 = 8: dense when 8 u_i >= the row's column range
    "dense_pred_min": [0, 12288, 6144, 3072],  # learned: predicted nnz(c_i) that sends a row to the slices
    "dense_keep": [0, -1],                # 0 = the count leaves its bitmaps for the compact fill, -1 = never
}
POLICY_PARAMS = {
    "hybrid": ["heap_max_u", "heap_block", "merge_batch", "smem_cap_max", "merge_wide_above", "merge_miss",
               "initial_cap", "dense_min_u", "dense_span", "dense_span_div", "dense_keep"],
    "learned": ["heap_max_u", "heap_block", "merge_batch", "smem_cap_max", "merge_wide_above", "merge_miss",
                "predictor_margin", "dense_min_u", "dense_span", "dense_span_div", "dense_pred_min", "dense_keep"],
    "upper_bound": ["heap_max_u", "heap_block", "merge_batch", "smem_cap_max", "merge_wide_above", "dense_min_u",
                    "dense_span", "dense_span_div", "dense_keep"],
}
MEMORY_SLACK = 1.05


def workload(name: str):
    """(A, B) host pairs of a named workload (the products bench.py times)."""
    import gen
    if name.startswith("rmat"):
        scale, avg = (int(x) for x in name[4:].split("x"))
        A = gen.rmat(scale, avg, seed=1)
        return [(A, A)]
    if name == "lap2d64":
        A = gen.lap2d(64)
        return [(A, A)]
    if name == "galerkin64":
        A = gen.lap3d27(64)
        P = gen.agg_P(64)
        return [(A, P), (gen.transpose(P), None)]  # R * (A*P): the second product takes the first's result
    if name == "batch512":
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
            return pool.map(gen.batch_pair, range(512), chunksize=1)
    raise ValueError(f"unknown workload {name}")


def base_opts(policy: str, predictor=None) -> dict:
    if policy == "learned":
        return predictor.opts()
    return {"alloc_policy": policy}


def apply(opts: dict, params: dict, predictor=None) -> dict:
    out = dict(opts)
    for k, v in params.items():
        if k == "predictor_margin":
            if v is not None:
                out["predictor_margin"] = float(v)
        elif v is not None:
            out[k] = v
    return out


class Runner:
    """Times one configuration of the whole product on device-resident inputs."""

    def __init__(self, pairs, device="cuda", value_type="f64"):
        import torch

        from .spgemm import CSR
        self.torch = torch
        self.chain = len(pairs) == 2 and pairs[1][1] is None
        self.batched = len(pairs) > 1 and not self.chain
        vdt = torch.float32 if value_type == "f32" else torch.float64
        self.A = [CSR.from_host(A, device=device, rowptr_dtype=torch.int32, dtype=vdt) for A, _ in pairs]
        self.B = [a if B is A else (None if B is None else CSR.from_host(B, device=device, rowptr_dtype=torch.int32,
                                                                         dtype=vdt))
                  for a, (A, B) in zip(self.A, pairs)]
        self.stream = torch.cuda.current_stream()

    def once(self, opts):
        from .spgemm import BatchPlan, Plan
        if self.chain:  # R * (A*P)
            p1 = Plan(self.A[0], self.B[0], stream=self.stream, **opts)
            p2 = Plan(self.A[1], p1.numeric(), stream=self.stream, **opts)
            p2.numeric()
            p2._keep = p1
            return _Chain(p1, p2)
        if self.batched:
            p = BatchPlan(self.A, self.B, stream=self.stream, **opts)
        else:
            p = Plan(self.A[0], self.B[0], stream=self.stream, **opts)
        p.numeric()
        return p


    def time(self, opts, reps: int = 3):
        torch = self.torch
        p = self.once(opts)  # warm-up (also loads kernels)
        peak = p.stats()["peak_bytes"]
        del p
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            p = self.once(opts)
            e1.record(self.stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            del p
        return statistics.median(times), peak


class _Chain:
    """Two plans of a chained product; stats() reports the larger peak."""

    def __init__(self, p1, p2):
        self.p1, self.p2 = p1, p2

    def stats(self):
        s1, s2 = self.p1.stats(), self.p2.stats()
        return {"peak_bytes": max(s1["peak_bytes"], s1["held_bytes"] + s2["peak_bytes"])}


def tune(runner: Runner, policy: str, predictor=None, rounds: int = 2, reps: int = 3, log=print) -> dict:
    """Coordinate descent over POLICY_PARAMS[policy]; returns the result record."""
    names = POLICY_PARAMS[policy]
    best = {k: SPACE[k][0] for k in names}
    opts0 = base_opts(policy, predictor)
    default_ms, default_peak = runner.time(apply(opts0, best), reps)
    best_ms = default_ms
    trials = [{"params": dict(best), "ms": default_ms, "peak_bytes": default_peak}]
    log(f"default {best}: {default_ms:.3f} ms, peak {default_peak / 1e9:.2f} GB")
    for r in range(rounds):
        changed = False
        for k in names:
            for v in SPACE[k]:
                if v == best[k]:
                    continue
                cand = dict(best, **{k: v})
                ms, peak = runner.time(apply(opts0, cand), reps)
                trials.append({"params": cand, "ms": ms, "peak_bytes": peak})
                ok = peak <= default_peak * MEMORY_SLACK
                log(f"  round {r} {k}={v}: {ms:.3f} ms, peak {peak / 1e9:.2f} GB{'' if ok else ' (memory)'}")
                if ok and ms < best_ms * 0.99:
                    best, best_ms, changed = cand, ms, True
        if not changed:
            break
    log(f"best {best}: {best_ms:.3f} ms (default {default_ms:.3f} ms)")
    return {"params": best, "ms": best_ms, "default_ms": default_ms, "default_peak_bytes": default_peak,
            "trials": len(trials), "reps": reps}


def load(workload_name: str, policy: str) -> dict | None:
    """Tuned parameters for (workload, policy), or None."""
    if not os.path.exists(TUNED):
        return None
    try:
        rec = json.load(open(TUNED)).get(workload_name, {}).get(policy)
    except (OSError, ValueError):
        return None
    return None if rec is None else rec.get("params")


def main():
    import torch

    from .predictor import Predictor
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True)
    ap.add_argument("--policy", default="learned", choices=list(POLICY_PARAMS))
    ap.add_argument("--rounds", type=int, default=2)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=TUNED)
    ap.add_argument("--value-type", default="f64", choices=["f64", "f32"],
                    help="f32: the single-precision library; stored under '<workload>:f32'")
    args = ap.parse_args()
    if not torch.cuda.is_available():
        raise SystemExit("autotune needs a CUDA device")
    t0 = time.time()
    pairs = workload(args.workload)
    runner = Runner(pairs, value_type=args.value_type)
    pred = Predictor.load(dtype=args.value_type) if args.policy == "learned" else None
    rec = tune(runner, args.policy, pred, rounds=args.rounds, reps=args.reps)
    rec["products"] = int(sum(np.diff(B.row_ptr)[A.col].sum() for A, B in pairs if B is not None))
    rec["device"] = torch.cuda.get_device_name()
    rec["tuning_seconds"] = round(time.time() - t0, 1)
    doc = json.load(open(args.out)) if os.path.exists(args.out) else {}
    key = args.workload + (":f32" if args.value_type == "f32" else "")
    doc.setdefault(key, {})[args.policy] = rec
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
