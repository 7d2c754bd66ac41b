"""Benchmark: FP64 CSR SpGEMM throughput (GFLOP/s = 2 * products / s) on one GB300.

Default workload: C = A*A, A = R-MAT with 2^20 rows/cols, 8 samples/row
(a,b,c,d = .57,.19,.19,.05, duplicates merged, values U(-1,1), seed 1), under the learned
preallocation; the same product is also timed under the paper's plain (hybrid) form and
the upper-bound policy, and the 512-pair batch is timed batched against 512 sequential
plain calls (`compare.batch512`).  A step is one full pass of the four-stage framework
(symbolic + numeric: stages 1-4, including the size read-backs and allocations the method
needs) on inputs that are already resident in device memory.  L2 is flushed (a 512 MB
write) between timed steps, outside the timed events.  Step times are medians.

Prints one JSON line.  `--impl reference` times the CPU oracle (the reference arm)
on the same workload: W untimed steps, then K timed ones, each a pass over the workload
or over a bounded seeded sample of it.  Under torchrun each rank runs an independent replica (the
method does not exchange data between problems), and rank 0 reports the
aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "rmat16x16": "C = A*A, A = R-MAT 2^16 x 2^16, 16 samples/row (.57,.19,.19,.05), U(-1,1), seed 1",
    "lap2d64": "C = A*A, A = 2D 5-point Laplacian on a 64x64 grid",
    "galerkin64": "Ac = R*(A*P), A = 27-point Laplacian on 64^3, P = 2x2x2 aggregation, R = P^T",
    "rmat20x8": "C = A*A, A = R-MAT 2^20 x 2^20, 8 samples/row, U(-1,1), seed 1",
    "rmat14x16": "C = A*A, A = R-MAT 2^14 x 2^14, 16 samples/row, U(-1,1), seed 1 (small profiling case)",
    "rmat18x4": "C = A*A, A = R-MAT 2^18 x 2^18, 4 samples/row, U(-1,1), seed 1 (profiling case of the 2^20 x 8 "
                "product's kernels, with its tuned parameters)",
    "batch512": "512 independent C_i = A_i*B_i, rows log-uniform in [256, 65536], family per pair from "
                "{banded, block-diagonal, Erdos-Renyi, R-MAT}, 4-32 nnz/row, U(-1,1), seed = pair index",
}


def make_workload(name):
    import gen
    if name == "rmat16x16":
        A = gen.rmat(16, 16, seed=1)
        return [(A, A)]
    if name == "lap2d64":
        A = gen.lap2d(64)
        return [(A, A)]
    if name == "rmat20x8":
        A = gen.rmat(20, 8, seed=1)
        return [(A, A)]
    if name == "rmat14x16":
        A = gen.rmat(14, 16, seed=1)
        return [(A, A)]
    if name == "rmat18x4":
        A = gen.rmat(18, 4, seed=1)
        return [(A, A)]
    if name == "batch512":
        return batch_pairs_parallel(512)
    if name == "galerkin64":
        A = gen.lap3d27(64)
        P = gen.agg_P(64)
        R = gen.transpose(P)
        return [(A, P), (R, None)]  # second product multiplies R by the first result
    raise ValueError(name)


def _batch_pair(i):
    import gen
    return gen.batch_pair(i)


def batch_pairs_parallel(n):
    """gen.batch_pairs(n), generated by a spawned process pool (pair i depends only on seed i)."""
    import multiprocessing as mp
    workers = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_batch_pair, range(n), chunksize=1)


class _Cat:
    """Row pointers of the block-diagonal concatenation of the batch's A (for the byte model)."""

    def __init__(self, mats):
        lens = np.concatenate([np.diff(M.row_ptr) for M in mats])
        self.row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        self.nrows = int(lens.size)
        self.nnz = int(self.row_ptr[-1])


def src_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {
    "merge": ["paper_1504_05022_gb300/csrc/merge.cu", "paper_1504_05022_gb300/csrc/merge_bm.cu",
              "paper_1504_05022_gb300/csrc/dense.cu", "paper_1504_05022_gb300/csrc/common.cuh"],
    "arrange": ["paper_1504_05022_gb300/csrc/arrange.cu", "paper_1504_05022_gb300/csrc/scan.cuh"],
    "esc": ["paper_1504_05022_gb300/csrc/esc.cu"],
    "heap": ["paper_1504_05022_gb300/csrc/heap.cu"],
    "bound": ["paper_1504_05022_gb300/csrc/stage12.cu", "paper_1504_05022_gb300/csrc/scan.cuh"],
    "bin": ["paper_1504_05022_gb300/csrc/stage12.cu"],
}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    INTERVAL_MS = 200

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        # the raw samples go to BENCH_CLOCKS_DIR when set (to keep them), else to a temporary file
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"spgemm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def wait_first_sample(self, timeout_s=5.0):
        """Waits until nvidia-smi has written its first sample (it is then polling steadily)."""
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < timeout_s:
            self.fh.flush()
            if os.path.exists(self.path) and os.path.getsize(self.path) > 0:
                return
            if self.proc.poll() is not None:
                return
            time.sleep(0.02)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # median over the samples taken under load (upper half of the clock distribution)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(A, B, u, rows_sel, row_nnz):
    """Bytes of A (12 B per entry + 16 B B.row_ptr pair per entry), touched B rows (12 B per
    product) and C~/C rows (12 B per output entry) for the rows in rows_sel."""
    la = np.diff(A.row_ptr)[rows_sel]
    return int(la.sum()) * 28 + int(u[rows_sel].sum()) * 12 + int(row_nnz[rows_sel].sum()) * 12


def policy_opts(policy, tuned_workload=None, value_type="f64"):
    """Library options of a policy name: 'hybrid' = the paper's plain path (256-entry start,
    x2 relaunches), 'upper_bound', 'learned' = trained predictor (committed weights).  With
    tuned_workload, the autotuner's parameters for that workload and policy are applied
    (when paper_1504_05022_gb300/tuned.json has them)."""
    pred = None
    if policy == "learned":
        from paper_1504_05022_gb300.predictor import Predictor
        pred = Predictor.load(dtype=value_type)
        opts = pred.opts()
    else:
        opts = {"alloc_policy": policy}
    if MERGE_KERNEL != "auto":
        opts["merge_kernel"] = MERGE_KERNEL
    if tuned_workload:
        from paper_1504_05022_gb300 import autotune
        params = autotune.load(tuned_workload, policy)
        if params:
            opts = autotune.apply(opts, params)
    return opts, pred


MERGE_KERNEL = "auto"  # form of the bin-37 kernel (--merge-kernel)


# profiling cases that run with the tuned parameters of the workload they stand for
TUNED_AS = {"rmat18x4": "rmat20x8"}


def tuned_params(args, policy):
    if not args.tuned:
        return None
    from paper_1504_05022_gb300 import autotune
    return autotune.load(TUNED_AS.get(args.workload, args.workload), policy)


def measure(args, spg, pairs, dev, stream, policy, flush, world, sample_clocks=False, tuned=False,
            value_type="f64"):
    """W warm-up steps, then K timed steps (CUDA events on the launching stream, L2 flushed
    between steps outside the events).  Returns the per-step figures.  value_type "f32": the
    same product in single precision (values rounded to float, the float library)."""
    import torch
    tw = None
    if tuned and args.tuned:  # single precision: its own tuned entry when there is one
        from paper_1504_05022_gb300 import autotune
        tw = TUNED_AS.get(args.workload, args.workload)
        if value_type == "f32" and autotune.load(tw + ":f32", policy):
            tw = tw + ":f32"
    opts, keep = policy_opts(policy, tw, value_type)
    spg.pool_trim(dev.index)  # every policy starts from a pool holding no memory of the previous one
    timing_opts = dict(opts, record_timing=True)  # per-kernel split, taken in one extra untimed step
    vdt = torch.float32 if value_type == "f32" else torch.float64
    Ad = [spg.CSR.from_host(A, device=dev, rowptr_dtype=torch.int32, dtype=vdt) for A, _ in pairs]
    Bd = [spg.CSR.from_host(B, device=dev, rowptr_dtype=torch.int32, dtype=vdt)
          if B is not None and B is not A else None for A, B in pairs]

    def step(o=opts):
        prev = None
        plans = []
        for i in range(len(pairs)):
            A_ = Ad[i]
            if pairs[i][1] is None:          # chained: R * (previous result)
                B_ = prev
            elif pairs[i][1] is pairs[i][0]:  # A*A
                B_ = A_
            else:
                B_ = Bd[i]
            plan = spg.Plan(A_, B_, stream=stream, **o)
            prev = plan.numeric()
            plans.append(plan)
        return plans, prev

    # the clock sampler starts before the warm-up: its start-up (NVML initialisation in
    # nvidia-smi) stalls CUDA calls for milliseconds and must not fall on a timed step
    clk = ClockSampler(dev.index) if sample_clocks else None
    if clk:
        clk.__enter__()
        clk.wait_first_sample()
    for _ in range(args.warmup):
        plans, C = step()
        del plans, C
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    kms, launches = {}, 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        plans, C = step()
        ev[k][1].record(stream)
        torch.cuda.synchronize()
        # (no loop variable: a name left bound to a plan would keep its result alive into the next step)
        launches += sum(sum(q.stats()["launches"].values()) for q in plans)
        if k < args.steps - 1:
            del plans, C
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if clk:
        clk.__exit__(None, None, None)
    times = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    flush.fill_(-1.0)
    torch.cuda.synchronize()
    tplans, tC = step(timing_opts)  # the same step once more, with CUDA events around every kernel
    torch.cuda.synchronize()
    for p in tplans:
        for name, ms in p.stats()["kernel_ms"].items():
            kms[name] = kms.get(name, 0.0) + ms
    del tplans, tC
    st_all = [p.stats() for p in plans]
    arrays = [p.arrays() for p in plans]
    sum_u = sum(p.upper_bound_nnz for p in plans)
    value, ms_step = job_gflops(sum_u, float(np.median(times)), world, dev)
    res = {"policy": policy, "ms_per_step": ms_step, "value": value, "ms_steps": [round(t, 3) for t in times],
           "kms": kms, "launches": launches, "wall_s": t_wall,
           "st_all": st_all, "arrays": arrays, "sum_u": sum_u, "nnz_C": int(st_all[-1]["nnz_c"]),
           "heap_max_u": opts.get("heap_max_u"),
           "peak_bytes": int(sum(s["peak_bytes"] for s in st_all)),
           "merge_rounds": int(sum(s["merge_rounds"] for s in st_all)),
           "rows_fallback": int(sum(s["rows_fallback"] for s in st_all)),
           "rows_bin37": int(sum(s["bin_count"][37] for s in st_all)),
           "clocks": clk.summary() if clk else None}
    del plans, C, keep
    torch.cuda.synchronize()
    return res


def job_gflops(products, ms, world, device):
    """Whole-job GFLOP/s over `world` ranks (2 * products of all ranks / the slowest rank's
    step time) and that time.  Every rank must call it; device is where the collective's
    tensors live (a CUDA device for NCCL, the CPU for gloo)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        u = torch.tensor([float(products)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, products = float(t.item()), float(u.item())
    return 2.0 * products / (ms * 1e-3) / 1e9, ms


def time_steps(args, stream, flush, step):
    """W untimed warm-up calls of step(), then K calls each bracketed by CUDA events on
    `stream`, L2 flushed (512 MB write) before each, outside the events.  step() returns an
    object kept alive until the next call.  Returns this rank's median milliseconds per step."""
    import torch
    keep = None
    for _ in range(args.warmup):
        keep = step()
        del keep
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    times = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        ev[k][0].record(stream)
        keep = step()
        ev[k][1].record(stream)
        torch.cuda.synchronize()
        times.append(ev[k][0].elapsed_time(ev[k][1]))
        if k < args.steps - 1:
            del keep
            keep = None
    return float(np.median(times)), keep


def galerkin_graph(args, spg, dev, stream, flush, opts, world):
    """Galerkin chain Ac = R*(A*P) in both timings: the values-only replay of the two plans
    captured in one CUDA graph (the structure of A*P and Ac is reused), and the other
    association (R*A)*P as two plain calls."""
    import gen
    import torch
    A = gen.lap3d27(64)
    P = gen.agg_P(64)
    R = gen.transpose(P)
    Ad, Pd, Rd = (spg.CSR.from_host(M, device=dev, rowptr_dtype=torch.int32) for M in (A, P, R))
    stream = torch.cuda.Stream(dev)  # a graph is captured from a created stream, not the legacy one
    torch.cuda.synchronize()
    Ac, p1, p2 = spg.galerkin(Rd, Ad, Pd, stream=stream, **opts)
    products = p1.upper_bound_nnz + p2.upper_bound_nnz
    g = spg.ReplayGraph([p1, p2])

    def replay():
        g.launch()

    ms_graph, _ = time_steps(args, stream, flush, replay)
    v_graph, ms_graph = job_gflops(products, ms_graph, world, dev)
    p2.check()

    def ra_p():
        q1 = spg.Plan(Rd, Ad, stream=stream, **opts)
        RA = q1.numeric()
        q2 = spg.Plan(RA, Pd, stream=stream, **opts)
        q2.numeric()
        return q1, q2, RA

    ms_rap, keep = time_steps(args, stream, flush, ra_p)
    prod_rap = keep[0].upper_bound_nnz + keep[1].upper_bound_nnz
    v_rap, ms_rap = job_gflops(prod_rap, ms_rap, world, dev)
    nnz_ac = int(Ac.nnz)
    del keep, g, Ac, p1, p2
    torch.cuda.synchronize()
    # the whole chain (stages 1-4 of both products, every size on the device) in one CUDA graph
    cap = A.nnz  # nnz(A*P) <= sum u = nnz(A) (one entry per row of P); nnz(Ac) <= nnz(A*P)
    d1, d2, dg = spg.galerkin_device(Rd, Ad, Pd, cap, cap, stream=stream)
    ms_full, _ = time_steps(args, stream, flush, dg.launch)
    v_full, ms_full = job_gflops(products, ms_full, world, dev)
    full_ok = int(d2.result().nnz) == nnz_ac
    held = d1.held_bytes + d2.held_bytes
    del d1, d2, dg
    torch.cuda.synchronize()
    return {"graph_full_chain": {"value": v_full, "unit": "GFLOP/s", "ms_per_step": ms_full, "products": int(products),
                                 "held_bytes": held, "nnz_Ac_matches": full_ok,
                                 "note": "both products, stages 1-4 each, every size on the device (precise method, "
                                         "persistent per-bin kernels), in one CUDA graph"},
            "graph_replay": {"value": v_graph, "unit": "GFLOP/s",
                             "ms_per_step": ms_graph, "products": int(products), "launches_per_step": None,
                             "note": "values-only replay of R*(A*P) (structure of A*P and Ac reused) in one CUDA graph"},
            "rA_then_P": {"value": v_rap, "unit": "GFLOP/s",
                          "ms_per_step": ms_rap, "products": int(prod_rap)},
            "nnz_Ac": nnz_ac}


class BatchRig:
    """The 512 batched pairs on the device, and the two ways of computing them that the metric
    compares: one batched pipeline (block-diagonal concatenation, in waves) and 512 sequential
    plain calls."""

    def __init__(self, args, world, device, pairs=None):
        # generated by spawned workers (pair i depends only on seed i)
        self.pairs = make_workload("batch512") if pairs is None else pairs
        import torch

        import paper_1504_05022_gb300 as spg
        spg.load_library()
        self.spg, self.args, self.world = spg, args, world
        self.dev = torch.device(f"cuda:{device}")
        torch.cuda.set_device(self.dev)
        self.stream = torch.cuda.current_stream(self.dev)
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=self.dev)
        self.As = [spg.CSR.from_host(A, device=self.dev, rowptr_dtype=torch.int32) for A, _ in self.pairs]
        self.Bs = [spg.CSR.from_host(B, device=self.dev, rowptr_dtype=torch.int32) for _, B in self.pairs]
        self.products = int(sum(_products_ab(A, B) for A, B in self.pairs))

    def batched(self, policy, clocks=False, wave_mproducts=0, tuned=False):
        """One BatchPlan per step.  Returns (figures, the last step's plan, objects to keep alive)."""
        self.spg.pool_trim(self.dev.index)
        import torch
        args, spg = self.args, self.spg
        opts, keep = policy_opts(policy, "batch512" if tuned and args.tuned else None)
        opts = dict(opts, wave_mproducts=wave_mproducts)

        def step(o=opts):
            bp = spg.BatchPlan(self.As, self.Bs, stream=self.stream, **o)
            bp.numeric()
            return bp
        clk = ClockSampler(self.dev.index) if clocks else None
        if clk:
            clk.__enter__()
            clk.wait_first_sample()
        ms, bp = time_steps(args, self.stream, self.flush, step)
        value, ms = job_gflops(self.products, ms, self.world, self.dev)
        if clk:
            clk.__exit__(None, None, None)
        st = bp.stats()
        self.flush.fill_(-1.0)
        torch.cuda.synchronize()
        tp = step(dict(opts, record_timing=True))  # once more with CUDA events around every kernel
        torch.cuda.synchronize()
        kms = tp.stats()["kernel_ms"]
        del tp
        out = {"value": value, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
               "peak_bytes": int(st["peak_bytes"]), "held_bytes_after": int(st["held_bytes"]),
               "launches_per_step": int(sum(st["launches"].values())), "kms": kms,
               "rows_bin37": int(st["bin_count"][37]), "rows_fallback": int(st["rows_fallback"]),
               "merge_rounds": int(st["merge_rounds"]), "item_rounds": int(st["item_rounds"]),
               "nnz_C": int(st["nnz_c"]), "waves": bp.n_waves, "clocks": clk.summary() if clk else None}
        return out, bp, keep

    def sequential(self, policy):
        """The 512 pairs as 512 plain calls, one after another, on one stream."""
        self.spg.pool_trim(self.dev.index)
        args, spg = self.args, self.spg
        opts, keep = policy_opts(policy)

        def step():
            plans = []
            for A, B in zip(self.As, self.Bs):
                p = spg.Plan(A, B, stream=self.stream, **opts)
                p.numeric()
                plans.append(p)
            return plans
        ms, plans = time_steps(args, self.stream, self.flush, step)
        value, ms = job_gflops(self.products, ms, self.world, self.dev)
        held, peak, launches = 0, 0, 0
        for p in plans:  # results stay resident, so call i peaks on top of results 0..i-1
            st = p.stats()
            peak = max(peak, held + st["peak_bytes"])
            held += st["held_bytes"]
            launches += sum(st["launches"].values())
        del plans, keep
        return {"value": value, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                "peak_bytes": int(peak), "launches_per_step": int(launches)}

    def replay_graph(self, policy):
        """Values-only replay (structure reused) of the batched plan, captured in one CUDA graph."""
        self.spg.pool_trim(self.dev.index)
        import torch
        args, spg = self.args, self.spg
        opts, keep_g = policy_opts(policy, "batch512" if args.tuned else None)
        gstream = torch.cuda.Stream(self.dev)  # a graph is captured from a created stream, not the legacy one
        torch.cuda.synchronize()
        gp = spg.BatchPlan(self.As, self.Bs, stream=gstream, **opts)
        gp.numeric()
        g = spg.ReplayGraph([gp])
        ms_g, _ = time_steps(args, gstream, self.flush, g.launch)
        v_g, ms_g = job_gflops(self.products, ms_g, self.world, self.dev)
        gp.check()
        del g, gp, keep_g
        torch.cuda.synchronize()
        return {"value": v_g, "ms_per_step": ms_g,
                "note": "values-only replay (structure reused) of the batched plan, one CUDA graph"}

    def device_graph(self, capacity):
        """The whole batch -- concatenation and stages 1-4, every size on the device (precise
        method, persistent per-bin kernels) -- captured in one CUDA graph."""
        self.spg.pool_trim(self.dev.index)
        import torch
        args, spg = self.args, self.spg
        gstream = torch.cuda.Stream(self.dev)
        torch.cuda.synchronize()
        dp = spg.DevicePlan(self.As, self.Bs, capacity, stream=gstream)
        g = spg.DeviceGraph([dp])
        ms_g, _ = time_steps(args, gstream, self.flush, g.launch)
        v_g, ms_g = job_gflops(self.products, ms_g, self.world, self.dev)
        nnz = sum(int(C.nnz) for C in dp.result())
        held = dp.held_bytes
        del g, dp
        torch.cuda.synchronize()
        return {"value": v_g, "ms_per_step": ms_g, "steps": args.steps, "warmup": args.warmup,
                "peak_bytes": held, "nnz_C": nnz,
                "note": "concatenation and stages 1-4 of the whole batch, every size on the device (precise method, "
                        "persistent per-bin kernels), one CUDA graph"}

    def release(self):
        import torch
        del self.As, self.Bs, self.flush
        torch.cuda.synchronize()
        torch.cuda.empty_cache()


def batch_compare(args, world, device):
    """The batched half of the metric on the 512-pair workload, for the default line: the batched
    learned pipeline against 512 sequential calls of the paper's plain form (hybrid)."""
    rig = BatchRig(args, world, device)
    head = "learned" if _weights_exist() else "hybrid"
    main, bp, keep = rig.batched(head, tuned=True)
    del bp, keep
    main.pop("clocks", None)
    seq = rig.sequential("hybrid")
    full = rig.device_graph(main["nnz_C"])
    out = {"workload": "batch512", "description": WORKLOADS["batch512"], "products_per_step": rig.products,
           "batched_" + head: main, "sequential_hybrid": seq, "graph_full_chain": full,
           "speedup_batched_over_sequential": main["value"] / seq["value"],
           "peak_ratio_batched_to_sequential": main["peak_bytes"] / seq["peak_bytes"]}
    rig.release()
    return out


def _weights_exist():
    from paper_1504_05022_gb300.predictor import WEIGHTS
    return os.path.exists(WEIGHTS)


def run_batch(args, world, device):
    """512 independent products: one batched pipeline (block-diagonal concatenation) under the
    learned and the plain policy, 512 sequential plain calls, and the batched plan's
    values-only replay captured in a CUDA graph."""
    import torch
    rig = BatchRig(args, world, device)
    pairs = rig.pairs
    res = {}
    head = args.policy
    main, bp, keep = rig.batched(head, clocks=True, tuned=True)
    arrays = bp.arrays()
    order = bp.pair_order()
    del bp
    torch.cuda.synchronize()
    for p in ("hybrid",):
        if p != head:
            r, b2, k2 = rig.batched(p)
            del b2, k2
            res["batched_" + p] = r
    torch.cuda.synchronize()
    r, b2, k2 = rig.batched(head, wave_mproducts=-1, tuned=True)  # one wave: fewer launches, more memory
    del b2, k2
    res[f"batched_{head}_one_wave"] = r
    torch.cuda.synchronize()
    res["sequential_hybrid"] = rig.sequential("hybrid")
    torch.cuda.synchronize()
    res["graph_replay"] = rig.replay_graph(head)
    res["graph_full_chain"] = rig.device_graph(main["nnz_C"])
    products = rig.products
    m = {"policy": head, "kms": main["kms"], "st_all": [{"launches": {}}], "arrays": [arrays],
         "ms_per_step": main["ms_per_step"]}
    cat_a = _Cat([pairs[i][0] for i in order])  # rows in the order of the plan's arrays
    cat_b = _Cat([pairs[i][1] for i in order])
    rl = roofline(args, [(cat_a, cat_b)], m)
    rl["launches_per_step"] = None
    main_clocks = main.pop("clocks")
    out = {
        "metric": "FP64 SpGEMM GFLOP/s (2*products/s)",
        "value": main["value"], "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded generator)",
        "config": {"workload": "batch512", "description": WORKLOADS["batch512"], "alloc_policy": head,
                   "tuned": tuned_params(args, head),
                   "mode": "batched (block-diagonal concatenation, waves of <= 1024M products)",
                   "waves": main["waves"], "pairs": len(pairs),
                   "products_per_step": products, "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "roofline": rl,
        "e2e": {"value": None, "unit": "GFLOP/s",
                "note": "not measured for this workload: the 512 results need more pinned host memory than a bench run should take"},
        "gpu_launches": int(main["launches_per_step"] * args.steps),
        "kernel_ms_per_step": main["kms"],
        "memory": {"peak_bytes": main["peak_bytes"], "held_bytes_after": main["held_bytes_after"],
                   "rows_bin37": main["rows_bin37"], "rows_fallback": main["rows_fallback"],
                   "misprediction_rate": (main["rows_fallback"] / main["rows_bin37"])
                   if head == "learned" and main["rows_bin37"] else None},
        "compare": res,
        "clocks": main_clocks,
    }
    c_bytes = int(arrays["row_nnz"].astype(np.int64).sum()) * 12 + 8 * (int(arrays["u"].shape[0]) + len(pairs))
    out["memory"]["c_bytes"] = c_bytes
    out["memory"]["comparison"] = memory_comparison(
        pairs, c_bytes, "batched_" + head, main,
        {k: v for k, v in res.items() if isinstance(v, dict) and "peak_bytes" in v})
    rig.release()
    return out, pairs


def _products_ab(A, B):
    blen = np.diff(B.row_ptr)
    return int(blen[A.col].sum())


def roofline(args, pairs, m):
    """Roofline of the kernel class with the largest measured time (HBM-bound model)."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    kms = m["kms"]
    dom = max(kms, key=lambda k: kms[k]) if kms else "merge"
    dom_ms = kms.get(dom, 0.0)
    dom_launches = sum(s["launches"].get(dom, 0) for s in m["st_all"])
    bytes_dom = 0
    flops_dom = 0
    for (A, B), arr in zip(pairs, m["arrays"]):
        if B is None:
            continue
        u = arr["u"]
        rn = arr["row_nnz"].astype(np.int64)
        bins = arr["bin"]
        if dom == "arrange":
            bytes_dom += int(rn.sum()) * 24 + 8 * (u.shape[0] + 1)
        elif dom in ("bound", "bin", "scan"):
            bytes_dom += A.nnz * 12 + 16 * u.shape[0]
        else:
            hmax = m.get("heap_max_u") or 32  # bins above it (up to 36) run the bitmap ESC kernel
            sel = {"merge": bins == 37, "esc": (bins > hmax) & (bins <= 36), "heap": (bins >= 2) & (bins <= hmax)}.get(
                dom, np.ones(u.shape[0], dtype=bool))
            bytes_dom += algorithmic_bytes(A, B, u, np.nonzero(sel)[0], rn)
            flops_dom += 2 * int(u[sel].astype(np.int64).sum())  # a multiply and an add per product
    achieved = bytes_dom / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else None
    # FP64 ceiling: 2 FP64 FMA per clock per SM (the 1.25 TFLOP/s nominal rate at 2,070 MHz), 152 SMs,
    # at the SM clock sampled during the timed steps
    sm_mhz = (m.get("clocks") or {}).get("sm_mhz") or 2070.0
    fp64_peak = 2 * 2 * 152 * sm_mhz * 1e6 / 1e9
    fp64 = None
    if flops_dom and dom_ms > 0:
        ach = flops_dom / (dom_ms * 1e-3) / 1e9
        fp64 = {"achieved": ach, "peak": fp64_peak, "unit": "GFLOP/s", "frac": ach / fp64_peak,
                "flops_per_step": flops_dom, "arithmetic_intensity": flops_dom / max(1, bytes_dom),
                "ridge": fp64_peak / hbm_peak,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 2 flop x 152 SMs x sampled SM clock "
                               "(a DFMA micro-benchmark measured 1.60/clk/SM at an assumed 2,070 MHz)"}
    traffic = None
    tj = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tj):
        try:
            t = json.load(open(tj))
            ent = t.get(args.workload, {}).get(m["policy"], {}).get(dom)
            if ent and ent.get("source_digest") == src_digest(KERNEL_SOURCES.get(dom, [])):
                traffic = ent.get("bytes_per_step")
        except Exception:
            traffic = None
    # compulsory bytes: A, B and C read or written once each, over the whole step time
    comp = 0
    for (A, B), arr in zip(pairs, m["arrays"]):
        if B is None:
            continue
        comp += A.nnz * 12 + (A.nrows + 1) * 4 + int(arr["row_nnz"].astype(np.int64).sum()) * 12 + (A.nrows + 1) * 8
        if B is not A:
            comp += B.nnz * 12 + (B.nrows + 1) * 4
    comp_gbs = comp / (m["ms_per_step"] * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "compulsory_bytes_per_step": comp, "compulsory_gbs": comp_gbs, "compulsory_frac": comp_gbs / hbm_peak,
            "frac": (achieved / hbm_peak) if achieved else None, "traffic": traffic, "peak_source": peak_src,
            "nominal_peak": NOMINAL_HBM_GBS, "frac_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
            "algorithmic_bytes_per_step": bytes_dom, "kernel_ms_per_step": dom_ms,
            "launches_per_step": dom_launches, "fp64": fp64,
            "note": "achieved = algorithmic bytes of the kernel class per step / its summed CUDA-event time per step; "
                    "the class's arithmetic intensity is below the FP64/HBM ridge, so HBM is its roofline bound"}


def run_ours(args, rank, world, device):
    import torch

    import paper_1504_05022_gb300 as spg
    from paper_1504_05022_gb300.predictor import WEIGHTS

    spg.load_library()
    pairs = make_workload(args.workload)
    dev = torch.device(f"cuda:{device}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    head = args.policy
    if head == "learned" and not os.path.exists(WEIGHTS):
        head = "hybrid"
    # the paper's plain form (hybrid) and its upper-bound allocation, for the memory comparison
    others = [p for p in ("hybrid", "upper_bound", "precise") if p != head] if not args.single_policy else []
    main_m = measure(args, spg, pairs, dev, stream, head, flush, world, sample_clocks=True, tuned=True)
    cmp = {p: measure(args, spg, pairs, dev, stream, p, flush, world) for p in others}
    if not args.single_policy:
        # the same product in single precision (the paper's SpSGEMM), same policy and parameters
        cmp[head + "_f32"] = measure(args, spg, pairs, dev, stream, head, flush, world, tuned=True, value_type="f32")
    e2e_opts, e2e_keep = policy_opts(head, TUNED_AS.get(args.workload, args.workload) if args.tuned else None)  # keeps the predictor alive
    e2e = None if args.no_e2e else run_e2e(args, spg, pairs, dev, stream, e2e_opts, world)
    chain = galerkin_graph(args, spg, dev, stream, flush, e2e_opts, world) if args.workload == "galerkin64" else None
    del e2e_keep

    def brief(m):
        return {"value": m["value"], "ms_per_step": m["ms_per_step"], "peak_bytes": m["peak_bytes"],
                "merge_rounds": m["merge_rounds"], "rows_fallback": m["rows_fallback"],
                "kernel_ms_per_step": m["kms"]}

    out = {
        "metric": "FP64 SpGEMM GFLOP/s (2*products/s)",
        "value": main_m["value"], "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main_m["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded generator)",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                   "alloc_policy": head, "tuned": tuned_params(args, head), "merge_kernel": args.merge_kernel,
                   "products_per_step": main_m["sum_u"], "nnz_C": main_m["nnz_C"],
                   "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": roofline(args, pairs, main_m),
        "e2e": e2e,
        "gpu_launches": int(main_m["launches"]),
        "wall_s_timed": main_m["wall_s"],
        "ms_steps": main_m["ms_steps"],
        "kernel_ms_per_step": main_m["kms"],
        "memory": {"peak_bytes": main_m["peak_bytes"],
                   "c_bytes": int(main_m["nnz_C"]) * 12 + 8 * (int(main_m["arrays"][-1]["u"].shape[0]) + 1),
                   "rows_bin37": main_m["rows_bin37"],
                   "rows_fallback": main_m["rows_fallback"],
                   "misprediction_rate": (main_m["rows_fallback"] / main_m["rows_bin37"])
                   if head == "learned" and main_m["rows_bin37"] else None,
                   "merge_rounds": main_m["merge_rounds"]},
        "compare": {p: brief(m) for p, m in cmp.items()},
        "clocks": main_m["clocks"],
    }
    out["memory"]["comparison"] = memory_comparison(pairs, out["memory"]["c_bytes"], head, main_m,
                                                    {k: m for k, m in cmp.items() if not k.endswith("_f32")})
    if chain is not None:
        out["compare"].update(chain)
    return out, pairs


def memory_comparison(pairs, c_bytes, head, main_m, cmp):
    """Global memory of the allocation methods, as the paper compares them for C = A*A (the
    precise, hybrid and upper-bound methods, Section 5.5): each policy's figure is the inputs
    plus the plan's measured device high-water mark (temporaries and C).  The precise method
    runs as a policy of its own (count first, then C exactly, no temporary matrix); its ratio
    is the denominator.  inputs_plus_C is the floor no method can go below."""
    inputs = 0
    for A, B in pairs:
        inputs += A.nnz * 12 + (A.nrows + 1) * 4
        if B is not None and B is not A:
            inputs += B.nnz * 12 + (B.nrows + 1) * 4
    mem = {"unit": "bytes, inputs included", "inputs_plus_C": inputs + int(c_bytes)}
    for name, m in [(head, main_m)] + list(cmp.items()):
        mem[name] = inputs + int(m["peak_bytes"])
    base_key = next((k for k in mem if k.endswith("precise")), "inputs_plus_C")
    mem["ratio_to_precise"] = {k: v / mem[base_key] for k, v in mem.items() if k not in ("unit", base_key)}
    mem["precise_source"] = "measured run of the precise policy" if base_key != "inputs_plus_C" else \
        "inputs plus C (the precise policy was not run)"
    return mem


NOMINAL_HBM_GBS = 8000.0  # the round nominal HBM3e figure the roofline is also quoted against
STAGE_BYTES = 1 << 30  # pinned staging buffer for results larger than this
PIECE_BYTES = 64 << 20  # size of the copies that run beside a product


def row_blocks(A, B, max_blocks=8, block_bytes=4 << 30):
    """Row ranges [r0, r1) of A, consecutive and covering every row, that split the products of
    A*B into about equal parts: one block per block_bytes of products at 12 bytes each, at most
    max_blocks, none empty."""
    blen = np.diff(B.row_ptr)
    cs = np.concatenate([[0], np.cumsum(blen[A.col], dtype=np.int64)])
    u = cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]  # products per row
    u_sum = int(u.sum())
    nb = int(min(max_blocks, max(1, -(-u_sum * 12 // block_bytes))))
    cu = np.concatenate([[0], np.cumsum(u)])
    cuts = [0] + [int(np.searchsorted(cu, u_sum * b / nb)) for b in range(1, nb)] + [A.nrows]
    cuts = sorted(set(min(max(c, 0), A.nrows) for c in cuts))
    return [(r0, r1) for r0, r1 in zip(cuts[:-1], cuts[1:]) if r1 > r0]


def run_e2e(args, spg, pairs, dev, stream, opts, world=1):
    """Same metric through the public API with host buffers: every step copies A from pinned
    host memory to the device, computes C = A*A and reads every byte of C (row pointers,
    columns, values) back to the host.

    C is computed as NB row blocks C_b = A[rows of b] * A (each block one plan, blocks of about
    equal product counts; NB grows with the result, up to 8) on the compute stream, and each
    block's copy to the host runs on a second stream while the next block is computed.  A
    result of at most STAGE_BYTES lands in pinned host arrays; a larger one streams through one
    pinned staging buffer of STAGE_BYTES in chunks, each chunk overwriting the previous one (the
    host keeps no copy), so a run pins a bounded amount of host memory whatever the size of C.
    One step at a time, each bracketed by a device synchronisation; the value is the median
    step.  one_block_ms_per_step times the same step as one plan with the copy after it."""
    import torch
    if len(pairs) != 1 or pairs[0][1] is not pairs[0][0]:
        return None
    A = pairs[0][0]
    hp = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
          for x in (A.row_ptr.astype(np.int32), A.col, A.val)]
    u_sum = int(_products(A))
    blocks = []  # (r0, r1, first entry, pinned rebased row pointers)
    for r0, r1 in row_blocks(A, A):
        rp = A.row_ptr[r0:r1 + 1]
        blocks.append((r0, r1, int(rp[0]), torch.from_numpy((rp - rp[0]).astype(np.int32)).pin_memory()))
    h2d = sum(t.numel() * t.element_size() for t in hp)
    if len(blocks) > 1:
        h2d += sum(b[3].numel() * 4 for b in blocks)
    reps = max(3, min(args.steps, 10))
    copy_stream = torch.cuda.Stream(dev)
    state = {"out": None, "staging": None}

    def read_back(srcs, s, single):
        total = sum(t.numel() * t.element_size() for t in srcs)
        with torch.cuda.stream(s):
            if single and total <= STAGE_BYTES:
                if state["out"] is None or [h.numel() for h in state["out"]] != [t.numel() for t in srcs]:
                    state["out"] = [torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in srcs]
                for h, d in zip(state["out"], srcs):
                    h.copy_(d, non_blocking=True)
                return total, "pinned host arrays"
            if state["staging"] is None:
                state["staging"] = torch.empty(STAGE_BYTES, dtype=torch.uint8).pin_memory()
            # beside a running product, copies of PIECE_BYTES: the product's own small reads of
            # sizes wait for the copy in flight, not for a whole block's result
            piece = STAGE_BYTES if single else PIECE_BYTES
            for d in srcs:
                b = d.view(torch.uint8)
                for off in range(0, b.numel(), piece):
                    n = min(piece, b.numel() - off)
                    state["staging"][:n].copy_(b[off:off + n], non_blocking=True)
        return total, f"streamed through one {STAGE_BYTES >> 20} MiB pinned staging buffer"

    def step_blocks():
        keep, d2h, how = [], 0, None
        with torch.cuda.stream(stream):
            rp, col, val = (t.to(dev, non_blocking=True) for t in hp)
            Ad = spg.CSR(rp, col, val, (A.nrows, A.ncols))
            for r0, r1, e0, brp in blocks:
                e1 = int(A.row_ptr[r1])
                Ab = spg.CSR(brp.to(dev, non_blocking=True), col[e0:e1], val[e0:e1], (r1 - r0, A.ncols))
                plan = spg.Plan(Ab, Ad, stream=stream, **opts)
                C = plan.numeric()
                done = torch.cuda.Event()
                done.record(stream)
                copy_stream.wait_event(done)
                nbytes, how = read_back((C.row_ptr, C.col, C.val), copy_stream, False)
                d2h += nbytes
                keep.append((plan, C, Ab))  # alive until its copy has run
        return keep, d2h, how

    def step_one():
        with torch.cuda.stream(stream):
            rp, col, val = (t.to(dev, non_blocking=True) for t in hp)
            Ad = spg.CSR(rp, col, val, (A.nrows, A.ncols))
            C = spg.Plan(Ad, Ad, stream=stream, **opts).numeric()
            nbytes, how = read_back((C.row_ptr, C.col, C.val), stream, True)
        return (C, Ad), nbytes, how

    def timed(step):
        times, d2h, how = [], 0, None
        for k in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            keep, d2h, how = step()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            del keep
            if k > 0:
                times.append(dt)
        return float(np.median(times)) * 1e3, d2h, how

    spg.pool_trim(dev.index)
    ms_one, d2h, how_one = timed(step_one)
    how = how_one
    if len(blocks) > 1:
        spg.pool_trim(dev.index)
        ms, d2h, how = timed(step_blocks)
    else:
        ms = ms_one
    state.clear()
    value, ms = job_gflops(u_sum, ms, world, dev)
    return {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms, "steps": reps, "row_blocks": len(blocks),
            "one_block_ms_per_step": ms_one,
            "note": f"median of {reps} steps after 1 untimed, one at a time; A copied from pinned host memory; "
                    f"C as {len(blocks)} row block(s), each block's copy to the host on a second stream beside the "
                    f"next block's product; C {how}"}


def _products(A):
    blen = np.diff(A.row_ptr)
    return blen[A.col].sum()


def oracle_sample(args, pairs, cap_products):
    """One pass of the oracle over a bounded sample of the workload: the whole workload when
    it has at most cap_products products, else seeded random rows (or whole pairs of a batch)
    up to that count.  Returns (step, products, threads, sample description)."""
    import oracle
    nthreads = oracle.num_threads()
    if args.workload == "batch512":
        order = np.random.default_rng(0).permutation(len(pairs))
        sel, prods = [], 0
        for i in order:
            u = _products_ab(*pairs[i])
            if prods + u > cap_products and sel:
                continue
            sel.append(int(i))
            prods += u

        def step():
            for i in sel:
                oracle.spgemm_rows(pairs[i][0], pairs[i][1], None, nthreads=nthreads)
        return step, prods, nthreads, f"{len(sel)} of {len(pairs)} pairs (seeded random order, products capped)"
    A, B = pairs[0]
    B = A if B is None else B
    blen = np.diff(B.row_ptr)
    cs = np.concatenate([[0], np.cumsum(blen[A.col])])
    u = cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]
    total_u = int(u.sum())
    rows = None
    sample = "full workload"
    if len(pairs) == 2 and pairs[1][1] is None:
        sample = "the chain's first product, A*P"
    if total_u > cap_products:
        perm = np.random.default_rng(0).permutation(A.nrows)
        cu = np.cumsum(u[perm])
        rows = np.sort(perm[: int(np.searchsorted(cu, cap_products)) + 1])
        sample = f"{rows.size} of {A.nrows} rows (random, seed 0)"
    prods = total_u if rows is None else int(u[rows].sum())

    def step():
        oracle.spgemm_rows(A, B, rows, nthreads=nthreads)
    return step, prods, nthreads, sample


def run_cpu_baseline(args, budget_s=20.0, pairs=None):
    """The oracle, as it stands, on the host cores: repeated passes over the workload (or a
    bounded sample of it), median time, GFLOP/s on the products computed."""
    import oracle
    pairs = make_workload(args.workload) if pairs is None else pairs
    # keep one pass under ~budget/3 seconds assuming >= 20M products/s/thread
    cap_products = int(20e6 * oracle.num_threads() * budget_s / 3)
    step, prods, nthreads, sample = oracle_sample(args, pairs, cap_products)
    times = []
    t_start = time.perf_counter()
    while len(times) < 5 and (time.perf_counter() - t_start) < budget_s:
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    t = float(np.median(times))
    out = {"value": 2.0 * prods / t / 1e9, "unit": "GFLOP/s", "cores": nthreads, "kind": "oracle",
           "sample": f"{sample}; {prods} products; median of {len(times)} passes", "ms_per_pass": t * 1e3}
    if args.workload != "batch512":
        # one core, on a smaller row sample (about 80 M products)
        A, B = pairs[0]
        B = A if B is None else B
        blen = np.diff(B.row_ptr)
        cs = np.concatenate([[0], np.cumsum(blen[A.col])])
        u = cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]
        perm1 = np.random.default_rng(1).permutation(A.nrows)
        cs1 = np.cumsum(u[perm1])
        rows1 = np.sort(perm1[: int(np.searchsorted(cs1, 80_000_000)) + 1])
        t1 = time.perf_counter()
        oracle.spgemm_rows(A, B, rows1, nthreads=1)
        t1 = time.perf_counter() - t1
        out["one_core"] = {"value": 2.0 * int(u[rows1].sum()) / t1 / 1e9, "unit": "GFLOP/s",
                           "sample": f"{rows1.size} random rows (seed 1), {int(u[rows1].sum())} products, one pass"}
    return out


def run_reference(args, total_s=150.0):
    """The reference arm: the oracle on the host cores, W untimed steps, then exactly K timed
    steps, each one pass over a bounded sample of the workload sized so that the whole run
    takes about total_s seconds or less (at >= 20M products/s/thread)."""
    import oracle
    pairs = make_workload(args.workload)
    per_step = min(20.0, total_s / max(1, args.steps + args.warmup))
    step, prods, nthreads, sample = oracle_sample(args, pairs, int(20e6 * oracle.num_threads() * per_step))
    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    total = float(sum(times))
    value = 2.0 * prods * len(times) / total / 1e9
    return {"value": value, "unit": "GFLOP/s", "cores": nthreads, "kind": "oracle",
            "sample": f"{sample}; {prods} products per step; {len(times)} timed steps after {args.warmup} untimed",
            "ms_per_step": total / len(times) * 1e3}


def run_merge_micro(args):
    """The merge evaluation of Section 4.2: 2^25 keys in groups of two ascending runs of
    length l, merged by the ranking merge, merge path and bitonic merge (one CTA per group,
    best of 64-1024 threads), with no value, 32-bit and 64-bit values.  CUDA-event time of
    one launch, median of 5 after a warm-up; merged elements per second."""
    import torch

    import paper_1504_05022_gb300 as spg
    spg.load_library()
    n = 1 << 25
    gen_ = torch.Generator(device="cuda").manual_seed(0)
    out = []
    for vb in (0, 4, 8):
        for lg in range(5, 14):
            l = 1 << lg
            if 2 * l * (4 + vb) > 200 * 1024:
                continue
            keys = torch.randint(0, 1 << 30, (n // (2 * l), 2, l), device="cuda", dtype=torch.int32, generator=gen_)
            keys = keys.sort(dim=2).values.reshape(-1).contiguous()
            vals = None
            if vb == 4:
                vals = torch.arange(n, device="cuda", dtype=torch.int32)
            elif vb == 8:
                vals = torch.arange(n, device="cuda", dtype=torch.float64)
            row = {"value_bytes": vb, "l": l}
            for method in ("ranking", "merge_path", "bitonic"):
                best = None
                for threads in (64, 128, 256, 512, 1024):
                    spg.merge_micro(keys, l, method=method, threads=threads, vals=vals)
                    ts = []
                    for _ in range(5):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        spg.merge_micro(keys, l, method=method, threads=threads, vals=vals)
                        e1.record()
                        torch.cuda.synchronize()
                        ts.append(e0.elapsed_time(e1))
                    ms = float(np.median(ts))
                    if best is None or ms < best[0]:
                        best = (ms, threads)
                row[method] = {"gelem_s": n / (best[0] * 1e-3) / 1e9, "ms": best[0], "threads": best[1]}
            row["fastest"] = max(("ranking", "merge_path", "bitonic"), key=lambda k: row[k]["gelem_s"])
            out.append(row)
            del keys, vals
    head = next(r for r in out if r["value_bytes"] == 8 and r["l"] == 256)
    return {"metric": "merge micro-benchmark (Section 4.2): merged elements/s, merge path, l = 256, "
                      "32-bit keys with 64-bit values", "value": head["merge_path"]["gelem_s"] * 1e9,
            "unit": "elements/s", "higher_is_better": True, "n_gpus": 1, "dtype": "i32 keys",
            "data": "synthetic (seeded generator)",
            "config": {"workload": "merge_micro", "elements": n, "ls": sorted({r["l"] for r in out}),
                       "threads": [64, 128, 256, 512, 1024]},
            "results": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat20x8", choices=list(WORKLOADS))
    ap.add_argument("--policy", default="learned", choices=["hybrid", "upper_bound", "learned"])
    ap.add_argument("--single-policy", action="store_true", help="do not also time the plain hybrid path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch-compare", action="store_true",
                    help="R-MAT 2^20 line: do not also time the 512-pair batch (batched against sequential calls)")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end figure (profiling runs: every product of the run is then a whole one)")
    ap.add_argument("--no-tuned", dest="tuned", action="store_false",
                    help="do not apply the autotuner's parameters to the reported policy")
    ap.add_argument("--merge-kernel", default="auto", choices=["auto", "merge_path", "bitmap"],
                    help="form of the bin-37 kernel for every policy")
    ap.add_argument("--merge-micro", action="store_true",
                    help="run the merge evaluation of Section 4.2 instead and print its line")
    args = ap.parse_args()
    if args.merge_micro:
        print(json.dumps(run_merge_micro(args)))
        return
    global MERGE_KERNEL
    MERGE_KERNEL = args.merge_kernel
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        cb = run_reference(args)
        out = {"metric": "FP64 SpGEMM GFLOP/s (2*products/s)", "value": cb["value"], "unit": "GFLOP/s",
               "impl": "reference", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": cb["ms_per_step"], "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
               "config": {"workload": args.workload, "description": WORKLOADS[args.workload]},
               "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    pairs = None
    if args.workload == "batch512":
        out, pairs = run_batch(args, world, local)
    else:
        out, pairs = run_ours(args, rank, world, local)
        if args.workload == "rmat20x8" and not args.no_batch_compare and not args.single_policy:
            # the batched half of the metric: 512 pairs, batched pipeline against sequential plain calls
            out["compare"]["batch512"] = batch_compare(args, world, local)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = run_cpu_baseline(args, pairs=pairs)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
