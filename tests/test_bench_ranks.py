"""Whole-job aggregation of bench.py over ranks (the torchrun replica path), on CPU with
gloo and two processes: the slowest rank's time and the products of all ranks."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, os.environ["REPO"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + os.environ["PORT"],
                        rank=int(os.environ["RANK"]), world_size=2)
r = dist.get_rank()
value, ms = bench.job_gflops(products=1_000_000 * (r + 1), ms=2.0 + 3.0 * r, world=2, device="cpu")
print(json.dumps({"rank": r, "value": value, "ms": ms}))
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_gflops_over_two_gloo_ranks():
    pytest.importorskip("torch")
    import json
    port = str(_free_port())
    procs = [subprocess.Popen([sys.executable, "-c", CHILD], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              env=dict(os.environ, REPO=ROOT, PORT=port, RANK=str(r)), text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        # slowest rank: 5 ms; all ranks: 3M products -> 2 * 3e6 / 5e-3 s = 1.2 GFLOP/s
        assert o["ms"] == 5.0
        assert abs(o["value"] - 1.2) < 1e-12


def test_job_gflops_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    v, ms = bench.job_gflops(5e8, 10.0, 1, "cpu")
    assert ms == 10.0 and abs(v - 100.0) < 1e-9
