"""Full-size parity at the benchmark's largest configurations, in the launch configuration
bench.py times (learned policy with the committed weights and tuned parameters): every row
pointer of C against the oracle's row counts, and every entry of sampled rows (random rows,
the longest rows, random rows of bin 37) against the oracle's rows (structure exact, values
within 1e-12 * sum |a b|)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import gen
from tests.helpers import REL_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_05022_gb300 as spg
    spg.load_library()
    return spg


def _learned_opts(workload):
    from paper_1504_05022_gb300 import autotune
    from paper_1504_05022_gb300.predictor import Predictor
    pred = Predictor.load()
    return autotune.apply(pred.opts(), autotune.load(workload, "learned") or {}), pred


def _products(A, B):
    blen = np.diff(B.row_ptr)
    cs = np.concatenate([[0], np.cumsum(blen[A.col])])
    return cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]


def _sample_rows(u, bins, rng, n_random=1500, n_long=20, n_bin37=300):
    m = u.shape[0]
    rows = [rng.choice(m, min(n_random, m), replace=False), np.argsort(u)[-n_long:]]
    b37 = np.nonzero(bins == 37)[0]
    if b37.size:
        rows.append(rng.choice(b37, min(n_bin37, b37.size), replace=False))
    return np.unique(np.concatenate(rows))


def _check_rows(oracle_mod, A, B, C, rows, label):
    rp = C.row_ptr.cpu().numpy()
    starts, ends = rp[rows], rp[rows + 1]
    idx = np.concatenate([np.arange(s, e, dtype=np.int64) for s, e in zip(starts, ends)])
    it = torch.from_numpy(idx).to(C.col.device)
    gc = C.col[it].cpu().numpy()
    gv = C.val[it].cpu().numpy()
    off, col, val, den = oracle_mod.spgemm_rows(A, B, rows)
    assert np.array_equal(np.diff(off), ends - starts), label
    assert np.array_equal(gc, col), label
    bad = np.abs(gv - val) > REL_TOL * den
    assert not bad.any(), f"{label}: {int(bad.sum())} values outside the tolerance"


def test_config4_rmat20x8_full_size(spg, oracle_mod):
    A = gen.rmat(20, 8, seed=1)
    opts, keep = _learned_opts("rmat20x8")
    Ad = spg.CSR.from_host(A, rowptr_dtype=torch.int32)
    plan = spg.Plan(Ad, Ad, **opts)
    C = plan.numeric()
    torch.cuda.synchronize()
    u = _products(A, A)
    assert plan.upper_bound_nnz == int(u.sum())
    counts = oracle_mod.row_counts(A, A)
    assert np.array_equal(np.diff(C.row_ptr.cpu().numpy()), counts)
    assert C.nnz == int(counts.sum()) > 2**31          # int64 row pointers are needed
    rows = _sample_rows(u, plan.arrays()["bin"], np.random.default_rng(4))
    _check_rows(oracle_mod, A, A, C, rows, "R-MAT 2^20 x 8")
    st = plan.stats()
    assert st["rows_split"] > 0                          # hub rows took the long-row path
    del keep


def test_config5_batch512_full_size(spg, oracle_mod):
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        pairs = pool.map(gen.batch_pair, range(512), chunksize=1)
    opts, keep = _learned_opts("batch512")
    As = [spg.CSR.from_host(A, rowptr_dtype=torch.int32) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B, rowptr_dtype=torch.int32) for _, B in pairs]
    plan = spg.BatchPlan(As, Bs, **opts)
    Cs = plan.numeric()
    torch.cuda.synchronize()
    assert plan.n_waves > 1
    assert plan.upper_bound_nnz == sum(int(_products(A, B).sum()) for A, B in pairs)
    for i, ((A, B), C) in enumerate(zip(pairs, Cs)):
        assert C.shape == (A.nrows, B.ncols)
        assert np.array_equal(np.diff(C.row_ptr.cpu().numpy()), oracle_mod.row_counts(A, B)), f"pair {i}"
    rng = np.random.default_rng(9)
    for i in rng.choice(len(pairs), 12, replace=False):
        A, B = pairs[i]
        u = _products(A, B)
        rows = _sample_rows(u, np.where(u > 512, 37, 0), rng, n_random=300, n_long=5, n_bin37=100)
        _check_rows(oracle_mod, A, B, Cs[i], rows, f"pair {i}")
    del keep
