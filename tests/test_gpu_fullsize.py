"""Full-size parity at the benchmark's largest configurations, in the launch configuration
bench.py times (learned policy with the committed weights and tuned parameters): every entry
of C against the oracle (structure exact, values within 1e-12 * sum |a b|).  The oracle
computes C block of rows by block of rows (about 200 M products each), so the host never
holds all of it; each block is compared with the GPU's rows on the device."""
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


def _check_all_rows(oracle_mod, A, B, C, label, block_products=200_000_000):
    """Every row of C against the oracle, in row blocks of about block_products products."""
    u = _products(A, B)
    cu = np.cumsum(u)
    rp = C.row_ptr.cpu().numpy()
    dev = C.col.device
    r0 = 0
    while r0 < A.nrows:
        r1 = int(np.searchsorted(cu, (cu[r0 - 1] if r0 else 0) + block_products, side="right"))
        r1 = min(A.nrows, max(r1, r0 + 1))
        off, col, val, den = oracle_mod.spgemm_rows(A, B, np.arange(r0, r1, dtype=np.int64))
        where = f"{label}, rows {r0}..{r1 - 1}"
        assert np.array_equal(np.diff(rp[r0:r1 + 1]), np.diff(off)), f"{where}: row sizes differ"
        s, e = int(rp[r0]), int(rp[r1])
        assert torch.equal(C.col[s:e], torch.from_numpy(col).to(dev)), f"{where}: columns differ"
        err = (C.val[s:e] - torch.from_numpy(val).to(dev)).abs()
        bad = int((err > REL_TOL * torch.from_numpy(den).to(dev)).sum())
        assert bad == 0, f"{where}: {bad} values outside the tolerance"
        r0 = r1


def test_config4_rmat20x8_full_size(spg, oracle_mod):
    A = gen.rmat(20, 8, seed=1)
    opts, keep = _learned_opts("rmat20x8")
    Ad = spg.CSR.from_host(A, rowptr_dtype=torch.int32)
    plan = spg.Plan(Ad, Ad, **opts)
    C = plan.numeric()
    torch.cuda.synchronize()
    u = _products(A, A)
    assert plan.upper_bound_nnz == int(u.sum())
    assert C.nnz > 2**31                                 # int64 row pointers are needed
    _check_all_rows(oracle_mod, A, A, C, "R-MAT 2^20 x 8")
    st = plan.stats()
    assert st["rows_dense"] > 0                          # the rows with many products took the slices
    assert st["bin_count"][37] > st["rows_dense"]        # and the merge kernel the other long rows
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
        _check_all_rows(oracle_mod, A, B, C, f"pair {i}")
    del keep
