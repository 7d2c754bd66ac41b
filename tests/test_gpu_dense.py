"""GPU parity of the dense-slice kernels (bin-37 rows with many products): every result
against the oracle (structure exact, values within 1e-12 * sum |a b|, integer inputs
exact), for one and several column slices, ragged last slices, empty slices, cancellation,
every allocation policy, values-only replay and batched products."""
import numpy as np
import pytest

import gen
from tests.helpers import assert_csr_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_05022_gb300 as spg
    spg.load_library()
    return spg


def _run(spg, A, B, **opts):
    Ad = spg.CSR.from_host(A)
    Bd = Ad if B is A else spg.CSR.from_host(B)
    plan = spg.Plan(Ad, Bd, **opts)
    C = plan.numeric()
    torch.cuda.synchronize()
    return plan, C, Ad


def _check(oracle_mod, A, B, C, exact=False, label=""):
    ref = oracle_mod.spgemm(A, B)
    rp, col, val = C.to_host()
    assert C.shape == (A.nrows, B.ncols)
    assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, exact=exact, label=label)
    return ref


def _products(A, B):
    blen = np.diff(B.row_ptr)
    cs = np.concatenate([[0], np.cumsum(blen[A.col])])
    return cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]


def _col_range(A, B):
    """Per row of A*B: first and last-plus-one column of the B rows it selects."""
    blen = np.diff(B.row_ptr)
    col = B.col.astype(np.int64)
    first = np.where(blen > 0, col[np.minimum(B.row_ptr[:-1], max(B.nnz - 1, 0))], np.iinfo(np.int64).max)
    last = np.where(blen > 0, col[np.maximum(B.row_ptr[1:] - 1, 0)], -1)
    lo = np.full(A.nrows, np.iinfo(np.int64).max)
    hi = np.full(A.nrows, -1)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    np.minimum.at(lo, rows, first[A.col])
    np.maximum.at(hi, rows, last[A.col])
    return lo, hi + 1


def _policy_opts(policy):
    from paper_1504_05022_gb300.predictor import Predictor
    if policy == "learned":
        keep = Predictor.load()
        return keep.opts(), keep
    return {"alloc_policy": policy}, None


@pytest.mark.parametrize("span,slices", [(0, 1), (2048, 4), (1024, 8)])
@pytest.mark.parametrize("policy", ["hybrid", "upper_bound", "learned"])
@pytest.mark.parametrize("dmin", [0, 600])
def test_dense_slices_parity(spg, oracle_mod, span, slices, policy, dmin):
    """R-MAT 2^13 x 16 (8,192 columns) with 1, 4 or 8 slices; dense rows from u >= 1,024
    (ncols / 8) or u >= 600 (nearly every bin-37 row)."""
    A = gen.rmat(13, 16, seed=61)
    opts, keep = _policy_opts(policy)
    plan, C, _ = _run(spg, A, A, dense_min_u=dmin, dense_span=span, **opts)
    _check(oracle_mod, A, A, C, label=f"dense {span}/{policy}/{dmin}")
    st = plan.stats()
    u = _products(A, A)
    if dmin > 0:
        expect = int((u >= dmin).sum())
    else:  # 8 u_i >= the width of the row's reachable column range
        lo, hi = _col_range(A, A)
        expect = int(((u > 512) & (8 * u >= hi - lo)).sum())
    assert st["rows_dense"] == expect > 0
    assert st["dense_slices"] == slices
    plan.check()
    del keep


def test_dense_rectangular_ragged_last_slice(spg, oracle_mod):
    """B with 5,001 columns in 5 slices of 1,024 (the last one holds 905)."""
    A = gen.rmat(12, 24, seed=62)
    B = gen.erdos_renyi(4096, 40, seed=63, ncols=5001)
    plan, C, _ = _run(spg, A, B, dense_min_u=600, dense_span=1024)
    _check(oracle_mod, A, B, C, label="ragged")
    st = plan.stats()
    assert st["rows_dense"] > 0 and st["dense_slices"] == 5
    plan.check()


def test_dense_empty_slices_and_integer_values(spg, oracle_mod):
    """B's columns all lie in the first of 8 slices (the other seven count nothing and are
    skipped); integer values, so the result is exact."""
    rng = np.random.default_rng(64)
    n = 2000
    A = gen.random_sparse(300, n, 0.3, 65, integer_values=True)
    r = np.repeat(np.arange(n), 8)
    c = np.concatenate([np.sort(rng.choice(900, 8, replace=False)) for _ in range(n)])
    B = gen.from_coo(n, 8000, r, c, rng.integers(-4, 5, r.size).astype(np.float64))
    plan, C, _ = _run(spg, A, B, dense_min_u=600, dense_span=1024)
    _check(oracle_mod, A, B, C, exact=True, label="empty slices")
    st = plan.stats()
    assert st["rows_dense"] == int((_products(A, B) >= 600).sum()) > 0 and st["dense_slices"] == 8
    plan.check()


def test_dense_cancellation_keeps_structural_zeros(spg, oracle_mod):
    """Row 0 of A = [1, 1, ...] times B whose rows come in +/- pairs: every column of row 0
    sums to exactly 0 and must still be stored."""
    n, w = 1024, 600
    rows, cols, vals = [], [], []
    for k in range(n):
        cc = np.arange(w) + (k // 2) % 7
        rows.append(np.full(w, k))
        cols.append(cc)
        vals.append(np.full(w, 1.0 if k % 2 == 0 else -1.0))
    B = gen.from_coo(n, w + 8, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    A = gen.from_coo(2, n, np.concatenate([np.zeros(n, np.int64), np.ones(4, np.int64)]),
                     np.concatenate([np.arange(n), np.arange(4)]), np.ones(n + 4))
    plan, C, _ = _run(spg, A, B, dense_min_u=513, dense_span=1024)
    ref = _check(oracle_mod, A, B, C, exact=True, label="cancellation")
    rp, col, val = C.to_host()
    assert rp[1] == w + 6 and np.all(val[:rp[1]] == 0.0)
    assert plan.stats()["rows_dense"] >= 1


@pytest.mark.parametrize("policy", ["hybrid", "learned"])
def test_dense_replay_and_graph(spg, oracle_mod, policy):
    """Values-only replay recomputes the dense rows (and the others) for new values of A,
    alone and from a CUDA graph."""
    A = gen.rmat(13, 16, seed=66)
    opts, keep = _policy_opts(policy)
    plan, C, Ad = _run(spg, A, A, dense_span=2048, **opts)
    assert plan.stats()["rows_dense"] > 0
    rng = np.random.default_rng(67)
    for r in range(2):
        A2 = gen.HostCSR(A.nrows, A.ncols, A.row_ptr, A.col, A.val * rng.uniform(0.5, 2.0, A.nnz))
        Ad.val.copy_(torch.from_numpy(A2.val))
        plan.replay()
        torch.cuda.synchronize()
        plan.check()
        # B is A's device copy, so both operands changed
        _check(oracle_mod, A2, A2, C, label=f"replay {r}/{policy}")
    s = torch.cuda.Stream()
    plan2, C2, Ad2 = None, None, None
    with torch.cuda.stream(s):
        Ad2 = spg.CSR.from_host(A)
        plan2 = spg.Plan(Ad2, Ad2, stream=s, dense_span=2048, **opts)
        C2 = plan2.numeric()
    s.synchronize()
    graph = spg.ReplayGraph([plan2])
    A3 = gen.HostCSR(A.nrows, A.ncols, A.row_ptr, A.col, A.val * 2.0)
    Ad2.val.copy_(torch.from_numpy(A3.val))
    s.synchronize()
    graph.launch()
    s.synchronize()
    _check(oracle_mod, A3, A3, C2, label=f"graph/{policy}")
    del keep


@pytest.mark.parametrize("policy", ["hybrid", "learned"])
def test_dense_batched(spg, oracle_mod, policy):
    """Batched pairs of different widths (local column numbers): dense rows of every pair
    are sliced over the widest B and give each pair's own C."""
    pairs = []
    for i, (m, ncols) in enumerate([(2048, 6000), (1024, 2500), (4096, 9000), (512, 700)]):
        A = gen.rmat(int(np.log2(m)), 16, seed=70 + i)
        B = gen.erdos_renyi(m, 24, seed=80 + i, ncols=ncols)
        pairs.append((A, B))
    opts, keep = _policy_opts(policy)
    As = [spg.CSR.from_host(A) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B) for _, B in pairs]
    plan = spg.BatchPlan(As, Bs, dense_min_u=600, dense_span=2048, wave_mproducts=-1, **opts)
    Cs = plan.numeric()
    torch.cuda.synchronize()
    assert plan.stats()["rows_dense"] > 0
    for i, ((A, B), C) in enumerate(zip(pairs, Cs)):
        _check(oracle_mod, A, B, C, label=f"batched dense {i}/{policy}")
    plan.check()
    del keep


def test_dense_off_for_merge_path_and_level1(spg, oracle_mod):
    A = gen.rmat(12, 16, seed=68)
    for kw in ({"merge_kernel": "merge_path"}, {"long_rows": "level1"}, {"dense_min_u": -1}):
        plan, C, _ = _run(spg, A, A, **kw)
        assert plan.stats()["rows_dense"] == 0, kw
        _check(oracle_mod, A, A, C, label=str(kw))


@pytest.mark.parametrize("policy", ["hybrid", "precise"])
@pytest.mark.parametrize("span", [0, 16384])
def test_dense_compact_form_and_replay(spg, oracle_mod, policy, span):
    """Slices too wide for one sum per column (R-MAT 2^15 x 16: one slice of 32,768 columns, or
    two of 16,384 in the single-pass form): the bitmap, rank directory and compact sums; then a
    values-only replay of the same plan."""
    A = gen.rmat(15, 16, seed=64)
    Ad = spg.CSR.from_host(A)
    plan = spg.Plan(Ad, Ad, alloc_policy=policy, dense_span=span)
    C = plan.numeric()
    torch.cuda.synchronize()
    _check(oracle_mod, A, A, C, label=f"compact {policy}/{span}")
    st = plan.stats()
    assert st["rows_dense"] > 0 and st["dense_slices"] == (1 if span == 0 else 2)
    rng = np.random.default_rng(65)
    A2 = gen.HostCSR(A.nrows, A.ncols, A.row_ptr, A.col, rng.uniform(-1, 1, A.nnz))
    Ad.val.copy_(torch.from_numpy(A2.val))
    plan.replay()
    torch.cuda.synchronize()
    plan.check()
    _check(oracle_mod, A2, A2, C, label=f"compact replay {policy}/{span}")


def test_learned_kernel_choice_sends_long_rows_to_the_slices(spg, oracle_mod):
    """With dense_pred_min, the rows the network predicts to be long are computed by the
    dense-slice kernels instead of the merge kernel; C is unchanged."""
    from paper_1504_05022_gb300.predictor import Predictor
    A = gen.rmat(14, 8, seed=66)
    Ad = spg.CSR.from_host(A)
    pred = Predictor.load()
    base = spg.Plan(Ad, Ad, **pred.opts())
    C0 = base.numeric()
    torch.cuda.synchronize()
    st0 = base.stats()
    plan = spg.Plan(Ad, Ad, dense_pred_min=1024, **pred.opts())
    C = plan.numeric()
    torch.cuda.synchronize()
    _check(oracle_mod, A, A, C, label="learned kernel choice")
    st = plan.stats()
    assert st["rows_dense"] > st0["rows_dense"]
    assert st["item_rounds"] < st0["item_rounds"]
    plan.check()


def _kept_bytes(st, W):
    """Bytes of the kept bitmaps: ceil(W / 32) + 1 words rounded up to 4, per (row, slice)."""
    return st["rows_dense"] * st["dense_slices"] * 4 * (((W + 31) // 32 + 4) & ~3)


@pytest.mark.parametrize("case", ["square", "rect", "flags"])
@pytest.mark.parametrize("policy", ["hybrid", "learned", "precise"])
def test_dense_kept_bitmaps(spg, oracle_mod, case, policy):
    """Slices too wide for the single-pass fill are filled in the compact form; the counting pass
    may leave each (row, slice)'s column bitmap in device memory for it, instead of the fill
    marking the columns again (dense_keep): counted with a bitmap (slices wider than 32,768
    columns), or with flag bytes turned into a bitmap (the "flags" case, 32,768 columns).  C is the oracle's with the bitmaps kept and without; the precise policy keeps
    them only when asked, and its peak then grows by exactly their size; a values-only replay
    afterwards (the bitmaps are gone) is exact too."""
    if case == "square":
        A = B = gen.rmat(16, 8, seed=71)  # one slice of 65,536 columns
        kw = {}
        W = 65536
    elif case == "flags":
        A = B = gen.rmat(15, 16, seed=75)  # one slice of 32,768 columns
        kw = {}
        W = 32768
    else:
        A = gen.rmat(13, 24, seed=72)
        B = gen.erdos_renyi(8192, 40, seed=73, ncols=100001)
        kw = {"dense_span": 65536, "dense_min_u": 600}  # two slices of 50,016 columns
        W = 50016
    opts, _keep = _policy_opts(policy)
    peaks = {}
    for keep in (-1, 0, 1):
        plan, C, Ad = _run(spg, A, B, dense_keep=keep, **kw, **opts)
        _check(oracle_mod, A, B, C, label=f"kept bitmaps {case}/{policy}/{keep}")
        st = plan.stats()
        assert st["rows_dense"] > 0 and st["dense_slices"] == (2 if case == "rect" else 1)
        peaks[keep] = st["peak_bytes"]
        if keep == 1 and case == "square":
            rng = np.random.default_rng(74)
            A2 = gen.HostCSR(A.nrows, A.ncols, A.row_ptr, A.col, rng.uniform(-1, 1, A.nnz))
            Ad.val.copy_(torch.from_numpy(A2.val))
            plan.replay()
            torch.cuda.synchronize()
            plan.check()
            _check(oracle_mod, A2, A2, C, label=f"kept bitmaps replay {policy}")
    kb = _kept_bytes(st, W)
    if policy == "precise":
        assert peaks[0] == peaks[-1]
        assert peaks[1] - peaks[-1] == kb
    else:
        assert peaks[0] == peaks[1]
        assert peaks[-1] <= peaks[0] <= peaks[-1] + kb
