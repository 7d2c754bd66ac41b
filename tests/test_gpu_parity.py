"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Structure (row_ptr, col) must match bit-exactly; values within
|c - ref| <= 1e-12 * sum_k |a_ik b_kj|, or bit-exactly where all values are
small integers.  Stage 1 and stage 2 outputs are integers and must match the
oracle's restatements of Algorithms 2 and 3 exactly."""
import numpy as np
import pytest

import gen
from tests.helpers import REL_TOL, assert_csr_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_05022_gb300 as spg
    spg.load_library()
    return spg


def run(spg, A, B, rowptr_dtype=torch.int64, **opts):
    Ad = spg.CSR.from_host(A, rowptr_dtype=rowptr_dtype)
    Bd = Ad if B is A else spg.CSR.from_host(B, rowptr_dtype=rowptr_dtype)
    plan = spg.Plan(Ad, Bd, **opts)
    C = plan.numeric()
    torch.cuda.synchronize()
    return plan, C


def check(oracle_mod, A, B, C, exact=False, label=""):
    ref = oracle_mod.spgemm(A, B)
    rp, col, val = C.to_host()
    assert C.shape == (A.nrows, B.ncols)
    assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, exact=exact, label=label)
    return ref


def test_lap2d_64_bit_exact(spg, oracle_mod):
    A = gen.lap2d(64)
    plan, C = run(spg, A, A, rowptr_dtype=torch.int32, check_inputs=True)
    assert C.nnz == 51972
    check(oracle_mod, A, A, C, exact=True, label="lap2d64")
    assert plan.upper_bound_nnz == 100104


@pytest.mark.parametrize("policy", ["hybrid", "upper_bound"])
@pytest.mark.parametrize("scale,avg", [(8, 4), (10, 16), (12, 8), (12, 32)])
def test_rmat_small(spg, oracle_mod, policy, scale, avg):
    A = gen.rmat(scale, avg, seed=scale + avg)
    plan, C = run(spg, A, A, alloc_policy=policy)
    check(oracle_mod, A, A, C, label=f"rmat{scale}x{avg}/{policy}")


@pytest.mark.parametrize("name,mk", [
    ("lap2d", lambda: (gen.lap2d(40), None)),
    ("rmat", lambda: (gen.rmat(11, 16, seed=4), None)),
    ("er_rect", lambda: (gen.erdos_renyi(700, 9, seed=2, ncols=900), gen.erdos_renyi(900, 30, seed=3, ncols=500))),
    ("blockdiag", lambda: (gen.blockdiag(1000, 40, seed=1), None)),
])
def test_stage1_stage2_bit_exact(spg, oracle_mod, name, mk):
    A, B = mk()
    B = A if B is None else B
    for policy in ("hybrid", "upper_bound"):
        plan, _ = run(spg, A, B, alloc_policy=policy, dense_min_u=-1)  # Algorithm 3's sizes
        arr = plan.arrays()
        u = oracle_mod.upper_bound(A, B)
        assert np.array_equal(arr["u"], u), name
        b, sz, cnt, rows, total = oracle_mod.binning(u)
        assert np.array_equal(arr["bin"].astype(np.int32), b)
        assert np.array_equal(arr["bin_rows"], rows)           # stable order inside each bin
        assert np.array_equal(np.diff(arr["bin_start"]), cnt)
        caps = np.diff(arr["ctilde_row_ptr"])
        if policy == "hybrid":
            assert np.array_equal(caps, sz)                     # Algorithm 3 sizes
            assert int(arr["ctilde_row_ptr"][-1]) == total
        else:
            assert np.array_equal(caps, u)
        assert plan.upper_bound_nnz == int(u.sum())
        st = plan.stats()
        assert st["sum_u"] == int(u.sum()) and st["bin_count"] == cnt.tolist()
        ref = oracle_mod.spgemm(A, B)
        assert np.array_equal(arr["row_nnz"].astype(np.int64), np.diff(ref.row_ptr))


@pytest.mark.parametrize("long_rows", ["split", "level1"])
@pytest.mark.parametrize("initial_cap,smem_cap_max,batch", [
    (32, 256, 32), (64, 512, 64), (256, 1024, 256), (256, 0, 2048), (128, 2048, 512)])
def test_progressive_split_and_level1_paths(spg, oracle_mod, initial_cap, smem_cap_max, batch, long_rows):
    """Small capacities force every long row through several relaunches and, past
    smem_cap_max, through column splitting or the level-1 sequence."""
    A = gen.rmat(12, 16, seed=7)
    plan, C = run(spg, A, A, initial_cap=initial_cap, smem_cap_max=smem_cap_max, merge_batch=batch,
                  long_rows=long_rows, dense_min_u=-1)
    check(oracle_mod, A, A, C, label=f"cap{initial_cap}/{smem_cap_max}/{batch}/{long_rows}")
    st = plan.stats()
    assert st["merge_rounds"] >= 2 and st["rows_relaunched"] > 0
    if smem_cap_max and smem_cap_max <= 1024:
        if long_rows == "split":
            assert st["rows_split"] > 0 and st["rows_level1"] == 0
        else:
            assert st["rows_level1"] > 0 and st["rows_split"] == 0


def _rows_with_u(targets, ncols_b, seed, dup=False):
    """A (len(targets) rows) and B such that row i of A*B has exactly targets[i] products.
    B row k has length k+1 (k < 600); dup=True makes every B row use the same columns, so many
    products collide (all-duplicates rows)."""
    rng = np.random.default_rng(seed)
    nb = 600
    rows, cols = [], []
    for k in range(nb):
        L = k + 1
        c = np.arange(L) if dup else np.sort(rng.choice(ncols_b, size=L, replace=False))
        rows.append(np.full(L, k))
        cols.append(c)
    B = gen.from_coo(nb, ncols_b, np.concatenate(rows), np.concatenate(cols), None)
    B.val = rng.uniform(-1, 1, B.nnz)
    ar, ac = [], []
    for i, t in enumerate(targets):
        # greedy: pick distinct B rows whose lengths sum to t
        left, k = t, nb - 1
        picked = []
        while left > 0:
            k = min(k, left - 1)
            picked.append(k)
            left -= k + 1
            k -= 1
        ar += [i] * len(picked)
        ac += picked
    A = gen.from_coo(len(targets), nb, np.array(ar, dtype=np.int64), np.array(ac, dtype=np.int64), None)
    A.val = rng.uniform(-1, 1, A.nnz)
    return A, B


def test_config2_level1_mode(spg, oracle_mod):
    A = gen.rmat(16, 16, seed=1)
    plan, C = run(spg, A, A, rowptr_dtype=torch.int32, long_rows="level1")
    check(oracle_mod, A, A, C, label="cfg2-level1")
    assert plan.stats()["rows_level1"] > 0


@pytest.mark.parametrize("dup", [False, True])
def test_bin_edges(spg, oracle_mod, dup):
    targets = [0, 1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513,
               1000, 4096, 20000, 70000]
    A, B = _rows_with_u(targets, 3000, seed=11, dup=dup)
    u = oracle_mod.upper_bound(A, B)
    assert u.tolist() == targets
    for policy in ("hybrid", "upper_bound"):
        plan, C = run(spg, A, B, alloc_policy=policy)
        check(oracle_mod, A, B, C, label=f"edges dup={dup} {policy}")


def test_rectangular_empty_and_degenerate(spg, oracle_mod):
    cases = [
        (gen.random_sparse(50, 70, 0.1, 1, empty_rows=0.3), gen.random_sparse(70, 40, 0.1, 2, empty_rows=0.3)),
        (gen.random_sparse(1, 1, 1.0, 3), gen.random_sparse(1, 1, 1.0, 4)),
        (gen.random_sparse(30, 20, 0.0, 5), gen.random_sparse(20, 30, 0.2, 6)),     # A empty
        (gen.random_sparse(30, 20, 0.2, 7), gen.random_sparse(20, 30, 0.0, 8)),     # B empty
        (gen.random_sparse(0, 20, 0.2, 9), gen.random_sparse(20, 30, 0.2, 10)),     # no rows
        (gen.random_sparse(25, 0, 0.2, 11), gen.random_sparse(0, 30, 0.2, 12)),     # inner dim 0
        (gen.random_sparse(25, 20, 0.3, 13), gen.random_sparse(20, 0, 0.2, 14)),    # no columns
        (gen.random_sparse(300, 5000, 0.01, 15), gen.random_sparse(5000, 3, 0.5, 16)),  # long A rows
    ]
    for i, (A, B) in enumerate(cases):
        for rdt in (torch.int32, torch.int64):
            plan, C = run(spg, A, B, rowptr_dtype=rdt)
            check(oracle_mod, A, B, C, label=f"case{i}")


def test_integer_values_bit_exact(spg, oracle_mod):
    A = gen.random_sparse(400, 300, 0.05, 21, integer_values=True)
    B = gen.random_sparse(300, 500, 0.08, 22, integer_values=True)
    _, C = run(spg, A, B)
    check(oracle_mod, A, B, C, exact=True, label="int")


def test_cancellation_keeps_structural_zeros(spg, oracle_mod):
    # A = [[1, 1], [0, 3]], B = [[2, 0], [-2, 1]]: c_00 = 1*2 + 1*(-2) = 0 stays a structural entry
    A = gen.from_coo(2, 2, np.array([0, 0, 1]), np.array([0, 1, 1]), np.array([1.0, 1.0, 3.0]))
    B = gen.from_coo(2, 2, np.array([0, 1, 1]), np.array([0, 0, 1]), np.array([2.0, -2.0, 1.0]))
    _, C = run(spg, A, B)
    rp, col, val = C.to_host()
    assert rp.tolist() == [0, 2, 4] and col.tolist() == [0, 1, 0, 1]
    assert val.tolist() == [0.0, 1.0, -6.0, 3.0]


def test_check_inputs_rejects_malformed(spg):
    good = gen.random_sparse(20, 20, 0.2, 1)
    for mutate in ("unsorted", "duplicate", "out_of_range"):
        bad = gen.HostCSR(good.nrows, good.ncols, good.row_ptr.copy(), good.col.copy(), good.val.copy())
        r = int(np.argmax(np.diff(bad.row_ptr) >= 2))
        s = int(bad.row_ptr[r])
        if mutate == "unsorted":
            bad.col[s], bad.col[s + 1] = bad.col[s + 1], bad.col[s]
        elif mutate == "duplicate":
            bad.col[s + 1] = bad.col[s]
        else:
            bad.col[s] = 20 + 5
        Ad = spg.CSR.from_host(bad)
        Bd = spg.CSR.from_host(good)
        with pytest.raises(spg.SpgemmError) as ei:
            spg.Plan(Ad, Bd, check_inputs=True)
        assert ei.value.code == 3
    with pytest.raises(ValueError):
        spg.spgemm(spg.CSR.from_host(good), spg.CSR.from_host(gen.random_sparse(21, 20, 0.2, 2)))


def test_repeat_is_structurally_identical(spg, oracle_mod):
    A = gen.rmat(11, 16, seed=9)
    _, C1 = run(spg, A, A)
    _, C2 = run(spg, A, A)
    r1, c1, v1 = C1.to_host()
    r2, c2, v2 = C2.to_host()
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
    ref = oracle_mod.spgemm(A, A)
    assert np.all(np.abs(v1 - v2) <= 2 * REL_TOL * ref.den)


@pytest.mark.parametrize("dense", [True, False])
def test_config2_rmat16_full(spg, oracle_mod, dense):
    """R-MAT 2^16 rows, 16 samples/row, A*A: every bin group; with the dense-slice rows, or
    with every bin-37 row through the progressive rounds and column splits."""
    A = gen.rmat(16, 16, seed=1)
    plan, C = run(spg, A, A, rowptr_dtype=torch.int32, record_timing=True, dense_min_u=0 if dense else -1)
    check(oracle_mod, A, A, C, label=f"cfg2 dense={dense}")
    st = plan.stats()
    if dense:
        assert st["rows_dense"] > 0 and st["dense_slices"] >= 1 and st["merge_rounds"] >= 1
    else:
        assert st["merge_rounds"] >= 3 and st["rows_split"] > 0 and st["rows_dense"] == 0
    assert all(st["bin_count"][b] > 0 for b in (0, 1, 2, 33, 34, 35, 36, 37))
    plan.check()


def test_config3_galerkin_closed_form(spg, oracle_mod):
    g = 64
    A = gen.lap3d27(g)
    P = gen.agg_P(g)
    R = gen.transpose(P)
    Ad, Pd, Rd = (spg.CSR.from_host(M, rowptr_dtype=torch.int32) for M in (A, P, R))
    AP = spg.spgemm(Ad, Pd)
    assert AP.nnz == 126 ** 3
    Ac = spg.spgemm(Rd, AP)
    torch.cuda.synchronize()
    assert Ac.nnz == 94 ** 3
    rp, col, val = Ac.to_host()
    assert set(np.unique(val).tolist()) == {152.0, -16.0, -4.0, -1.0}
    RA = spg.spgemm(Rd, Ad)
    Ac2 = spg.spgemm(RA, Pd)
    rp2, col2, val2 = Ac2.to_host()
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2) and np.array_equal(val, val2)
    # exact against the oracle too
    APh = oracle_mod.spgemm(A, P)
    ref = oracle_mod.spgemm(R, gen.HostCSR(APh.nrows, APh.ncols, APh.row_ptr, APh.col, APh.val))
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col) and np.array_equal(val, ref.val)


@pytest.mark.parametrize("policy", ["hybrid", "learned"])
def test_temporaries_released_after_numeric(spg, oracle_mod, policy):
    """C~, the merge pools and the stage-1/2 scratch are released when the product returns:
    the plan then holds C plus O(rows) tables, below its peak; a later product on the same
    stream reuses that memory and the first result stays intact."""
    from paper_1504_05022_gb300.predictor import Predictor
    A = gen.rmat(12, 16, seed=3)
    opts = Predictor.load().opts() if policy == "learned" else {"alloc_policy": policy}
    plan, C = run(spg, A, A, initial_cap=256, **opts)
    st = plan.stats()
    m = A.nrows
    c_bytes = C.nnz * 12 + (m + 1) * 8
    assert st["peak_bytes"] > st["held_bytes"] >= c_bytes
    assert st["held_bytes"] - c_bytes < 64 * m + (1 << 20) + 8 * A.nnz
    plan2, C2 = run(spg, A, A, **opts)  # allocates from the released memory
    check(oracle_mod, A, A, C, label=f"first result after release/{policy}")
    assert torch.equal(C.col, C2.col)


@pytest.mark.parametrize("heap_max_u", [2, 8, 17, 32])
def test_heap_esc_boundary(spg, oracle_mod, heap_max_u):
    """Rows of bins heap_max_u+1..32 go to the bitonic ESC kernel with 32 slots instead of the
    heap kernel: same structure and values within tolerance, and replay agrees."""
    A = gen.erdos_renyi(3000, 5, seed=4)   # u_i spread over bins 2..64
    plan, C = run(spg, A, A, heap_max_u=heap_max_u)
    ref = check(oracle_mod, A, A, C, label=f"heap_max_u={heap_max_u}")
    bins = plan.arrays()["bin"]
    assert ((bins >= 2) & (bins <= 32)).sum() > 1000
    st = plan.stats()
    if heap_max_u < 32:
        assert st["launches"]["esc"] >= 1
    plan.replay()
    torch.cuda.synchronize()
    check(oracle_mod, A, A, C, label=f"replay heap_max_u={heap_max_u}")
    del ref


def test_autotune_smoke(spg):
    """The tuner runs on a small product, keeps the memory bound and returns values of its space."""
    from paper_1504_05022_gb300 import autotune
    A = gen.rmat(11, 8, seed=5)
    runner = autotune.Runner([(A, A)])
    rec = autotune.tune(runner, "hybrid", rounds=1, reps=1, log=lambda *_: None)
    for k, v in rec["params"].items():
        assert v in autotune.SPACE[k]
    assert rec["ms"] <= rec["default_ms"]


@pytest.mark.parametrize("wide_above,smem_cap_max,policy", [(4096, 0, "hybrid"), (1 << 20, 0, "hybrid"),
                                                           (6144, 6144, "hybrid"), (1 << 20, 0, "learned")])
def test_merge_cta_width(spg, oracle_mod, wide_above, smem_cap_max, policy):
    """256-thread merge CTAs for larger result capacities (merge_wide_above) give the same C."""
    from paper_1504_05022_gb300.predictor import Predictor
    A = gen.rmat(13, 16, seed=31)
    keep = Predictor.load() if policy == "learned" else None
    opts = keep.opts() if keep else {"alloc_policy": policy}
    plan, C = run(spg, A, A, merge_wide_above=wide_above, smem_cap_max=smem_cap_max, dense_min_u=-1, **opts)
    check(oracle_mod, A, A, C, label=f"wide_above={wide_above}/{smem_cap_max}/{policy}")
    assert plan.stats()["bin_count"][37] > 0


@pytest.mark.parametrize("kernel", ["merge_path", "bitmap"])
@pytest.mark.parametrize("policy,initial_cap,smem_cap_max,batch,miss", [
    ("hybrid", 256, 0, 0, 0), ("hybrid", 64, 1024, 256, 256), ("learned", 256, 0, 0, 0),
    ("upper_bound", 256, 2048, 512, 512)])
def test_merge_kernel_forms(spg, oracle_mod, kernel, policy, initial_cap, smem_cap_max, batch, miss):
    """Both forms of the bin-37 kernel (merge-path and bitmap/rank) give the oracle's C,
    with progressive rounds, column splits and small miss buffers forced."""
    from paper_1504_05022_gb300.predictor import Predictor
    A = gen.rmat(13, 16, seed=41)
    keep = Predictor.load() if policy == "learned" else None
    opts = keep.opts() if keep else {"alloc_policy": policy}
    plan, C = run(spg, A, A, merge_kernel=kernel, initial_cap=initial_cap, smem_cap_max=smem_cap_max,
                  merge_batch=batch, merge_miss=miss, dense_min_u=-1, **opts)
    check(oracle_mod, A, A, C, label=f"{kernel}/{policy}/{initial_cap}/{smem_cap_max}/{miss}")
    st = plan.stats()
    assert st["bin_count"][37] > 0
    if smem_cap_max:
        assert st["rows_split"] > 0
    plan.check()


def test_bitmap_kernel_rectangular_and_split_children(spg, oracle_mod):
    """Bitmap form on a rectangular B (bitmap sized by B's columns) and on column slices
    whose origin is not 0."""
    A = gen.rmat(12, 24, seed=43)
    B = gen.erdos_renyi(4096, 12, seed=44, ncols=70000)
    plan, C = run(spg, A, B, merge_kernel="bitmap", smem_cap_max=1024, merge_batch=512, merge_miss=512,
                  dense_min_u=-1)
    check(oracle_mod, A, B, C, label="bitmap rectangular")
    assert plan.stats()["rows_split"] > 0


@pytest.mark.parametrize("policy,smem_cap_max", [("hybrid", 0), ("learned", 0), ("hybrid", 1024)])
def test_bitmap_kernel_wide_b_two_level(spg, oracle_mod, policy, smem_cap_max):
    """B with more columns than the flat bitmap holds: the two-level index (occupied
    32-column words, then their bits) gives the oracle's C, with splits forced too."""
    from paper_1504_05022_gb300.predictor import Predictor
    A = gen.rmat(12, 16, seed=51)
    B = gen.erdos_renyi(4096, 24, seed=52, ncols=300000)
    keep = Predictor.load() if policy == "learned" else None
    opts = keep.opts() if keep else {"alloc_policy": policy}
    plan, C = run(spg, A, B, smem_cap_max=smem_cap_max, merge_kernel="bitmap", dense_min_u=-1, **opts)
    check(oracle_mod, A, B, C, label=f"wide B/{policy}/{smem_cap_max}")
    st = plan.stats()
    assert st["bin_count"][37] > 0
    if smem_cap_max:
        assert st["rows_split"] > 0
    plan.replay()
    torch.cuda.synchronize()
    plan.check()
    check(oracle_mod, A, B, C, label=f"wide B replay/{policy}")


def test_bitmap_kernel_two_level_rmat(spg, oracle_mod):
    """Two-level index on an R-MAT product with 2^18 columns (hub rows, splits)."""
    A = gen.rmat(18, 4, seed=53)
    plan, C = run(spg, A, A, merge_kernel="bitmap", dense_min_u=-1)
    check(oracle_mod, A, A, C, label="two-level R-MAT 2^18")
    assert plan.stats()["bin_count"][37] > 0


def test_pool_trim_returns_memory_and_products_stay_exact(spg, oracle_mod):
    """The library's pool keeps freed blocks; pool_trim hands them back to the system, and the
    next product (which maps fresh memory) is still the oracle's."""
    A = gen.rmat(13, 16, seed=81)
    Ad = spg.CSR.from_host(A)
    C = spg.spgemm(Ad, Ad)
    check(oracle_mod, A, A, C, label="before trim")
    del C
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    spg.pool_trim()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0
    C = spg.spgemm(Ad, Ad)
    check(oracle_mod, A, A, C, label="after trim")
