"""The precise method (Section 3.1) and the products sized on the device, against the oracle.

- alloc_policy="precise": every row counted first, C allocated exactly, every row computed
  straight into it (no temporary matrix C~): structure bit-exact, values within 1e-12 * den,
  integer stencils exact.
- DevicePlan / DeviceGraph: the whole product (stages 1-4) enqueued with every size on the
  device, run again on new contents of the same input arrays -- new values and new structure
  of the same sizes -- and captured in one CUDA graph with a chained second product (the
  Galerkin chain R*(A*P) of the 27-point operator on a 64^3 grid)."""
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


def _check(oracle_mod, A, B, C, label, exact=False):
    ref = oracle_mod.spgemm(A, B)
    rp, col, val = C.to_host()
    assert C.shape == (A.nrows, B.ncols), label
    assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, exact=exact, label=label)
    return ref


def _permuted(M, seed, rows=True, cols=True):
    """P_r M P_c for random permutations: the same number of entries (and of rows and columns),
    another structure.  Columns sorted within rows."""
    rng = np.random.default_rng(seed)
    r = np.repeat(np.arange(M.nrows, dtype=np.int64), np.diff(M.row_ptr))
    c = M.col.astype(np.int64)
    if rows:
        r = rng.permutation(M.nrows)[r]
    if cols:
        c = rng.permutation(M.ncols)[c]
    return gen.from_coo(M.nrows, M.ncols, r, c, rng.uniform(-1, 1, M.nnz))


def _load_into(Md, M):
    """Copies host matrix M into the device arrays of Md (same sizes)."""
    Md.row_ptr.copy_(torch.from_numpy(np.ascontiguousarray(M.row_ptr)).to(Md.row_ptr.dtype))
    Md.col.copy_(torch.from_numpy(np.ascontiguousarray(M.col, dtype=np.int32)))
    Md.val.copy_(torch.from_numpy(np.ascontiguousarray(M.val)).to(Md.val.dtype))


@pytest.mark.parametrize("name", ["lap2d64", "rmat12x16", "rmat13x8", "banded", "rect"])
def test_precise_policy_matches_oracle(spg, oracle_mod, name):
    if name == "lap2d64":
        A = B = gen.lap2d(64)
    elif name == "rmat12x16":
        A = B = gen.rmat(12, 16, seed=31)
    elif name == "rmat13x8":
        A = B = gen.rmat(13, 8, seed=32)
    elif name == "banded":
        A = B = gen.banded(3000, 40, seed=33)
    else:
        A = gen.rmat(12, 24, seed=34)
        B = gen.erdos_renyi(4096, 30, seed=35, ncols=70001)
    Ad = spg.CSR.from_host(A, rowptr_dtype=torch.int32)
    Bd = Ad if B is A else spg.CSR.from_host(B)
    plan = spg.Plan(Ad, Bd, alloc_policy="precise")
    C = plan.numeric()
    torch.cuda.synchronize()
    _check(oracle_mod, A, B, C, f"precise {name}", exact=name == "lap2d64")
    st = plan.stats()
    assert st["nnz_ctilde"] == 0 and st["bytes_ctilde"] == 0   # no temporary matrix
    assert st["rows_dense"] == st["bin_count"][37]              # every bin-37 row by the column slices
    assert st["merge_rounds"] == 0 and st["rows_relaunched"] == 0
    plan.check()


def test_precise_peak_is_inputs_free_result_plus_tables(spg, oracle_mod):
    """The plan's high-water mark is C plus O(rows) tables: below the hybrid plan's."""
    A = gen.rmat(14, 16, seed=36)
    Ad = spg.CSR.from_host(A)
    peaks = {}
    for pol in ("precise", "hybrid"):
        plan = spg.Plan(Ad, Ad, alloc_policy=pol)
        C = plan.numeric()
        torch.cuda.synchronize()
        peaks[pol] = plan.stats()["peak_bytes"]
        if pol == "precise":
            _check(oracle_mod, A, A, C, "precise rmat14")
            c_bytes = C.nnz * 12 + (A.nrows + 1) * 8
            assert c_bytes <= peaks[pol] <= c_bytes + 80 * A.nrows + 16 * A.nnz + (64 << 20)
    assert peaks["precise"] < peaks["hybrid"]


def test_precise_replay(spg, oracle_mod):
    A = gen.rmat(12, 16, seed=37)
    Ad = spg.CSR.from_host(A)
    plan = spg.Plan(Ad, Ad, alloc_policy="precise")
    C = plan.numeric()
    rng = np.random.default_rng(38)
    A2 = gen.HostCSR(A.nrows, A.ncols, A.row_ptr, A.col, rng.uniform(-2, 2, A.nnz))
    Ad.val.copy_(torch.from_numpy(A2.val))
    plan.replay()
    torch.cuda.synchronize()
    plan.check()
    _check(oracle_mod, A2, A2, C, "precise replay")


def test_precise_rejects_too_wide_b(spg):
    A = gen.erdos_renyi(64, 4, seed=39, ncols=64)
    B = gen.erdos_renyi(64, 4, seed=40, ncols=9_000_000)  # beyond 64 slices of 131,072 columns
    with pytest.raises(spg.SpgemmError, match="SHAPE"):
        spg.Plan(spg.CSR.from_host(A), spg.CSR.from_host(B), alloc_policy="precise")


def test_device_plan_runs_on_new_structure(spg, oracle_mod):
    """One DevicePlan, three runs: the first matrix, then two matrices with the same sizes and
    another structure (rows and columns permuted) written into the same input arrays."""
    A = gen.rmat(12, 16, seed=41)
    Ad = spg.CSR.from_host(A, rowptr_dtype=torch.int32)
    s = torch.cuda.Stream()
    cap = int(oracle_mod.upper_bound(A, A).sum())
    dp = spg.DevicePlan(Ad, Ad, cap, stream=s)
    for k, M in enumerate([A, _permuted(A, 42), _permuted(A, 43, rows=False)]):
        s.synchronize()
        _load_into(Ad, M)
        torch.cuda.synchronize()
        dp.run()
        C = dp.result()
        _check(oracle_mod, M, M, C, f"device plan run {k}")


def test_device_plan_capacity_exceeded(spg, oracle_mod):
    """A result larger than the capacity is reported and C is left empty (row pointers 0), so
    a chained product reads an empty matrix; the plan works again with a result that fits."""
    A = gen.rmat(11, 16, seed=44)
    Ad = spg.CSR.from_host(A)
    s = torch.cuda.Stream()
    nnz = int(oracle_mod.row_counts(A, A).sum())
    dp = spg.DevicePlan(Ad, Ad, nnz - 1, stream=s)
    dp2 = spg.DevicePlan(Ad, dp.as_input(), nnz, stream=s)
    dp.run()
    dp2.run()
    with pytest.raises(spg.SpgemmError, match="OOM"):
        dp.result()
    assert int(dp.as_input().row_ptr.abs().sum()) == 0
    C2 = dp2.result()
    assert C2.nnz == 0
    dp3 = spg.DevicePlan(Ad, Ad, nnz, stream=s)
    dp3.run()
    _check(oracle_mod, A, A, dp3.result(), "capacity exact")


def _int_values(M, seed):
    rng = np.random.default_rng(seed)
    v = rng.integers(-3, 4, size=M.nnz).astype(np.float64)
    v[v == 0] = 5.0
    return gen.HostCSR(M.nrows, M.ncols, M.row_ptr, M.col, v)


def _random_aggregation(g, seed):
    """A piecewise-constant prolongator with the shape and the entry count of agg_P(g) (one 1.0
    per fine row) that sends every fine point to a random aggregate: another structure."""
    n, nc = g ** 3, (g // 2) ** 3
    rng = np.random.default_rng(seed)
    return gen.from_coo(n, nc, np.arange(n, dtype=np.int64), rng.integers(0, nc, n).astype(np.int64),
                        np.ones(n))


def test_galerkin_chain_in_one_graph_from_fresh_inputs(spg, oracle_mod):
    """R*(A*P) for the 27-point operator on a 64^3 grid, both products -- stages 1-4 each, every
    size on the device -- captured in one CUDA graph before anything was computed, launched,
    and compared with the oracle exactly (integer values).  Then the same graph on new inputs
    written into the same arrays: new integer values, and a prolongator of another structure
    (random aggregates) with its transpose."""
    g = 64
    A, P = gen.lap3d27(g), gen.agg_P(g)
    R = gen.transpose(P)
    s = torch.cuda.Stream()
    Ad, Pd, Rd = (spg.CSR.from_host(M) for M in (A, P, R))
    cap = A.nnz  # nnz(A*P) <= sum_i u_i = nnz(A) (one entry per row of P), and nnz(Ac) <= nnz(A*P)
    p1, p2, graph = spg.galerkin_device(Rd, Ad, Pd, cap, cap, stream=s)
    cases = [(A, P, R), (_int_values(A, 50), _int_values(P, 51), _int_values(R, 52))]
    P3 = _random_aggregation(g, 53)
    cases.append((_int_values(A, 54), P3, _int_values(gen.transpose(P3), 55)))
    for k, (Ak, Pk, Rk) in enumerate(cases):
        s.synchronize()
        for Md, M in ((Ad, Ak), (Pd, Pk), (Rd, Rk)):
            _load_into(Md, M)
        torch.cuda.synchronize()
        graph.launch()
        Ac = p2.result()
        AP = oracle_mod.spgemm(Ak, Pk)
        ref = oracle_mod.spgemm(Rk, gen.HostCSR(AP.nrows, AP.ncols, AP.row_ptr, AP.col, AP.val))
        rp, col, val = Ac.to_host()
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col), f"chain {k}"
        assert np.array_equal(val, ref.val), f"chain {k}"          # integers: exact
        if k == 0:
            assert Ac.nnz == 94 ** 3


def test_batched_device_plan_in_a_graph(spg, oracle_mod):
    """A batch of pairs of uneven sizes as one device-sized product in one CUDA graph,
    relaunched on new values: every C_i against the oracle."""
    pairs = [gen.batch_pair(i) for i in (3, 17, 40, 77, 101, 130)]
    pairs = [(A, B) for A, B in pairs if A.nrows <= 20000][:4]
    assert len(pairs) >= 2
    As = [spg.CSR.from_host(A, rowptr_dtype=torch.int32) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B, rowptr_dtype=torch.int32) for _, B in pairs]
    cap = sum(int(oracle_mod.row_counts(A, B).sum()) for A, B in pairs)
    s = torch.cuda.Stream()
    dp = spg.DevicePlan(As, Bs, cap, stream=s)
    graph = spg.DeviceGraph([dp])
    for k in range(2):
        if k:
            rng = np.random.default_rng(60)
            new = []
            for (A, B), Ad_, Bd_ in zip(pairs, As, Bs):
                A2 = gen.HostCSR(A.nrows, A.ncols, A.row_ptr, A.col, rng.uniform(-1, 1, A.nnz))
                B2 = gen.HostCSR(B.nrows, B.ncols, B.row_ptr, B.col, rng.uniform(-1, 1, B.nnz))
                Ad_.val.copy_(torch.from_numpy(A2.val))
                Bd_.val.copy_(torch.from_numpy(B2.val))
                new.append((A2, B2))
            pairs = new
            torch.cuda.synchronize()
        graph.launch()
        Cs = dp.result()
        for i, ((A, B), C) in enumerate(zip(pairs, Cs)):
            _check(oracle_mod, A, B, C, f"batched device plan {k}/{i}")
