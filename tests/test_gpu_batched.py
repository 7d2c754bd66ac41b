"""Batched products, values-only replay, CUDA graphs and the Galerkin chain, against the
CPU oracle (structure bit-exact, values within 1e-12 * sum |a b|; integer stencils exact)."""
import ctypes

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


def _check(oracle_mod, A, B, C, label):
    ref = oracle_mod.spgemm(A, B)
    rp, col, val = C.to_host()
    assert C.shape == (A.nrows, B.ncols)
    assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, label=label)


@pytest.mark.parametrize("policy", ["hybrid", "upper_bound"])
def test_batched_matches_oracle(spg, oracle_mod, policy):
    pairs = gen.batch_pairs(40, m_lo=16, m_hi=3000, seed0=100)
    pairs.append((gen.random_sparse(0, 5, 0.2, 1), gen.random_sparse(5, 7, 0.2, 2)))   # a pair without rows
    pairs.append((gen.random_sparse(9, 4, 0.0, 3), gen.random_sparse(4, 6, 0.3, 4)))   # a pair without products
    As = [spg.CSR.from_host(A) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B, rowptr_dtype=torch.int32) for _, B in pairs]
    Cs = spg.spgemm_batched(As, Bs, alloc_policy=policy)
    torch.cuda.synchronize()
    assert len(Cs) == len(pairs)
    for i, ((A, B), C) in enumerate(zip(pairs, Cs)):
        _check(oracle_mod, A, B, C, f"pair {i}")


def test_batched_equals_sequential(spg):
    pairs = gen.batch_pairs(12, m_lo=500, m_hi=5000, seed0=7)
    As = [spg.CSR.from_host(A) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B) for _, B in pairs]
    Cs = spg.spgemm_batched(As, Bs)
    for A, B, C in zip(As, Bs, Cs):
        D = spg.spgemm(A, B)
        torch.cuda.synchronize()
        assert torch.equal(C.row_ptr, D.row_ptr) and torch.equal(C.col, D.col)
        assert torch.allclose(C.val, D.val, rtol=1e-12, atol=1e-12)


def _scaled(M, seed):
    rng = np.random.default_rng(seed)
    return gen.HostCSR(M.nrows, M.ncols, M.row_ptr, M.col, M.val * rng.uniform(0.5, 2.0, M.nnz))


@pytest.mark.parametrize("policy", ["hybrid", "learned"])
def test_replay_recomputes_values(spg, oracle_mod, policy):
    from paper_1504_05022_gb300.predictor import Predictor
    A = gen.rmat(13, 16, seed=11)
    Ad = spg.CSR.from_host(A)
    keep = None
    opts = {"alloc_policy": policy}
    if policy == "learned":
        keep = Predictor.load()
        opts = keep.opts()
    plan = spg.Plan(Ad, Ad, smem_cap_max=2048, dense_min_u=-1, **opts)   # small capacity: many column splits
    C = plan.numeric()
    torch.cuda.synchronize()
    assert plan.stats()["rows_split"] > 0
    for r in range(2):
        A2 = _scaled(A, 50 + r)
        Ad.val.copy_(torch.from_numpy(A2.val))
        plan.replay()
        torch.cuda.synchronize()
        plan.check()
        _check(oracle_mod, A2, A2, C, f"replay {r}")
    del keep


def test_batched_replay(spg, oracle_mod):
    pairs = gen.batch_pairs(10, m_lo=100, m_hi=4000, seed0=3)
    As = [spg.CSR.from_host(A) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B) for _, B in pairs]
    plan = spg.BatchPlan(As, Bs)
    Cs = plan.numeric()
    new = [(_scaled(A, 2 * i), _scaled(B, 2 * i + 1)) for i, (A, B) in enumerate(pairs)]
    for (A2, B2), Ad, Bd in zip(new, As, Bs):
        Ad.val.copy_(torch.from_numpy(A2.val))
        Bd.val.copy_(torch.from_numpy(B2.val))
    plan.replay()
    torch.cuda.synchronize()
    plan.check()
    for i, ((A2, B2), C) in enumerate(zip(new, Cs)):
        _check(oracle_mod, A2, B2, C, f"batched replay {i}")


def _int_values(M, seed, lo=-3, hi=4):
    """M with new small nonzero integer values drawn from the seed (same structure), so every
    product and sum is exact in FP64."""
    rng = np.random.default_rng(seed)
    v = rng.integers(lo, hi, size=M.nnz).astype(np.float64)
    v[v == 0] = 5.0
    return gen.HostCSR(M.nrows, M.ncols, M.row_ptr, M.col, v)


def test_galerkin_graph_exact(spg, oracle_mod):
    """R*(A*P) on the 27-point 32^3 operator, then its values-only replay from one CUDA graph for
    new integer values of R, A and P (the same structure): each replay equals the oracle's
    R*(A*P) of those values exactly."""
    g = 32
    A, P = gen.lap3d27(g), gen.agg_P(g)
    R = gen.transpose(P)
    s = torch.cuda.Stream()
    Ad, Pd, Rd = (spg.CSR.from_host(M) for M in (A, P, R))
    with torch.cuda.stream(s):
        Ac, p1, p2 = spg.galerkin(Rd, Ad, Pd, stream=s)
    s.synchronize()
    rp, col, val = Ac.to_host()
    assert Ac.nnz == (3 * (g // 2) - 2) ** 3
    assert set(np.unique(val).tolist()) == {152.0, -16.0, -4.0, -1.0}
    graph = spg.ReplayGraph([p1, p2])
    for k in range(3):
        A2, P2, R2 = _int_values(A, 100 + k), _int_values(P, 200 + k), _int_values(R, 300 + k)
        for Md, M2 in ((Ad, A2), (Pd, P2), (Rd, R2)):
            Md.val.copy_(torch.from_numpy(M2.val))
        s.synchronize()
        graph.launch()
        s.synchronize()
        AP = oracle_mod.spgemm(A2, P2)
        ref = oracle_mod.spgemm(R2, gen.HostCSR(AP.nrows, AP.ncols, AP.row_ptr, AP.col, AP.val))
        rp2, col2, val2 = Ac.to_host()
        assert np.array_equal(rp2, ref.row_ptr) and np.array_equal(col2, ref.col)
        assert np.array_equal(val2, ref.val), f"replay {k}"    # integers: exact
    p2.check()


def test_galerkin_c_entry_point(spg):
    from paper_1504_05022_gb300 import _lib
    L = _lib.load()
    g = 16
    A, P = gen.lap3d27(g), gen.agg_P(g)
    R = gen.transpose(P)
    Ad, Pd, Rd = (spg.CSR.from_host(M) for M in (A, P, R))
    ins = [M._c_in() for M in (Rd, Ad, Pd)]
    p1, p2 = ctypes.c_void_p(), ctypes.c_void_p()
    out = _lib.CsrOut()
    rc = L.spgemm_galerkin(ctypes.byref(ins[0]), ctypes.byref(ins[1]), ctypes.byref(ins[2]), None,
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(p1),
                           ctypes.byref(p2), ctypes.byref(out))
    assert rc == 0
    torch.cuda.synchronize()
    assert out.nnz == (3 * (g // 2) - 2) ** 3
    import importlib
    mod = importlib.import_module("paper_1504_05022_gb300.spgemm")
    vals = torch.as_tensor(mod._PlanArray(out.val, out.nnz, "<f8", None, 0), device="cuda").cpu().numpy()
    assert set(np.unique(vals).tolist()) == {152.0, -16.0, -4.0, -1.0}
    L.spgemm_free(p2)
    L.spgemm_free(p1)


def test_replay_refused_for_level1(spg):
    A = gen.rmat(12, 16, seed=7)
    Ad = spg.CSR.from_host(A)
    plan = spg.Plan(Ad, Ad, smem_cap_max=256, long_rows="level1")
    plan.numeric()
    with pytest.raises(spg.SpgemmError) as ei:
        plan.replay()
    assert ei.value.code == 1


def _greedy_waves(prods, budget):
    starts, acc = [0], 0
    for i, p in enumerate(sorted(prods, reverse=True)):
        if acc > 0 and acc + p > budget:
            starts.append(i)
            acc = 0
        acc += p
    return len(starts)


@pytest.mark.parametrize("policy", ["hybrid", "learned"])
def test_batched_waves(spg, oracle_mod, policy):
    """Pairs grouped into waves of at most 1M products: same results as the oracle, the
    waves the greedy grouping gives, a peak no higher than one wave over all pairs, and
    values-only replay of every wave captured in one CUDA graph."""
    from paper_1504_05022_gb300.predictor import Predictor
    pairs = gen.batch_pairs(24, m_lo=200, m_hi=6000, seed0=300)
    prods = [int(np.diff(B.row_ptr)[A.col].sum()) for A, B in pairs]
    keep = Predictor.load() if policy == "learned" else None
    opts = keep.opts() if keep else {"alloc_policy": policy}
    s = torch.cuda.Stream()
    As = [spg.CSR.from_host(A) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B, rowptr_dtype=torch.int32) for _, B in pairs]
    torch.cuda.synchronize()
    plan = spg.BatchPlan(As, Bs, stream=s, wave_mproducts=1, **opts)
    assert plan.upper_bound_nnz == sum(prods)
    assert plan.n_waves == _greedy_waves(prods, 1_000_000) > 1
    Cs = plan.numeric()
    s.synchronize()
    for i, ((A, B), C) in enumerate(zip(pairs, Cs)):
        _check(oracle_mod, A, B, C, f"wave pair {i}")
    st = plan.stats()
    assert st["sum_u"] == sum(prods) and st["nnz_c"] == sum(C.nnz for C in Cs)
    one = spg.BatchPlan(As, Bs, stream=s, wave_mproducts=-1, **opts)
    assert one.n_waves == 1
    one.numeric()
    s.synchronize()
    assert st["peak_bytes"] <= one.stats()["peak_bytes"]
    ar = plan.arrays()
    order = plan.pair_order()
    assert sorted(order) == list(range(len(pairs)))
    assert all(prods[order[q]] >= prods[order[q + 1]] for q in range(len(pairs) - 1))
    assert ar["u"].shape[0] == sum(pairs[i][0].nrows for i in order) and ar["u"].sum() == sum(prods)
    new = [(_scaled(A, 7 * i), _scaled(B, 7 * i + 1)) for i, (A, B) in enumerate(pairs)]
    for (A2, B2), Ad, Bd in zip(new, As, Bs):
        Ad.val.copy_(torch.from_numpy(A2.val))
        Bd.val.copy_(torch.from_numpy(B2.val))
    torch.cuda.synchronize()
    g = spg.ReplayGraph([plan])
    g.launch()
    s.synchronize()
    plan.check()
    for i, ((A2, B2), C) in enumerate(zip(new, Cs)):
        _check(oracle_mod, A2, B2, C, f"wave replay {i}")
    del g, keep


@pytest.mark.parametrize("stencil,g,dim", [("lap2d9", 256, 2), ("lap3d7", 32, 3), ("lap3d27", 32, 3)])
@pytest.mark.parametrize("policy", ["hybrid", "learned"])
def test_galerkin_hierarchy_exact(spg, oracle_mod, stencil, g, dim, policy):
    """A piecewise-constant aggregation hierarchy A_{l+1} = P_l^T (A_l P_l) down to a 4^dim grid,
    each level's product fed by the previous one on the device: every level equals the oracle's
    exactly (integer-valued operators), and all levels' plans replayed from one CUDA graph after
    scaling the finest operator scale every level."""
    from paper_1504_05022_gb300.predictor import Predictor
    A = getattr(gen, stencil)(g)
    Ps = gen.galerkin_levels(g, dim)
    opts = Predictor.load().opts() if policy == "learned" else {"alloc_policy": policy}
    s = torch.cuda.Stream()
    Ad = spg.CSR.from_host(A)
    cur, plans, levels, keep = Ad, [], [], []
    with torch.cuda.stream(s):
        for P in Ps:
            Pd, Rd = spg.CSR.from_host(P), spg.CSR.from_host(gen.transpose(P))
            cur, p1, p2 = spg.galerkin(Rd, cur, Pd, stream=s, **opts)
            plans += [p1, p2]
            levels.append(cur)
            keep += [Pd, Rd]
    s.synchronize()
    ref, host = A, []
    for P, Ac in zip(Ps, levels):
        AP = oracle_mod.spgemm(ref, P)
        Rc = oracle_mod.spgemm(gen.transpose(P), gen.HostCSR(AP.nrows, AP.ncols, AP.row_ptr, AP.col, AP.val))
        rp, col, val = Ac.to_host()
        assert np.array_equal(rp, Rc.row_ptr) and np.array_equal(col, Rc.col) and np.array_equal(val, Rc.val)
        host.append((rp, col, val))
        ref = gen.HostCSR(Rc.nrows, Rc.ncols, Rc.row_ptr, Rc.col, Rc.val)
    assert levels[-1].shape == (4 ** dim, 4 ** dim)
    graph = spg.ReplayGraph(plans)
    for scale in (2.0, -3.0):
        Ad.val.copy_(torch.from_numpy(A.val * scale))
        s.synchronize()
        graph.launch()
        s.synchronize()
        for Ac, (rp, col, val) in zip(levels, host):
            rp2, col2, val2 = Ac.to_host()
            assert np.array_equal(col2, col) and np.array_equal(val2, val * scale)
    for p in plans:
        p.check()
