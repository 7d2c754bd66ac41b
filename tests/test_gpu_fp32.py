"""GPU parity of the single-precision library (libspgemm_f32.so, the paper's SpSGEMM):
the same C ABI with float values.  The oracle computes in FP64 from the inputs rounded to
float, so the only error left is the kernels' float arithmetic.  Structure must match
exactly; a value c_ij with k_ij products (k_ij = the pattern product's count, from the oracle
on all-ones matrices) must satisfy |c_ij - ref_ij| <= gamma_{k_ij + 1} * sum_k |a_ik b_kj|,
gamma_n = n u / (1 - n u), u = 2^-24: the standard bound for a sum of k rounded products in
any order (one rounding per product and per addition).  Integer-valued inputs are exact."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def spg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_05022_gb300 as spg
    spg.load_library()
    return spg


def _f32(M):
    return gen.HostCSR(M.nrows, M.ncols, M.row_ptr, M.col, M.val.astype(np.float32).astype(np.float64))


def _ones(M):
    return gen.HostCSR(M.nrows, M.ncols, M.row_ptr, M.col, np.ones(M.nnz))


def _check(oracle_mod, A, B, C, exact=False, label=""):
    """A, B: the float-rounded host inputs; C: the device result (float32 values)."""
    ref = oracle_mod.spgemm(A, B)
    cnt = oracle_mod.spgemm(_ones(A), _ones(B))
    rp, col, val = C.to_host()
    assert C.val.dtype == torch.float32 and C.shape == (A.nrows, B.ncols), label
    assert np.array_equal(rp, ref.row_ptr), f"{label}: row_ptr"
    assert np.array_equal(col, ref.col), f"{label}: col"
    v = val.astype(np.float64)
    if exact:
        assert np.array_equal(v, ref.val), f"{label}: values"
        return
    n = cnt.val + 1.0
    gamma = n * U32 / (1.0 - n * U32)
    bad = np.abs(v - ref.val) > gamma * ref.den
    assert not bad.any(), f"{label}: {int(bad.sum())} values outside the float bound"


def _run(spg, A, B, **opts):
    Ad = spg.CSR.from_host(A, dtype=torch.float32)
    Bd = Ad if B is A else spg.CSR.from_host(B, dtype=torch.float32)
    plan = spg.Plan(Ad, Bd, **opts)
    C = plan.numeric()
    torch.cuda.synchronize()
    return plan, C, Ad


def test_f32_library_is_the_one_running(spg):
    from paper_1504_05022_gb300 import _lib
    A = _f32(gen.rmat(10, 8, seed=3))
    plan, C, _ = _run(spg, A, A)
    assert plan.L is _lib.load(dtype="f32") and plan.L is not _lib.load()
    assert C.val.dtype == torch.float32


def test_f32_lap2d_exact(spg, oracle_mod):
    A = _f32(gen.lap2d(64))
    plan, C, _ = _run(spg, A, A)
    assert C.nnz == 51972
    _check(oracle_mod, A, A, C, exact=True, label="lap2d64 f32")


@pytest.mark.parametrize("policy", ["hybrid", "upper_bound", "learned"])
@pytest.mark.parametrize("dense", [0, -1])
def test_f32_rmat(spg, oracle_mod, policy, dense):
    """Every bin group, the dense-slice rows (or none), progressive rounds and splits."""
    from paper_1504_05022_gb300.predictor import Predictor
    A = _f32(gen.rmat(13, 16, seed=91))
    keep = Predictor.load(dtype="f32") if policy == "learned" else None
    opts = keep.opts() if keep else {"alloc_policy": policy}
    plan, C, _ = _run(spg, A, A, dense_min_u=dense, smem_cap_max=2048, **opts)
    _check(oracle_mod, A, A, C, label=f"rmat13 f32 {policy} dense={dense}")
    st = plan.stats()
    assert (st["rows_dense"] > 0) == (dense == 0)
    if dense < 0:
        assert st["rows_split"] > 0
    plan.check()


@pytest.mark.parametrize("kw", [{"merge_kernel": "merge_path"}, {"long_rows": "level1", "smem_cap_max": 1024}])
def test_f32_merge_forms(spg, oracle_mod, kw):
    A = _f32(gen.rmat(12, 16, seed=92))
    plan, C, _ = _run(spg, A, A, **kw)
    _check(oracle_mod, A, A, C, label=f"f32 {kw}")


def test_f32_rectangular_and_replay(spg, oracle_mod):
    A = _f32(gen.rmat(12, 24, seed=93))
    B = _f32(gen.erdos_renyi(4096, 30, seed=94, ncols=5001))
    Ad = spg.CSR.from_host(A, dtype=torch.float32)
    Bd = spg.CSR.from_host(B, dtype=torch.float32)
    plan = spg.Plan(Ad, Bd, dense_span=1024)
    C = plan.numeric()
    torch.cuda.synchronize()
    _check(oracle_mod, A, B, C, label="rect f32")
    assert plan.stats()["rows_dense"] > 0
    rng = np.random.default_rng(95)
    A2 = _f32(gen.HostCSR(A.nrows, A.ncols, A.row_ptr, A.col, A.val * rng.uniform(0.5, 2.0, A.nnz)))
    Ad.val.copy_(torch.from_numpy(A2.val.astype(np.float32)))
    plan.replay()
    torch.cuda.synchronize()
    plan.check()
    _check(oracle_mod, A2, B, C, label="rect f32 replay")


def test_f32_batched(spg, oracle_mod):
    pairs = []
    for i, (m, ncols) in enumerate([(2048, 6000), (1024, 2500), (512, 700)]):
        pairs.append((_f32(gen.rmat(int(np.log2(m)), 16, seed=96 + i)),
                      _f32(gen.erdos_renyi(m, 24, seed=99 + i, ncols=ncols))))
    As = [spg.CSR.from_host(A, dtype=torch.float32) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B, dtype=torch.float32) for _, B in pairs]
    Cs = spg.spgemm_batched(As, Bs)
    torch.cuda.synchronize()
    for i, ((A, B), C) in enumerate(zip(pairs, Cs)):
        _check(oracle_mod, A, B, C, label=f"batched f32 {i}")


def test_value_types_must_match(spg):
    from paper_1504_05022_gb300.predictor import Predictor
    A = gen.rmat(8, 4, seed=5)
    A64 = spg.CSR.from_host(A)
    A32 = spg.CSR.from_host(A, dtype=torch.float32)
    with pytest.raises(TypeError):
        spg.Plan(A64, A32)
    with pytest.raises(TypeError):
        spg.Plan(A32, A32, **Predictor.load().opts())  # a double-precision predictor


@pytest.mark.parametrize("stencil,g,dim", [("lap2d9", 256, 2), ("lap3d7", 32, 3), ("lap3d27", 32, 3)])
@pytest.mark.parametrize("policy", ["hybrid", "learned"])
def test_f32_galerkin_hierarchy_exact(spg, oracle_mod, stencil, g, dim, policy):
    """The single-precision Galerkin products of the paper's AMG setting (Section 5.2 reports
    them in both precisions): a piecewise-constant aggregation hierarchy A_{l+1} = P_l^T (A_l P_l)
    down to a 4^dim grid, each level fed by the previous one on the device.  Every value of
    every level is an integer below 2^24, so each level equals the oracle's exactly."""
    from paper_1504_05022_gb300.predictor import Predictor
    A = getattr(gen, stencil)(g)
    Ps = gen.galerkin_levels(g, dim)
    opts = Predictor.load(dtype="f32").opts() if policy == "learned" else {"alloc_policy": policy}
    s = torch.cuda.Stream()
    cur = spg.CSR.from_host(A, dtype=torch.float32)
    levels, keep = [], []
    with torch.cuda.stream(s):
        for P in Ps:
            Pd = spg.CSR.from_host(P, dtype=torch.float32)
            Rd = spg.CSR.from_host(gen.transpose(P), dtype=torch.float32)
            cur, p1, p2 = spg.galerkin(Rd, cur, Pd, stream=s, **opts)
            levels.append(cur)
            keep += [Pd, Rd, p1, p2]
    s.synchronize()
    ref = A
    for lvl, (P, Ac) in enumerate(zip(Ps, levels)):
        AP = oracle_mod.spgemm(ref, P)
        Rc = oracle_mod.spgemm(gen.transpose(P), gen.HostCSR(AP.nrows, AP.ncols, AP.row_ptr, AP.col, AP.val))
        assert np.abs(Rc.val).max() < 2 ** 24
        rp, col, val = Ac.to_host()
        assert Ac.val.dtype == torch.float32
        assert np.array_equal(rp, Rc.row_ptr) and np.array_equal(col, Rc.col), f"level {lvl}"
        assert np.array_equal(val.astype(np.float64), Rc.val), f"level {lvl}"
        ref = gen.HostCSR(Rc.nrows, Rc.ncols, Rc.row_ptr, Rc.col, Rc.val)
    assert levels[-1].shape == (4 ** dim, 4 ** dim)
    for p in keep[2::4] + keep[3::4]:
        p.check()
