"""Pins for the CPU oracle (no GPU).

The oracle is only trusted because these tests tie it to facts that do not come
from the oracle itself:
  * the worked example of Section 2.1 (tests/golden/sec2_1_example.txt),
  * dense matrix multiplication (numpy, exact for small-integer values) and a
    pure-Python triple loop on tiny inputs, rectangular shapes, empty rows/cols,
  * the boolean product of the patterns (structure incl. cancelled values, Section 3.1),
  * the invariant C*1 = A*(B*1),
  * closed forms of the 2D 5-point Laplacian square and of the 3D 27-point
    Galerkin product with 2x2x2 aggregation (derived from the stencils, not by
    multiplying),
  * nnz(C^) = sum u_i = flops/2 (Section 3.1, Table 2 caption) by brute force,
  * scipy's sparse product as a library cross-check,
  * the bin edges stated in Section 4.1 for Algorithm 3.
Each planted mistake (a dropped term, a wrong sign, a wrong index) built into an
oracle mutant must fail at least one pin.
"""
import itertools

import numpy as np
import pytest

import gen
from tests.helpers import (REL_TOL, csr_pattern, csr_to_dense, dense,
                           load_golden, pattern)


def _oracle_dense(oracle_mod, A, B, variant=0):
    C = oracle_mod.spgemm(A, B, variant=variant)
    return C, csr_to_dense(C.row_ptr, C.col, C.val, A.nrows, B.ncols)


def _triple_loop(Ad, Bd):
    m, k = Ad.shape
    n = Bd.shape[1]
    C = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            s = 0.0
            for t in range(k):
                s += Ad[i, t] * Bd[t, j]
            C[i, j] = s
    return C


def test_worked_example_section_2_1(oracle_mod):
    g = load_golden("sec2_1_example.txt")
    A, B, Cref = g["A"], g["B"], g["C"]
    C = oracle_mod.spgemm(A, B)
    assert list(C.row_ptr) == list(Cref.row_ptr)
    assert list(C.col) == list(Cref.col)          # columns r, s, t
    assert list(C.val) == list(Cref.val)          # 10, 33, 53 exactly


SHAPES = [(1, 1, 1), (5, 7, 3), (7, 5, 9), (16, 16, 16), (13, 29, 11), (40, 3, 40), (3, 40, 2)]


@pytest.mark.parametrize("m,k,n", SHAPES)
@pytest.mark.parametrize("seed", [0, 1])
def test_dense_integer_exact(oracle_mod, m, k, n, seed):
    A = gen.random_sparse(m, k, 0.3, seed, integer_values=True, empty_rows=0.2)
    B = gen.random_sparse(k, n, 0.3, seed + 100, integer_values=True, empty_rows=0.2)
    C, Cd = _oracle_dense(oracle_mod, A, B)
    Ad, Bd = dense(A), dense(B)
    np.testing.assert_array_equal(Cd, Ad @ Bd)        # small integers: exact in FP64
    if m * n * k <= 4000:
        np.testing.assert_array_equal(Cd, _triple_loop(Ad, Bd))
    # structure == boolean product, including entries that cancel to 0.0
    np.testing.assert_array_equal(csr_pattern(C.row_ptr, C.col, m, n),
                                  (pattern(A) @ pattern(B) > 0).astype(np.int64))
    # columns ascending and unique in every row
    for i in range(m):
        c = C.col[C.row_ptr[i]:C.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_cancellation_keeps_structural_zero(oracle_mod):
    A = gen.from_coo(1, 2, np.array([0, 0]), np.array([0, 1]), np.array([1.0, 1.0]))
    B = gen.from_coo(2, 1, np.array([0, 1]), np.array([0, 0]), np.array([2.0, -2.0]))
    C = oracle_mod.spgemm(A, B)
    assert C.nnz == 1 and C.col[0] == 0 and C.val[0] == 0.0 and C.den[0] == 4.0


def test_empty_and_degenerate(oracle_mod):
    for (m, k, n) in [(0, 0, 0), (0, 5, 3), (4, 0, 3), (4, 5, 0), (3, 3, 3)]:
        A = gen.from_coo(m, k, np.array([], np.int64), np.array([], np.int64), np.array([]))
        B = gen.random_sparse(k, n, 0.5, 3)
        C = oracle_mod.spgemm(A, B)
        assert C.nnz == 0 and C.row_ptr.shape == (m + 1,)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_float_values_against_dense(oracle_mod, seed):
    A = gen.random_sparse(30, 40, 0.2, seed)
    B = gen.random_sparse(40, 25, 0.2, seed + 7)
    C, Cd = _oracle_dense(oracle_mod, A, B)
    ref = dense(A) @ dense(B)
    bound = REL_TOL * (np.abs(dense(A)) @ np.abs(dense(B)))
    assert np.all(np.abs(Cd - ref) <= bound + 1e-300)
    # den_ij = sum_k |a_ik b_kj|
    den = csr_to_dense(C.row_ptr, C.col, C.den, 30, 25)
    np.testing.assert_allclose(den, np.abs(dense(A)) @ np.abs(dense(B)), rtol=1e-14)


def test_row_sum_invariant_rmat(oracle_mod):
    A = gen.rmat(10, 8, seed=3)
    C = oracle_mod.spgemm(A, A)
    ones = np.ones(A.ncols)

    def spmv(M_rp, M_col, M_val, x):
        y = np.zeros(M_rp.shape[0] - 1)
        rows = np.repeat(np.arange(M_rp.shape[0] - 1), np.diff(M_rp))
        np.add.at(y, rows, M_val * x[M_col])
        return y

    lhs = spmv(C.row_ptr, C.col, C.val, ones)
    Bx = spmv(A.row_ptr, A.col, A.val, ones)
    rhs = spmv(A.row_ptr, A.col, A.val, Bx)
    absA = np.abs(A.val)
    bound = spmv(A.row_ptr, A.col, absA, spmv(A.row_ptr, A.col, absA, ones))
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * bound + 1e-300)


def _lap2d_expected(g):
    """Entries of A^2 for the 5-point stencil (diag 4, off -1) from the stencil itself:
    diagonal 16 + deg, +-e: -8, +-2e: 1, +-e1+-e2: 2 (deg = in-grid neighbours)."""
    def inside(x, y):
        return 0 <= x < g and 0 <= y < g
    exp = {}
    for y in range(g):
        for x in range(g):
            i = x + g * y
            deg = sum(inside(x + dx, y + dy) for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)))
            exp[(i, i)] = 16.0 + deg
            for dx, dy, v in [(1, 0, -8.0), (-1, 0, -8.0), (0, 1, -8.0), (0, -1, -8.0),
                              (2, 0, 1.0), (-2, 0, 1.0), (0, 2, 1.0), (0, -2, 1.0),
                              (1, 1, 2.0), (1, -1, 2.0), (-1, 1, 2.0), (-1, -1, 2.0)]:
                if inside(x + dx, y + dy):
                    exp[(i, x + dx + g * (y + dy))] = v
    return exp


def _as_dict(C):
    rows = np.repeat(np.arange(C.nrows), np.diff(C.row_ptr))
    return {(int(r), int(c)): float(v) for r, c, v in zip(rows, C.col, C.val)}


def test_lap2d_closed_form(oracle_mod):
    g = 64
    A = gen.lap2d(g)
    assert A.nnz == 20224
    C = oracle_mod.spgemm(A, A)
    # nnz(C) = g^2 + 4g(g-1) + 4g(g-2) + 4(g-1)^2
    assert C.nnz == g * g + 4 * g * (g - 1) + 4 * g * (g - 2) + 4 * (g - 1) ** 2 == 51972
    assert _as_dict(C) == _lap2d_expected(g)            # integers: bit-exact
    # sum u_i = sum_k (deg(k)+1)^2 = 100,104 = flops/2
    u = oracle_mod.upper_bound(A, A)
    assert int(u.sum()) == 100104


def _galerkin_expected(h):
    """Ac = P^T A P for the 27-point stencil with 2x2x2 aggregation, coarse grid h^3:
    per coarse neighbour the count of adjacent fine pairs is prod_d (4 if same coordinate else 1),
    diagonal 8*26 - 8*7 = 152."""
    exp = {}
    for Z, Y, X in itertools.product(range(h), repeat=3):
        I = X + h * (Y + h * Z)
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            x2, y2, z2 = X + dx, Y + dy, Z + dz
            if not (0 <= x2 < h and 0 <= y2 < h and 0 <= z2 < h):
                continue
            J = x2 + h * (y2 + h * z2)
            if J == I:
                exp[(I, J)] = 152.0
            else:
                same = (dx == 0) + (dy == 0) + (dz == 0)
                exp[(I, J)] = -float(4 ** same)
    return exp


def test_galerkin_closed_form_small(oracle_mod):
    g = 8
    A = gen.lap3d27(g)
    P = gen.agg_P(g)
    R = gen.transpose(P)
    AP = oracle_mod.spgemm(A, P)
    APc = gen.HostCSR(AP.nrows, AP.ncols, AP.row_ptr, AP.col, AP.val)
    Ac = oracle_mod.spgemm(R, APc)
    assert _as_dict(Ac) == _galerkin_expected(g // 2)
    # the other association order gives the same exact integers
    RA = oracle_mod.spgemm(R, A)
    Ac2 = oracle_mod.spgemm(gen.HostCSR(RA.nrows, RA.ncols, RA.row_ptr, RA.col, RA.val), P)
    assert np.array_equal(Ac2.row_ptr, Ac.row_ptr) and np.array_equal(Ac2.col, Ac.col)
    assert np.array_equal(Ac2.val, Ac.val)


def test_galerkin_closed_form_64(oracle_mod):
    g, h = 64, 32
    A = gen.lap3d27(g)
    assert A.nnz == 190 ** 3 == 6859000
    P = gen.agg_P(g)
    R = gen.transpose(P)
    AP = oracle_mod.spgemm(A, P)
    # fine x is adjacent to coarse X iff x in [2X-1, 2X+2] within the grid: 126 pairs per dimension
    assert AP.nnz == 126 ** 3 == 2000376
    Ac = oracle_mod.spgemm(R, gen.HostCSR(AP.nrows, AP.ncols, AP.row_ptr, AP.col, AP.val))
    assert Ac.nnz == 94 ** 3 == 830584
    vals = set(np.unique(Ac.val).tolist())
    assert vals == {152.0, -16.0, -4.0, -1.0}
    rows = np.repeat(np.arange(Ac.nrows), np.diff(Ac.row_ptr))
    diag = Ac.col == rows
    assert np.all(Ac.val[diag] == 152.0) and diag.sum() == h ** 3
    # interior coarse rows sum to exactly 0
    I = np.arange(h ** 3)
    X, Y, Z = I % h, (I // h) % h, I // (h * h)
    interior = (X > 0) & (X < h - 1) & (Y > 0) & (Y < h - 1) & (Z > 0) & (Z < h - 1)
    rs = np.zeros(h ** 3)
    np.add.at(rs, rows, Ac.val)
    assert np.all(rs[interior] == 0.0)


def test_upper_bound_is_product_count(oracle_mod):
    A = gen.rmat(9, 6, seed=5)
    B = gen.erdos_renyi(A.ncols, 5, seed=6)
    u = oracle_mod.upper_bound(A, B)
    # brute force: count products a_ij * b_jk per row
    blen = np.diff(B.row_ptr)
    for i in range(A.nrows):
        cols, _ = A.row(i)
        assert u[i] == sum(int(blen[j]) for j in cols)
    # nnz(C^) = sum u = flops / 2 >= nnz(C)
    C = oracle_mod.spgemm(A, B)
    assert u.sum() >= C.nnz
    assert np.all(u >= np.diff(C.row_ptr))


def test_scipy_cross_check(oracle_mod):
    sp = pytest.importorskip("scipy.sparse")
    A = gen.rmat(12, 8, seed=1)
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=A.shape)
    Cs = (S @ S).tocsr()
    Cs.sort_indices()
    C = oracle_mod.spgemm(A, A)
    # scipy keeps structural zeros from cancellation too; structure must be identical
    assert np.array_equal(np.asarray(Cs.indptr, np.int64), C.row_ptr)
    assert np.array_equal(Cs.indices, C.col)
    assert np.all(np.abs(Cs.data - C.val) <= REL_TOL * C.den + 1e-300)


# Bin edges of Algorithm 3 as stated in Section 4.1: sizes 0 and 1 get their own bins, sizes 2..32
# one bin each, then the ranges 33-64, 65-128, 129-256, 257-512, and everything above 512 goes to
# the last bin with a temporary row of 256 entries.
EDGES = [(0, 0, 0), (1, 1, 1), (2, 2, 2), (3, 3, 3), (17, 17, 17), (31, 31, 31), (32, 32, 32),
         (33, 33, 33), (64, 33, 64), (65, 34, 65), (128, 34, 128), (129, 35, 129), (256, 35, 256),
         (257, 36, 257), (512, 36, 512), (513, 37, 256), (100000, 37, 256), (2**40, 37, 256)]


def test_binning_edges(oracle_mod):
    u = np.array([e[0] for e in EDGES], dtype=np.int64)
    b, sz, cnt, rows, total = oracle_mod.binning(u)
    assert b.tolist() == [e[1] for e in EDGES]
    assert sz.tolist() == [e[2] for e in EDGES]
    assert total == sum(e[2] for e in EDGES)
    assert cnt.sum() == len(EDGES)


def test_binning_segments(oracle_mod):
    rng = np.random.default_rng(0)
    u = rng.integers(0, 2000, 5000)
    u[rng.random(5000) < 0.2] = 0
    u[rng.random(5000) < 0.1] = 1
    b, sz, cnt, rows, total = oracle_mod.binning(u)
    assert sorted(rows.tolist()) == list(range(5000))
    start = np.concatenate([[0], np.cumsum(cnt)])
    for k in range(38):
        seg = rows[start[k]:start[k + 1]]
        assert np.all(np.diff(seg) > 0)           # row order kept inside each bin
        assert np.all(b[seg] == k)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_planted_mistakes_fail_a_pin(oracle_mod, variant):
    """Each deliberately wrong oracle build must be caught by the pins above."""
    caught = []
    # dense / triple-loop pin with integer values
    A = gen.random_sparse(13, 29, 0.3, 0, integer_values=True)
    B = gen.random_sparse(29, 11, 0.3, 100, integer_values=True)
    _, Cd = _oracle_dense(oracle_mod, A, B, variant=variant)
    caught.append(not np.array_equal(Cd, dense(A) @ dense(B)))
    # closed-form pin
    A = gen.lap2d(16)
    caught.append(_as_dict(oracle_mod.spgemm(A, A, variant=variant)) != _lap2d_expected(16))
    assert all(caught)


def test_row_counts_match_full_product():
    import oracle
    A = gen.rmat(10, 8, seed=4)
    ref = oracle.spgemm(A, A)
    assert np.array_equal(oracle.row_counts(A, A), np.diff(ref.row_ptr))
    rows = np.array([5, 0, 1023, 7])
    assert np.array_equal(oracle.row_counts(A, A, rows), np.diff(ref.row_ptr)[rows])



def test_sampled_rows_and_thread_counts_are_bit_exact():
    """The full-size checks compare sampled rows: spgemm_rows on a subset (any order, with
    repeats) must give exactly those rows of the full product, and the result must not
    depend on the thread count (each row is summed in the same order by one thread)."""
    import oracle
    A = gen.rmat(11, 12, seed=8)
    ref = oracle.spgemm(A, A, nthreads=1)
    for nt in (2, 5, 0):
        C = oracle.spgemm(A, A, nthreads=nt)
        assert np.array_equal(C.row_ptr, ref.row_ptr) and np.array_equal(C.col, ref.col)
        assert np.array_equal(C.val, ref.val) and np.array_equal(C.den, ref.den)
    rows = np.array([2047, 0, 17, 17, 1024, 3])
    off, col, val, den = oracle.spgemm_rows(A, A, rows, nthreads=3)
    for j, i in enumerate(rows):
        s, e = ref.row_ptr[i], ref.row_ptr[i + 1]
        assert np.array_equal(col[off[j]:off[j + 1]], ref.col[s:e])
        assert np.array_equal(val[off[j]:off[j + 1]], ref.val[s:e])
        assert np.array_equal(den[off[j]:off[j + 1]], ref.den[s:e])
    with pytest.raises(ValueError):
        oracle.spgemm_rows(A, A, np.array([A.nrows]))

def _galerkin_oracle(A, P):
    import oracle
    R = gen.transpose(P)
    AP = oracle.spgemm(A, P)
    APm = gen.HostCSR(A.nrows, P.ncols, AP.row_ptr, AP.col, AP.val)
    return oracle.spgemm(R, APm)


def _coarse_entry(Ac, i, j):
    s, e = Ac.row_ptr[i], Ac.row_ptr[i + 1]
    hit = np.nonzero(Ac.col[s:e] == j)[0]
    return None if hit.size == 0 else Ac.val[s + hit[0]]


def test_galerkin_2d9_closed_form():
    """2D 9-point Laplacian with 2x2 aggregation: the coarse operator is a 9-point stencil on the
    (g/2)^2 grid, nnz (3g/2 - 2)^2; interior diagonal 4*(8 - 3) = 20, edge neighbours -2*2 = -4,
    corner neighbours -1, interior row sums 0."""
    g = 16
    Ac = _galerkin_oracle(gen.lap2d9(g), gen.agg_P2(g, 2))
    h = g // 2
    assert Ac.nnz == (3 * h - 2) ** 2
    i = 3 + h * 4
    assert _coarse_entry(Ac, i, i) == 20.0
    assert _coarse_entry(Ac, i, i + 1) == -4.0 and _coarse_entry(Ac, i, i + h) == -4.0
    assert _coarse_entry(Ac, i, i + h + 1) == -1.0 and _coarse_entry(Ac, i, i - h - 1) == -1.0
    assert Ac.val[Ac.row_ptr[i]:Ac.row_ptr[i + 1]].sum() == 0.0


def test_galerkin_3d7_closed_form():
    """3D 7-point Laplacian with 2x2x2 aggregation: a 7-point coarse stencil, nnz 7h^3 - 6h^2
    (h = g/2); diagonal 8*(6 - 3) = 24 everywhere (Dirichlet truncation keeps the fine diagonal),
    face neighbours -4 (four fine couplings across a block face)."""
    g = 12
    Ac = _galerkin_oracle(gen.lap3d7(g), gen.agg_P2(g, 3))
    h = g // 2
    assert Ac.nnz == 7 * h ** 3 - 6 * h ** 2
    diag = np.array([_coarse_entry(Ac, i, i) for i in range(h ** 3)])
    assert np.all(diag == 24.0)
    i = 2 + h * (2 + h * 2)
    for d in (1, h, h * h):
        assert _coarse_entry(Ac, i, i + d) == -4.0 and _coarse_entry(Ac, i, i - d) == -4.0


def test_aggregation_generators_agree():
    for g in (4, 8):
        assert np.array_equal(gen.agg_P2(g, 3).col, gen.agg_P(g).col)
    assert [(P.nrows, P.ncols) for P in gen.galerkin_levels(32, 3)] == \
        [(32 ** 3, 16 ** 3), (16 ** 3, 8 ** 3), (8 ** 3, 4 ** 3)]


def _hierarchy(A, Ps):
    import oracle
    out = []
    for P in Ps:
        AP = oracle.spgemm(A, P)
        APm = gen.HostCSR(A.nrows, P.ncols, AP.row_ptr, AP.col, AP.val)
        Ac = oracle.spgemm(gen.transpose(P), APm)
        A = gen.HostCSR(Ac.nrows, Ac.ncols, Ac.row_ptr, Ac.col, Ac.val)
        out.append(A)
    return out


def _offsets(M, h, dim):
    rows = np.repeat(np.arange(M.nrows), np.diff(M.row_ptr))
    d = [((M.col // h ** k) % h) - ((rows // h ** k) % h) for k in range(dim)]
    return np.stack(d, 1)


def test_galerkin_hierarchies_closed_form():
    """Every level of the piecewise-constant hierarchies, every entry.  Aggregation keeps the
    stencil shape and maps its values by a recursion that does not depend on the boundary
    (a block's own couplings and the couplings across a block face are the same for every
    block): 2D 9-point (diagonal d, edge e, corner c) -> (4d + 8e + 4c, 2e + 2c, c) from
    (8, -1, -1); 3D 7-point (diagonal d, face f) -> (8d + 24f, 4f) from (6, -1); 3D 27-point
    below."""
    g, (d, e, c) = 32, (8.0, -1.0, -1.0)
    for lvl, A in enumerate(_hierarchy(gen.lap2d9(g), gen.galerkin_levels(g, 2))):
        h = g >> (lvl + 1)
        d, e, c = 4 * d + 8 * e + 4 * c, 2 * e + 2 * c, c
        off = _offsets(A, h, 2)
        kind = np.abs(off).sum(1)
        assert A.nnz == (3 * h - 2) ** 2 and np.abs(off).max() == 1
        assert np.all(A.val[kind == 0] == d) and np.all(A.val[kind == 1] == e) and np.all(A.val[kind == 2] == c)
    assert (d, e, c) == (92.0, -22.0, -1.0)  # the 4 x 4 level: interior row sum 92 - 4*22 - 4 = 0
    g, (d, f) = 16, (6.0, -1.0)
    for lvl, A in enumerate(_hierarchy(gen.lap3d7(g), gen.galerkin_levels(g, 3))):
        h = g >> (lvl + 1)
        d, f = 8 * d + 24 * f, 4 * f
        off = _offsets(A, h, 3)
        kind = np.abs(off).sum(1)
        assert A.nnz == 7 * h ** 3 - 6 * h ** 2 and kind.max() == 1
        assert np.all(A.val[kind == 0] == d) and np.all(A.val[kind == 1] == f)
    assert (d, f) == (96.0, -16.0)  # the 4 x 4 x 4 level
    # 3D 27-point: (diagonal d, face f, edge e, corner c) -> (8d + 24f + 24e + 8c, 4f + 8e + 4c,
    # 2e + 2c, c) from (26, -1, -1, -1); the first level is the (152, -16, -4, -1) operator
    g, (d, f, e, c) = 16, (26.0, -1.0, -1.0, -1.0)
    for lvl, A in enumerate(_hierarchy(gen.lap3d27(g), gen.galerkin_levels(g, 3))):
        h = g >> (lvl + 1)
        d, f, e, c = 8 * d + 24 * f + 24 * e + 8 * c, 4 * f + 8 * e + 4 * c, 2 * e + 2 * c, c
        off = _offsets(A, h, 3)
        kind = np.abs(off).sum(1)
        assert A.nnz == (3 * h - 2) ** 3 and np.abs(off).max() == 1
        for k, want in enumerate((d, f, e, c)):
            assert np.all(A.val[kind == k] == want), (lvl, k)
        if lvl == 0:
            assert (d, f, e, c) == (152.0, -16.0, -4.0, -1.0)
    assert (d, f, e, c) == (728.0, -100.0, -10.0, -1.0)  # interior row sum 728 - 600 - 120 - 8 = 0
