"""Input generators: valid CSR (sorted, unique columns) with the documented sizes."""
import numpy as np

import gen


def test_lap2d_shape():
    A = gen.lap2d(64)
    A.validate()
    assert A.shape == (4096, 4096) and A.nnz == 20224
    assert set(np.unique(A.val).tolist()) == {4.0, -1.0}


def test_lap3d27_and_aggregation_shapes():
    A = gen.lap3d27(8)
    A.validate()
    assert A.nnz == 22 ** 3                       # (3g-2)^3 entries for a 27-point stencil
    P = gen.agg_P(8)
    P.validate()
    assert P.shape == (512, 64) and P.nnz == 512
    assert np.all(np.diff(P.row_ptr) == 1)
    R = gen.transpose(P)
    R.validate()
    assert R.shape == (64, 512) and np.all(np.diff(R.row_ptr) == 8)


def test_rmat_is_seeded_and_valid():
    A1 = gen.rmat(12, 16, seed=1)
    A2 = gen.rmat(12, 16, seed=1)
    A1.validate()
    assert np.array_equal(A1.col, A2.col) and np.array_equal(A1.val, A2.val)
    assert A1.nnz <= 16 * 4096
    assert np.all(np.abs(A1.val) <= 1.0)
    # power law: the first row (highest quadrant probability) is far longer than average
    assert np.diff(A1.row_ptr)[0] > 10 * A1.nnz / A1.nrows


def test_families_valid():
    for fam, param in [("banded", 7), ("blockdiag", 16), ("er", 12), ("rmat", 8)]:
        M = gen.family_matrix(fam, 1000, param, seed=3)
        M.validate()
        assert M.nrows >= 1000


def test_autotune_apply_and_load(tmp_path, monkeypatch):
    from paper_1504_05022_gb300 import autotune
    opts = autotune.apply({"alloc_policy": "learned", "predictor_margin": 1.3},
                          {"heap_max_u": 16, "predictor_margin": None, "merge_batch": 1024})
    assert opts == {"alloc_policy": "learned", "predictor_margin": 1.3, "heap_max_u": 16, "merge_batch": 1024}
    f = tmp_path / "tuned.json"
    f.write_text('{"w": {"hybrid": {"params": {"heap_block": 64}}}}')
    monkeypatch.setattr(autotune, "TUNED", str(f))
    assert autotune.load("w", "hybrid") == {"heap_block": 64}
    assert autotune.load("w", "learned") is None and autotune.load("x", "hybrid") is None


def test_rmat_headline_recipe():
    """The R-MAT 2^16 x 16 input of the headline product: its size after merging duplicates,
    its product count, first-level quadrant shares near (a, b, c, d) = (.57, .19, .19, .05)
    (duplicates, most frequent in the dense quadrant, lower its share a little) and values in
    (-1, 1)."""
    A = gen.rmat(16, 16, seed=1)
    assert A.nrows == A.ncols == 1 << 16
    assert A.nnz == 955_117
    assert int(np.diff(A.row_ptr)[A.col].astype(np.int64).sum()) == 402_077_751
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    h = A.nrows // 2
    q = [np.mean((rows < h) & (A.col < h)), np.mean((rows < h) & (A.col >= h)),
         np.mean((rows >= h) & (A.col < h)), np.mean((rows >= h) & (A.col >= h))]
    assert abs(q[0] - 0.57) < 0.03 and abs(q[1] - 0.19) < 0.015 and abs(q[2] - 0.19) < 0.015
    assert abs(q[3] - 0.05) < 0.01
    assert A.val.min() > -1.0 and A.val.max() < 1.0
