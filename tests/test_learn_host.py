"""Host side of the learned preallocation, on the CPU: the training recipe, the parameter
layout shared with the device kernels, the rounding of a predicted row size, and the stored
weights checked with the oracle on matrices the training held out (every seed s with s % 5 == 2).
The network's forward pass here is the oracle's (FP64); its row sizes are the oracle's exact
counts, so what is measured is the stored network itself."""
import json

import numpy as np
import pytest

import gen


@pytest.fixture(scope="module")
def weights():
    from paper_1504_05022_gb300.predictor import WEIGHTS
    with open(WEIGHTS) as f:
        return json.load(f)


def test_recipe_spans_the_families_and_sizes():
    from paper_1504_05022_gb300 import learn
    seen = {}
    for s in range(200):
        fam, n, p = learn.recipe(s)
        assert fam == learn.FAMILIES[s % 4] and n == 1 << (14 + (s // 4) % 5)
        lo, hi = {"banded": (3, 64), "blockdiag": (8, 64), "er": (4, 32), "rmat": (4, 16)}[fam]
        assert lo <= p <= hi
        seen.setdefault(fam, set()).add(n)
    assert set(seen) == set(learn.FAMILIES)
    assert all(sizes == {1 << k for k in range(14, 19)} for sizes in seen.values())
    assert learn.recipe(17) == learn.recipe(17)


def test_parameter_layout_matches_the_oracle_and_the_header():
    from oracle import mlp

    from paper_1504_05022_gb300 import _lib, learn
    mu, sigma = np.arange(8.0), np.linspace(1.0, 2.0, 8)
    th = learn.init_params(3, mu, sigma)
    assert th.size == mlp.N_TOTAL == _lib.MLP_NUM_TOTAL
    assert mlp.N_PARAMS == _lib.MLP_NUM_PARAMS
    parts = mlp.unpack(th.astype(np.float64))
    for b in ("b1", "b2", "b3"):
        assert not parts[b].any()
    assert np.allclose(parts["mu"], mu) and np.allclose(parts["sigma"], sigma)
    for w, fan_in in (("W1", 8), ("W2", 32), ("W3", 32)):  # He initialisation
        assert abs(parts[w].std() / np.sqrt(2.0 / fan_in) - 1.0) < 0.25
    nnz = np.array([0, 1, 2, 3, 4, 5, 1023, 1024, 1025, 1 << 20])
    assert np.array_equal(learn.size_class(nnz), mlp.size_class(nnz))


def test_predicted_size_rounding():
    from paper_1504_05022_gb300 import learn
    out = np.zeros((5, 17), dtype=np.float32)
    out[:, 16] = np.log2(1.0 + np.array([1000.0, 10.0, 4095.0, 0.0, 1e12]))
    got = learn.predicted_sizes(out, 1.0)
    # 1000 -> 1024 (a multiple of 32); 10 -> the 256-entry floor; 4095 -> 4096; 0 -> 256;
    # the regression is clipped at 30, 2^30 - 1 -> 2^30
    assert np.array_equal(got, [1024, 256, 4096, 256, 1 << 30])
    assert np.array_equal(learn.predicted_sizes(out, 1.5)[:1], [1504])  # ceil(1000 * 1.5 / 32) * 32
    assert np.all(learn.predicted_sizes(out, 2.0) >= got)


def test_stored_weights_are_well_formed(weights):
    from oracle import mlp
    th = np.array(weights["params"], dtype=np.float64)
    assert th.size == mlp.N_TOTAL and np.isfinite(th).all()
    assert (mlp.unpack(th)["sigma"] > 0).all()
    assert weights["margin"] >= 1.0
    table = {r["margin"]: r["miss_rate"] for r in weights["val_margin_table"]}
    assert table[weights["margin"]] <= weights["target_miss"]
    assert all(a >= b for a, b in zip(list(table.values()), list(table.values())[1:]))


@pytest.mark.parametrize("seed", [7, 27, 47])
def test_stored_weights_on_held_out_rmat(oracle_mod, weights, seed):
    """R-MAT matrices of the recipe that the training held out: at the stored margin at most
    a few percent of the long rows (u_i > 512) fall back to the progressive path, and the
    preallocation stays within 1.3x of the exact output (the validation table records 4.9%
    and 1.32x over all held-out matrices)."""
    from oracle import mlp

    from paper_1504_05022_gb300 import learn
    assert seed % 5 == 2
    fam, n, p = learn.recipe(seed)
    assert fam == "rmat"
    M = gen.family_matrix(fam, n, p, seed=seed)
    rows = np.nonzero(oracle_mod.upper_bound(M, M) > 512)[0]
    assert rows.size > 1000
    F = mlp.row_features(M, M)[rows]
    out, _ = mlp.forward(np.array(weights["params"], dtype=np.float32).astype(np.float64), F)
    nnz = oracle_mod.row_counts(M, M, rows)
    pred = learn.predicted_sizes(out, weights["margin"])
    miss = float((pred < nnz).mean())
    assert miss <= 0.05, miss
    assert pred.sum() / nnz.sum() <= 1.3
    # the class head agrees with the exact size class on most rows
    assert (out[:, :16].argmax(1) == mlp.size_class(nnz)).mean() >= 0.9
