"""Pins for the FP64 predictor reference (no GPU): central finite differences of
the loss, the zero-weight special case in closed form, the size-class edges and
the row features on a hand-built example."""
import numpy as np

import gen
from oracle import mlp


def _rand_batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 3, size=(n, mlp.N_IN)) + 5
    cls = rng.integers(0, mlp.NUM_CLASSES, n)
    y = rng.uniform(0, 12, n)
    return X, cls, y


def test_gradient_matches_central_differences():
    X, cls, y = _rand_batch(7, 0)
    theta = mlp.init_params(1, mu=X.mean(0), sigma=X.std(0) + 0.5)
    theta[:mlp.N_PARAMS] += np.random.default_rng(2).normal(0, 0.05, mlp.N_PARAMS)
    f0, g = mlp.loss_and_grad(theta, X, cls, y)
    rng = np.random.default_rng(3)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mlp.loss_and_grad(tp, X, cls, y)[0] - mlp.loss_and_grad(tm, X, cls, y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_zero_weights_closed_form():
    X, cls, y = _rand_batch(5, 4)
    theta = mlp.init_params(0)
    theta[:mlp.N_PARAMS] = 0.0
    p = mlp.unpack(theta)
    b3 = np.linspace(-1, 1, mlp.N_OUT)
    p["b3"][:] = b3
    loss, g = mlp.loss_and_grad(theta, X, cls, y)
    lse = np.log(np.exp(b3[:16]).sum())
    expect = sum(lse - b3[c] for c in cls) + 0.5 * ((b3[16] - y) ** 2).sum()
    assert abs(loss - expect) < 1e-12 * max(1, abs(expect))
    soft = np.exp(b3[:16] - lse)
    gb3 = np.zeros(mlp.N_OUT)
    for c in cls:
        gb3[:16] += soft
        gb3[c] -= 1
    gb3[16] = (b3[16] - y).sum()
    gp = mlp.unpack(np.concatenate([g, np.zeros(2 * mlp.N_IN)]))
    assert np.allclose(gp["b3"], gb3, atol=1e-12)
    # with zero hidden activations nothing flows into the first layers
    assert np.all(gp["W1"] == 0) and np.all(gp["W2"] == 0) and np.all(gp["W3"] == 0)


def test_size_class_edges():
    nnz = np.array([0, 1, 2, 3, 4, 5, 8, 9, 256, 257, 2 ** 15, 2 ** 15 + 1, 2 ** 20])
    assert mlp.size_class(nnz).tolist() == [0, 0, 1, 2, 2, 3, 3, 4, 8, 9, 15, 15, 15]


def test_row_features_hand_example():
    # A row 0 selects B rows 0 (cols 2,5) and 2 (cols 1,4,9); row 1 selects the empty B row 1;
    # row 2 is empty.
    A = gen.from_coo(3, 3, np.array([0, 0, 1]), np.array([0, 2, 1]), np.ones(3))
    B = gen.from_coo(3, 10, np.array([0, 0, 2, 2, 2]), np.array([2, 5, 1, 4, 9]), np.ones(5))
    F = mlp.row_features(A, B)
    g = np.log2(np.array([3.0, 4.0]))
    assert np.allclose(F[0], [np.log2(3), np.log2(6), g.min(), g.max(), g.mean(), g.std(),
                              np.log2(1 + (9 - 1 + 1)), np.log2(11)])
    assert np.allclose(F[1], [1.0, 0.0, 0, 0, 0, 0, 0, np.log2(11)])
    assert np.allclose(F[2], [0, 0, 0, 0, 0, 0, 0, np.log2(11)])
