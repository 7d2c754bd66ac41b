"""GPU checks of the learned preallocation against the FP64 reference in
oracle/mlp.py (features, forward, loss and gradient), and exactness of C under
the learned policy whatever the prediction (the exact path is the fallback)."""
import numpy as np
import pytest

import gen
from oracle import mlp
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


@pytest.mark.parametrize("mk", [lambda: (gen.rmat(11, 16, seed=2), None),
                                lambda: (gen.erdos_renyi(900, 7, seed=3, ncols=1300),
                                         gen.random_sparse(1300, 700, 0.01, 4, empty_rows=0.2))])
def test_row_features_match_reference(spg, mk):
    from paper_1504_05022_gb300.predictor import row_features
    A, B = mk()
    B = A if B is None else B
    Ad, Bd = spg.CSR.from_host(A), spg.CSR.from_host(B)
    X = row_features(Ad, Bd).cpu().numpy()
    ref = mlp.row_features(A, B)
    np.testing.assert_allclose(X, ref, rtol=2e-6, atol=1e-5)


def _params(seed, X):
    th = mlp.init_params(seed, mu=X.mean(0), sigma=X.std(0) + 0.1)
    th[:mlp.N_PARAMS] += np.random.default_rng(seed).normal(0, 0.05, mlp.N_PARAMS)
    return th


def test_forward_and_gradient_match_reference(spg):
    from paper_1504_05022_gb300.predictor import Trainer, mlp_forward
    rng = np.random.default_rng(0)
    n = 3000
    X = rng.normal(4, 2, size=(n, 8))
    cls = rng.integers(0, 16, n)
    y = rng.uniform(0, 14, n)
    th = _params(1, X)
    P = torch.from_numpy(th.astype(np.float32)).cuda()
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    out = mlp_forward(P, Xd).cpu().numpy()
    ref, _ = mlp.forward(th.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=1e-4, atol=1e-4)
    tr = Trainer(P)
    loss, grad = tr.loss_grad(Xd, torch.from_numpy(cls.astype(np.int32)).cuda(),
                              torch.from_numpy(y.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    rl, rg = mlp.loss_and_grad(th.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64),
                               cls, y.astype(np.float32).astype(np.float64))
    assert abs(loss.item() - rl) <= 1e-5 * abs(rl)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - rg) <= 1e-4 * np.linalg.norm(rg)


def test_adam_training_reduces_loss(spg):
    from paper_1504_05022_gb300.predictor import Trainer
    rng = np.random.default_rng(5)
    n = 4096
    X = rng.normal(0, 1, size=(n, 8))
    y = 3 + X[:, 0] * 2 - X[:, 1]                      # a learnable target
    cls = np.clip(np.round(y), 0, 15).astype(np.int32)
    th = _params(2, X)
    tr = Trainer(torch.from_numpy(th.astype(np.float32)).cuda(), lr=3e-3)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    cd = torch.from_numpy(cls).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    first = tr.step(Xd, cd, yd).item()
    for _ in range(300):
        last = tr.step(Xd, cd, yd).item()
    assert last < 0.3 * first


@pytest.mark.parametrize("margin", [0.01, 1.0, 50.0])
def test_learned_policy_is_exact(spg, oracle_mod, margin):
    """C is the same for any prediction: a too-small prediction only sends rows to the
    exact fallback (margin 0.01), a large one only costs memory (margin 50)."""
    from paper_1504_05022_gb300.predictor import Predictor, row_features
    A = gen.rmat(13, 16, seed=8)
    Ad = spg.CSR.from_host(A)
    X = row_features(Ad, Ad).cpu().numpy()
    th = mlp.init_params(3, mu=X.mean(0), sigma=X.std(0) + 0.1)
    w3 = 32 * 8 + 32 + 32 * 32 + 32
    th[w3:w3 + 17 * 32] = 0.0         # W3 = 0: the regression head outputs b3[16] for every row
    th[mlp.N_PARAMS - 1] = 9.0        # b3[16] = 9: 2^9 - 1 = 511 entries before the margin
    pred = Predictor(th, margin=margin)
    plan = spg.Plan(Ad, Ad, dense_min_u=-1, **pred.opts())  # every bin-37 row predicted
    C = plan.numeric()
    torch.cuda.synchronize()
    ref = oracle_mod.spgemm(A, A)
    rp, col, val = C.to_host()
    assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, label=f"learned m={margin}")
    st = plan.stats()
    n37 = st["bin_count"][37]
    assert n37 > 0
    nnz37 = np.diff(ref.row_ptr)[plan.arrays()["bin"] == 37]
    fb = st["rows_fallback"]

    def bounds(cap):
        # a row falls back when its result exceeds its slot, and may fall back up to a quarter
        # batch earlier (a batch only starts when all its products could be new entries)
        return int((nnz37 > cap).sum()), int((nnz37 > cap - cap // 4).sum())
    if margin == 0.01:    # every bin-37 row gets the minimum 256 entries
        lo, hi = bounds(256)
        assert lo <= fb <= hi and fb > 0
    if margin == 1.0:     # 512 entries
        lo, hi = bounds(512)
        assert lo <= fb <= hi
    if margin == 50.0:    # 25,568 entries (or u_i): nothing outgrows it
        assert fb == 0


def test_trained_weights_if_present(spg, oracle_mod):
    import os
    from paper_1504_05022_gb300.predictor import WEIGHTS, Predictor
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights committed")
    pred = Predictor.load()
    A = gen.rmat(15, 8, seed=77)                   # not in the training recipe (seed, size)
    Ad = spg.CSR.from_host(A)
    plan = spg.Plan(Ad, Ad, **pred.opts())
    C = plan.numeric()
    torch.cuda.synchronize()
    ref = oracle_mod.spgemm(A, A)
    rp, col, val = C.to_host()
    assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, label="trained")
    st = plan.stats()
    assert st["rows_fallback"] <= 0.25 * st["bin_count"][37]


@pytest.mark.parametrize("margin,long_rows", [(0.01, "split"), (1.0, "split"), (50.0, "split"), (50.0, "level1"),
                                              (1.0, "level1")])
def test_learned_fallback_levels_and_long_rows(spg, oracle_mod, margin, long_rows):
    """Largest capacity lowered to 1024 entries: rows that outgrow a small prediction climb the
    capacity levels (512, 1024) and then take the long-row path; rows predicted beyond the
    largest capacity (margin 50) go to the long-row path as soon as they reach it."""
    from paper_1504_05022_gb300.predictor import Predictor, row_features
    A = gen.rmat(12, 16, seed=21)
    Ad = spg.CSR.from_host(A)
    X = row_features(Ad, Ad).cpu().numpy()
    th = mlp.init_params(5, mu=X.mean(0), sigma=X.std(0) + 0.1)
    w3 = 32 * 8 + 32 + 32 * 32 + 32
    th[w3:w3 + 17 * 32] = 0.0
    th[mlp.N_PARAMS - 1] = 9.0        # 511 entries before the margin
    pred = Predictor(th, margin=margin)
    plan = spg.Plan(Ad, Ad, smem_cap_max=1024, long_rows=long_rows, dense_min_u=-1, **pred.opts())
    C = plan.numeric()
    torch.cuda.synchronize()
    ref = oracle_mod.spgemm(A, A)
    rp, col, val = C.to_host()
    assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, label=f"learned {margin}/{long_rows}")
    st = plan.stats()
    nnz37 = np.diff(ref.row_ptr)[plan.arrays()["bin"] == 37]
    assert (nnz37 > 1024).sum() > 0
    if long_rows == "split":
        assert st["rows_split"] > 0 and st["rows_level1"] == 0
    else:
        assert st["rows_level1"] > 0 and st["rows_split"] == 0
    if margin == 50.0:
        assert st["rows_fallback"] == 0
    plan.check()
