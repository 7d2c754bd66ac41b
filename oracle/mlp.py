"""FP64 reference of the row-size predictor (test infrastructure only).

The predictor is not part of the paper.  It is the learned replacement for the
paper's fixed bin-37 preallocation (Section 4.1 allocates 256 entries and doubles
on overflow): a small multilayer perceptron maps 8 features of a row of C to
  * logits over NUM_CLASSES size classes (class of nnz(c_i): 0 for nnz <= 1,
    otherwise ceil(log2(nnz)), clipped to NUM_CLASSES - 1), and
  * a regression of log2(1 + nnz(c_i)).

Layout of the parameter vector (float32 on the device, float64 here):
  W1[32x8] b1[32] W2[32x32] b2[32] W3[17x32] b3[17]   (1905 trainable values)
followed by mu[8] sigma[8] (input standardisation, not trained).
x_hat = (x - mu) / sigma;  h1 = relu(W1 x_hat + b1);  h2 = relu(W2 h1 + b2);
out = W3 h2 + b3;  loss = CE(softmax(out[:16]), class) + 0.5 (out[16] - y)^2.

Only tests/ import this module; the CUDA kernels are checked against it.
"""
from __future__ import annotations

import numpy as np

N_IN = 8
N_HID = 32
NUM_CLASSES = 16
N_OUT = NUM_CLASSES + 1
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 1905
N_TOTAL = N_PARAMS + 2 * N_IN                        # + mu, sigma


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    out["mu"] = theta[o:o + N_IN]
    out["sigma"] = theta[o + N_IN:o + 2 * N_IN]
    return out


def size_class(nnz: np.ndarray) -> np.ndarray:
    nnz = np.asarray(nnz, dtype=np.int64)
    c = np.zeros(nnz.shape, dtype=np.int64)
    big = nnz > 1
    c[big] = np.ceil(np.log2(nnz[big].astype(np.float64))).astype(np.int64)
    return np.minimum(c, NUM_CLASSES - 1)


def forward(theta: np.ndarray, X: np.ndarray):
    """Returns (out[n, 17], cache) in float64."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    xh = (np.asarray(X, dtype=np.float64) - p["mu"]) / p["sigma"]
    z1 = xh @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (p, xh, z1, h1, z2, h2)


def loss_and_grad(theta: np.ndarray, X: np.ndarray, cls: np.ndarray, y: np.ndarray):
    """Summed loss over the samples and its gradient w.r.t. the 1905 trainable values."""
    out, (p, xh, z1, h1, z2, h2) = forward(theta, X)
    logits = out[:, :NUM_CLASSES]
    reg = out[:, NUM_CLASSES]
    mx = logits.max(axis=1, keepdims=True)
    ex = np.exp(logits - mx)
    se = ex.sum(axis=1, keepdims=True)
    logp = logits - mx - np.log(se)
    n = X.shape[0]
    cls = np.asarray(cls, dtype=np.int64)
    y = np.asarray(y, dtype=np.float64)
    loss = -logp[np.arange(n), cls].sum() + 0.5 * ((reg - y) ** 2).sum()
    dout = np.zeros_like(out)
    dout[:, :NUM_CLASSES] = ex / se
    dout[np.arange(n), cls] -= 1.0
    dout[:, NUM_CLASSES] = reg - y
    gW3 = dout.T @ h2
    gb3 = dout.sum(axis=0)
    dh2 = dout @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ xh
    gb1 = dz1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return float(loss), grad


def init_params(seed: int, mu=None, sigma=None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            fan_in = shp[1]
            parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shp).ravel())
        else:
            parts.append(np.zeros(shp))
    mu = np.zeros(N_IN) if mu is None else np.asarray(mu, dtype=np.float64)
    sigma = np.ones(N_IN) if sigma is None else np.asarray(sigma, dtype=np.float64)
    return np.concatenate(parts + [mu, sigma])


def row_features(A, B) -> np.ndarray:
    """The 8 per-row features of C = A*B, in float64, written out from their definitions:
      0 log2(1 + nnz(a_i*))
      1 log2(1 + u_i), u_i = sum of nnz(b_k*) over the stored a_ik (Algorithm 2)
      2 min, 3 max, 4 mean, 5 standard deviation of log2(1 + nnz(b_k*)) over the stored a_ik
      6 log2(1 + colspan_i), colspan_i = (max over non-empty b_k* of its last column)
                                        - (min over non-empty b_k* of its first column) + 1
      7 log2(1 + ncols(B))
    Rows with an empty A row get 0 for features 2..6."""
    m = A.nrows
    F = np.zeros((m, N_IN), dtype=np.float64)
    blen = np.diff(B.row_ptr)
    for i in range(m):
        cols = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        F[i, 0] = np.log2(1.0 + cols.size)
        L = blen[cols].astype(np.float64)
        F[i, 1] = np.log2(1.0 + L.sum())
        if cols.size:
            g = np.log2(1.0 + L)
            F[i, 2], F[i, 3], F[i, 4] = g.min(), g.max(), g.mean()
            F[i, 5] = np.sqrt(max(0.0, (g * g).mean() - g.mean() ** 2))
            ne = cols[blen[cols] > 0]
            if ne.size:
                first = B.col[B.row_ptr[ne]]
                last = B.col[B.row_ptr[ne + 1] - 1]
                F[i, 6] = np.log2(1.0 + (int(last.max()) - int(first.min()) + 1))
        F[i, 7] = np.log2(1.0 + B.ncols)
    return F
