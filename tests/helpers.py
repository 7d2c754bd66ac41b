"""Shared test helpers: golden-fixture reader, dense conversions and parity checks.

Nothing here implements SpGEMM; the checks compare two results element by element."""
from __future__ import annotations

import os

import numpy as np

from gen import HostCSR, from_coo

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Value tolerance of the parity contract: |c_ij - ref_ij| <= REL_TOL * sum_k |a_ik b_kj|.
REL_TOL = 1e-12


def load_golden(name: str) -> dict:
    """Read a '# comment / shape X m n / X / row col value' fixture into HostCSR matrices."""
    mats, shapes, cur, entries = {}, {}, None, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "shape":
                shapes[parts[1]] = (int(parts[2]), int(parts[3]))
            elif len(parts) == 1:
                cur = parts[0]
                entries[cur] = []
            else:
                entries[cur].append((int(parts[0]), int(parts[1]), float(parts[2])))
    for k, ent in entries.items():
        m, n = shapes[k]
        r = np.array([e[0] for e in ent], dtype=np.int64)
        c = np.array([e[1] for e in ent], dtype=np.int64)
        v = np.array([e[2] for e in ent], dtype=np.float64)
        mats[k] = from_coo(m, n, r, c, v)
    return mats


def dense(M: HostCSR) -> np.ndarray:
    D = np.zeros((M.nrows, M.ncols), dtype=np.float64)
    for i in range(M.nrows):
        c, v = M.row(i)
        D[i, c] = v
    return D


def pattern(M: HostCSR) -> np.ndarray:
    P = np.zeros((M.nrows, M.ncols), dtype=np.int64)
    for i in range(M.nrows):
        c, _ = M.row(i)
        P[i, c] = 1
    return P


def csr_to_dense(rp, col, val, m, n) -> np.ndarray:
    D = np.zeros((m, n), dtype=np.float64)
    for i in range(m):
        s, e = int(rp[i]), int(rp[i + 1])
        D[i, col[s:e]] = val[s:e]
    return D


def csr_pattern(rp, col, m, n) -> np.ndarray:
    P = np.zeros((m, n), dtype=np.int64)
    for i in range(m):
        s, e = int(rp[i]), int(rp[i + 1])
        P[i, col[s:e]] = 1
    return P


def assert_csr_equal(rp, col, val, ref_rp, ref_col, ref_val, ref_den, rel_tol=REL_TOL, exact=False,
                     label=""):
    """Structure bit-exact; values within rel_tol * den (or bit-exact when exact=True)."""
    rp = np.asarray(rp, dtype=np.int64)
    ref_rp = np.asarray(ref_rp, dtype=np.int64)
    assert rp.shape == ref_rp.shape, f"{label}: row_ptr length {rp.shape} vs {ref_rp.shape}"
    bad = np.nonzero(rp != ref_rp)[0]
    assert bad.size == 0, f"{label}: row_ptr differs first at {bad[:5]}: {rp[bad[:5]]} vs {ref_rp[bad[:5]]}"
    nnz = int(ref_rp[-1])
    col = np.asarray(col)[:nnz]
    ref_col = np.asarray(ref_col)[:nnz]
    badc = np.nonzero(col != ref_col)[0]
    assert badc.size == 0, f"{label}: col differs at {badc[:5]} ({col[badc[:5]]} vs {ref_col[badc[:5]]})"
    val = np.asarray(val, dtype=np.float64)[:nnz]
    ref_val = np.asarray(ref_val, dtype=np.float64)[:nnz]
    if exact:
        badv = np.nonzero(val != ref_val)[0]
        assert badv.size == 0, f"{label}: values differ at {badv[:5]}: {val[badv[:5]]} vs {ref_val[badv[:5]]}"
    else:
        den = np.asarray(ref_den, dtype=np.float64)[:nnz]
        err = np.abs(val - ref_val)
        lim = rel_tol * den
        badv = np.nonzero(err > lim)[0]
        assert badv.size == 0, (f"{label}: {badv.size} values out of tolerance, e.g. at {badv[:5]}: "
                                f"{val[badv[:5]]} vs {ref_val[badv[:5]]} (den {den[badv[:5]]})")
