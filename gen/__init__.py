"""Seeded synthetic CSR inputs shaped like the workloads of Liu & Vinter's SpGEMM paper.

This module builds input matrices only.  It holds none of the SpGEMM arithmetic
(no products, no accumulation), so both the CPU oracle and the CUDA path can take
their inputs from here without sharing any of the method.

Every generator returns a :class:`HostCSR` with sorted, duplicate-free column
indices per row (the CSR convention assumed in Section 3.2 of the paper), int64
row pointers, int32 column indices and float64 values.

Workloads (all seeded, all synthetic):

* ``lap2d(g)``      2D 5-point Laplacian on a g x g grid, diagonal 4, off-diagonal -1,
                    Dirichlet truncation (stands in for the 2D 5-point Poisson system
                    matrix of the Galerkin experiment, Section 5.2).
* ``lap3d27(g)``    3D 27-point Laplacian on a g^3 grid, diagonal 26, off-diagonal -1
                    (the 3D 27-point Poisson matrix of Section 5.2).
* ``agg_P(g)``      piecewise-constant prolongation over 2x2x2 aggregates (one 1.0 per
                    row); ``transpose`` gives the restriction R = P^T.
* ``rmat(...)``     R-MAT power-law matrix (stands in for the irregular University of
                    Florida matrices of Table 2, which are not available here).
* ``banded``, ``blockdiag``, ``erdos_renyi``: the other matrix families used to
                    train the row-size predictor and to fill batched workloads.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "HostCSR", "from_coo", "transpose", "lap2d", "lap3d27", "agg_P", "rmat",
    "banded", "blockdiag", "erdos_renyi", "random_sparse", "family_matrix", "batch_pairs",
]


@dataclass
class HostCSR:
    """A CSR matrix in host memory: row_ptr (nrows+1, int64), col (nnz, int32), val (nnz, float64)."""

    nrows: int
    ncols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def shape(self):
        return (self.nrows, self.ncols)

    def row(self, i: int):
        s, e = int(self.row_ptr[i]), int(self.row_ptr[i + 1])
        return self.col[s:e], self.val[s:e]

    def validate(self) -> None:
        rp = self.row_ptr
        assert rp.dtype == np.int64 and self.col.dtype == np.int32 and self.val.dtype == np.float64
        assert rp.shape == (self.nrows + 1,) and rp[0] == 0
        assert np.all(np.diff(rp) >= 0)
        assert self.col.shape == (self.nnz,) and self.val.shape == (self.nnz,)
        if self.nnz:
            assert self.col.min() >= 0 and self.col.max() < self.ncols
            # strictly increasing within each row
            d = np.diff(self.col.astype(np.int64))
            starts = rp[1:-1]
            inner = np.ones(self.nnz - 1, dtype=bool)
            b = starts[(starts > 0) & (starts < self.nnz)] - 1
            inner[b] = False
            assert np.all(d[inner] > 0), "columns must be sorted and unique within a row"

    def with_row_ptr32(self) -> np.ndarray:
        assert self.nnz < 2**31
        return self.row_ptr.astype(np.int32)


def from_coo(nrows: int, ncols: int, r: np.ndarray, c: np.ndarray, v: np.ndarray | None,
             merge: str = "first") -> HostCSR:
    """Build a CSR from coordinates.  Duplicate coordinates are merged by keeping one entry
    (``merge='first'``: the value of the first occurrence in sorted order is kept; values are
    normally drawn after deduplication, so this only matters for callers passing values)."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    key = r * np.int64(max(ncols, 1)) + c
    order = np.argsort(key, kind="stable")
    key = key[order]
    keep = np.ones(key.shape[0], dtype=bool)
    keep[1:] = key[1:] != key[:-1]
    key = key[keep]
    rr = key // max(ncols, 1)
    cc = key - rr * max(ncols, 1)
    if v is None:
        vv = np.ones(key.shape[0], dtype=np.float64)
    else:
        vv = np.asarray(v, dtype=np.float64)[order][keep]
    counts = np.bincount(rr, minlength=nrows).astype(np.int64)
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return HostCSR(nrows, ncols, rp, cc.astype(np.int32), vv)


def transpose(M: HostCSR) -> HostCSR:
    """Structural transpose (used to form the restriction R = P^T)."""
    counts = np.diff(M.row_ptr)
    rows = np.repeat(np.arange(M.nrows, dtype=np.int64), counts)
    return from_coo(M.ncols, M.nrows, M.col.astype(np.int64), rows, M.val)


def _stencil(g: int, dim: int, offsets, diag: float, off: float) -> HostCSR:
    n = g ** dim
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // (g ** d)) % g for d in range(dim)]  # x fastest: index = x + g*y (+ g^2*z)
    rows, cols, vals = [], [], []
    for o in offsets:
        ok = np.ones(n, dtype=bool)
        for d in range(dim):
            cd = coords[d] + o[d]
            ok &= (cd >= 0) & (cd < g)
        src = idx[ok]
        dst = src + sum(o[d] * g ** d for d in range(dim))
        rows.append(src)
        cols.append(dst)
        vals.append(np.full(src.shape[0], diag if all(x == 0 for x in o) else off))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    return from_coo(n, n, r, c, v)


def lap2d(g: int) -> HostCSR:
    """2D 5-point Laplacian, g x g grid, diagonal 4.0, off-diagonal -1.0, no wrap-around."""
    offs = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]
    return _stencil(g, 2, offs, 4.0, -1.0)


def lap3d27(g: int) -> HostCSR:
    """3D 27-point Laplacian, g^3 grid, diagonal 26.0 (also on the boundary), off-diagonal -1.0."""
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return _stencil(g, 3, offs, 26.0, -1.0)


def lap2d9(g: int) -> HostCSR:
    """2D 9-point Laplacian, g x g grid, diagonal 8.0, off-diagonal -1.0, no wrap-around."""
    offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return _stencil(g, 2, offs, 8.0, -1.0)


def lap3d7(g: int) -> HostCSR:
    """3D 7-point Laplacian, g^3 grid, diagonal 6.0, off-diagonal -1.0, no wrap-around."""
    offs = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    return _stencil(g, 3, offs, 6.0, -1.0)


def agg_P2(g: int, dim: int) -> HostCSR:
    """Piecewise-constant aggregation over 2^dim blocks of a g^dim grid (g even): fine point
    x + g*y (+ g^2*z) maps to aggregate (x/2) + (g/2)*(y/2) (+ (g/2)^2*(z/2)); one 1.0 per row."""
    assert g % 2 == 0 and dim in (2, 3)
    n = g ** dim
    h = g // 2
    idx = np.arange(n, dtype=np.int64)
    agg = np.zeros(n, dtype=np.int64)
    for d in range(dim):
        agg += ((idx // g ** d) % g // 2) * h ** d
    return from_coo(n, h ** dim, idx, agg, np.ones(n))


def galerkin_levels(g: int, dim: int, coarsest: int = 4):
    """Aggregation operators of a piecewise-constant hierarchy on a g^dim grid: P_l for
    levels l = 0, 1, ... while the grid is larger than `coarsest` (halved each level)."""
    Ps = []
    while g > coarsest:
        Ps.append(agg_P2(g, dim))
        g //= 2
    return Ps


def agg_P(g: int) -> HostCSR:
    """Piecewise-constant aggregation over 2x2x2 blocks of a g^3 grid (g even).

    Fine point x + g*y + g^2*z maps to aggregate (x/2) + (g/2)*(y/2) + (g/2)^2*(z/2); P has one
    1.0 per row, shape g^3 x (g/2)^3."""
    assert g % 2 == 0
    n = g ** 3
    h = g // 2
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % g, (idx // g) % g, idx // (g * g)
    agg = (x // 2) + h * ((y // 2) + h * (z // 2))
    return from_coo(n, h ** 3, idx, agg, np.ones(n))


def rmat(scale: int, avg: int, seed: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         vlo: float = -1.0, vhi: float = 1.0) -> HostCSR:
    """R-MAT matrix with 2^scale rows/cols.

    Draws exactly avg * 2^scale edge samples by recursive quadrant choice (probabilities
    a, b, c, d = 1-a-b-c at each of the `scale` levels, most significant bit first), keeps
    self-loops, merges duplicate samples, then draws one value uniform(vlo, vhi) per unique
    entry in CSR order from the same generator."""
    n = 1 << scale
    m = avg * n
    rng = np.random.default_rng(seed)
    r = np.zeros(m, dtype=np.int64)
    cc = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for lvl in range(scale):
        u = rng.random(m)
        bit = np.int64(1 << (scale - 1 - lvl))
        col_bit = ((u >= a) & (u < ab)) | (u >= abc)
        row_bit = u >= ab
        cc += bit * col_bit
        r += bit * row_bit
    M = from_coo(n, n, r, cc, None)
    M.val = rng.uniform(vlo, vhi, M.nnz)
    return M


def banded(n: int, w: int, seed: int) -> HostCSR:
    """Banded matrix: row i holds columns max(0,i-w//2) .. min(n-1, i+w//2), values U(-1,1)."""
    rng = np.random.default_rng(seed)
    half = w // 2
    offs = np.arange(-half, w - half, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), offs.shape[0])
    cols = rows + np.tile(offs, n)
    ok = (cols >= 0) & (cols < n)
    M = from_coo(n, n, rows[ok], cols[ok], None)
    M.val = rng.uniform(-1.0, 1.0, M.nnz)
    return M


def blockdiag(n: int, bs: int, seed: int) -> HostCSR:
    """Block-diagonal matrix with dense bs x bs blocks (last block truncated), values U(-1,1)."""
    rng = np.random.default_rng(seed)
    rows_l, cols_l = [], []
    for s in range(0, n, bs):
        e = min(n, s + bs)
        rr = np.repeat(np.arange(s, e, dtype=np.int64), e - s)
        cc = np.tile(np.arange(s, e, dtype=np.int64), e - s)
        rows_l.append(rr)
        cols_l.append(cc)
    M = from_coo(n, n, np.concatenate(rows_l), np.concatenate(cols_l), None)
    M.val = rng.uniform(-1.0, 1.0, M.nnz)
    return M


def erdos_renyi(n: int, deg: int, seed: int, ncols: int | None = None) -> HostCSR:
    """Erdos-Renyi style matrix: deg uniform column samples per row (duplicates merged)."""
    ncols = n if ncols is None else ncols
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    cols = rng.integers(0, ncols, size=n * deg, dtype=np.int64)
    M = from_coo(n, ncols, rows, cols, None)
    M.val = rng.uniform(-1.0, 1.0, M.nnz)
    return M


def random_sparse(nrows: int, ncols: int, density: float, seed: int, integer_values: bool = False,
                  empty_rows: float = 0.0) -> HostCSR:
    """Uniform random sparsity for small tests; optionally small-integer values (exact in FP64)
    and a fraction of forced-empty rows."""
    rng = np.random.default_rng(seed)
    mask = rng.random((nrows, ncols)) < density
    if empty_rows > 0 and nrows:
        er = rng.random(nrows) < empty_rows
        mask[er, :] = False
    r, c = np.nonzero(mask)
    M = from_coo(nrows, ncols, r, c, None)
    if integer_values:
        M.val = rng.integers(-4, 5, M.nnz).astype(np.float64)
    else:
        M.val = rng.uniform(-1.0, 1.0, M.nnz)
    return M


def family_matrix(family: str, n: int, param: int, seed: int) -> HostCSR:
    """One matrix of a named family: 'banded' (width), 'blockdiag' (block size),
    'er' (nnz per row) or 'rmat' (avg nnz per row; n rounded up to a power of two)."""
    if family == "banded":
        return banded(n, param, seed)
    if family == "blockdiag":
        return blockdiag(n, param, seed)
    if family == "er":
        return erdos_renyi(n, param, seed)
    if family == "rmat":
        scale = max(1, int(np.ceil(np.log2(max(n, 2)))))
        M = rmat(scale, param, seed)
        if M.nrows == n:
            return M
        # leading n x n block of the 2^scale R-MAT matrix
        rows = np.repeat(np.arange(M.nrows, dtype=np.int64), np.diff(M.row_ptr))
        keep = (rows < n) & (M.col < n)
        S = from_coo(n, n, rows[keep], M.col[keep].astype(np.int64), M.val[keep])
        return S
    raise ValueError(family)


BATCH_FAMILIES = ("banded", "blockdiag", "er", "rmat")


def batch_pairs(n_pairs: int = 512, m_lo: int = 256, m_hi: int = 65536, avg_lo: int = 4, avg_hi: int = 32,
                seed0: int = 0):
    """Independent square pairs (A_i, B_i): for pair i (seeded with seed0 + i) the size is
    log-uniform in [m_lo, m_hi], the family is drawn from banded / block-diagonal /
    Erdos-Renyi / R-MAT, the nonzeros per row from [avg_lo, avg_hi]; A_i and B_i are two
    seeded matrices of that family and size.  Values U(-1, 1)."""
    return [batch_pair(seed0 + i, m_lo, m_hi, avg_lo, avg_hi) for i in range(n_pairs)]


def batch_pair(seed: int, m_lo: int = 256, m_hi: int = 65536, avg_lo: int = 4, avg_hi: int = 32):
    """Pair number `seed` of batch_pairs (generated on its own, e.g. in a worker process)."""
    rng = np.random.default_rng(seed)
    m = int(round(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi)))))
    fam = BATCH_FAMILIES[int(rng.integers(len(BATCH_FAMILIES)))]
    avg = int(rng.integers(avg_lo, avg_hi + 1))
    A = family_matrix(fam, m, avg, seed=2 * seed)
    B = family_matrix(fam, m, avg, seed=2 * seed + 1)
    return A, B
