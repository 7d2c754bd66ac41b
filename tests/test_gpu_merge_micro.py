"""GPU tests of the merge evaluation of Section 4.2 (spgemm_merge_micro): every method merges
every group of two ascending runs into the sorted group, with values moving with their keys,
for run lengths from 1 to 4,096, every CTA size and every value width.  Keys within a group
are distinct, so the expected output is unique; with repeated keys the keys must still come
out sorted (and, for the ranking merge and merge path, the first run's element first)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_05022_gb300 as spg
    spg.load_library()
    return spg


def _groups(groups, l, seed, distinct=True):
    rng = np.random.default_rng(seed)
    if distinct:
        keys = np.stack([rng.choice(1 << 30, 2 * l, replace=False) for _ in range(groups)]).astype(np.int32)
    else:
        keys = rng.integers(0, max(2, l // 4), size=(groups, 2 * l)).astype(np.int32)
    keys[:, :l].sort(axis=1)
    keys[:, l:].sort(axis=1)
    return keys


def _expected(keys, vals):
    order = np.argsort(keys, axis=1, kind="stable")  # stable: the first run's element first on ties
    return np.take_along_axis(keys, order, 1), None if vals is None else np.take_along_axis(vals, order, 1)


@pytest.mark.parametrize("method", ["ranking", "merge_path", "bitonic"])
@pytest.mark.parametrize("vb", [0, 4, 8])
@pytest.mark.parametrize("l,threads", [(1, 64), (32, 64), (256, 256), (1024, 1024), (4096, 512), (128, 1024)])
def test_merge_micro_distinct_keys(spg, method, vb, l, threads):
    groups = max(2, 8192 // l)
    keys = _groups(groups, l, seed=l + vb)
    vals = None
    if vb:
        vals = np.arange(keys.size).reshape(keys.shape)
        vals = vals.astype(np.int32) if vb == 4 else vals.astype(np.float64) * 0.5
    dk = torch.from_numpy(keys.ravel()).cuda()
    dv = None if vals is None else torch.from_numpy(vals.ravel()).cuda()
    ok, ov = spg.merge_micro(dk, l, method=method, threads=threads, vals=dv)
    torch.cuda.synchronize()
    ek, ev = _expected(keys, vals)
    assert np.array_equal(ok.cpu().numpy().reshape(keys.shape), ek)
    if vb:
        assert np.array_equal(ov.cpu().numpy().reshape(keys.shape), ev)


@pytest.mark.parametrize("method", ["ranking", "merge_path", "bitonic"])
def test_merge_micro_repeated_keys(spg, method):
    l = 512
    keys = _groups(16, l, seed=3, distinct=False)
    vals = np.arange(keys.size, dtype=np.int32).reshape(keys.shape)
    ok, ov = spg.merge_micro(torch.from_numpy(keys.ravel()).cuda(), l, method=method, threads=256,
                             vals=torch.from_numpy(vals.ravel()).cuda())
    torch.cuda.synchronize()
    ok = ok.cpu().numpy().reshape(keys.shape)
    ov = ov.cpu().numpy().reshape(keys.shape)
    ek, ev = _expected(keys, vals)
    assert np.array_equal(ok, ek)
    if method != "bitonic":
        assert np.array_equal(ov, ev)
    else:  # every value still travels with its key
        assert np.array_equal(np.take_along_axis(keys.reshape(-1), ov.reshape(-1), 0).reshape(keys.shape), ok)


def test_merge_micro_rejects_bad_arguments(spg):
    k = torch.zeros(1000, dtype=torch.int32, device="cuda")
    for kw in ({"l": 3}, {"l": 256}, {"l": 4, "threads": 96}, {"l": 1 << 16}):
        with pytest.raises(spg.SpgemmError):
            spg.merge_micro(k if kw.get("l") != 256 else k[:1000], kw["l"], threads=kw.get("threads", 256))
