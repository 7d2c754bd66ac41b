"""The allocation-free row-pointer scan gives the same row pointers as the regular path.

spgemm_rowptr_scan_noalloc exists for callers that cannot allocate device memory
(an arena owns it, or an allocation's implicit synchronisation is not allowed).
Its scratch is a fixed device array inside the library, so this file checks,
through the C ABI, that two calls in a row reproduce C.row_ptr of the regular
spgemm_numeric path bit for bit, and that oversized inputs are refused before
any work is launched."""
import ctypes

import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_05022_gb300 as spg
    spg.load_library()
    return spg


def _noalloc_rowptr(lib, row_nnz_ptr, m, stream):
    out = torch.full((m + 1,), -7, dtype=torch.int64, device="cuda")
    rc = lib.spgemm_rowptr_scan_noalloc(ctypes.c_void_p(row_nnz_ptr), m, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    return out


def test_noalloc_rowptr_matches_regular_path_twice(spg):
    from paper_1504_05022_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    for A in (gen.rmat(14, 16, seed=5), gen.lap2d(300)):
        Ad = spg.CSR.from_host(A)
        plan = spg.Plan(Ad, Ad, stream=stream)
        C = plan.numeric()
        arrs = _lib.PlanArrays()
        assert lib.spgemm_plan_arrays_get(ctypes.c_void_p(plan.handle.ptr), ctypes.byref(arrs)) == 0
        m = A.nrows
        for _ in range(2):  # two calls in a row share the same scratch
            rp = _noalloc_rowptr(lib, arrs.row_nnz, m, stream)
            torch.cuda.synchronize()
            assert torch.equal(rp, C.row_ptr)
        del plan, C


def test_noalloc_rowptr_small_and_empty(spg):
    from paper_1504_05022_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    assert lib.spgemm_rowptr_scan_noalloc(None, 0, ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert out.item() == 0
    rng = np.random.default_rng(3)
    for m in (1, 2047, 2048, 2049, 100_000):
        sizes = torch.from_numpy(rng.integers(0, 50, m).astype(np.int32)).cuda()
        rp = _noalloc_rowptr(lib, sizes.data_ptr(), m, stream)
        torch.cuda.synchronize()
        ref = np.concatenate([[0], np.cumsum(sizes.cpu().numpy().astype(np.int64))])
        assert np.array_equal(rp.cpu().numpy(), ref)


def test_noalloc_rowptr_rejects_oversized(spg):
    from paper_1504_05022_gb300 import _lib
    lib = _lib.load()
    mx = lib.spgemm_rowptr_scan_noalloc_max_rows()
    assert mx == 32768 * 2048
    dummy = torch.zeros(2, dtype=torch.int64, device="cuda")
    # refused on the host before any kernel is enqueued
    assert lib.spgemm_rowptr_scan_noalloc(ctypes.c_void_p(dummy.data_ptr()), mx + 1,
                                          ctypes.c_void_p(dummy.data_ptr()), None) == 2
    assert lib.spgemm_rowptr_scan_noalloc(None, 5, ctypes.c_void_p(dummy.data_ptr()), None) == 1
