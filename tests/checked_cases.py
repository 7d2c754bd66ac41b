"""Products run by the bounds-checked build (SPGEMM_CHECKED=1, in a process of its own):
every kernel path on small cases, each C compared with the oracle, and the build's status
word read after each.  Prints one line per case; exits non-zero on the first failure.
Test infrastructure, run by tests/test_gpu_check_build.py."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import ctypes  # noqa: E402

import torch  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402
from tests.helpers import assert_csr_equal  # noqa: E402


def main():
    assert os.environ.get("SPGEMM_CHECKED") == "1"
    from paper_1504_05022_gb300 import _build, _lib
    _build.build_check()
    oracle.build()
    import paper_1504_05022_gb300 as spg
    L = spg.load_library()
    assert L._name.endswith("libspgemm_check.so"), L._name
    code = ctypes.c_int64(0)

    def status():
        torch.cuda.synchronize()
        _lib.check(L.spgemm_check_status(ctypes.byref(code), 1), "spgemm_check_status")
        return code.value

    assert status() == 0  # a checked build with nothing recorded yet
    from paper_1504_05022_gb300.predictor import Predictor
    pred = Predictor.load()
    cases = [
        ("lap2d64", gen.lap2d(64), None, {}),
        ("rmat12x16 hybrid", gen.rmat(12, 16, seed=101), None, {}),
        ("rmat13x16 learned", gen.rmat(13, 16, seed=102), None, pred.opts()),
        ("rmat13x16 upper bound, heap 8", gen.rmat(13, 16, seed=103), None, {"alloc_policy": "upper_bound", "heap_max_u": 8}),
        ("rmat14x8 precise", gen.rmat(14, 8, seed=104), None, {"alloc_policy": "precise"}),
        ("rmat12x16 split at small capacities", gen.rmat(12, 16, seed=105), None, {"smem_cap_max": 1024, "dense_min_u": -1}),
        ("rmat12x16 merge path", gen.rmat(12, 16, seed=106), None, {"merge_kernel": "merge_path"}),
        ("rmat16x4 compact slices, kept bitmaps", gen.rmat(16, 4, seed=107), None, {"dense_min_u": 1024}),
        ("rmat16x4 compact slices, bitmaps not kept", gen.rmat(16, 4, seed=108), None,
         {"dense_min_u": 1024, "dense_keep": -1}),
        ("rect two-level bitmap", gen.rmat(12, 24, seed=109), gen.erdos_renyi(4096, 30, seed=110, ncols=300001),
         {"dense_min_u": -1}),
        ("rect wide slices", gen.rmat(12, 24, seed=111), gen.erdos_renyi(4096, 30, seed=112, ncols=100001),
         {"dense_min_u": 600, "dense_span": 65536}),
    ]
    for label, A, B, opts in cases:
        B = A if B is None else B
        Ad = spg.CSR.from_host(A)
        Bd = Ad if B is A else spg.CSR.from_host(B)
        plan = spg.Plan(Ad, Bd, **opts)
        C = plan.numeric()
        ref = oracle.spgemm(A, B)
        rp, col, val = C.to_host()
        assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, label=label)
        plan.replay()  # the values-only kernels too
        plan.check()
        s = status()
        print(f"{label}: nnz(C) {C.nnz}, status {s}", flush=True)
        assert s == 0, f"{label}: a bounds check failed at site {s}"
    pairs = [gen.batch_pair(i) for i in (3, 17, 40)]
    As = [spg.CSR.from_host(A) for A, _ in pairs]
    Bs = [spg.CSR.from_host(B) for _, B in pairs]
    Cs = spg.spgemm_batched(As, Bs)
    for (A, B), C in zip(pairs, Cs):
        ref = oracle.spgemm(A, B)
        rp, col, val = C.to_host()
        assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, label="batched")
    s = status()
    print(f"batched: status {s}", flush=True)
    assert s == 0, f"batched: a bounds check failed at site {s}"
    print("all clean")


if __name__ == "__main__":
    main()
