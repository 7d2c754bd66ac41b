"""What the trained network gains over the method without it (the learned preallocation against
the paper's allocation methods, Section 3.1), on matrices the training held out.

The committed weights were trained on rows logged from 200 seeded matrices; every seed s with
s % 5 == 2 was held out.  Here the product A*A of held-out R-MAT matrices (seeds 7 and 27 of
the training recipe, 2^15 rows) and of a 2^18-row R-MAT the recipe never drew (seed 7, 8
samples per row) is computed three ways:

- hybrid: the paper's plain form, every bin-37 row starting at 256 entries and relaunched at
  twice the size whenever it overflows (Section 4.1);
- upper_bound: every row sized by its product count u_i (Section 3.1);
- learned: the bin-37 rows sized by the network's prediction, the exact path as fallback.

C must be the oracle's under every policy.  Against the paper's plain method (hybrid), the
learned plan must hold less device memory at its peak and run fewer bin-37 work items over all
its rounds (each relaunch of a row runs it again); at most 5% of the rows it sized may outgrow
their prediction.  Against the upper-bound method the gain depends on how loose the bound is
for the rows the network sizes: on the 2^18-row R-MAT (the regime of the 2^20-row benchmark)
the learned peak must be below the upper bound's; on the 2^15-row recipe matrices, whose long
rows' bounds are nearly tight (the network cannot save what the bound does not waste), it may
not exceed it by more than 1%."""
import os

import numpy as np
import pytest
import torch

import gen
from tests.helpers import assert_csr_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_1504_05022_gb300 as spg
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    spg.load_library()
    return spg


def _held_out(s):
    from paper_1504_05022_gb300 import learn
    fam, n, p = learn.recipe(s)
    assert s % 5 == 2 and fam == "rmat"
    return gen.family_matrix(fam, n, p, seed=s)


# case -> (matrix, whether the learned peak must be strictly below the upper bound's)
CASES = {"recipe seed 7 (2^15 rows)": (lambda: _held_out(7), False),
         "recipe seed 27 (2^15 rows)": (lambda: _held_out(27), False),
         "R-MAT 2^18 x 8, seed 7": (lambda: gen.rmat(18, 8, seed=7), True)}


@pytest.mark.parametrize("case", list(CASES))
def test_learned_preallocation_gains_over_plain_methods(spg, oracle_mod, case):
    from paper_1504_05022_gb300.predictor import WEIGHTS, Predictor
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights committed")
    make, strict = CASES[case]
    A = make()
    ref = oracle_mod.spgemm(A, A)
    Ad = spg.CSR.from_host(A)
    pred = Predictor.load()
    st = {}
    for policy, opts in (("hybrid", {"alloc_policy": "hybrid"}), ("upper_bound", {"alloc_policy": "upper_bound"}),
                         ("learned", pred.opts())):
        plan = spg.Plan(Ad, Ad, **opts)
        C = plan.numeric()
        torch.cuda.synchronize()
        rp, col, val = C.to_host()
        assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, label=f"{case} {policy}")
        plan.check()
        st[policy] = plan.stats()
        if policy == "learned":
            arr = plan.arrays()
        del plan, C
    b37 = arr["bin"] == 37
    loose = float(arr["u"][b37].sum()) / float(np.diff(ref.row_ptr)[b37].sum())
    h, ub, ln = st["hybrid"], st["upper_bound"], st["learned"]
    sized = ln["bin_count"][37] - ln["rows_dense"]  # the bin-37 rows the network sized
    print(f"\n{case}: bin37 {ln['bin_count'][37]} (dense {ln['rows_dense']}), "
          f"peak hybrid/ub/learned {h['peak_bytes']}/{ub['peak_bytes']}/{ln['peak_bytes']}, "
          f"item rounds hybrid/learned {h['item_rounds']}/{ln['item_rounds']}, "
          f"launches hybrid/learned {h['merge_rounds']}/{ln['merge_rounds']}, "
          f"C~ bytes hybrid/ub/learned {h['bytes_ctilde']}/{ub['bytes_ctilde']}/{ln['bytes_ctilde']}, "
          f"fallback {ln['rows_fallback']} of {sized}, sum u / nnz over bin 37 {loose:.2f}")
    assert sized > 100
    assert ln["peak_bytes"] < h["peak_bytes"]
    assert ln["item_rounds"] < h["item_rounds"]
    assert ln["rows_fallback"] <= 0.05 * sized
    if strict:
        assert ln["peak_bytes"] < ub["peak_bytes"]
    else:
        assert ln["peak_bytes"] <= 1.01 * ub["peak_bytes"]
