"""Allocation failures injected on the host: a per-plan cap on device memory (opts.max_bytes)
makes an allocation fail as if the device were full.  Every policy reports SPGEMM_ERR_OOM from
the stage whose allocation failed, a failed plan gives all its memory back when it is freed, and
the library keeps working: a plan allowed its full peak computes the oracle's C."""
import pytest

import gen
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


def _opts(policy):
    if policy == "learned":
        from paper_1504_05022_gb300.predictor import Predictor
        pred = Predictor.load()
        return pred.opts(), pred
    return {"alloc_policy": policy}, None


def _free_after_trim(spg):
    torch.cuda.synchronize()
    spg.pool_trim()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("policy", ["hybrid", "upper_bound", "learned", "precise"])
def test_allocation_cap_reports_oom_and_leaks_nothing(spg, oracle_mod, policy):
    A = gen.rmat(14, 16, seed=91)  # with bin-37 rows, column slices and merge rounds
    Ad = spg.CSR.from_host(A)
    opts, _keep = _opts(policy)
    free0 = _free_after_trim(spg)  # after the inputs and the weights are on the device
    plan = spg.Plan(Ad, Ad, **opts)
    C = plan.numeric()
    torch.cuda.synchronize()
    peak = plan.stats()["peak_bytes"]
    del plan, C
    stages = set()
    for frac in (0.0, 0.05, 0.3, 0.6, 0.9, 0.99):
        cap = max(1, int(frac * peak))
        try:
            plan = spg.Plan(Ad, Ad, max_bytes=cap, **opts)
        except spg.SpgemmError as e:
            assert "OOM" in str(e), str(e)
            stages.add("symbolic")
            continue
        with pytest.raises(spg.SpgemmError, match="OOM"):
            plan.numeric()
        stages.add("numeric")
        assert plan.stats()["held_bytes"] <= cap
        del plan
    assert stages == {"symbolic", "numeric"}, stages
    # everything the failed plans held went back to the pool, and from there to the system
    assert _free_after_trim(spg) >= free0 - (8 << 20)
    plan = spg.Plan(Ad, Ad, max_bytes=peak, **opts)
    C = plan.numeric()
    torch.cuda.synchronize()
    ref = oracle_mod.spgemm(A, A)
    rp, col, val = C.to_host()
    assert_csr_equal(rp, col, val, ref.row_ptr, ref.col, ref.val, ref.den, label=f"{policy} at its peak")
