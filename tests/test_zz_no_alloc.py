"""lqt_scan_value_noalloc: the value scan for callers that may not allocate
device memory while they run (its scratch is a fixed array inside the library
instead of a caller workspace).  Called through the C ABI and checked against
lqt_scan_value, which takes a workspace, on two calls in a row.  Collected
last so that a failure here leaves every other test already run."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9


def relerr(a, b):
    """Per-boundary relative error (the measure of test_gpu_parity.py)."""
    a = a.detach().cpu().numpy().reshape(a.shape[0], -1)
    b = b.detach().cpu().numpy().reshape(b.shape[0], -1)
    r = np.linalg.norm(b, axis=1)
    return float((np.linalg.norm(a - b, axis=1) / np.maximum(r, max(1e-8 * r.max(), 1e-300))).max())


@pytest.mark.parametrize("make", [lambda: W.point_mass_2d(T=4099, K=4),
                                  lambda: W.general_time_varying(3, 2, 2, T=517, K=2, seed=61),
                                  lambda: W.batched_member(9, T=500, n=16),
                                  lambda: W.batched_member(10, T=1951, n=16)],
                         ids=["point_mass_T4099", "general_n3_T517", "n16_T500_team_scan", "n16_T1951_at_limit"])
def test_noalloc_scan_matches_workspace_scan_twice(make):
    import paper_2212_11744_gb300 as lqt
    p = make()
    dp = lqt.DeviceProblem(p)
    el = lqt.lqt_build_elements(dp)
    ref = lqt.lqt_scan_value(dp, el)
    for _ in range(2):
        got = lqt.lqt_scan_value_noalloc(dp, el)
        torch.cuda.synchronize()
        assert lqt.lqt_get_status() == 0
        for k in ("S", "v", "zeta"):
            assert relerr(got[k], ref[k]) <= TOL, k


def test_noalloc_rejects_problems_beyond_its_scratch():
    import paper_2212_11744_gb300 as lqt
    from paper_2212_11744_gb300 import _abi
    # one sub-interval above the largest T the header states for n = 4
    p = W.point_mass_2d(T=26878, K=1)
    dp = lqt.DeviceProblem(p)
    assert lqt.lqt_workspace_size(dp, lqt.LQT_WS_VALUE) > _abi.LQT_STATIC_SCRATCH_BYTES
    el = {k: torch.zeros(1, dtype=torch.float64, device="cuda") for k in ("A", "b", "C", "eta", "J", "zeta")}
    with pytest.raises(lqt.LQTError) as e:
        lqt.lqt_scan_value_noalloc(dp, el, out={"S": el["A"], "v": el["b"], "zeta": el["zeta"]})
    assert e.value.code == _abi.LQT_EWORKSPACE
