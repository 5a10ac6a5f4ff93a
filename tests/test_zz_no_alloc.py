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
    a = a.detach().cpu().numpy()
    b = b.detach().cpu().numpy()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))


@pytest.mark.parametrize("make", [lambda: W.point_mass_2d(T=4099, K=4),
                                  lambda: W.general_time_varying(3, 2, 2, T=517, K=2, seed=61)],
                         ids=["point_mass_T4099", "general_n3_T517"])
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
    p = W.point_mass_2d(T=1 << 20, K=1)
    dp = lqt.DeviceProblem(p)
    assert lqt.lqt_workspace_size(dp, lqt.LQT_WS_VALUE) > _abi.LQT_STATIC_SCRATCH_BYTES
    el = {k: torch.zeros(1, dtype=torch.float64, device="cuda") for k in ("A", "b", "C", "eta", "J", "zeta")}
    with pytest.raises(lqt.LQTError) as e:
        lqt.lqt_scan_value_noalloc(dp, el, out={"S": el["A"], "v": el["b"], "zeta": el["zeta"]})
    assert e.value.code == _abi.LQT_EWORKSPACE
