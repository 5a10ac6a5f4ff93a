"""Mixed-precision path (lqt_solve_mixed: FP32 products in the combinations,
FP64 LU solves and FP64 element build) against the FP64 oracle: relative
error per output within the 1e-4 target, and clearly above FP64 rounding (the
FP32 products are really used)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))


CASES = [
    ("point_mass_T4096", lambda: W.point_mass_2d(T=4096, K=4)),
    ("double_integrator_T1024", lambda: W.double_integrator()),
    ("batched_member_n8_T500", lambda: W.batched_member(11, T=500, n=8)),
    ("batched_member_n16_T300", lambda: W.batched_member(12, T=300, n=16)),
    ("large_state_n64_T128", lambda: W.large_state_n64(T=128)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_mixed_within_target(name, make):
    import paper_2212_11744_gb300 as lqt
    p = make()
    ref = oracle.solve(p)
    dp = lqt.DeviceProblem(p)
    mixed = lqt.lqt_solve_mixed(dp)
    full = lqt.lqt_solve(dp)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    errs = {k: rel(mixed[k].cpu().numpy(), ref[k]) for k in ("S", "v", "zeta", "x", "u")}
    assert max(errs.values()) <= 1e-4, errs
    full_err = max(rel(full[k].cpu().numpy(), ref[k]) for k in ("S", "v", "x"))
    assert max(errs[k] for k in ("S", "v", "x")) > 10 * full_err, (errs, full_err)
