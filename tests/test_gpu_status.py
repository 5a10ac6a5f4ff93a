"""The device status word's singular-system report: a combination whose
system W = I + C J is singular to working precision (an LU pivot at most
2^-40 of its row's scale max(1, max_j |W_ij|)) sets LQT_ESINGULAR; a
well-conditioned one, even with W as small as 1e-9 I, does not.  With PSD C
and J this cannot happen (App. B: the eigenvalues of I + C J are >= 1), so
the elements here are built by hand with an indefinite J: element 0 has
A = C = I, element 1 (the last) J = j I.  Both the thread path (n = 2) and the
warp path (n = 16) of the value scan."""
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [2, 16])
@pytest.mark.parametrize("j,expect", [(-0.5, "ok"), (-(1.0 - 1e-9), "ok"), (-(1.0 - 1e-14), "singular"),
                                      (-1.0, "singular_or_nonfinite")],
                         ids=["W=0.5I", "W=1e-9I", "W=1e-14I", "W=0"])
def test_near_singular_combination_is_reported(n, j, expect):
    import paper_2212_11744_gb300 as lqt
    from paper_2212_11744_gb300 import _abi
    p = W.general_time_varying(n, max(1, n // 2), n, T=1, K=1, seed=5)
    dp = lqt.DeviceProblem(p)
    f64 = dict(dtype=torch.float64, device="cuda")
    eye = torch.eye(n, **f64)
    zero = torch.zeros(n, n, **f64)
    el = {"A": torch.stack([eye, zero]), "b": torch.zeros(2, n, **f64), "C": torch.stack([eye, zero]),
          "eta": torch.zeros(2, n, **f64), "J": torch.stack([zero, j * eye]), "zeta": torch.zeros(2, **f64)}
    assert lqt.lqt_get_status() == 0
    out = lqt.lqt_scan_value(dp, el)
    torch.cuda.synchronize()
    st = lqt.lqt_get_status()
    if expect == "ok":
        assert st == 0, lqt.lqt_strerror(st)
        assert torch.allclose(out["S"][0], (j / (1.0 + j)) * eye, rtol=1e-6)
    elif expect == "singular":
        assert st == _abi.LQT_ESINGULAR, lqt.lqt_strerror(st)
    else:
        assert st in (_abi.LQT_ESINGULAR, _abi.LQT_ENONFINITE), lqt.lqt_strerror(st)
    assert lqt.lqt_get_status() == 0
