"""Mixed-precision path (lqt_solve_mixed: FP32 products in the combinations,
FP64 LU solves and FP64 element build) against the FP64 oracle: relative
error per output within the 1e-4 target, and clearly above FP64 rounding (the
FP32 products are really used).  Error measure: max |mixed - oracle| over the
whole output tensor divided by max |oracle| (a stated accuracy target, not a
parity bound: FP32 rounding is absolute in scale, so a per-boundary relative
measure would be dominated by boundaries where u or x pass near zero)."""
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


@pytest.mark.slow
def test_mixed_point_mass_full_size_against_oracle():
    """The FP32-product path on the point-mass workload at its full size
    (T = 2^20, K = 4), every output at every boundary against the full FP64
    oracle: each within the 1e-4 relative target (max-norm measure above)."""
    import paper_2212_11744_gb300 as lqt
    p = W.point_mass_2d(T=1 << 20, K=4)
    dp = lqt.DeviceProblem(p)
    mixed = lqt.lqt_solve_mixed(dp)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    got = {k: mixed[k].cpu().numpy() for k in ("S", "v", "zeta", "x", "u")}
    cost = float(mixed["cost"][0])
    del mixed, dp
    ref = oracle.solve(p)
    errs = {k: rel(got[k], ref[k]) for k in got}
    assert max(errs.values()) <= 1e-4, errs
    assert abs(cost - ref["cost"]) <= 1e-4 * abs(ref["cost"])


@pytest.mark.slow
def test_mixed_large_state_full_size_against_oracle():
    """The FP32-product path on the n = 64, m = 16 workload at its full size
    (T = 2^16, K = 2).  The oracle cannot fold all 2^16 elements of n = 64 in
    seconds, so three checks, each within the 1e-4 target:
    * values at the last 256 boundaries against the oracle's solve of the
      last 256 sub-intervals with the terminal cost (the values at those
      boundaries depend on nothing else): the error accumulated by 256
      combinations of the scan;
    * states at the first 257 boundaries against the oracle's rollout over the
      first 256 sub-intervals (its own elements) with the values of the FP64
      path (itself checked against the oracle in test_gpu_parity.py);
    * at sampled boundaries k, (S, v, zeta)_k against the oracle's element k
      combined with the mixed path's own values at k + 1, and the control law."""
    import paper_2212_11744_gb300 as lqt
    p = W.large_state_n64(T=1 << 16)
    n, T = p.n, p.T
    dp = lqt.DeviceProblem(p)
    mixed = lqt.lqt_solve_mixed(dp)
    full = lqt.lqt_solve(dp)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    got = {k: mixed[k].cpu().numpy() for k in ("S", "v", "zeta", "x", "u")}
    S64, v64 = full["S"].cpu().numpy(), full["v"].cpu().numpy()
    del mixed, full, dp
    Ts = 256
    tail = oracle.solve(W.window(p, T - Ts, Ts))
    errs = {k: rel(got[k][T - Ts:], tail[k]) for k in ("S", "v", "zeta")}
    head = W.window(p, 0, Ts)
    el = oracle.build_elements(head, 0, Ts + 1)
    x_ref, u_ref = oracle.trajectory(head, el, S64[:Ts + 1], v64[:Ts + 1], p.x0)
    errs["x"] = rel(got["x"][:Ts + 1], x_ref)
    errs["u"] = rel(got["u"][:Ts + 1], u_ref)
    assert max(errs.values()) <= 1e-4, errs
    S, v, z = got["S"], got["v"], got["zeta"]
    L, U = p.L.values[0], p.U.values[0]
    for k in (0, 4097, T // 2 + 3, T - 1):
        e = {kk: vv[0] for kk, vv in oracle.build_elements(p, k, k + 1).items()}
        val = {"A": np.zeros((n, n)), "b": np.zeros(n), "C": np.zeros((n, n)), "eta": v[k + 1], "J": S[k + 1],
               "zeta": z[k + 1]}
        c = oracle.combine(n, e, val)
        assert rel(S[k], c["J"]) <= 1e-4, k
        assert rel(v[k], c["eta"]) <= 1e-4, k
        assert abs(z[k] - float(c["zeta"])) <= 1e-4 * abs(float(c["zeta"])), k
        assert rel(got["u"][k], np.linalg.solve(U, L.T @ (v[k] - S[k] @ got["x"][k]))) <= 1e-4, k


def test_mixed_n64_T4096_against_fp64_path():
    """The n = 64 workload at T = 4096 (every CTA slot of the CTA-per-element
    scan busy): the FP32-product path against the FP64 path (itself checked
    against the oracle at T = 64, 129 and at sampled boundaries of T = 2^16)
    within the 1e-4 target; the mixed solve runs first."""
    import paper_2212_11744_gb300 as lqt
    p = W.large_state_n64(T=4096)
    dp = lqt.DeviceProblem(p)
    mixed = lqt.lqt_solve_mixed(dp)
    torch.cuda.synchronize()
    full = lqt.lqt_solve(dp)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    errs = {k: rel(mixed[k].cpu().numpy(), full[k].cpu().numpy()) for k in ("S", "v", "zeta", "x", "u")}
    assert max(errs.values()) <= 1e-4, errs
