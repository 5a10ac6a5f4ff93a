"""Method 2 (forward-ODE elements, prefix scan, eq. Opt_trajectory_method2)
through the C ABI against the oracle.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_gpu_parity import TOL, relerr, to_np

pytestmark = pytest.mark.gpu

CASES = [
    ("double_integrator_T1024_K10", lambda: W.double_integrator(T=1024, K=10)),
    ("point_mass_T1000_K4", lambda: W.point_mass_2d(T=1000, K=4)),
    ("general_n3_m2_nr2_T37", lambda: W.general_time_varying(3, 2, 2, T=37, K=3, seed=21)),
    ("general_mixed_modes_T45", lambda: W.general_time_varying(
        4, 2, 3, T=45, K=2, seed=22, modes={"r": W.PER_INTERVAL, "X": W.CONST, "F": W.PER_INTERVAL,
                                             "L": W.CONST, "U": W.PER_INTERVAL})),
    ("general_nonuniform_T29", lambda: W.general_time_varying(2, 1, 2, T=29, K=4, seed=23, nonuniform=True)),
    ("scalar_n1_T50", lambda: W.general_time_varying(1, 1, 1, T=50, K=5, seed=24)),
    ("n8_m4_T300", lambda: W.batched_member(5, T=300, n=8)),
    ("n8_m8_T33", lambda: W.general_time_varying(8, 8, 8, T=33, K=2, seed=25, tf=1.0)),
    ("T1", lambda: W.general_time_varying(3, 1, 3, T=1, K=4, seed=26, tf=0.5)),
    ("T2", lambda: W.general_time_varying(2, 2, 2, T=2, K=1, seed=27)),
    ("T3", lambda: W.general_time_varying(4, 2, 4, T=3, K=2, seed=28)),
    # n = 16 (one warp per element and per combination) and n = 64 (one CTA)
    ("n16_m8_T40_general", lambda: W.general_time_varying(16, 8, 16, T=40, K=2, seed=81, tf=1.0)),
    ("n16_batched_member_T300", lambda: W.batched_member(7, T=300, n=16)),
    ("n16_m1_T3", lambda: W.general_time_varying(16, 1, 16, T=3, K=2, seed=82, tf=0.5)),
    ("n64_m16_T64", lambda: W.large_state_n64(T=64)),
    ("n64_m16_T129_ragged", lambda: W.large_state_n64(T=129)),
]
IDS = [c[0] for c in CASES]


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name,make", CASES, ids=IDS)
def test_forward_elements_match_oracle(name, make):
    import paper_2212_11744_gb300 as lqt
    p = make()
    ref = oracle.build_elements_forward(p)
    got = lqt.lqt_build_elements_forward(lqt.DeviceProblem(p))
    torch.cuda.synchronize()
    for k in ("A", "b", "C", "eta", "J", "zeta"):
        assert relerr(to_np(got[k]), ref[k]) <= 1e-11, k


@pytest.mark.parametrize("name,make", CASES, ids=IDS)
def test_trajectory_method2_on_oracle_inputs(name, make):
    """Same forward elements and values on both sides (the oracle's)."""
    import paper_2212_11744_gb300 as lqt
    p = make()
    sol = oracle.solve(p)
    fe = oracle.build_elements_forward(p)
    ref = oracle.trajectory_method2(p, sol["S"], sol["v"])
    dp = lqt.DeviceProblem(p)
    got = lqt.lqt_trajectory_method2(dp, {k: dev(fe[k]) for k in fe}, {"S": dev(sol["S"]), "v": dev(sol["v"])})
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    for k in ("x", "u"):
        assert relerr(to_np(got[k]), ref[k]) <= TOL, k


@pytest.mark.parametrize("name,make", CASES, ids=IDS)
def test_solve_method2_matches_oracle(name, make):
    import paper_2212_11744_gb300 as lqt
    p = make()
    sol = oracle.solve(p)
    ref = oracle.trajectory_method2(p, sol["S"], sol["v"])
    got = lqt.lqt_solve_method2(lqt.DeviceProblem(p))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    for k in ("S", "v", "zeta"):
        assert relerr(to_np(got[k]), sol[k]) <= TOL, k
    for k in ("x", "u"):
        assert relerr(to_np(got[k]), ref[k]) <= TOL, k
    assert abs(float(got["cost"][0]) - sol["cost"]) <= TOL * max(1.0, abs(sol["cost"]))


@pytest.mark.slow
def test_method2_agrees_with_method1_at_full_size():
    """Point mass at T = 2^20, K = 4: Method 2 and Method 1 (lqt_solve) are two
    discretisations of the same optimal states; at h = 2.4e-5 they agree to far
    below 1e-9 (their difference is RK4 truncation, O(h^4))."""
    import paper_2212_11744_gb300 as lqt
    p = W.point_mass_2d(T=1 << 20, K=4)
    dp = lqt.DeviceProblem(p)
    m1 = lqt.lqt_solve(dp)
    m2 = lqt.lqt_solve_method2(dp)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    for k in ("S", "v", "zeta", "x", "u"):
        assert relerr(to_np(m2[k]), to_np(m1[k])) <= TOL, k


def test_method2_n16_level0_chunks_of_four():
    """n = 16 at T = 5000: the level-0 chunks hold 4 forward elements (the
    fold inside a chunk runs 4 combinations), 1250 chunks with a ragged
    prefix tree above them."""
    import paper_2212_11744_gb300 as lqt
    p = W.batched_member(7, T=5000, n=16)
    sol = oracle.solve(p)
    ref = oracle.trajectory_method2(p, sol["S"], sol["v"])
    got = lqt.lqt_solve_method2(lqt.DeviceProblem(p))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    for k in ("S", "v", "zeta"):
        assert relerr(to_np(got[k]), sol[k]) <= TOL, k
    for k in ("x", "u"):
        assert relerr(to_np(got[k]), ref[k]) <= TOL, k
