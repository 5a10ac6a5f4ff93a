"""Time-invariant element build (lqt_build_elements_invariant, lqt_solve_invariant
and the batched flag) against the oracle's general element build, through the
C ABI.  The specialisation changes the arithmetic's organisation, not its steps,
so the elements match the oracle's at the general build's 1e-11 and the
solutions at 1e-9."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_gpu_parity import TOL, relerr, to_np

pytestmark = pytest.mark.gpu

ALL_CONST = {"F": W.CONST, "L": W.CONST, "H": W.CONST, "X": W.CONST, "U": W.CONST}

CASES = [
    ("double_integrator_T1024_K10", lambda: W.double_integrator(T=1024, K=10)),
    ("general_n3_H_c_stage_r", lambda: W.general_time_varying(3, 2, 2, T=41, K=3, seed=51, tf=1.5, modes=ALL_CONST)),
    ("general_n4_interval_r", lambda: W.general_time_varying(
        4, 2, 4, T=29, K=2, seed=52, tf=1.2, modes=dict(ALL_CONST, r=W.PER_INTERVAL, c=W.PER_INTERVAL))),
    ("scalar_n1", lambda: W.general_time_varying(1, 1, 1, T=50, K=5, seed=53, modes=ALL_CONST)),
    ("batched_member_n2", lambda: W.batched_member(11, T=300, n=2)),
    ("batched_member_n4", lambda: W.batched_member(12, T=257, n=4)),
    ("batched_member_n8", lambda: W.batched_member(13, T=301, n=8)),
    ("batched_member_n16", lambda: W.batched_member(14, T=129, n=16)),
    ("T1", lambda: W.general_time_varying(3, 1, 3, T=1, K=4, seed=54, tf=0.5, modes=ALL_CONST)),
    ("general_n16_m8_H_c", lambda: W.general_time_varying(16, 8, 16, T=33, K=2, seed=56, tf=0.8, modes=ALL_CONST)),
    ("large_state_n64_T64", lambda: W.large_state_n64(T=64)),
    ("large_state_n64_T129", lambda: W.large_state_n64(T=129)),
]
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("name,make", CASES, ids=IDS)
def test_invariant_elements_match_oracle(name, make):
    import paper_2212_11744_gb300 as lqt
    p = make()
    ref = oracle.build_elements(p)
    got = lqt.lqt_build_elements_invariant(lqt.DeviceProblem(p))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    for k in ("A", "b", "C", "eta", "J", "zeta"):
        assert relerr(to_np(got[k]), ref[k]) <= 1e-11, k


@pytest.mark.parametrize("name,make", CASES, ids=IDS)
def test_solve_invariant_matches_oracle(name, make):
    import paper_2212_11744_gb300 as lqt
    p = make()
    ref = oracle.solve(p)
    got = lqt.lqt_solve_invariant(lqt.DeviceProblem(p))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    for k in ("S", "v", "zeta", "x", "u"):
        assert relerr(to_np(got[k]), ref[k]) <= TOL, k
    assert abs(float(got["cost"][0]) - ref["cost"]) <= TOL * max(1.0, abs(ref["cost"]))


def test_nonuniform_grid_is_reported():
    import paper_2212_11744_gb300 as lqt
    p = W.general_time_varying(2, 1, 2, T=29, K=4, seed=23, nonuniform=True, modes=ALL_CONST)
    lqt.lqt_build_elements_invariant(lqt.DeviceProblem(p))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == lqt._abi.LQT_EINVAL
    assert lqt.lqt_get_status() == 0


def test_time_varying_coefficients_are_rejected_on_host():
    import paper_2212_11744_gb300 as lqt
    p = W.general_time_varying(3, 2, 2, T=9, K=2, seed=55)  # everything per stage
    with pytest.raises(lqt.LQTError) as e:
        lqt.lqt_solve_invariant(lqt.DeviceProblem(p))
    assert e.value.code == lqt._abi.LQT_EUNSUPPORTED


@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_batched_invariant_build_matches_oracle(n):
    from paper_2212_11744_gb300.batch import Batch
    probs = [W.batched_member(500 + 10 * n + i, T=T, n=n) for i, T in enumerate([37, 123, 300, 64])]
    bt = Batch(probs)
    general = bt.solve()
    bt.set_invariant_build(True)
    out = bt.solve()
    torch.cuda.synchronize()
    import paper_2212_11744_gb300 as lqt
    assert lqt.lqt_get_status() == 0
    for k in ("S", "v", "zeta", "x"):
        assert relerr(to_np(out[k]), to_np(general[k])) <= 1e-10, k
    for b, p in enumerate(probs):
        ref = oracle.solve(p)
        got = bt.problem_slice(out, b)
        for k in ("S", "v", "zeta", "x", "u"):
            assert relerr(got[k].cpu().numpy(), ref[k]) <= TOL, (b, k)


def test_long_uniform_grid_is_accepted():
    """A linspace over [0, 1310.72] with 2^16 sub-intervals: lengths differ by
    up to 1.05e-11 relative through the rounding of t alone, which is not a
    non-uniform grid.  The shared A, C, J are integrated with the first
    sub-interval's length, the oracle's with each one's own, so they agree to
    that relative spread (bound 1e-10), the rest as in the cases above."""
    import paper_2212_11744_gb300 as lqt
    p = W.batched_member(17, T=1 << 16, n=2)
    p.t = W.uniform_grid(0.0, 0.02 * p.T, p.T)
    ref = oracle.build_elements(p)
    got = lqt.lqt_build_elements_invariant(lqt.DeviceProblem(p))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    for k in ("A", "b", "C", "eta", "J", "zeta"):
        assert relerr(to_np(got[k]), ref[k]) <= 1e-10, k
