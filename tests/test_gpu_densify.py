"""lqt_densify (values, states and controls at every RK4 sub-step) against the
oracle's densification, through the C ABI.  Tolerance and error measure as in
test_gpu_parity.py (relative 1e-9 per output tensor)."""
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
    # K = 8: at K <= 4 this problem's Riccati RK4 (the sequential method, and so
    # the densification) is unstable at its right end, while the element
    # build is not
    ("general_mixed_modes_T45_K8", lambda: W.resample(W.general_time_varying(
        4, 2, 3, T=45, K=2, seed=22, modes={"r": W.PER_INTERVAL, "X": W.CONST, "F": W.PER_INTERVAL,
                                             "L": W.CONST, "U": W.PER_INTERVAL}), 8)),
    ("general_nonuniform_T29", lambda: W.general_time_varying(2, 1, 2, T=29, K=4, seed=23, nonuniform=True)),
    ("scalar_n1_T50_K16", lambda: W.resample(W.general_time_varying(1, 1, 1, T=50, K=5, seed=24), 16)),
    ("n8_m4_T300", lambda: W.batched_member(5, T=300, n=8)),
    # (seed 25, t_f = 1 is unstable for the Riccati RK4 at every K <= 8; this one is not)
    ("n8_m8_T33", lambda: W.general_time_varying(8, 8, 8, T=33, K=4, seed=26, tf=0.5)),
    ("T1_K1", lambda: W.general_time_varying(3, 1, 3, T=1, K=1, seed=26, tf=0.5)),
]


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_densify_of_oracle_boundary_solution(name, make):
    """Both sides densify the same (oracle) boundary solution."""
    import paper_2212_11744_gb300 as lqt
    p = make()
    sol = oracle.solve(p)
    ref = oracle.densify(p, sol)
    dp = lqt.DeviceProblem(p)
    got = lqt.lqt_densify(dp, {k: dev(sol[k]) for k in ("S", "v", "zeta", "x")})
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    errs = {k: relerr(to_np(got[k]), ref[k]) for k in ("S", "v", "zeta", "x", "u")}
    assert all(e <= TOL for e in errs.values()), errs
    # boundary points are the given solution, bit for bit
    for k in ("S", "v", "zeta", "x"):
        assert np.array_equal(to_np(got[k])[::p.K], sol[k]), k


@pytest.mark.parametrize("name,make", CASES[:3] + CASES[6:7], ids=[c[0] for c in CASES[:3] + CASES[6:7]])
def test_solve_then_densify_matches_oracle(name, make):
    import paper_2212_11744_gb300 as lqt
    p = make()
    ref = oracle.densify(p, oracle.solve(p))
    dp = lqt.DeviceProblem(p)
    got = lqt.lqt_densify(dp, lqt.lqt_solve(dp))
    torch.cuda.synchronize()
    errs = {k: relerr(to_np(got[k]), ref[k]) for k in ("S", "v", "zeta", "x", "u")}
    assert all(e <= TOL for e in errs.values()), errs


def test_densify_full_point_mass_sampled():
    """Point mass at T = 2^20, K = 4 (the benchmarked size): the GPU chain
    solve -> densify at 64 sampled sub-intervals against the oracle densifying
    the GPU's own boundary solution of those sub-intervals one by one (each
    sub-interval's densification depends only on its two boundary values)."""
    import paper_2212_11744_gb300 as lqt
    p = W.point_mass_2d(T=1 << 20, K=4)
    dp = lqt.DeviceProblem(p)
    sol = lqt.lqt_solve(dp)
    d = lqt.lqt_densify(dp, sol)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    rng = np.random.default_rng(9)
    js = np.sort(rng.choice(p.T, 64, replace=False))
    S, v, z, x = (to_np(sol[k]) for k in ("S", "v", "zeta", "x"))
    worst = 0.0
    for j in js:
        sub = W.window(p, int(j), 1)
        loc = {"S": S[j:j + 2], "v": v[j:j + 2], "zeta": z[j:j + 2], "x": x[j:j + 2]}
        ref = oracle.densify(sub, loc)
        K = p.K
        for k in ("S", "v", "zeta", "x", "u"):
            g = to_np(d[k][j * K:(j + 1) * K + 1])
            worst = max(worst, relerr(g, ref[k]))
    assert worst <= TOL, worst


def test_unstable_step_is_reported():
    """The same problem at K = 2: the Riccati RK4 diverges in the last
    sub-interval (the oracle's states there are not finite).  The status word
    reports exactly whether the GPU's outputs contain a non-finite value."""
    import paper_2212_11744_gb300 as lqt
    p = W.general_time_varying(4, 2, 3, T=45, K=2, seed=22, modes={"r": W.PER_INTERVAL, "X": W.CONST,
                                                                     "F": W.PER_INTERVAL, "L": W.CONST,
                                                                     "U": W.PER_INTERVAL})
    sol = oracle.solve(p)
    assert not np.isfinite(oracle.densify(p, sol)["x"]).all()
    dp = lqt.DeviceProblem(p)
    got = lqt.lqt_densify(dp, {k: dev(sol[k]) for k in ("S", "v", "zeta", "x")})
    torch.cuda.synchronize()
    finite = all(bool(torch.isfinite(got[k]).all()) for k in ("S", "v", "zeta", "x"))
    assert not finite or float(got["S"].abs().max()) > 1e5  # diverged either way
    assert lqt.lqt_get_status() == (0 if finite else lqt._abi.LQT_ENONFINITE)
    assert lqt.lqt_get_status() == 0
