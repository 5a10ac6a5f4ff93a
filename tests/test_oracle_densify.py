"""Pins of the oracle's within-block densification (values, states and
controls at every RK4 sub-step), on the CPU.

* One block is the sequential method: densifying a single sub-interval of K
  steps from its end values reproduces, at every sub-step, the sequential
  sweep (O2) run on the same fine grid as K sub-intervals of one step (the
  coefficient samples are the same arrays).
* Against an adaptive DOP853 solution of the Riccati and closed-loop ODEs at
  every sub-step time, converging at order 4.
* At block boundaries the densified arrays are the boundary solution itself.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.test_oracle_pins import rel, riccati_reference


def split_steps(p):
    """The same problem with every RK4 step as a sub-interval of its own
    (T K sub-intervals, K = 1), on identical coefficient arrays."""
    K = p.K
    co = {}
    for k, c in p.coefs().items():
        if c is None:
            co[k] = None
        elif c.mode == W.PER_INTERVAL:
            co[k] = W.Coef(np.repeat(c.values, K, axis=0), W.PER_INTERVAL)
        else:
            co[k] = c  # CONST, and PER_STAGE (2 K T + 1 = 2 (T K) + 1 samples on the same times)
    return W.Problem(name=p.name + "_split", n=p.n, m=p.m, nr=p.nr, T=p.T * K, K=1, t=oracle.fine_times(p),
                     Hf=p.Hf, Xf=p.Xf, rf=p.rf, x0=p.x0, extra=p.extra, funcs=p.funcs, **co)


def one_block(K):
    base = W.general_time_varying(3, 2, 2, T=1, K=K, seed=21, tf=0.8)
    return base


@pytest.mark.parametrize("K", [4, 8])
def test_single_block_densification_is_the_sequential_method(K):
    p = one_block(K)
    boundary = oracle.sequential(p)
    d = oracle.densify(p, boundary)
    ref = oracle.sequential(split_steps(p))
    for k in ("S", "v", "zeta", "x", "u"):
        assert rel(d[k], ref[k]) < 1e-13, (k, rel(d[k], ref[k]))


def test_boundaries_are_the_given_solution():
    p = W.point_mass_2d(T=32, K=4)
    sol = oracle.solve(p)
    d = oracle.densify(p, sol)
    for k in ("S", "v", "zeta", "x", "u"):
        assert np.array_equal(d[k][::p.K], sol[k]), k


@pytest.mark.parametrize("modes", [None, {"r": W.PER_INTERVAL, "F": W.PER_INTERVAL}])
def test_densified_solution_against_adaptive_reference(modes):
    """Every term time-varying (non-symmetric F, H with n_r != n, drift c).
    The O1 boundary solution densified at every sub-step against DOP853 at the
    same times: order 4, and < 2e-9 at K = 32."""
    base = W.general_time_varying(3, 2, 2, T=4, K=2, seed=12, tf=1.2, modes=modes)
    errs = []
    for K in (4, 8, 16, 32):
        p = W.resample(base, K)
        d = oracle.densify(p, oracle.solve(p))
        ref = riccati_reference(split_steps(p))
        errs.append(max(rel(d[k], ref[k]) for k in ("S", "v", "zeta", "x", "u")))
    assert errs[-1] < 2e-9, errs
    assert all(10 < errs[i] / errs[i + 1] < 40 for i in range(len(errs) - 1)), errs
