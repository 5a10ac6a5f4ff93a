"""Pins of the oracle's Method 2 path (forward-HJB elements, prefix fold,
eq. Opt_trajectory_method2), on the CPU.

* Forward-ODE elements of a constant-coefficient interval against the matrix
  exponential of the Pontryagin system (the same closed form that pins the
  backward-ODE elements), at order 4.
* Forward- and backward-ODE elements describe the same conditional value
  function: they agree, zeta included, to RK4 truncation (order 4).
* The prefix fold against a right-associated fold of the same elements
  (associativity) and, for constant coefficients, against the closed form of
  the whole interval [t_0, t_k].
* Method 2 states and controls against Method 1 (the scan path) and against
  an adaptive solution of the closed loop, at order 4.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.test_oracle_pins import hamiltonian_element, rand_psd, rel, riccati_reference


def const_problem(n, m, nr, K, dt, T=1, seed=0):
    rng = np.random.default_rng(300 + seed)
    F = rng.standard_normal((n, n)) * 0.7
    L = rng.standard_normal((n, m))
    c = rng.standard_normal(n)
    H = rng.standard_normal((nr, n))
    X = rand_psd(rng, nr) + 0.3 * np.eye(nr)
    U = rand_psd(rng, m) + 0.3 * np.eye(m)
    r = rng.standard_normal(nr)
    p = W.Problem(name="const", n=n, m=m, nr=nr, T=T, K=K, t=np.linspace(0.0, dt * T, T + 1), F=W.const(F),
                  L=W.const(L), c=W.const(c), H=W.const(H), X=W.const(X), U=W.const(U), r=W.const(r),
                  Xf=np.eye(nr), x0=rng.standard_normal(n))
    return p, (F, L, c, H, X, U, r)


@pytest.mark.parametrize("n,m,nr", [(1, 1, 1), (3, 2, 2), (4, 2, 3)])
def test_forward_element_matches_matrix_exponential(n, m, nr):
    errs = []
    for K in (4, 8, 16, 256):
        p, co = const_problem(n, m, nr, K, 0.4, seed=n)
        ref = hamiltonian_element(*co, 0.4)
        e = oracle.build_elements_forward(p, 0, 1)
        errs.append(max(rel(e[k][0], ref[k]) for k in ("A", "b", "C", "eta", "J")))
    assert errs[-1] < 1e-9, errs
    assert 10 < errs[0] / errs[1] < 22 and 10 < errs[1] / errs[2] < 22, errs
    assert 3e4 < errs[2] / errs[3] < 1e5, errs


def test_forward_and_backward_elements_agree_at_order_4():
    base = W.general_time_varying(3, 2, 2, T=6, K=2, seed=31, tf=1.2)
    errs = []
    for K in (4, 8, 16, 32):
        p = W.resample(base, K)
        fe = oracle.build_elements_forward(p)
        be = oracle.build_elements(p, 0, p.T)
        errs.append(max(rel(fe[k], be[k]) for k in ("A", "b", "C", "eta", "J", "zeta")))
    assert errs[-1] < 5e-8, errs
    assert all(12 < errs[i] / errs[i + 1] < 20 for i in range(len(errs) - 1)), errs


def test_prefix_fold_associativity_and_closed_form():
    p, co = const_problem(3, 2, 2, K=64, dt=0.25, T=6, seed=5)
    el = oracle.build_elements_forward(p)
    pre = oracle.prefix(3, el)
    # p_0 is the identity element
    assert np.array_equal(pre["A"][0], np.eye(3)) and np.abs(pre["C"][0]).max() == 0.0
    # right-associated fold of a_0..a_{k-1}
    for k in (1, 3, 6):
        acc = {f: el[f][k - 1] for f in el}
        for j in range(k - 2, -1, -1):
            acc = oracle.combine(3, {f: el[f][j] for f in el}, acc)
        assert max(rel(pre[f][k], acc[f]) for f in ("A", "b", "C", "eta", "J", "zeta")) < 1e-12
        # constant coefficients: the composite is the element of [t_0, t_k]
        ref = hamiltonian_element(*co, 0.25 * k)
        assert max(rel(pre[f][k], ref[f]) for f in ("A", "b", "C", "eta", "J")) < 1e-9


def test_method2_states_against_method1_and_adaptive_reference():
    base = W.general_time_varying(3, 2, 2, T=8, K=2, seed=11, tf=1.5)
    ref = riccati_reference(base)
    e1, e2 = [], []
    for K in (4, 8, 16, 32):
        p = W.resample(base, K)
        sol = oracle.solve(p)
        m2 = oracle.trajectory_method2(p, sol["S"], sol["v"])
        e1.append(max(rel(m2["x"], sol["x"]), rel(m2["u"], sol["u"])))
        e2.append(max(rel(m2["x"], ref["x"]), rel(m2["u"], ref["u"])))
        assert np.array_equal(m2["x"][0], p.x0)
    for e in (e1, e2):
        assert e[-1] < 1e-9, e
        assert all(12 < e[i] / e[i + 1] < 20 for i in range(len(e) - 1)), e
