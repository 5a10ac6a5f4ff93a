"""Pins of the oracle's grid method for the nonlinear scalar example (Sec. VI-B,
App. E), on the CPU.

* App. E's interpolated minimum is exact for quadratics (the refinement uses
  the quadratic through three grid points).
* Without the refinement the grid combination is the plain min-plus product
  (against a brute-force numpy evaluation), associative to rounding.
* With a linear drift the problem is a discrete-time LQ problem (explicit Euler
  steps): every function the grid method minimises is then quadratic, so its
  values at interior grid points equal the discrete Riccati solution, which
  the test computes independently.
* The doubling order of the values (the GPU's) against the sequential fold:
  equal up to rounding without the refinement, and up to the interpolation
  error with it.
* The nonlinear example against the sequential upwind finite-difference
  method of the paper's comparison (an independent discretisation of the same
  HJB equation), to their discretisation error.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def lq_problem(G=121, T=12, x_range=6.0, interp=True):
    g = W.falling_body(G=G, T=T, x_range=x_range, interp=interp)
    g.d2 = 0.0  # dx/dt = 1 + u: linear, so the problem is LQ
    return g


def test_interpolated_minimum_is_exact_for_quadratics():
    g = W.falling_body(G=41, T=1)
    x = g.grid()
    rng = np.random.default_rng(3)
    for _ in range(10):
        a1, a2 = rng.uniform(0.5, 3.0, 2)
        p1, p2 = rng.uniform(-2.0, 2.0, 2)
        c1, c2 = rng.standard_normal(2)
        gv = a1 * (x - p1) ** 2 + c1
        fv = a2 * (x - p2) ** 2 + c2
        xs = (a1 * p1 + a2 * p2) / (a1 + a2)
        exact = a1 * (xs - p1) ** 2 + c1 + a2 * (xs - p2) ** 2 + c2
        M = np.tile(gv, (g.G, 1))
        got = oracle.grid_apply(g, M, fv)
        assert np.abs(got - exact).max() <= 1e-12 * max(1.0, abs(exact))


def test_ties_take_the_lowest_index():
    """Two grid minimisers with exactly equal sums, each the middle of three
    points on its own parabola: the refined minimum is that of the parabola
    at the lower index (the reading for ties), known in closed form
    c - a delta^2 for the parabola a (x - x_k - delta)^2 + c - a delta^2."""
    g = W.falling_body(G=41, T=1)
    dx, G = g.dx, g.G
    c = 1.25

    def parabola_points(a, delta):
        return [c + a * ((s * dx - delta) ** 2 - delta ** 2) for s in (-1, 0, 1)]

    k1, k2 = 12, 29
    a1, d1 = 2.0, 0.3 * dx
    a2, d2 = 0.5, -0.4 * dx
    row = np.full(G, 50.0)
    row[k1 - 1:k1 + 2] = parabola_points(a1, d1)
    row[k2 - 1:k2 + 2] = parabola_points(a2, d2)
    assert row[k1] == row[k2] == c and row.min() == c
    M = np.tile(row, (G, 1))
    got = oracle.grid_apply(g, M, np.zeros(G))
    expect = c - a1 * d1 ** 2
    assert np.abs(got - expect).max() <= 1e-12, (got[0], expect, c - a2 * d2 ** 2)
    # reversed rows put the other parabola at the lower index
    got_rev = oracle.grid_apply(g, M[:, ::-1].copy(), np.zeros(G))
    assert np.abs(got_rev - (c - a2 * d2 ** 2)).max() <= 1e-12


def test_plain_combination_is_min_plus_and_associative():
    g = W.falling_body(G=13, T=1, interp=False)
    rng = np.random.default_rng(4)
    A, B, C = (rng.uniform(0.0, 5.0, (13, 13)) for _ in range(3))
    AB = oracle.grid_combine(g, A, B)
    assert np.array_equal(AB, (A[:, :, None] + B[None, :, :]).min(axis=1))
    left = oracle.grid_combine(g, AB, C)
    right = oracle.grid_combine(g, A, oracle.grid_combine(g, B, C))
    assert np.abs(left - right).max() <= 1e-14 * np.abs(left).max()
    brute = (A[:, :, None, None] + B[None, :, :, None] + C[None, None, :, :]).min(axis=(1, 2))
    assert np.abs(left - brute).max() <= 1e-14 * np.abs(brute).max()


def discrete_lq_values(g):
    """V_k(x) = min_u dt (q x^2 + rho u^2)/2 + V_{k+1}(x + dt (d0 + d1 x + u)),
    V_N = qf x^2/2, N = T * substeps, for quadratic V = S x^2/2 - v x + z:
    minimiser u = (v' - S' a)/(rho + S' dt) with a = x + dt (d0 + d1 x).  The
    coefficients of each V_k are read off three exact evaluations."""
    dt = g.tau / g.substeps
    S, v, z = g.qf, 0.0, 0.0
    out = [(S, v, z)]
    for _ in range(g.T):
        for _ in range(g.substeps):
            def V(x, S=S, v=v, z=z):
                a = x + dt * (g.d0 + g.d1 * x)
                u = (v - S * a) / (g.rho + S * dt)
                y = a + dt * u
                return dt * 0.5 * (g.q * x * x + g.rho * u * u) + 0.5 * S * y * y - v * y + z
            f0, f1, fm = V(0.0), V(1.0), V(-1.0)
            S, v, z = f1 + fm - 2.0 * f0, -(f1 - fm) / 2.0, f0
        out.append((S, v, z))
    out.reverse()
    return out


def test_linear_drift_grid_method_equals_discrete_riccati():
    g = lq_problem()
    x = g.grid()
    Vb = oracle.grid_block(g)
    coef = discrete_lq_values(g)
    inner = np.abs(x) <= 2.0
    for values in (oracle.grid_values(g, Vb), oracle.grid_values_sequential(g, Vb)):
        for k, (S, v, z) in enumerate(coef):
            ref = 0.5 * S * x * x - v * x + z
            err = np.abs(values[k] - ref)[inner].max() / np.abs(ref[inner]).max()
            assert err <= 1e-10, (k, err)


def test_doubling_order_against_sequential_fold():
    plain = W.falling_body(G=61, T=13, interp=False)
    Vb = oracle.grid_block(plain)
    a, b = oracle.grid_values(plain, Vb), oracle.grid_values_sequential(plain, Vb)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    errs = []
    for G in (61, 121, 241):
        g = W.falling_body(G=G, T=13)
        Vb = oracle.grid_block(g)
        a, b = oracle.grid_values(g, Vb), oracle.grid_values_sequential(g, Vb)
        inner = np.abs(g.grid()) <= 3.0
        errs.append(np.abs(a - b)[:, inner].max() / np.abs(b[:, inner]).max())
    assert errs[-1] < 1e-4 and errs[0] > errs[-1], errs


def upwind_values(g, steps_per_block):
    """The sequential method of the comparison: an explicit upwind
    finite-difference scheme for -V_t = min_u l(x, u) + V_x f(x, u) on the
    grid (one-sided derivative against the flow, the minimising control
    u = -V_x / rho), stepped backward from V(t_f) = phi."""
    x = g.grid()
    dt = g.tau / steps_per_block
    V = 0.5 * g.qf * x * x
    out = [V.copy()]
    for _ in range(g.T):
        for _ in range(steps_per_block):
            fwd = np.empty_like(V); bwd = np.empty_like(V)
            fwd[:-1] = (V[1:] - V[:-1]) / g.dx; fwd[-1] = fwd[-2]
            bwd[1:] = (V[1:] - V[:-1]) / g.dx; bwd[0] = bwd[1]
            drift = g.d0 + g.d1 * x + g.d2 * x * x
            best = None
            for Vx in (fwd, bwd):
                u = -Vx / g.rho
                f = drift + u
                ok = (f >= 0) if Vx is fwd else (f <= 0)
                h = 0.5 * (g.q * x * x + g.rho * u * u) + Vx * f
                h = np.where(ok, h, np.inf)
                best = h if best is None else np.minimum(best, h)
            best = np.where(np.isfinite(best), best, 0.5 * g.q * x * x + (g.d0 + g.d1 * x + g.d2 * x * x) * fwd)
            V = V + dt * best
        out.append(V.copy())
    out.reverse()
    return np.array(out)


def test_nonlinear_example_against_upwind_method():
    g = W.falling_body(G=241, T=10)
    Vb = oracle.grid_block(g)
    vals = oracle.grid_values(g, Vb)
    up = upwind_values(g, steps_per_block=200)
    inner = np.abs(g.grid()) <= 2.0
    err = np.abs(vals - up)[:, inner].max() / np.abs(up[:, inner]).max()
    assert err < 2e-2, err
