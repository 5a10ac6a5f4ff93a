"""Pins of the oracle against facts that the paper and the mathematics fix.

Each test ties the oracle to something other than itself: the paper's worked
scan example, closed forms, a matrix exponential, an adaptive high-order ODE
solver, direct quadrature of the cost, brute-force minimisation, grid dynamic
programming, invariants of the combination rule.  CPU only.
"""
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sl
import scipy.optimize as so

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers (test side only)
# ---------------------------------------------------------------------------

def rand_psd(rng, n, rank=None, scale=1.0):
    rank = n if rank is None else rank
    G = rng.standard_normal((n, rank))
    return scale * G @ G.T / max(rank, 1)


def rand_element(rng, n, c_pd=True):
    return {
        "A": rng.standard_normal((n, n)),
        "b": rng.standard_normal(n),
        "C": rand_psd(rng, n) + (0.5 * np.eye(n) if c_pd else 0.0),
        "eta": rng.standard_normal(n),
        "J": rand_psd(rng, n),
        "zeta": np.array(rng.standard_normal()),
    }


def identity_element(n):
    return {"A": np.eye(n), "b": np.zeros(n), "C": np.zeros((n, n)), "eta": np.zeros(n),
            "J": np.zeros((n, n)), "zeta": np.array(0.0)}


def V_closed(e, x, z):
    """Conditional value function with invertible C (Sec. IV-A, eq. LQT_V_form2b)."""
    d = z - e["A"] @ x - e["b"]
    return float(e["zeta"] + 0.5 * x @ e["J"] @ x - x @ e["eta"] + 0.5 * d @ np.linalg.solve(e["C"], d))


def rel(a, b, floor=1e-8):
    a = np.asarray(a); b = np.asarray(b)
    den = max(np.abs(b).max(), floor)
    return np.abs(a - b).max() / den


def scalar_problem(a, ell, q, rho, Sf, T, K, tf=1.0, r=0.0, rf=0.0):
    """n = m = 1 constant-coefficient LQT: dx/dt = a x + ell u, l = q/2 (r-x)^2 + rho/2 u^2."""
    t = W.uniform_grid(0.0, tf, T)
    return W.Problem(name="scalar", n=1, m=1, nr=1, T=T, K=K, t=t,
                     F=W.const([[a]]), L=W.const([[ell]]), X=W.const([[q]]), U=W.const([[rho]]),
                     r=W.const([r]) if r else None, Xf=np.array([[Sf]]), rf=np.array([rf]) if rf else None,
                     x0=np.array([0.7]))


def scalar_riccati_closed_form(a, ell, q, rho, Sf, tau):
    """S(t_f - tau) for dS/dtau = 2 a S + q - beta S^2, beta = ell^2/rho (textbook
    closed form via the substitution S = s_plus + 1/w)."""
    beta = ell * ell / rho
    g = np.sqrt(a * a + beta * q)
    sp = (a + g) / beta
    if Sf == sp:
        return np.full_like(tau, sp)
    w0 = 1.0 / (Sf - sp)
    w = (w0 + beta / (2 * g)) * np.exp(2 * g * tau) - beta / (2 * g)
    return sp + 1.0 / w


def riccati_reference(p, rtol=1e-12, atol=1e-13):
    """Adaptive DOP853 solution of the paper's sequential equations (Sec. II-B,
    eqs. LQT_differential_S_v, LQT_optimal_control, optimal_trajectory_ODE_LQT)
    with the continuous-time coefficients, plus the running cost so that the
    optimal cost can be checked by quadrature."""
    n, m, nr = p.n, p.m, p.nr
    fF, fL, fX, fU = p.fn("F"), p.fn("L"), p.fn("X"), p.fn("U")
    fc, fH, fr = p.fn("c"), p.fn("H"), p.fn("r")

    def coefs(tt):
        tt = np.array([tt])
        F = fF(tt)[0]; L = fL(tt)[0]; X = fX(tt)[0]; U = fU(tt)[0]
        c = fc(tt)[0] if fc else np.zeros(n)
        H = fH(tt)[0] if fH else np.eye(n)
        r = fr(tt)[0] if fr else np.zeros(nr)
        return F, L, X, U, c, H, r

    def back(tt, y):
        F, L, X, U, c, H, r = coefs(tt)
        S = y[:n * n].reshape(n, n); v = y[n * n:n * n + n]
        B = L @ np.linalg.solve(U, L.T)
        dS = -F.T @ S - S @ F - H.T @ X @ H + S @ B @ S
        dv = -H.T @ X @ r + S @ c - F.T @ v + S @ B @ v
        dz = -0.5 * r @ X @ r + 0.5 * v @ B @ v + v @ c
        return np.concatenate([dS.ravel(), dv, [dz]])

    Hf = p.Hf if p.Hf is not None else np.eye(n)
    rf = p.rf if p.rf is not None else np.zeros(nr)
    yT = np.concatenate([(Hf.T @ p.Xf @ Hf).ravel(), Hf.T @ p.Xf @ rf, [0.5 * rf @ p.Xf @ rf]])
    # integrate piecewise so that piecewise-constant coefficients are never straddled
    tpts = p.t
    sols = []
    y = yT
    for j in range(p.T - 1, -1, -1):
        s = si.solve_ivp(back, (tpts[j + 1], tpts[j]), y, method="DOP853", rtol=rtol, atol=atol,
                         dense_output=True)
        sols.append((tpts[j], tpts[j + 1], s.sol))
        y = s.y[:, -1]
    sols.reverse()
    Sv = np.stack([sols[j][2](tpts[j]) for j in range(p.T)] + [yT])

    def Sv_at(tt, j):
        return sols[j][2](tt)

    def fwd(tt, w, j):
        F, L, X, U, c, H, r = coefs(tt)
        x = w[:n]
        y = Sv_at(tt, j)
        S = y[:n * n].reshape(n, n); v = y[n * n:n * n + n]
        u = -np.linalg.solve(U, L.T @ (S @ x - v))
        e = r - H @ x
        dcost = 0.5 * e @ X @ e + 0.5 * u @ U @ u
        return np.concatenate([F @ x + L @ u + c, [dcost]])

    xs = [p.x0.copy()]
    w = np.concatenate([p.x0, [0.0]])
    for j in range(p.T):
        s = si.solve_ivp(lambda tt, ww: fwd(tt, ww, j), (tpts[j], tpts[j + 1]), w, method="DOP853", rtol=rtol,
                         atol=atol)
        w = s.y[:, -1]
        xs.append(w[:n].copy())
    xT = w[:n]
    e = Hf @ xT - rf
    total_cost = w[n] + 0.5 * e @ p.Xf @ e
    S = Sv[:, :n * n].reshape(-1, n, n)
    v = Sv[:, n * n:n * n + n]
    zeta = Sv[:, -1]
    x = np.stack(xs)
    # control law eq. LQT_optimal_control at every boundary
    u = []
    for j in range(p.T + 1):
        F, L, X, U, c, H, r = coefs(tpts[j])
        u.append(-np.linalg.solve(U, L.T @ (S[j] @ x[j] - v[j])))
    return {"S": S, "v": v, "zeta": zeta, "x": x, "u": np.stack(u), "cost": total_cost}


# ---------------------------------------------------------------------------
# scan structure: the paper's worked example (Sec. II-C)
# ---------------------------------------------------------------------------

def load_golden_scan():
    rows = [list(map(float, ln.split())) for ln in open(os.path.join(GOLDEN, "scan_worked_example.txt"))
            if ln.strip() and not ln.startswith("#")]
    return np.array(rows[0]), np.array(rows[1]), np.array(rows[2])


def test_scan_worked_example_through_lqt_combination():
    """With n = 1, A = 1, C = J = b = 0, the LQT combination adds the eta's, so the
    oracle's right-to-left fold must give the paper's reverse sums and its
    trajectory recursion (x_{j+1} = x_j + b_j with b_j = a_j) the prefix sums."""
    a, pre, suf = load_golden_scan()
    T = len(a)
    el = {"A": np.ones((T, 1, 1)), "b": np.zeros((T, 1)), "C": np.zeros((T, 1, 1)), "eta": a[:, None].copy(),
          "J": np.zeros((T, 1, 1)), "zeta": np.zeros(T)}
    S, v, z = oracle.suffix_values(1, el)
    assert np.array_equal(v[:, 0], suf)
    assert np.array_equal(S[:, 0, 0], np.zeros(T))
    # prefix: T blocks with b_j = a_j; elements + S = v = 0
    p = scalar_problem(0.0, 1.0, 1.0, 1.0, 1.0, T=T, K=1)
    el2 = {"A": np.ones((T + 1, 1, 1)), "b": np.concatenate([a, [0.0]])[:, None], "C": np.zeros((T + 1, 1, 1)),
           "eta": np.zeros((T + 1, 1)), "J": np.zeros((T + 1, 1, 1)), "zeta": np.zeros(T + 1)}
    x, _ = oracle.trajectory(p, el2, np.zeros((T + 1, 1, 1)), np.zeros((T + 1, 1)), np.zeros(1))
    assert np.array_equal(x[1:, 0], pre)


# ---------------------------------------------------------------------------
# the combination rule (Sec. IV-A, eq. lqt_comb) and App. B
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_identity_element(n):
    """A=I, b=C=eta=J=0 is the neutral element (Sec. IV-A, zero-length interval)."""
    rng = np.random.default_rng(n)
    e = rand_element(rng, n)
    I = identity_element(n)
    for out in (oracle.combine(n, e, I), oracle.combine(n, I, e)):
        for k in e:
            np.testing.assert_allclose(out[k], e[k], rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_associativity(n):
    rng = np.random.default_rng(10 + n)
    for trial in range(5):
        a, b, c = (rand_element(rng, n, c_pd=False) for _ in range(3))
        l = oracle.combine(n, oracle.combine(n, a, b), c)
        r = oracle.combine(n, a, oracle.combine(n, b, c))
        for k in a:
            assert rel(l[k], r[k]) < 1e-11, (k, rel(l[k], r[k]))


@pytest.mark.parametrize("n", [2, 3])
def test_combination_equals_minimisation_over_intermediate_state(n):
    """Definition Assoc_operator_HJB: (V1 (x) V2)(x, y) = min_z V1(x,z) + V2(z,y).
    With invertible C the closed form (eq. LQT_V_form2b) is evaluated at random
    x, y and the minimum over z is found numerically (BFGS, no use of the lemma)."""
    rng = np.random.default_rng(20 + n)
    e1, e2 = rand_element(rng, n), rand_element(rng, n)
    e = oracle.combine(n, e1, e2)
    for _ in range(4):
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        f = lambda z: V_closed(e1, x, z) + V_closed(e2, z, y)
        res = so.minimize(f, np.zeros(n), method="BFGS", options={"gtol": 1e-11})
        assert abs(res.fun - V_closed(e, x, y)) < 1e-8 * max(1.0, abs(res.fun))


def test_combination_scalar_grid_minimum():
    """n = 1: minimum over a dense grid of z with the three-point quadratic
    refinement of App. E, against the combined element's closed form."""
    rng = np.random.default_rng(7)
    e1, e2 = rand_element(rng, 1), rand_element(rng, 1)
    e = oracle.combine(1, e1, e2)
    z = np.linspace(-30, 30, 600001)
    dz = z[1] - z[0]
    for x, y in ((0.3, -0.4), (1.2, 0.8), (-2.0, 1.5)):
        X, Y = np.array([x]), np.array([y])
        g = e1["zeta"] + 0.5 * e1["J"][0, 0] * x * x - x * e1["eta"][0] + \
            0.5 * (z - e1["A"][0, 0] * x - e1["b"][0]) ** 2 / e1["C"][0, 0]
        f = e2["zeta"] + 0.5 * e2["J"][0, 0] * z * z - z * e2["eta"][0] + \
            0.5 * (y - e2["A"][0, 0] * z - e2["b"][0]) ** 2 / e2["C"][0, 0]
        s = g + f
        i = int(np.argmin(s))
        assert 0 < i < len(z) - 1
        a_ = (s[i + 1] + s[i - 1] - 2 * s[i]) / (2 * dz * dz)
        b_ = (s[i + 1] - s[i - 1]) / (2 * dz)
        best = s[i] - b_ * b_ / (4 * a_)
        assert abs(best - V_closed(e, X, Y)) < 1e-9 * max(1.0, abs(best))


def test_invertibility_lemma():
    """App. B: for symmetric PSD C, J the eigenvalues of I + C J are real and >= 1,
    also for rank-deficient C, J."""
    rng = np.random.default_rng(3)
    for n in (1, 2, 3, 4, 8, 16):
        for rank in {0, 1, n // 2, n}:
            C = rand_psd(rng, n, rank=rank, scale=10.0) if rank else np.zeros((n, n))
            J = rand_psd(rng, n, rank=max(rank, 1), scale=10.0)
            ev = np.linalg.eigvals(np.eye(n) + C @ J)
            assert np.abs(ev.imag).max() < 1e-8 * max(1.0, np.abs(ev).max())
            assert ev.real.min() > 1.0 - 1e-9


# ---------------------------------------------------------------------------
# element construction (Sec. IV-B) and the sequential method (Sec. VI-A)
# ---------------------------------------------------------------------------

def test_scalar_riccati_closed_form():
    """The Riccati ODE of Sec. II-B with constant scalar coefficients has a closed
    form; the scan route (O1) and the sequential sweep (O2) both converge to it
    at order 4."""
    a, ell, q, rho, Sf = 0.3, 1.2, 2.0, 0.5, 0.1
    errs1, errs2 = [], []
    for K in (2, 4, 8):
        p = scalar_problem(a, ell, q, rho, Sf, T=20, K=K, tf=2.0)
        ref = scalar_riccati_closed_form(a, ell, q, rho, Sf, p.t[-1] - p.t)
        o1, o2 = oracle.solve(p), oracle.sequential(p)
        errs1.append(np.abs(o1["S"][:, 0, 0] - ref).max())
        errs2.append(np.abs(o2["S"][:, 0, 0] - ref).max())
    for errs in (errs1, errs2):
        ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
        assert all(12 < r < 20 for r in ratios), ratios
    p = scalar_problem(a, ell, q, rho, Sf, T=40, K=32, tf=2.0)
    ref = scalar_riccati_closed_form(a, ell, q, rho, Sf, p.t[-1] - p.t)
    assert np.abs(oracle.solve(p)["S"][:, 0, 0] - ref).max() < 1e-11
    assert np.abs(oracle.sequential(p)["S"][:, 0, 0] - ref).max() < 1e-11


def test_scalar_riccati_fixed_point():
    """S_f at the stable root s_+ = (a + sqrt(a^2 + beta q))/beta: the Riccati
    right-hand side vanishes there, so the sequential sweep stays at s_+ to
    rounding, and the scan route converges to it at order 4."""
    a, ell, q, rho = -0.4, 1.0, 1.5, 0.7
    beta = ell * ell / rho
    sp = (a + np.sqrt(a * a + beta * q)) / beta
    errs = []
    for K in (4, 8, 16):
        p = scalar_problem(a, ell, q, rho, sp, T=16, K=K, tf=3.0)
        assert np.abs(oracle.sequential(p)["S"][:, 0, 0] - sp).max() < 1e-14
        errs.append(np.abs(oracle.solve(p)["S"][:, 0, 0] - sp).max())
    assert all(12 < errs[i] / errs[i + 1] < 20 for i in range(len(errs) - 1)), errs


def hamiltonian_element(F, L, c, H, X, U, r, dt):
    """Element of one constant-coefficient interval of length dt from the matrix
    exponential of the Pontryagin system d/dt[x; p; 1] = [[F, -B, c], [-Q, -F^T, q],
    [0, 0, 0]] [x; p; 1] (B = L U^-1 L^T, Q = H^T X H, q = H^T X r).  Writing its
    blocks Phi_xx, Phi_xp, Phi_px, Phi_pp, phi_x, phi_p and matching the gradients
    of the closed form (eq. LQT_V_form2b) with the boundary costates gives
    C = -Phi_xp Phi_pp^-1, A = Phi_xx - Phi_xp Phi_pp^-1 Phi_px,
    b = phi_x - Phi_xp Phi_pp^-1 phi_p, J = -A^T Phi_px, eta = A^T phi_p."""
    n = F.shape[0]
    B = L @ np.linalg.solve(U, L.T)
    Q = H.T @ X @ H
    q = H.T @ X @ r
    M = np.zeros((2 * n + 1, 2 * n + 1))
    M[:n, :n] = F; M[:n, n:2 * n] = -B; M[:n, -1] = c
    M[n:2 * n, :n] = -Q; M[n:2 * n, n:2 * n] = -F.T; M[n:2 * n, -1] = q
    Phi = sl.expm(M * dt)
    Pxx, Pxp, Px = Phi[:n, :n], Phi[:n, n:2 * n], Phi[:n, -1]
    Ppx, Ppp, Pp = Phi[n:2 * n, :n], Phi[n:2 * n, n:2 * n], Phi[n:2 * n, -1]
    W_ = Pxp @ np.linalg.inv(Ppp)
    A = Pxx - W_ @ Ppx
    return {"A": A, "b": Px - W_ @ Pp, "C": -W_, "J": -A.T @ Ppx, "eta": A.T @ Pp}


@pytest.mark.parametrize("n,m,nr", [(1, 1, 1), (3, 2, 2), (4, 2, 3)])
def test_constant_coefficient_element_matches_matrix_exponential(n, m, nr):
    rng = np.random.default_rng(100 + n)
    F = rng.standard_normal((n, n)) * 0.7
    L = rng.standard_normal((n, m))
    c = rng.standard_normal(n)
    H = rng.standard_normal((nr, n))
    X = rand_psd(rng, nr) + 0.3 * np.eye(nr)
    U = rand_psd(rng, m) + 0.3 * np.eye(m)
    r = rng.standard_normal(nr)
    dt = 0.4
    ref = hamiltonian_element(F, L, c, H, X, U, r, dt)
    errs = []
    for K in (4, 8, 16, 256):
        p = W.Problem(name="const", n=n, m=m, nr=nr, T=1, K=K, t=np.array([0.0, dt]), F=W.const(F),
                      L=W.const(L), c=W.const(c), H=W.const(H), X=W.const(X), U=W.const(U), r=W.const(r),
                      Xf=np.eye(nr), x0=np.zeros(n))
        e = oracle.build_elements(p, 0, 1)
        errs.append(max(rel(e[k][0], ref[k]) for k in ("A", "b", "C", "eta", "J")))
    assert errs[-1] < 1e-10, errs
    assert 10 < errs[0] / errs[1] < 22 and 10 < errs[1] / errs[2] < 22, errs
    assert 3e4 < errs[2] / errs[3] < 1e5, errs  # 16x smaller step: 16^4


def test_lqr_special_case_zero_affine_terms():
    """Sec. II-B: with c = 0 and r = rf = 0 the problem is an LQR; the affine
    parts v, eta, b and zeta vanish identically."""
    p = W.general_time_varying(3, 2, 3, T=12, K=3, seed=8)
    p.c = None; p.r = None; p.rf = None
    o = oracle.solve(p, keep_elements=True)
    e = o["elements"]
    assert np.abs(e["b"]).max() == 0.0 and np.abs(e["eta"]).max() == 0.0 and np.abs(e["zeta"]).max() == 0.0
    assert np.abs(o["v"]).max() == 0.0 and np.abs(o["zeta"]).max() == 0.0
    s = oracle.sequential(p)
    assert np.abs(s["v"]).max() == 0.0 and np.abs(s["zeta"]).max() == 0.0


def test_semigroup_of_elements():
    """Theorem HJB-comb: V(.,s;.,t) = V(.,s;.,tau) (x) V(.,tau;.,t).  One block with
    2K steps against the combination of its two halves with K steps each: the
    difference is RK4 truncation only and falls at order 4."""
    base = W.general_time_varying(3, 2, 2, T=1, K=2, seed=9, tf=0.6)
    diffs = []
    for K in (8, 16, 32, 64):
        whole = W.resample(base, 2 * K)
        halves = W.refine(W.resample(base, K), 2)
        ew = oracle.build_elements(whole, 0, 1)
        eh = oracle.build_elements(halves, 0, 2)
        comb = oracle.combine(3, {k: eh[k][0] for k in eh}, {k: eh[k][1] for k in eh})
        diffs.append(max(rel(comb[k], ew[k][0]) for k in ("A", "b", "C", "eta", "J", "zeta")))
    assert diffs[-1] < 2e-10, diffs
    assert all(13 < diffs[i] / diffs[i + 1] < 20 for i in range(len(diffs) - 1)), diffs


@pytest.mark.parametrize("modes", [None, {"r": W.PER_INTERVAL, "X": W.CONST, "F": W.PER_INTERVAL}])
def test_time_varying_against_adaptive_reference(modes):
    """Every term active (non-symmetric F, output matrix H with nr != n, drift c,
    time-varying L, U, X, r).  S, v, zeta, x, u at every t_i from the scan route (O1)
    and the sequential sweep (O2) against an adaptive DOP853 solution of the
    paper's sequential equations; the optimal cost V(x0,t0) against direct
    quadrature of the cost along the reference trajectory."""
    base = W.general_time_varying(3, 2, 2, T=8, K=2, seed=11, tf=1.5, modes=modes)
    ref = riccati_reference(base)
    assert abs(ref["cost"] - (ref["zeta"][0] + 0.5 * base.x0 @ ref["S"][0] @ base.x0 - ref["v"][0] @ base.x0)) \
        < 1e-8 * abs(ref["cost"])
    e1, e2, eu2 = [], [], []
    for K in (8, 16, 32, 64):
        p = W.resample(base, K)
        o1, o2 = oracle.solve(p), oracle.sequential(p)
        e1.append(max(rel(o1[k], ref[k]) for k in ("S", "v", "zeta", "x", "u")))
        e2.append(max(rel(o2[k], ref[k]) for k in ("S", "v", "zeta", "x")))
        eu2.append(rel(o2["u"], ref["u"]))
        c1 = abs(o1["cost"] - ref["cost"]) / abs(ref["cost"])
        c2 = abs(o2["cost"] - ref["cost"]) / abs(ref["cost"])
        if K == 64:
            assert c1 < 1e-10 and c2 < 1e-8, (c1, c2)
    assert e1[-1] < 1e-10, e1
    assert e2[-1] < 1e-8, e2
    for e in (e1, e2):
        # order 4 while the error is above the reference solver's own ~1e-11 floor
        assert all(10 < e[i] / e[i + 1] < 22 for i in range(len(e) - 1) if e[i + 1] > 1e-10), e
    # O2's controls at the coarsest grid are still pre-asymptotic (ratio ~30)
    assert eu2[-1] < 2e-8, eu2
    assert all(10 < eu2[i] / eu2[i + 1] < 40 for i in range(len(eu2) - 1)), eu2


def test_scan_and_sequential_agree_at_every_boundary():
    """The parallel (scan) route and the sequential Riccati sweep agree at
    every t_i, to discretisation error that vanishes at order 4 (the 2-D point
    mass on a short horizon)."""
    base = W.point_mass_2d(T=32, K=4)
    base.t = W.uniform_grid(0.0, 4.0, 32)
    errs = []
    for K in (8, 16, 32, 64):
        p = W.resample(base, K)
        o1, o2 = oracle.solve(p), oracle.sequential(p)
        errs.append(max(rel(o1[k], o2[k]) for k in ("S", "v", "x", "u")))
    assert errs[-1] < 2e-9
    assert all(12 < errs[i] / errs[i + 1] < 20 for i in range(len(errs) - 1)), errs


# ---------------------------------------------------------------------------
# 1-D grid dynamic programming (Bellman's principle on a state grid)
# ---------------------------------------------------------------------------

def grid_dp_values(a, q, rho, r_fn, qf, rf, tf, dt, out_times, xg, ug):
    """Backward dynamic programming on a state grid for the scalar problem
    dx/dt = a x + u, l = q/2 (x - r(t))^2 + rho/2 u^2, phi = qf/2 (x - rf)^2.
    Each step takes the minimum over a control grid of l dt + V(x + f dt), with
    V between nodes from the three-point quadratic through the nearest nodes and
    the minimum over u refined with the three-point quadratic of App. E.  Uses
    midpoint (second-order) quadrature of the running cost and an RK2 state map
    so that Richardson extrapolation in dt is meaningful."""
    dx = xg[1] - xg[0]
    V = 0.5 * qf * (xg - rf) ** 2
    nsteps = int(round(tf / dt))
    out = {}
    times = [tf - k * dt for k in range(nsteps + 1)]
    want = {int(round((tf - tt) / dt)): tt for tt in out_times}
    if 0 in want:
        out[want[0]] = V.copy()
    X_, U_ = np.meshgrid(xg, ug, indexing="ij")
    for k in range(1, nsteps + 1):
        t0 = times[k]
        tm = t0 + 0.5 * dt
        # RK2 (midpoint) state map over [t0, t0+dt] with constant u
        xm = X_ + 0.5 * dt * (a * X_ + U_)
        xn = X_ + dt * (a * xm + U_)
        cost = dt * (0.5 * q * (xm - r_fn(tm)) ** 2 + 0.5 * rho * U_ ** 2)
        # quadratic interpolation of V at xn from the nearest three nodes
        i = np.clip(np.rint((xn - xg[0]) / dx).astype(int), 1, len(xg) - 2)
        s = (xn - xg[i]) / dx
        Vn = V[i] + 0.5 * s * (V[i + 1] - V[i - 1]) + 0.5 * s * s * (V[i + 1] - 2 * V[i] + V[i - 1])
        tot = cost + Vn
        j = np.clip(np.argmin(tot, axis=1), 1, len(ug) - 2)
        rows = np.arange(len(xg))
        g0, g1, g2 = tot[rows, j - 1], tot[rows, j], tot[rows, j + 1]
        du = ug[1] - ug[0]
        aa = (g2 + g0 - 2 * g1) / (2 * du * du)
        bb = (g2 - g0) / (2 * du)
        V = g1 - np.where(aa > 0, bb * bb / (4 * np.where(aa > 0, aa, 1.0)), 0.0)
        if k in want:
            out[want[k]] = V.copy()
    return out


@pytest.mark.slow
def test_grid_dynamic_programming_1d():
    """The value function on a 1-D state grid from backward dynamic programming
    (Richardson-extrapolated in dt) has the quadratic form zeta + S x^2/2 - v x
    with the oracle's S, v, zeta at the block boundaries."""
    a, q, rho, qf, rf, tf = -0.5, 2.0, 0.5, 3.0, 0.4, 1.0
    r_fn = lambda tt: np.sin(2.0 * tt)
    T = 4
    t = W.uniform_grid(0.0, tf, T)
    p = W.Problem(name="dp", n=1, m=1, nr=1, T=T, K=32, t=t, F=W.const([[a]]), L=W.const([[1.0]]),
                  X=W.const([[q]]), U=W.const([[rho]]),
                  r=W.Coef(r_fn(W.stage_times(t, 32))[:, None], W.PER_STAGE),
                  Xf=np.array([[qf]]), rf=np.array([rf]), x0=np.array([0.5]))
    o = oracle.solve(p)
    xg = np.linspace(-4.0, 4.0, 401)
    ug = np.linspace(-14.0, 14.0, 141)
    fits = []
    for dt in (1.0 / 400, 1.0 / 800):
        vals = grid_dp_values(a, q, rho, r_fn, qf, rf, tf, dt, list(t), xg, ug)
        inner = np.abs(xg) <= 1.5
        fit = []
        for tt in t:
            Vg = vals[tt][inner]
            Amat = np.stack([np.ones(inner.sum()), 0.5 * xg[inner] ** 2, -xg[inner]], axis=1)
            fit.append(np.linalg.lstsq(Amat, Vg, rcond=None)[0])
        fits.append(np.array(fit))
    extrap = 2 * fits[1] - fits[0]  # (zeta, S, v) per boundary
    for i in range(T + 1):
        got = np.array([o["zeta"][i], o["S"][i, 0, 0], o["v"][i, 0]])
        assert np.abs(extrap[i] - got).max() < 2e-4 * max(1.0, np.abs(got).max()), (i, extrap[i], got)


def test_time_invariant_blocks_share_A_C_J():
    """Sec. VI-B (a time-invariant model has one conditional value function per
    block length): with F, L, H, X, U constant and a uniform grid, the oracle's
    elements have the same A, C, J in every block (to rounding: the block
    lengths of a linspace grid differ in their last bits), while b, eta, zeta
    follow the time-varying r and c.
    The time-invariant build computes A, C, J once and only b, eta, zeta per
    block, so its elements must equal the general build's."""
    p = W.general_time_varying(3, 2, 2, T=9, K=3, seed=41, tf=1.8,
                               modes={"F": W.CONST, "L": W.CONST, "H": W.CONST, "X": W.CONST, "U": W.CONST})
    e = oracle.build_elements(p, 0, p.T)
    for k in ("A", "C", "J"):
        assert max(rel(e[k][j], e[k][0]) for j in range(p.T)) < 1e-14, k
    for k in ("b", "eta", "zeta"):
        assert not np.allclose(e[k][1], e[k][0]), k
