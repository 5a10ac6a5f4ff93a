"""Differentiable restatement of oracle O1 in plain PyTorch CPU FP64 ops.

TEST INFRASTRUCTURE ONLY (the oracle of the gradients).  It computes exactly
what lqt_oracle.c's O1 computes -- K classical RK4 steps per sub-interval of the
backward conditional HJB ODEs (Sec. IV-B, Theorem Backward_HJB_LQT), the
terminal element (Sec. IV-D), the sequential right-to-left fold with the LQT
combination (Sec. IV-A, eq. lqt_comb), the one-sub-interval Method 2 rollout
(Sec. IV-E) and the optimal cost V(x0, t0) -- written with torch tensor ops so
that torch.autograd yields the sequential reverse-mode adjoint of that whole
computation.  The element build is vectorised over sub-intervals (each
sub-interval's arithmetic is independent); the fold and the rollout are plain
Python loops in the order of the C oracle.

Supported here: H = identity (nr = n), Hf = identity, c = 0; F, L, X, U constant
or per interval; r constant, per interval or per half-step sample.
"""
from __future__ import annotations

import torch

CONST, PER_INTERVAL, PER_STAGE = 0, 1, 2


def _sym(a):
    return 0.5 * (a + a.transpose(-1, -2))


def _at_stage(values, mode, T, K, p):
    """Coefficient samples for every sub-interval at half-step p: [T, ...]."""
    if mode == CONST:
        return values[0].expand((T,) + values.shape[1:])
    if mode == PER_INTERVAL:
        return values
    idx = torch.arange(T) * (2 * K) + p
    return values[idx]


def element_rhs(A, b, C, eta, J, z, F, Bm, Q, q, rho):
    """Theorem Backward_HJB_LQT (c = 0) plus the zeta equation, batched."""
    BJ = Bm @ J
    dA = A @ BJ - A @ F
    Beta = (Bm @ eta.unsqueeze(-1)).squeeze(-1)
    db = -(A @ Beta.unsqueeze(-1)).squeeze(-1)
    dC = _sym(-(A @ Bm) @ A.transpose(-1, -2))
    deta = -q - (F.transpose(-1, -2) @ eta.unsqueeze(-1)).squeeze(-1) + (J @ Beta.unsqueeze(-1)).squeeze(-1)
    JF = J @ F
    dJ = _sym(-((F.transpose(-1, -2) @ J) + JF) + J @ BJ - Q)
    dz = -0.5 * rho + 0.5 * (eta * Beta).sum(-1)
    return dA, db, dC, deta, dJ, dz


def build_elements(prob, F, L, X, U, r):
    """Elements 0..T-1 (RK4) and the terminal element T, as tensors with a
    leading T+1 axis.  F, L, X, U, r are sample tensors in their modes."""
    n, T, K = prob.n, prob.T, prob.K
    t = torch.as_tensor(prob.t, dtype=torch.float64)
    h = (t[1:] - t[:-1]) / K
    modes = {k: getattr(prob, k).mode for k in ("F", "L", "X", "U")}
    rmode = prob.r.mode if prob.r is not None else CONST
    A = torch.eye(n, dtype=torch.float64).expand(T, n, n).clone()
    b = torch.zeros(T, n, dtype=torch.float64)
    C = torch.zeros(T, n, n, dtype=torch.float64)
    eta = torch.zeros(T, n, dtype=torch.float64)
    J = torch.zeros(T, n, n, dtype=torch.float64)
    z = torch.zeros(T, dtype=torch.float64)

    def coefs(p):
        Fs = _at_stage(F, modes["F"], T, K, p)
        Ls = _at_stage(L, modes["L"], T, K, p)
        Xs = _at_stage(X, modes["X"], T, K, p)
        Us = _at_stage(U, modes["U"], T, K, p)
        rs = _at_stage(r, rmode, T, K, p) if r is not None else torch.zeros(T, n, dtype=torch.float64)
        Bm = _sym(Ls @ torch.linalg.solve(Us, Ls.transpose(-1, -2)))
        Q = _sym(Xs)
        Xr = (Xs @ rs.unsqueeze(-1)).squeeze(-1)
        return Fs, Bm, Q, Xr, (rs * Xr).sum(-1)

    hh = h.view(T, 1, 1)
    hv = h.view(T, 1)
    for i in range(K - 1, -1, -1):
        cs = [coefs(2 * i + 2), coefs(2 * i + 1), coefs(2 * i)]

        def f(state, c):
            return element_rhs(*state, *c)

        y = (A, b, C, eta, J, z)
        scal = (hh, hv, hh, hv, hh, h)
        k1 = f(y, cs[0])
        y2 = tuple(a - 0.5 * s * k for a, s, k in zip(y, scal, k1))
        k2 = f(y2, cs[1])
        y3 = tuple(a - 0.5 * s * k for a, s, k in zip(y, scal, k2))
        k3 = f(y3, cs[1])
        y4 = tuple(a - s * k for a, s, k in zip(y, scal, k3))
        k4 = f(y4, cs[2])
        A, b, C, eta, J, z = (a - (s / 6.0) * (w + 2.0 * x + 2.0 * yk + v)
                              for a, s, w, x, yk, v in zip(y, scal, k1, k2, k3, k4))
    return (A, b, C, eta, J, z)


def terminal(Xf, rf, n):
    Jt = _sym(Xf)
    et = Xf @ rf if rf is not None else torch.zeros(n, dtype=torch.float64)
    zt = 0.5 * (rf @ (Xf @ rf)) if rf is not None else torch.zeros((), dtype=torch.float64)
    return torch.zeros(n, n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64), \
        torch.zeros(n, n, dtype=torch.float64), et, Jt, zt


def combine(e1, e2):
    """Sec. IV-A, eq. lqt_comb, with the zeta term (single elements)."""
    A1, b1, C1, eta1, J1, z1 = e1
    A2, b2, C2, eta2, J2, z2 = e2
    n = A1.shape[0]
    I = torch.eye(n, dtype=torch.float64)
    M = torch.linalg.solve(I + C1 @ J2, I)
    Mt = M.T
    A = A2 @ M @ A1
    z0 = M @ (b1 + C1 @ eta2)
    b = A2 @ z0 + b2
    C = _sym(A2 @ M @ C1 @ A2.T + C2)
    eta = A1.T @ Mt @ (eta2 - J2 @ b1) + eta1
    J = _sym(A1.T @ Mt @ J2 @ A1 + J1)
    lam = J2 @ z0 - eta2
    zeta = z1 + z2 + 0.5 * lam @ (C1 @ lam) + 0.5 * z0 @ (J2 @ z0) - z0 @ eta2
    return A, b, C, eta, J, zeta


def solve(prob, F, L, X, U, r, Xf, rf, x0):
    """O1 forward with autograd: returns dict of S [T+1,n,n], v, zeta, x, cost."""
    n, T = prob.n, prob.T
    el = build_elements(prob, F, L, X, U, r)
    term = terminal(Xf, rf, n)
    s = term
    Ss, vs, zs = [None] * (T + 1), [None] * (T + 1), [None] * (T + 1)
    Ss[T], vs[T], zs[T] = s[4], s[3], s[5]
    for k in range(T - 1, -1, -1):
        ek = tuple(a[k] for a in el)
        s = combine(ek, s)
        Ss[k], vs[k], zs[k] = s[4], s[3], s[5]
    I = torch.eye(n, dtype=torch.float64)
    xs = [x0]
    for j in range(T):
        A, b, C = el[0][j], el[1][j], el[2][j]
        W = I + C @ Ss[j + 1]
        xs.append(torch.linalg.solve(W, A @ xs[-1] + b + C @ vs[j + 1]))
    S = torch.stack(Ss)
    v = torch.stack(vs)
    zeta = torch.stack(zs)
    x = torch.stack(xs)
    cost = zeta[0] + 0.5 * x0 @ (S[0] @ x0) - v[0] @ x0
    return {"S": S, "v": v, "zeta": zeta, "x": x, "cost": cost}
