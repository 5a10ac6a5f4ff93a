"""lqt_backward (and the autograd Function over it) against the oracle's
sequential reverse mode (torch.autograd through the PyTorch restatement of
oracle O1) and against central finite differences of the C oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import lqt_torch as LT

pytestmark = pytest.mark.gpu

TOL = 1e-9


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))


def cpu(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64)


def oracle_grads(p, wS, wv, wz, wx, wc):
    """Gradients of L = <wS,S> + <wv,v> + <wz,zeta> + <wx,x> + wc*cost from the
    oracle's reverse mode."""
    F = cpu(p.F.values).requires_grad_()
    L = cpu(p.L.values).requires_grad_()
    X = cpu(p.X.values).requires_grad_()
    U = cpu(p.U.values).requires_grad_()
    r = cpu(p.r.values).requires_grad_()
    Xf = cpu(p.Xf).requires_grad_()
    rf = cpu(p.rf).requires_grad_() if p.rf is not None else None
    x0 = cpu(p.x0).requires_grad_()
    o = LT.solve(p, F, L, X, U, r, Xf, rf, x0)
    loss = (o["S"] * cpu(wS)).sum() + (o["v"] * cpu(wv)).sum() + (o["zeta"] * cpu(wz)).sum() + \
        (o["x"] * cpu(wx)).sum() + wc * o["cost"]
    loss.backward()
    g = {"F": F.grad, "L": L.grad, "X": X.grad, "U": U.grad, "r": r.grad, "Xf": Xf.grad, "x0": x0.grad}
    if rf is not None:
        g["rf"] = rf.grad
    return {k: v.numpy() for k, v in g.items()}


def gpu_grads(p, wS, wv, wz, wx, wc):
    import paper_2212_11744_gb300 as lqt
    dp = lqt.DeviceProblem(p)
    fwd = lqt.lqt_solve(dp)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g = lqt.lqt_backward(dp, fwd, gS=dev(wS), gv=dev(wv), gzeta=dev(wz), gx=dev(wx), g_cost=wc)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    return {k: v.cpu().numpy() for k, v in g.items() if v is not None}


def weights(p, seed):
    rng = np.random.default_rng(seed)
    T1, n = p.T + 1, p.n
    return (rng.standard_normal((T1, n, n)), rng.standard_normal((T1, n)), rng.standard_normal(T1),
            rng.standard_normal((T1, n)), 1.3)


def drop_c_h(p):
    p.c = None
    p.H = None
    p.Hf = None
    return p


CASES = [
    ("differentiable_n8_T256", lambda: W.differentiable_n8(T=256)),
    ("general_n4_modes_T61", lambda: drop_c_h(W.general_time_varying(
        4, 2, 4, T=61, K=3, seed=71, tf=1.2,
        modes={"F": W.PER_INTERVAL, "L": W.CONST, "X": W.PER_INTERVAL, "U": W.PER_INTERVAL, "r": W.PER_STAGE}))),
    ("general_n3_const_T40", lambda: drop_c_h(W.general_time_varying(
        3, 1, 3, T=40, K=2, seed=72, tf=1.0,
        modes={"F": W.CONST, "L": W.CONST, "X": W.CONST, "U": W.CONST, "r": W.PER_INTERVAL}))),
    ("scalar_n1_T33", lambda: drop_c_h(W.general_time_varying(
        1, 1, 1, T=33, K=4, seed=73, tf=1.0,
        modes={"F": W.CONST, "L": W.PER_INTERVAL, "X": W.CONST, "U": W.CONST, "r": W.PER_STAGE}))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_backward_matches_oracle_reverse_mode(name, make):
    p = make()
    w = weights(p, 5)
    ref = oracle_grads(p, *w)
    got = gpu_grads(p, *w)
    for k, v in ref.items():
        e = rel(got[k], v)
        assert e <= TOL, (name, k, e)


def test_autograd_function_cost_and_terminal_state():
    """The differentiable workload's loss through LQTSolve.apply: total optimal cost plus
    |x(t_f) - x_target|^2, gradients against the oracle's reverse mode."""
    from paper_2212_11744_gb300.autograd import LQTSolve
    p = W.differentiable_n8(T=128)
    xt = p.extra["x_target"]
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda").requires_grad_()
    args = [dev(p.F.values), dev(p.L.values), dev(p.X.values), dev(p.U.values), dev(p.r.values), dev(p.Xf), None,
            dev(p.x0)]
    S, v, z, x, cost = LQTSolve.apply(p, *args)
    loss = cost + ((x[-1] - torch.tensor(xt, device="cuda")) ** 2).sum()
    loss.backward()
    wx = np.zeros((p.T + 1, p.n))
    o_fwd = oracle.solve(p)
    wx[-1] = 2.0 * (o_fwd["x"][-1] - xt)
    ref = oracle_grads(p, np.zeros((p.T + 1, p.n, p.n)), np.zeros((p.T + 1, p.n)), np.zeros(p.T + 1), wx, 1.0)
    names = ["F", "L", "X", "U", "r", "Xf", None, "x0"]
    for a, k in zip(args, names):
        if k is None:
            continue
        assert rel(a.grad.cpu().numpy(), ref[k]) <= TOL, k


@pytest.mark.slow
def test_differentiable_n8_full_size_gradients_fd_and_reverse_mode():
    """n = 8, T = 2^14: loss = cost + |x_T - x_target|^2 with Xf tied to X,
    parameters diag(X), diag(U), r (T x 8) and F.  The GPU gradient's
    directional derivatives along 32 seeded random directions against central
    finite differences of the C oracle (h = 1e-6, rel 1e-5), and the full
    gradient against the oracle's reverse mode (rel 1e-9)."""
    import paper_2212_11744_gb300 as lqt
    p = W.differentiable_n8(T=1 << 14)
    xt = p.extra["x_target"]
    n, m, T = p.n, p.m, p.T
    qd, rd = np.diag(p.X.values[0]).copy(), np.diag(p.U.values[0]).copy()
    F0, r0 = p.F.values[0].copy(), p.r.values.copy()

    def with_params(q, rho, r, F):
        pp = W.differentiable_n8(T=T)
        pp.X.values[0] = np.diag(q)
        pp.Xf = np.diag(q)
        pp.U.values[0] = np.diag(rho)
        pp.r.values[:] = r
        pp.F.values[0] = F
        return pp

    def loss_oracle(q, rho, r, F):
        o = oracle.solve(with_params(q, rho, r, F))
        return o["cost"] + float(((o["x"][-1] - xt) ** 2).sum())

    # GPU gradient
    dp = lqt.DeviceProblem(p)
    fwd = lqt.lqt_solve(dp)
    gx = torch.zeros(T + 1, n, dtype=torch.float64, device="cuda")
    gx[-1] = 2.0 * (fwd["x"][-1] - torch.tensor(xt, device="cuda"))
    g = lqt.lqt_backward(dp, fwd, gx=gx, g_cost=1.0)
    torch.cuda.synchronize()
    gq = np.diag(g["X"][0].cpu().numpy()) + np.diag(g["Xf"].cpu().numpy())
    grho = np.diag(g["U"][0].cpu().numpy())
    gr = g["r"].cpu().numpy()
    gF = g["F"][0].cpu().numpy()
    # reverse mode of the oracle (same loss, Xf tied)
    q_t = cpu(qd).requires_grad_()
    rho_t = cpu(rd).requires_grad_()
    r_t = cpu(r0).requires_grad_()
    F_t = cpu(F0).requires_grad_()
    o = LT.solve(p, F_t[None], cpu(p.L.values), torch.diag(q_t)[None], torch.diag(rho_t)[None], r_t,
                 torch.diag(q_t), None, cpu(p.x0))
    lo = o["cost"] + ((o["x"][-1] - cpu(xt)) ** 2).sum()
    lo.backward()
    assert rel(gq, q_t.grad.numpy()) <= TOL
    assert rel(grho, rho_t.grad.numpy()) <= TOL
    assert rel(gr, r_t.grad.numpy()) <= TOL
    assert rel(gF, F_t.grad.numpy()) <= TOL
    # finite differences along random directions.  Each direction is a seeded
    # Gaussian in (diag X, diag U, F) plus a Gaussian on 64 random reference
    # samples, normalised to unit length: the directional derivative is then of
    # order one, so that the h = 1e-6 central difference is not swamped by the
    # ~1e-14 relative rounding of the loss (a dense unit direction over all
    # 131072 reference entries gives derivatives ~1e-2, where central
    # differences at h = 1e-6 carry ~1e-5 relative rounding error).
    rng = np.random.default_rng(4242)
    h = 1e-6
    # the rounding of a central difference: the loss carries a relative
    # rounding of its own (measured here as the gap between two independent
    # evaluations of it, the C oracle and the torch restatement, floored at
    # 4 ulp), and the difference of two such values divided by 2h carries
    # twice that over 2h
    L0 = loss_oracle(qd, rd, r0, F0)
    noise = max(abs(L0 - float(lo.detach())), 4 * np.finfo(float).eps * abs(L0))
    fd_round = 2 * noise / (2 * h)
    worst = 0.0
    for _ in range(32):
        dq, drho, dF = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal((n, n))
        dr = np.zeros_like(r0)
        rows = rng.choice(T, 64, replace=False)
        dr[rows] = rng.standard_normal((64, n))
        nrm = np.sqrt((dq ** 2).sum() + (drho ** 2).sum() + (dr ** 2).sum() + (dF ** 2).sum())
        dq, drho, dr, dF = dq / nrm, drho / nrm, dr / nrm, dF / nrm
        fd = (loss_oracle(qd + h * dq, rd + h * drho, r0 + h * dr, F0 + h * dF) -
              loss_oracle(qd - h * dq, rd - h * drho, r0 - h * dr, F0 - h * dF)) / (2 * h)
        an = (gq * dq).sum() + (grho * drho).sum() + (gr * dr).sum() + (gF * dF).sum()
        # rel. 1e-5 of the derivative, plus the difference's own rounding
        worst = max(worst, abs(an - fd) / (1e-5 * abs(fd) + fd_round))
    assert worst <= 1.0, (worst, fd_round)


def test_backward_full_size_against_gpu_central_differences():
    """n = 8, T = 2^14 (the adjoint workload): the gradient's directional
    derivative along 4 seeded directions in (diag X, F, r) against central
    differences of the GPU's own forward solve (h = 1e-6, rel 1e-5 plus the
    difference's rounding, from the loss's measured rounding as in the oracle
    finite-difference test)."""
    import paper_2212_11744_gb300 as lqt
    p = W.differentiable_n8(T=1 << 14)
    xt = torch.tensor(p.extra["x_target"], device="cuda")
    dp = lqt.DeviceProblem(p)
    fwd = lqt.lqt_solve(dp)
    gx = torch.zeros(p.T + 1, p.n, dtype=torch.float64, device="cuda")
    gx[-1] = 2.0 * (fwd["x"][-1] - xt)
    g = lqt.lqt_backward(dp, fwd, gx=gx, g_cost=1.0)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    for k, v in g.items():
        assert bool(torch.isfinite(v).all()), k

    def loss(dq, dF, dr, h):
        q = p.X.values[0].copy(); q[np.diag_indices(p.n)] += h * dq
        pp = W.differentiable_n8(T=p.T)
        pp.X.values[0] = q
        pp.F.values[0] = p.F.values[0] + h * dF
        pp.r.values[:] = p.r.values + h * dr
        o = lqt.lqt_solve(lqt.DeviceProblem(pp))
        return float(o["cost"][0]) + float(((o["x"][-1] - xt) ** 2).sum())

    # the loss's rounding: its GPU value against the oracle's (floored at 4
    # ulp); a central difference carries twice that over 2h
    L0 = loss(np.zeros(p.n), np.zeros((p.n, p.n)), np.zeros_like(p.r.values), 0.0)
    o = oracle.solve(p)
    noise = max(abs(L0 - (o["cost"] + float(((o["x"][-1] - p.extra["x_target"]) ** 2).sum()))),
                4 * np.finfo(float).eps * abs(L0))
    fd_round = 2 * noise / 2e-6
    rng = np.random.default_rng(77)
    worst = 0.0
    for _ in range(4):
        dq, dF = rng.standard_normal(p.n), rng.standard_normal((p.n, p.n))
        dr = np.zeros_like(p.r.values)
        rows = rng.choice(p.T, 64, replace=False)
        dr[rows] = rng.standard_normal((64, p.n))
        nrm = np.sqrt((dq ** 2).sum() + (dF ** 2).sum() + (dr ** 2).sum())
        dq, dF, dr = dq / nrm, dF / nrm, dr / nrm
        fd = (loss(dq, dF, dr, 1e-6) - loss(dq, dF, dr, -1e-6)) / 2e-6
        an = float((np.diag(g["X"][0].cpu().numpy()) * dq).sum() + (g["F"][0].cpu().numpy() * dF).sum() +
                   (g["r"].cpu().numpy() * dr).sum())
        worst = max(worst, abs(an - fd) / (1e-5 * abs(fd) + fd_round))
    assert worst <= 1.0, (worst, fd_round)
