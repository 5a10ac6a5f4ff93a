"""Pins of the reverse-mode oracle (oracle/lqt_torch.py), on the CPU.

The GPU adjoint is checked against torch.autograd through lqt_torch, so
lqt_torch itself is pinned here against two things other than itself:
  * its forward values equal those of the C oracle (a separate implementation
    in another language, pinned in test_oracle_pins.py) to rounding;
  * its gradients equal central finite differences of the C oracle along
    seeded directions over every differentiable input (F, L, X, U, r, Xf, rf,
    x0) to the finite-difference error.
"""
import copy

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import lqt_torch as LT


def t64(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))


CASES = {
    "double_integrator_T32": lambda: W.truncate(W.double_integrator(), 32),
    "point_mass_T16": lambda: W.truncate(W.point_mass_2d(T=1 << 10), 16),
    "differentiable_n8_T12": lambda: W.differentiable_n8(T=12),
    "batched_n4_T20": lambda: W.batched_member(7, T=20, n=4),
}


def torch_forward(p, params=None):
    pr = params or {
        "F": t64(p.F.values), "L": t64(p.L.values), "X": t64(p.X.values), "U": t64(p.U.values),
        "r": t64(p.r.values), "Xf": t64(p.Xf), "rf": t64(p.rf) if p.rf is not None else None, "x0": t64(p.x0),
    }
    return LT.solve(p, pr["F"], pr["L"], pr["X"], pr["U"], pr["r"], pr["Xf"], pr["rf"], pr["x0"]), pr


@pytest.mark.parametrize("name", sorted(CASES))
def test_torch_forward_equals_c_oracle(name):
    p = CASES[name]()
    o, _ = torch_forward(p)
    ref = oracle.solve(p)
    for k in ("S", "v", "zeta", "x"):
        assert rel(o[k].detach().numpy(), ref[k]) < 1e-12, k
    assert abs(float(o["cost"]) - ref["cost"]) <= 1e-12 * max(1.0, abs(ref["cost"]))


def _with(p, name, value):
    q = copy.deepcopy(p)
    if name in ("F", "L", "X", "U", "r"):
        getattr(q, name).values = np.ascontiguousarray(value)
    else:
        setattr(q, name, np.ascontiguousarray(value))
    return q


@pytest.mark.parametrize("name", sorted(CASES))
def test_torch_gradients_equal_central_differences_of_c_oracle(name):
    """Loss = cost + <w, x> + <wS, S> + <wv, v> (weights seeded): directional
    derivatives of the autograd gradient along 6 seeded unit directions in the
    joint input space against (L(p + h d) - L(p - h d)) / 2h of the C oracle,
    h = 1e-5 (truncation ~h^2, rounding ~1e-16/h)."""
    p = CASES[name]()
    rng = np.random.default_rng(77)
    T, n = p.T, p.n
    wx = rng.standard_normal((T + 1, n))
    wS = rng.standard_normal((T + 1, n, n)) * 0.1
    wv = rng.standard_normal((T + 1, n)) * 0.1

    def loss_c(q):
        o = oracle.solve(q)
        return o["cost"] + float((o["x"] * wx).sum()) + float((o["S"] * wS).sum()) + float((o["v"] * wv).sum())

    _, pr = torch_forward(p)
    names = [k for k in ("F", "L", "X", "U", "r", "Xf", "rf", "x0") if pr[k] is not None]
    leaves = {k: pr[k].clone().requires_grad_() for k in names}
    full = dict(pr)
    full.update(leaves)
    o, _ = torch_forward(p, full)
    loss = o["cost"] + (o["x"] * t64(wx)).sum() + (o["S"] * t64(wS)).sum() + (o["v"] * t64(wv)).sum()
    loss.backward()
    grads = {k: leaves[k].grad.numpy() for k in names}
    base = {k: pr[k].numpy() for k in names}

    h = 1e-5
    worst = 0.0
    for _ in range(6):
        d = {k: rng.standard_normal(base[k].shape) for k in names}
        # keep X, U, Xf symmetric so that the perturbed problems stay valid
        for k in ("X", "U", "Xf"):
            d[k] = 0.5 * (d[k] + np.swapaxes(d[k], -1, -2))
        nrm = np.sqrt(sum((v ** 2).sum() for v in d.values()))
        d = {k: v / nrm for k, v in d.items()}
        qp, qm = p, p
        for k in names:
            qp = _with(qp, k, base[k] + h * d[k])
            qm = _with(qm, k, base[k] - h * d[k])
        fd = (loss_c(qp) - loss_c(qm)) / (2 * h)
        an = sum(float((grads[k] * d[k]).sum()) for k in names)
        worst = max(worst, abs(an - fd) / max(abs(fd), 1e-3))
    assert worst < 1e-6, worst
