"""Seeded synthetic LQT problems shaped like the paper's tracking workloads.

This module only makes inputs: time grids, coefficient samples and initial
states.  It holds none of the method's arithmetic, so both the oracle tests and
the GPU path can take their inputs from it.

A problem is the continuous-time LQT of Sec. II-B of the paper,
    dx/dt = F x + L u + c,
    l(x,u,t) = 1/2 (r - H x)^T X (r - H x) + 1/2 u^T U u,
    phi(x)   = 1/2 (Hf x - rf)^T Xf (Hf x - rf),
on [t0, tf] split into T sub-intervals with K RK4 steps each.  Each
time-varying coefficient is given in one of three sampling modes:

    CONST         one sample
    PER_INTERVAL  T samples; sample j holds on the whole of sub-interval j
    PER_STAGE     2*K*T+1 samples on the half-step grid t_j + p*h_j/2,
                  p = 0..2K, the ends of neighbouring sub-intervals shared
                  (global index 2*K*j + p)
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

CONST, PER_INTERVAL, PER_STAGE = 0, 1, 2
MODE_NAMES = {CONST: "CONST", PER_INTERVAL: "PER_INTERVAL", PER_STAGE: "PER_STAGE"}


@dataclass
class Coef:
    values: np.ndarray  # [samples, *shape] float64, C-contiguous
    mode: int

    def __post_init__(self):
        self.values = np.ascontiguousarray(self.values, dtype=np.float64)


@dataclass
class Problem:
    name: str
    n: int
    m: int
    nr: int
    T: int
    K: int
    t: np.ndarray  # [T+1] block boundaries
    F: Coef
    L: Coef
    X: Coef
    U: Coef
    c: Optional[Coef] = None  # None: zero
    H: Optional[Coef] = None  # None: identity (nr == n)
    r: Optional[Coef] = None  # None: zero
    Hf: Optional[np.ndarray] = None  # None: identity
    Xf: np.ndarray = None
    rf: Optional[np.ndarray] = None  # None: zero
    x0: np.ndarray = None
    extra: dict = field(default_factory=dict)
    # continuous-time definitions of every coefficient, for checks that need
    # values off the sample grid: name -> callable(times[N]) -> [N, *shape]
    funcs: dict = field(default_factory=dict)

    def coefs(self):
        return {k: getattr(self, k) for k in ("F", "L", "c", "H", "X", "U", "r")}

    def fn(self, name: str) -> Optional[Callable]:
        """Continuous-time definition of a coefficient (None for an absent one):
        CONST ones are constant, PER_INTERVAL ones piecewise constant, PER_STAGE
        ones come from `funcs`."""
        c = getattr(self, name)
        if c is None:
            return None
        if c.mode == CONST:
            v = c.values[0]
            return lambda tt: np.broadcast_to(v, (len(np.atleast_1d(tt)),) + v.shape)
        if c.mode == PER_INTERVAL:
            return piecewise_constant(self.t, c.values)
        return self.funcs[name]

    def nbytes_inputs(self) -> int:
        tot = self.t.nbytes + self.x0.nbytes
        for c in self.coefs().values():
            if c is not None:
                tot += c.values.nbytes
        return tot


def uniform_grid(t0: float, tf: float, T: int) -> np.ndarray:
    return np.linspace(t0, tf, T + 1, dtype=np.float64)


def stage_times(t: np.ndarray, K: int) -> np.ndarray:
    """The 2*K*T+1 half-step times t_j + p*h_j/2 (p = 0..2K-1 per block, then t_T)."""
    T = len(t) - 1
    p = np.arange(2 * K, dtype=np.float64) / (2 * K)
    inner = t[:-1, None] + (t[1:] - t[:-1])[:, None] * p[None, :]
    return np.concatenate([inner.reshape(-1), t[-1:]])


def const(a) -> Coef:
    a = np.asarray(a, dtype=np.float64)
    return Coef(a[None, ...], CONST)


def sample_fn(fn: Callable, t: np.ndarray, K: int, mode: int) -> Coef:
    """Sample a continuous coefficient function on the grid of `mode`."""
    if mode == CONST:
        return Coef(fn(t[:1]), CONST)
    if mode == PER_STAGE:
        return Coef(fn(stage_times(t, K)), PER_STAGE)
    if mode == PER_INTERVAL:
        return Coef(fn(t[:-1]), PER_INTERVAL)
    raise ValueError(mode)


def _sinusoid_sum(rng, count):
    amp = rng.uniform(0.5, 2.0, count)
    freq = rng.uniform(0.1, 1.0, count)
    phase = rng.uniform(0.0, 2 * np.pi, count)

    def f(tt):
        tt = np.asarray(tt, dtype=np.float64)
        return (amp[None, :] * np.sin(2 * np.pi * freq[None, :] * tt[:, None] + phase[None, :])).sum(axis=1)

    return f


def piecewise_constant(t: np.ndarray, values: np.ndarray) -> Callable:
    """Function of time that takes values[j] on [t_j, t_{j+1}) (and values[-1] at t_T)."""

    def f(tt):
        idx = np.clip(np.searchsorted(t, np.asarray(tt), side="right") - 1, 0, len(values) - 1)
        return values[idx]

    return f


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------


def double_integrator(T: int = 1024, K: int = 10, seed: int = 1001) -> Problem:
    """n=2 double integrator, m=1, t in [0,10]; X=diag(1,0.1), U=0.01, Xf=10 I;
    position reference = seeded sum of 3 sinusoids (amplitude U[0.5,2],
    frequency U[0.1,1] Hz, phase U[0,2pi)), zero velocity; x0 ~ N(0, I)."""
    rng = np.random.default_rng(seed)
    pos = _sinusoid_sum(rng, 3)
    x0 = rng.standard_normal(2)

    def rfun(tt):
        tt = np.asarray(tt, dtype=np.float64)
        return np.stack([pos(tt), np.zeros_like(tt)], axis=1)

    t = uniform_grid(0.0, 10.0, T)
    F = np.array([[0.0, 1.0], [0.0, 0.0]])
    L = np.array([[0.0], [1.0]])
    X = np.diag([1.0, 0.1])
    U = np.array([[0.01]])
    return Problem(
        name=f"double_integrator_n2_T{T}_K{K}", n=2, m=1, nr=2, T=T, K=K, t=t,
        F=const(F), L=const(L), X=const(X), U=const(U), r=sample_fn(rfun, t, K, PER_STAGE),
        Xf=10.0 * np.eye(2), rf=rfun(np.array([10.0]))[0], x0=x0,
        funcs={"r": rfun},
    )


def point_mass_2d(T: int = 1 << 20, K: int = 4, seed: int = 1002) -> Problem:
    """n=4 point mass (position, velocity) with the paper's F and L (Sec. VI-A),
    m=2, t in [0,100], U=0.1 I, X(t) = diag(1,1,0.01,0.01)(1+0.5 sin t) on the
    half-step grid, reference = 5 sinusoids per position axis with zero velocity,
    Xf = I, rf = r(100), x0 ~ N(0, I)."""
    rng = np.random.default_rng(seed)
    px = _sinusoid_sum(rng, 5)
    py = _sinusoid_sum(rng, 5)
    x0 = rng.standard_normal(4)
    F = np.zeros((4, 4)); F[0, 2] = 1.0; F[1, 3] = 1.0
    L = np.zeros((4, 2)); L[2, 0] = 1.0; L[3, 1] = 1.0
    U = 0.1 * np.eye(2)
    Xd = np.diag([1.0, 1.0, 0.01, 0.01])

    def rfun(tt):
        tt = np.asarray(tt, dtype=np.float64)
        z = np.zeros_like(tt)
        return np.stack([px(tt), py(tt), z, z], axis=1)

    def Xfun(tt):
        tt = np.asarray(tt, dtype=np.float64)
        return Xd[None, :, :] * (1.0 + 0.5 * np.sin(tt))[:, None, None]

    t = uniform_grid(0.0, 100.0, T)
    return Problem(
        name=f"point_mass_2d_n4_T{T}_K{K}", n=4, m=2, nr=4, T=T, K=K, t=t,
        F=const(F), L=const(L), X=sample_fn(Xfun, t, K, PER_STAGE), U=const(U),
        r=sample_fn(rfun, t, K, PER_STAGE), Xf=np.eye(4), rf=rfun(np.array([100.0]))[0], x0=x0,
        funcs={"X": Xfun, "r": rfun},
    )


def _rotation_dynamics(rng, n, lo, hi):
    P, _ = np.linalg.qr(rng.standard_normal((n, n)))
    D = np.zeros((n, n))
    for i in range(n // 2):
        a = rng.uniform(lo, hi)
        w = rng.uniform(0.0, 1.0)
        D[2 * i:2 * i + 2, 2 * i:2 * i + 2] = [[a, w], [-w, a]]
    if n % 2:
        D[-1, -1] = rng.uniform(lo, hi)
    return P @ D @ P.T


def _box_filtered_reference(rng, T, n, width):
    raw = rng.standard_normal((T + width - 1, n))
    kern = np.ones(width) / width
    return np.stack([np.convolve(raw[:, i], kern, mode="valid") for i in range(n)], axis=1)


def batched_member(b: int, T: Optional[int] = None, n: Optional[int] = None) -> Problem:
    """Member b of the 4096-problem batch: n uniform in {2,4,8,16}, m = n/2,
    T uniform in [256, 8192]; F = P blkdiag([[a,w],[-w,a]]) P^T with a ~ U[-1,0.2],
    w ~ U[0,1]; L ~ N(0,1/n); X = G G^T + 0.1 I, U = H H^T + 0.1 I; reference N(0,1)
    smoothed by a length-32 box filter, one sample per sub-interval; sub-interval
    length 0.05, K = 4, Xf = X, rf = r_{T-1}, x0 ~ N(0,I).  T and n may be
    overridden (for small test cases) without changing the other draws."""
    rng = np.random.default_rng(3000 + b)
    n_draw = int(rng.choice([2, 4, 8, 16]))
    T_draw = int(rng.integers(256, 8193))
    n = n_draw if n is None else n
    T = T_draw if T is None else T
    m = max(1, n // 2)
    F = _rotation_dynamics(rng, n, -1.0, 0.2)
    L = rng.standard_normal((n, m)) / np.sqrt(n)
    G = rng.standard_normal((n, n))
    X = G @ G.T + 0.1 * np.eye(n)
    Hm = rng.standard_normal((m, m))
    U = Hm @ Hm.T + 0.1 * np.eye(m)
    r = _box_filtered_reference(rng, T, n, 32)
    x0 = rng.standard_normal(n)
    t = uniform_grid(0.0, 0.05 * T, T)
    return Problem(
        name=f"batched_member{b}_n{n}_T{T}", n=n, m=m, nr=n, T=T, K=4, t=t,
        F=const(F), L=const(L), X=const(X), U=const(U), r=Coef(r, PER_INTERVAL),
        Xf=X.copy(), rf=r[-1].copy(), x0=x0,
    )


def differentiable_n8(T: int = 1 << 14, seed: int = 4001) -> Problem:
    """n=8, m=4, sub-interval length 0.01, K=4; stable F (a ~ U[-1,-0.1]),
    L ~ N(0,1/n), X = diag(U[0.5,2]), U = diag(U[0.05,0.5]); reference T x 8
    box-32 smoothed, one sample per sub-interval; Xf = X, rf = 0; x_target ~ N(0,I)
    is returned in extra["x_target"]."""
    rng = np.random.default_rng(seed)
    n, m = 8, 4
    F = _rotation_dynamics(rng, n, -1.0, -0.1)
    L = rng.standard_normal((n, m)) / np.sqrt(n)
    X = np.diag(rng.uniform(0.5, 2.0, n))
    U = np.diag(rng.uniform(0.05, 0.5, m))
    r = _box_filtered_reference(rng, T, n, 32)
    x0 = rng.standard_normal(n)
    x_target = rng.standard_normal(n)
    t = uniform_grid(0.0, 0.01 * T, T)
    return Problem(
        name=f"differentiable_n8_T{T}", n=n, m=m, nr=n, T=T, K=4, t=t,
        F=const(F), L=const(L), X=const(X), U=const(U), r=Coef(r, PER_INTERVAL),
        Xf=X.copy(), rf=None, x0=x0, extra={"x_target": x_target},
    )


def large_state_n64(T: int = 1 << 16, seed: int = 5001) -> Problem:
    """n=64, m=16, K=2, sub-interval length 0.02; F = -0.5 I + N(0,1/64),
    L ~ N(0,1/64), X = I, U = 0.1 I; reference box-64 smoothed, one sample per
    sub-interval; Xf = I, rf = r_{T-1}; x0 ~ N(0,I)."""
    rng = np.random.default_rng(seed)
    n, m = 64, 16
    F = -0.5 * np.eye(n) + rng.standard_normal((n, n)) / 8.0
    L = rng.standard_normal((n, m)) / 8.0
    r = _box_filtered_reference(rng, T, n, 64)
    x0 = rng.standard_normal(n)
    t = uniform_grid(0.0, 0.02 * T, T)
    return Problem(
        name=f"large_state_n64_T{T}", n=n, m=m, nr=n, T=T, K=2, t=t,
        F=const(F), L=const(L), X=const(np.eye(n)), U=const(0.1 * np.eye(m)), r=Coef(r, PER_INTERVAL),
        Xf=np.eye(n), rf=r[-1].copy(), x0=x0,
    )


def general_time_varying(n: int, m: int, nr: int, T: int, K: int, seed: int, tf: float = 2.0,
                         modes: Optional[dict] = None, nonuniform: bool = False) -> Problem:
    """A problem where every coefficient is a smooth function of time, with a
    non-symmetric F, an output matrix H (nr x n), a drift c and full X, U, so that
    every term of the method is exercised.  `modes` picks the sampling mode per
    coefficient (default PER_STAGE for all)."""
    rng = np.random.default_rng(seed)
    modes = dict(modes or {})
    F0 = rng.standard_normal((n, n)) * 0.6; F1 = rng.standard_normal((n, n)) * 0.3
    L0 = rng.standard_normal((n, m)); L1 = rng.standard_normal((n, m)) * 0.3
    c0 = rng.standard_normal(n); c1 = rng.standard_normal(n) * 0.5
    H0 = rng.standard_normal((nr, n)); H1 = rng.standard_normal((nr, n)) * 0.2
    GX = rng.standard_normal((nr, nr)); GU = rng.standard_normal((m, m))
    X0 = GX @ GX.T / nr + 0.2 * np.eye(nr)
    U0 = GU @ GU.T / m + 0.3 * np.eye(m)
    ra = rng.standard_normal(nr); rw = rng.uniform(0.5, 3.0, nr); rp = rng.uniform(0, 2 * np.pi, nr)
    w = rng.uniform(0.5, 2.0, 6)

    fns = {
        "F": lambda tt: F0[None] + F1[None] * np.sin(w[0] * np.asarray(tt))[:, None, None],
        "L": lambda tt: L0[None] + L1[None] * np.cos(w[1] * np.asarray(tt))[:, None, None],
        "c": lambda tt: c0[None] * np.cos(w[2] * np.asarray(tt))[:, None] + c1[None],
        "H": lambda tt: H0[None] + H1[None] * np.sin(w[3] * np.asarray(tt))[:, None, None],
        "X": lambda tt: X0[None] * (1.0 + 0.5 * np.sin(w[4] * np.asarray(tt)))[:, None, None],
        "U": lambda tt: U0[None] * (1.0 + 0.3 * np.cos(w[5] * np.asarray(tt)))[:, None, None],
        "r": lambda tt: ra[None] * np.sin(rw[None] * np.asarray(tt)[:, None] + rp[None]),
    }
    if nonuniform:
        d = rng.uniform(0.5, 1.5, T)
        t = np.concatenate([[0.0], np.cumsum(d)]) * (tf / d.sum())
        t[-1] = tf
    else:
        t = uniform_grid(0.0, tf, T)
    co = {}
    for k, fn in fns.items():
        mode = modes.get(k, PER_STAGE)
        co[k] = sample_fn(fn, t, K, mode)
    GF = rng.standard_normal((nr, nr))
    Xf = GF @ GF.T / nr + 0.5 * np.eye(nr)
    Hf = rng.standard_normal((nr, n))
    rf = rng.standard_normal(nr)
    x0 = rng.standard_normal(n)
    return Problem(
        name=f"general_n{n}_m{m}_nr{nr}_T{T}_K{K}", n=n, m=m, nr=nr, T=T, K=K, t=t,
        F=co["F"], L=co["L"], X=co["X"], U=co["U"], c=co["c"], H=co["H"], r=co["r"],
        Hf=Hf, Xf=Xf, rf=rf, x0=x0, funcs=fns,
    )


def resample(p: Problem, K: int) -> Problem:
    """The same continuous problem with K RK4 steps per sub-interval (coefficients
    re-sampled from their continuous definitions)."""
    co = {}
    for k, c in p.coefs().items():
        if c is None:
            co[k] = None
        elif c.mode == PER_STAGE:
            co[k] = Coef(p.funcs[k](stage_times(p.t, K)), PER_STAGE)
        else:
            co[k] = c
    return Problem(name=p.name + f"_K{K}", n=p.n, m=p.m, nr=p.nr, T=p.T, K=K, t=p.t, Hf=p.Hf, Xf=p.Xf, rf=p.rf,
                   x0=p.x0, extra=p.extra, funcs=p.funcs, **co)


def refine(p: Problem, factor: int) -> Problem:
    """The same continuous problem on `factor` times as many sub-intervals (each
    split evenly), with the same K; PER_INTERVAL coefficients are repeated."""
    T = p.T * factor
    t = np.concatenate([np.linspace(p.t[j], p.t[j + 1], factor + 1)[:-1] for j in range(p.T)] + [p.t[-1:]])
    co = {}
    for k, c in p.coefs().items():
        if c is None:
            co[k] = None
        elif c.mode == PER_STAGE:
            co[k] = Coef(p.funcs[k](stage_times(t, p.K)), PER_STAGE)
        elif c.mode == PER_INTERVAL:
            co[k] = Coef(np.repeat(c.values, factor, axis=0), PER_INTERVAL)
        else:
            co[k] = c
    return Problem(name=p.name + f"_x{factor}", n=p.n, m=p.m, nr=p.nr, T=T, K=p.K, t=t, Hf=p.Hf, Xf=p.Xf,
                   rf=p.rf, x0=p.x0, extra=p.extra, funcs=p.funcs, **co)


def truncate(p: Problem, Ts: int) -> Problem:
    """The first Ts sub-intervals of p as a problem of its own (same grid, same
    coefficient samples, same terminal cost placed at t_Ts).  Used to time a
    bounded sample of a workload with the same work per sub-interval."""
    K = p.K
    co = {}
    for k, c in p.coefs().items():
        if c is None:
            co[k] = None
        elif c.mode == PER_STAGE:
            co[k] = Coef(c.values[: 2 * K * Ts + 1], PER_STAGE)
        elif c.mode == PER_INTERVAL:
            co[k] = Coef(c.values[:Ts], PER_INTERVAL)
        else:
            co[k] = c
    return Problem(name=p.name + f"_first{Ts}", n=p.n, m=p.m, nr=p.nr, T=Ts, K=K, t=p.t[: Ts + 1].copy(), Hf=p.Hf,
                   Xf=p.Xf, rf=p.rf, x0=p.x0, extra=p.extra, funcs=p.funcs, **co)


def window(p: Problem, j0: int, count: int) -> Problem:
    """Sub-intervals j0 .. j0+count-1 of p as a problem of its own (same grid
    points and coefficient samples; the terminal cost of p placed at the
    window's end).  Used to check single sub-intervals of a large problem."""
    K = p.K
    co = {}
    for k, c in p.coefs().items():
        if c is None:
            co[k] = None
        elif c.mode == PER_STAGE:
            co[k] = Coef(c.values[2 * K * j0: 2 * K * (j0 + count) + 1], PER_STAGE)
        elif c.mode == PER_INTERVAL:
            co[k] = Coef(c.values[j0:j0 + count], PER_INTERVAL)
        else:
            co[k] = c
    return Problem(name=p.name + f"_w{j0}+{count}", n=p.n, m=p.m, nr=p.nr, T=count, K=K,
                   t=p.t[j0:j0 + count + 1].copy(), Hf=p.Hf, Xf=p.Xf, rf=p.rf, x0=p.x0, extra=p.extra,
                   funcs=p.funcs, **co)



@dataclass
class GridProblem:
    """Scalar control-affine problem dx/dt = d0 + d1 x + d2 x^2 + u with cost
    q x^2/2 + rho u^2/2 and terminal cost qf x^2/2 on a uniform state grid,
    blocks of length tau with `substeps` Euler steps each, T blocks."""
    G: int
    x_min: float
    dx: float
    d0: float
    d1: float
    d2: float
    q: float
    rho: float
    qf: float
    tau: float
    substeps: int
    T: int
    interp: bool = True

    def grid(self) -> np.ndarray:
        return self.x_min + self.dx * np.arange(self.G)


def falling_body(G: int = 201, T: int = 100, x_range: float = 6.0, interp: bool = True) -> GridProblem:
    """The nonlinear example of Sec. VI-B: dx/dt = 1 - x^2/10 + u (velocity of a
    falling body with air resistance, controlled by the force u), running cost
    (x^2 + u^2)/2, terminal cost 2 x^2; blocks of 1/10 time unit with 10 steps
    each; state grid [-x_range, x_range] with G points."""
    dx = 2.0 * x_range / (G - 1)
    return GridProblem(G=G, x_min=-x_range, dx=dx, d0=1.0, d1=0.0, d2=-0.1, q=1.0, rho=1.0, qf=4.0, tau=0.1,
                       substeps=10, T=T, interp=interp)
