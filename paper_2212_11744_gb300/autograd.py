"""torch.autograd.Function over lqt_solve / lqt_backward.

    S, v, zeta, x, cost = LQTSolve.apply(problem, F, L, X, U, r, Xf, rf, x0)

`problem` supplies the dimensions, time grid and sampling modes; F, L, X, U, r
(sample tensors in those modes), Xf, rf, x0 are device tensors and carry the
gradients.  Forward and backward both run in the CUDA library.
"""
from __future__ import annotations

import torch

from . import DeviceProblem, lqt_backward, lqt_solve


class _View:
    """A problem whose coefficient arrays are the given device tensors."""

    def __init__(self, template, F, L, X, U, r, Xf, rf, x0):
        class C:
            def __init__(self, values, mode):
                self.values, self.mode = values, mode

        self.n, self.m, self.nr, self.T, self.K = template.n, template.m, template.nr, template.T, template.K
        self.t = template.t
        self.F = C(F, template.F.mode)
        self.L = C(L, template.L.mode)
        self.X = C(X, template.X.mode)
        self.U = C(U, template.U.mode)
        self.r = C(r, template.r.mode) if r is not None else None
        self.c = None
        self.H = None
        self.Hf = None
        self.Xf, self.rf, self.x0 = Xf, rf, x0


class _DeviceView(DeviceProblem):
    """DeviceProblem built from tensors already on the device (no copies of
    them; the time grid is copied)."""

    def __init__(self, view, device):
        import ctypes as ct

        from ._abi import lqt_coef, lqt_problem
        self.keep = []
        self.device = torch.device(device)
        self.n, self.m, self.nr, self.T, self.K = view.n, view.m, view.nr, view.T, view.K
        t = torch.as_tensor(view.t, dtype=torch.float64, device=self.device).contiguous()
        self.keep.append(t)
        s = lqt_problem()
        s.n, s.m, s.nr, s.T, s.K = self.n, self.m, self.nr, self.T, self.K
        s.t = t.data_ptr()

        def cz(x):
            if x is None:
                return None
            x = x.detach().contiguous()
            self.keep.append(x)
            return x.data_ptr()

        for name in ("F", "L", "c", "H", "X", "U", "r"):
            co = getattr(view, name)
            setattr(s, name, lqt_coef(None, 0) if co is None else lqt_coef(cz(co.values), int(co.mode)))
        s.Hf = None
        s.Xf = cz(view.Xf)
        s.rf = cz(view.rf)
        self.x0 = view.x0.detach().contiguous()
        self.keep.append(self.x0)
        self.struct = s


class LQTSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, template, F, L, X, U, r, Xf, rf, x0):
        view = _View(template, F, L, X, U, r, Xf, rf, x0)
        dp = _DeviceView(view, F.device)
        out = lqt_solve(dp)
        ctx.dp = dp
        ctx.out = out
        ctx.has = (r is not None, rf is not None)
        return out["S"], out["v"], out["zeta"], out["x"], out["cost"][0]

    @staticmethod
    def backward(ctx, gS, gv, gzeta, gx, gcost):
        dp, out = ctx.dp, ctx.out
        g_cost = float(gcost) if gcost is not None else 0.0
        g = lqt_backward(dp, out, gS=gS.contiguous() if gS is not None else None,
                         gv=gv.contiguous() if gv is not None else None,
                         gzeta=gzeta.contiguous() if gzeta is not None else None,
                         gx=gx.contiguous() if gx is not None else None, g_cost=g_cost)
        return (None, g["F"], g["L"], g["X"], g["U"], g["r"] if ctx.has[0] else None, g["Xf"],
                g["rf"] if ctx.has[1] else None, g["x0"])
