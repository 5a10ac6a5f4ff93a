"""GB300-native temporally parallel continuous-time LQT solver.

Python binding of the C ABI in include/lqt.h, with the same entry-point names.
Every step of the solve runs in the CUDA library (csrc/); this module only
moves arrays to the device (PyTorch is used for device memory and streams) and
fills the C structs.

    import paper_2212_11744_gb300 as lqt
    dp = lqt.DeviceProblem(problem)        # problem: n, m, nr, T, K, t, F, L, ...
    out = lqt.lqt_solve(dp)                # dict of device tensors S, v, zeta, x, u, cost
"""
from __future__ import annotations

import ctypes as ct
from typing import Optional

import numpy as np
import torch

from . import _abi
from ._abi import (LQT_CONST, LQT_PER_INTERVAL, LQT_PER_STAGE, LQT_WS_BACKWARD, LQT_WS_BUILD, LQT_WS_DENSIFY,
                   LQT_WS_INVARIANT, LQT_WS_METHOD2, LQT_WS_SEQUENTIAL, LQT_WS_SOLVE, LQT_WS_SOLVE_INVARIANT,
                   LQT_WS_SOLVE_METHOD2, LQT_WS_TRAJ,
                   LQT_WS_VALUE, LQTError, lqt_coef, lqt_elements, lqt_grid_problem, lqt_problem)

__all__ = [
    "DeviceProblem", "HostProblem", "lqt_workspace_size", "lqt_build_elements", "lqt_scan_value",
    "lqt_scan_trajectory", "lqt_scan_value_noalloc", "lqt_densify", "lqt_solve", "lqt_solve_mixed",
    "lqt_solve_sequential", "lqt_solve_host", "lqt_host_staging_size", "lqt_build_elements_forward",
    "lqt_trajectory_method2", "lqt_solve_method2", "lqt_build_elements_invariant", "lqt_solve_invariant",
    "lqt_get_status", "lqt_strerror", "lqt_last_launch_count", "LQTError", "library_path", "lqt_backward",
    "grid_struct", "lqt_grid_workspace_size", "lqt_grid_block", "lqt_grid_combine", "lqt_grid_values",
    "lqt_probe_fma_rate",
]

_COEFS = ("F", "L", "c", "H", "X", "U", "r")


def library_path() -> str:
    return _abi.LIB_PATH


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


class _Marshal:
    """Copies a problem's arrays into tensors (device or pinned host) and fills lqt_problem."""

    def __init__(self, p, device, pinned: bool):
        self.keep = []
        self.n, self.m, self.nr, self.T, self.K = int(p.n), int(p.m), int(p.nr), int(p.T), int(p.K)

        def put(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            t = torch.from_numpy(a)
            if device is not None:
                t = t.to(device)
            elif pinned:
                t = t.pin_memory()
            self.keep.append(t)
            return t

        s = lqt_problem()
        s.n, s.m, s.nr, s.T, s.K = self.n, self.m, self.nr, self.T, self.K
        s.t = _ptr(put(p.t))
        for name in _COEFS:
            co = getattr(p, name)
            if co is None:
                setattr(s, name, lqt_coef(None, 0))
            else:
                setattr(s, name, lqt_coef(_ptr(put(co.values)), int(co.mode)))
        s.Hf = _ptr(put(p.Hf))
        s.Xf = _ptr(put(p.Xf))
        s.rf = _ptr(put(p.rf))
        self.x0 = put(p.x0) if getattr(p, "x0", None) is not None else None
        self.struct = s

    def ref(self):
        return ct.byref(self.struct)


class DeviceProblem(_Marshal):
    """A problem with every array resident on the GPU."""

    def __init__(self, problem, device: str = "cuda"):
        super().__init__(problem, torch.device(device), False)
        self.device = torch.device(device)


class HostProblem(_Marshal):
    """A problem whose arrays stay in (pinned) host memory, for lqt_solve_host."""

    def __init__(self, problem, pinned: bool = True):
        super().__init__(problem, None, pinned)


def lqt_strerror(code: int) -> str:
    return _abi.strerror(code)


def lqt_last_launch_count() -> int:
    return int(_abi.lib().lqt_last_launch_count())


def lqt_workspace_size(dp: _Marshal, which: int) -> int:
    return int(_abi.lib().lqt_workspace_size(dp.ref(), which))


def _workspace(dp: DeviceProblem, which: int, ws: Optional[torch.Tensor]):
    need = lqt_workspace_size(dp, which)
    if need == 0:
        raise LQTError(_abi.LQT_EINVAL, "lqt_workspace_size")
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=dp.device)
    return ws


def _empty(dp, *shape):
    return torch.empty(*shape, dtype=torch.float64, device=dp.device)


def _elements_struct(el: dict) -> lqt_elements:
    return lqt_elements(_ptr(el["A"]), _ptr(el["b"]), _ptr(el["C"]), _ptr(el["eta"]), _ptr(el["J"]),
                        _ptr(el.get("zeta")))


def new_elements(dp: DeviceProblem) -> dict:
    n, T1 = dp.n, dp.T + 1
    return {"A": _empty(dp, T1, n, n), "b": _empty(dp, T1, n), "C": _empty(dp, T1, n, n), "eta": _empty(dp, T1, n),
            "J": _empty(dp, T1, n, n), "zeta": _empty(dp, T1)}


def lqt_build_elements(dp: DeviceProblem, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    out = new_elements(dp) if out is None else out
    ws = _workspace(dp, LQT_WS_BUILD, ws)
    es = _elements_struct(out)
    _abi.check(_abi.lib().lqt_build_elements(dp.ref(), ct.byref(es), ws.data_ptr(), ws.numel(),
                                             _stream_handle(stream)), "lqt_build_elements")
    return out


def lqt_build_elements_forward(dp: DeviceProblem, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    """The T forward-ODE elements (Sec. IV-C), arrays of T entries."""
    n, T = dp.n, dp.T
    out = out or {"A": _empty(dp, T, n, n), "b": _empty(dp, T, n), "C": _empty(dp, T, n, n),
                  "eta": _empty(dp, T, n), "J": _empty(dp, T, n, n), "zeta": _empty(dp, T)}
    ws = _workspace(dp, LQT_WS_BUILD, ws)
    es = _elements_struct(out)
    _abi.check(_abi.lib().lqt_build_elements_forward(dp.ref(), ct.byref(es), ws.data_ptr(), ws.numel(),
                                                     _stream_handle(stream)), "lqt_build_elements_forward")
    return out


def lqt_build_elements_invariant(dp: DeviceProblem, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    """The T+1 elements by the time-invariant build (constant F, L, U, X, H;
    uniform grid)."""
    out = new_elements(dp) if out is None else out
    ws = _workspace(dp, LQT_WS_INVARIANT, ws)
    es = _elements_struct(out)
    _abi.check(_abi.lib().lqt_build_elements_invariant(dp.ref(), ct.byref(es), ws.data_ptr(), ws.numel(),
                                                       _stream_handle(stream)), "lqt_build_elements_invariant")
    return out


def lqt_solve_invariant(dp: DeviceProblem, x0=None, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    """lqt_solve with the time-invariant element build."""
    x0 = dp.x0 if x0 is None else x0
    out = new_solution(dp) if out is None else out
    ws = _workspace(dp, LQT_WS_SOLVE_INVARIANT, ws)
    _abi.check(_abi.lib().lqt_solve_invariant(dp.ref(), _ptr(x0), _ptr(out["S"]), _ptr(out["v"]),
                                              _ptr(out.get("zeta")), _ptr(out["x"]), _ptr(out.get("u")),
                                              _ptr(out.get("cost")), ws.data_ptr(), ws.numel(),
                                              _stream_handle(stream)), "lqt_solve_invariant")
    return out


def lqt_trajectory_method2(dp: DeviceProblem, fwd: dict, sol: dict, x0=None, out: Optional[dict] = None, ws=None,
                           stream=None) -> dict:
    """States and controls by Method 2 from forward-ODE elements `fwd` and the
    values sol["S"], sol["v"]."""
    x0 = dp.x0 if x0 is None else x0
    n, m, T1 = dp.n, dp.m, dp.T + 1
    out = out or {"x": _empty(dp, T1, n), "u": _empty(dp, T1, m)}
    ws = _workspace(dp, LQT_WS_METHOD2, ws)
    es = _elements_struct(fwd)
    _abi.check(_abi.lib().lqt_trajectory_method2(dp.ref(), ct.byref(es), _ptr(sol["S"]), _ptr(sol["v"]), _ptr(x0),
                                                 _ptr(out["x"]), _ptr(out.get("u")), ws.data_ptr(), ws.numel(),
                                                 _stream_handle(stream)), "lqt_trajectory_method2")
    return out


def lqt_solve_method2(dp: DeviceProblem, x0=None, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    """lqt_solve with the states by Method 2 (forward-ODE elements, prefix scan)."""
    x0 = dp.x0 if x0 is None else x0
    out = new_solution(dp) if out is None else out
    ws = _workspace(dp, LQT_WS_SOLVE_METHOD2, ws)
    _abi.check(_abi.lib().lqt_solve_method2(dp.ref(), _ptr(x0), _ptr(out["S"]), _ptr(out["v"]), _ptr(out.get("zeta")),
                                            _ptr(out["x"]), _ptr(out.get("u")), _ptr(out.get("cost")), ws.data_ptr(),
                                            ws.numel(), _stream_handle(stream)), "lqt_solve_method2")
    return out


def lqt_scan_value(dp: DeviceProblem, elements: dict, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    n, T1 = dp.n, dp.T + 1
    out = out or {"S": _empty(dp, T1, n, n), "v": _empty(dp, T1, n), "zeta": _empty(dp, T1)}
    ws = _workspace(dp, LQT_WS_VALUE, ws)
    es = _elements_struct(elements)
    _abi.check(_abi.lib().lqt_scan_value(dp.ref(), ct.byref(es), _ptr(out["S"]), _ptr(out["v"]),
                                         _ptr(out.get("zeta")), ws.data_ptr(), ws.numel(), _stream_handle(stream)),
               "lqt_scan_value")
    return out


def lqt_scan_value_noalloc(dp: DeviceProblem, elements: dict, out: Optional[dict] = None, stream=None) -> dict:
    """lqt_scan_value without a workspace: the scratch is a fixed array inside
    the library (see include/lqt.h for its size limit and its sharing rules)."""
    n, T1 = dp.n, dp.T + 1
    out = out or {"S": _empty(dp, T1, n, n), "v": _empty(dp, T1, n), "zeta": _empty(dp, T1)}
    es = _elements_struct(elements)
    _abi.check(_abi.lib().lqt_scan_value_noalloc(dp.ref(), ct.byref(es), _ptr(out["S"]), _ptr(out["v"]),
                                                 _ptr(out.get("zeta")), _stream_handle(stream)),
               "lqt_scan_value_noalloc")
    return out


def lqt_scan_trajectory(dp: DeviceProblem, elements: dict, S, v, x0=None, out: Optional[dict] = None, ws=None,
                        stream=None) -> dict:
    n, m, T1 = dp.n, dp.m, dp.T + 1
    x0 = dp.x0 if x0 is None else x0
    out = out or {"x": _empty(dp, T1, n), "u": _empty(dp, T1, m)}
    ws = _workspace(dp, LQT_WS_TRAJ, ws)
    es = _elements_struct(elements)
    _abi.check(_abi.lib().lqt_scan_trajectory(dp.ref(), ct.byref(es), _ptr(S), _ptr(v), _ptr(x0), _ptr(out["x"]),
                                              _ptr(out.get("u")), ws.data_ptr(), ws.numel(), _stream_handle(stream)),
               "lqt_scan_trajectory")
    return out


def new_solution(dp: DeviceProblem) -> dict:
    n, m, T1 = dp.n, dp.m, dp.T + 1
    return {"S": _empty(dp, T1, n, n), "v": _empty(dp, T1, n), "zeta": _empty(dp, T1), "x": _empty(dp, T1, n),
            "u": _empty(dp, T1, m), "cost": _empty(dp, 1)}


def lqt_solve(dp: DeviceProblem, x0=None, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    x0 = dp.x0 if x0 is None else x0
    out = new_solution(dp) if out is None else out
    ws = _workspace(dp, LQT_WS_SOLVE, ws)
    _abi.check(_abi.lib().lqt_solve(dp.ref(), _ptr(x0), _ptr(out["S"]), _ptr(out["v"]), _ptr(out.get("zeta")),
                                    _ptr(out["x"]), _ptr(out.get("u")), _ptr(out.get("cost")), ws.data_ptr(),
                                    ws.numel(), _stream_handle(stream)), "lqt_solve")
    return out


def lqt_solve_mixed(dp: DeviceProblem, x0=None, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    """lqt_solve with the combination products in FP32 (LU solves and the
    element build in FP64)."""
    x0 = dp.x0 if x0 is None else x0
    out = new_solution(dp) if out is None else out
    ws = _workspace(dp, LQT_WS_SOLVE, ws)
    _abi.check(_abi.lib().lqt_solve_mixed(dp.ref(), _ptr(x0), _ptr(out["S"]), _ptr(out["v"]), _ptr(out.get("zeta")),
                                          _ptr(out["x"]), _ptr(out.get("u")), _ptr(out.get("cost")), ws.data_ptr(),
                                          ws.numel(), _stream_handle(stream)), "lqt_solve_mixed")
    return out


def lqt_solve_sequential(dp: DeviceProblem, x0=None, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    x0 = dp.x0 if x0 is None else x0
    out = new_solution(dp) if out is None else out
    ws = _workspace(dp, LQT_WS_SEQUENTIAL, ws)
    _abi.check(_abi.lib().lqt_solve_sequential(dp.ref(), _ptr(x0), _ptr(out["S"]), _ptr(out["v"]),
                                               _ptr(out.get("zeta")), _ptr(out["x"]), _ptr(out.get("u")),
                                               _ptr(out.get("cost")), ws.data_ptr(), ws.numel(),
                                               _stream_handle(stream)), "lqt_solve_sequential")
    return out


def new_dense(dp: DeviceProblem) -> dict:
    n, m, G = dp.n, dp.m, dp.T * dp.K + 1
    return {"S": _empty(dp, G, n, n), "v": _empty(dp, G, n), "zeta": _empty(dp, G), "x": _empty(dp, G, n),
            "u": _empty(dp, G, m)}


def lqt_densify(dp: DeviceProblem, sol: dict, out: Optional[dict] = None, ws=None, stream=None) -> dict:
    """Solution at every RK4 sub-step from the boundary solution `sol` (the
    S, v, zeta, x of lqt_solve): arrays of T K + 1 points."""
    out = new_dense(dp) if out is None else out
    ws = _workspace(dp, LQT_WS_DENSIFY, ws)
    _abi.check(_abi.lib().lqt_densify(dp.ref(), _ptr(sol["S"]), _ptr(sol["v"]), _ptr(sol["zeta"]), _ptr(sol["x"]),
                                      _ptr(out["S"]), _ptr(out["v"]), _ptr(out["zeta"]), _ptr(out["x"]),
                                      _ptr(out.get("u")), ws.data_ptr(), ws.numel(), _stream_handle(stream)),
               "lqt_densify")
    return out


def lqt_backward(dp: DeviceProblem, fwd: dict, gS=None, gv=None, gzeta=None, gx=None, g_cost: float = 0.0,
                 x0=None, ws=None, stream=None) -> dict:
    """Gradients of a scalar loss with respect to F, L, X, U, r (in their sample
    layouts), Xf, rf and x0, given lqt_solve's outputs `fwd` and the loss's
    gradients with respect to them (see lqt_backward in include/lqt.h)."""
    x0 = dp.x0 if x0 is None else x0
    s = dp.struct
    n, m = dp.n, dp.m

    def samples(c, per):
        if c.ptr is None:
            return None
        cnt = {LQT_CONST: 1, LQT_PER_INTERVAL: dp.T, LQT_PER_STAGE: 2 * dp.K * dp.T + 1}[c.mode]
        return _empty(dp, cnt, *per)

    out = {"F": samples(s.F, (n, n)), "L": samples(s.L, (n, m)), "X": samples(s.X, (dp.nr, dp.nr)),
           "U": samples(s.U, (m, m)), "r": samples(s.r, (dp.nr,)), "Xf": _empty(dp, dp.nr, dp.nr),
           "rf": _empty(dp, dp.nr), "x0": _empty(dp, n)}
    ws = _workspace(dp, LQT_WS_BACKWARD, ws)
    _abi.check(_abi.lib().lqt_backward(
        dp.ref(), _ptr(x0), _ptr(fwd["S"]), _ptr(fwd["v"]), _ptr(fwd["x"]), _ptr(gS), _ptr(gv), _ptr(gzeta), _ptr(gx),
        None, float(g_cost), _ptr(out["F"]), _ptr(out["L"]), _ptr(out["X"]), _ptr(out["U"]), _ptr(out["r"]),
        _ptr(out["Xf"]), _ptr(out["rf"]), _ptr(out["x0"]), ws.data_ptr(), ws.numel(), _stream_handle(stream)),
        "lqt_backward")
    return out


def grid_struct(g) -> lqt_grid_problem:
    """lqt_grid_problem from any object with the fields G, x_min, dx, d0, d1,
    d2, q, rho, qf, tau, substeps, T, interp."""
    return lqt_grid_problem(int(g.G), float(g.x_min), float(g.dx), float(g.d0), float(g.d1), float(g.d2),
                            float(g.q), float(g.rho), float(g.qf), float(g.tau), int(g.substeps), int(g.T),
                            int(bool(g.interp)))


def lqt_grid_workspace_size(g, which: int) -> int:
    return int(_abi.lib().lqt_grid_workspace_size(ct.byref(grid_struct(g)), which))


def _grid_workspace(g, which: int, ws, device):
    need = lqt_grid_workspace_size(g, which)
    if need == 0:
        raise LQTError(_abi.LQT_EINVAL, "lqt_grid_workspace_size")
    return torch.empty(need, dtype=torch.uint8, device=device) if ws is None else ws


def lqt_grid_block(g, out: Optional[torch.Tensor] = None, ws=None, device="cuda", stream=None) -> torch.Tensor:
    """The block's conditional value function on the grid (G x G)."""
    out = torch.empty(g.G, g.G, dtype=torch.float64, device=device) if out is None else out
    ws = _grid_workspace(g, 0, ws, out.device)
    _abi.check(_abi.lib().lqt_grid_block(ct.byref(grid_struct(g)), out.data_ptr(), ws.data_ptr(), ws.numel(),
                                         _stream_handle(stream)), "lqt_grid_block")
    return out


def lqt_grid_combine(g, A: torch.Tensor, B: torch.Tensor, out: Optional[torch.Tensor] = None,
                     stream=None) -> torch.Tensor:
    """A (x) B: min over the grid of the intermediate state (App. E refinement
    when g.interp)."""
    out = torch.empty_like(A) if out is None else out
    _abi.check(_abi.lib().lqt_grid_combine(ct.byref(grid_struct(g)), A.data_ptr(), B.data_ptr(), out.data_ptr(),
                                           _stream_handle(stream)), "lqt_grid_combine")
    return out


def lqt_grid_values(g, Vblock: torch.Tensor, out: Optional[torch.Tensor] = None, ws=None,
                    stream=None) -> torch.Tensor:
    """V(., t_k) for k = 0..T, shape (T+1, G)."""
    out = torch.empty(g.T + 1, g.G, dtype=torch.float64, device=Vblock.device) if out is None else out
    ws = _grid_workspace(g, 1, ws, Vblock.device)
    _abi.check(_abi.lib().lqt_grid_values(ct.byref(grid_struct(g)), Vblock.data_ptr(), out.data_ptr(),
                                          ws.data_ptr(), ws.numel(), _stream_handle(stream)), "lqt_grid_values")
    return out


def lqt_probe_fma_rate(precision: int, blocks: int, threads: int, iters: int, active_lanes: int = 32,
                       out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Launches the FMA-pipe probe (timing is the caller's); returns its scratch."""
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda") if out is None else out
    _abi.check(_abi.lib().lqt_probe_fma_rate(precision, blocks, threads, iters, active_lanes, out.data_ptr(),
                                             _stream_handle(stream)), "lqt_probe_fma_rate")
    return out


def lqt_host_staging_size(hp: HostProblem) -> int:
    return int(_abi.lib().lqt_host_staging_size(hp.ref()))


def host_solution(hp: HostProblem, pinned: bool = True) -> dict:
    n, m, T1 = hp.n, hp.m, hp.T + 1

    def e(*shape):
        t = torch.empty(*shape, dtype=torch.float64)
        return t.pin_memory() if pinned else t

    return {"S": e(T1, n, n), "v": e(T1, n), "zeta": e(T1), "x": e(T1, n), "u": e(T1, m), "cost": e(1)}


def lqt_solve_host(hp: HostProblem, ws: torch.Tensor, out: Optional[dict] = None, x0=None, stream=None) -> dict:
    """Host buffers in and out; `ws` is a device uint8 tensor of at least
    lqt_workspace_size(hp, LQT_WS_SOLVE) + lqt_host_staging_size(hp) bytes."""
    x0 = hp.x0 if x0 is None else x0
    out = host_solution(hp) if out is None else out
    _abi.check(_abi.lib().lqt_solve_host(hp.ref(), _ptr(x0), _ptr(out["S"]), _ptr(out["v"]), _ptr(out.get("zeta")),
                                         _ptr(out["x"]), _ptr(out.get("u")), _ptr(out.get("cost")), ws.data_ptr(),
                                         ws.numel(), _stream_handle(stream)), "lqt_solve_host")
    return out


def lqt_get_status(stream=None, timeout_ms: int = 10000) -> int:
    return int(_abi.lib().lqt_get_status(_stream_handle(stream), timeout_ms))
