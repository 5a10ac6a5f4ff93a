"""Oracle for the temporally parallel continuous-time LQT solver.

TEST INFRASTRUCTURE ONLY: this package is the plain, sequential FP64 CPU
restatement of the method (lqt_oracle.c) that the GPU results are checked
against.  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark import it; the library path never does.  It shares no code with the
CUDA sources.

Python side: ctypes marshalling of a `workloads.Problem` into the C struct, and
unpacking of the packed elements.  Every number is computed in lqt_oracle.c.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lqt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblqt_oracle.so")
_lib = None

_dp = ct.POINTER(ct.c_double)


class _GridProblem(ct.Structure):
    _fields_ = [("G", ct.c_int), ("x_min", ct.c_double), ("dx", ct.c_double), ("d0", ct.c_double),
                ("d1", ct.c_double), ("d2", ct.c_double), ("q", ct.c_double), ("rho", ct.c_double),
                ("qf", ct.c_double), ("tau", ct.c_double), ("substeps", ct.c_int), ("T", ct.c_long),
                ("interp", ct.c_int)]


class _Problem(ct.Structure):
    _fields_ = [
        ("n", ct.c_int), ("m", ct.c_int), ("nr", ct.c_int), ("T", ct.c_long), ("K", ct.c_int),
        ("t", _dp),
        ("F", _dp), ("F_mode", ct.c_int),
        ("L", _dp), ("L_mode", ct.c_int),
        ("c", _dp), ("c_mode", ct.c_int),
        ("H", _dp), ("H_mode", ct.c_int),
        ("X", _dp), ("X_mode", ct.c_int),
        ("U", _dp), ("U_mode", ct.c_int),
        ("r", _dp), ("r_mode", ct.c_int),
        ("Hf", _dp), ("Xf", _dp), ("rf", _dp),
    ]


def build(force: bool = False) -> str:
    """Compile lqt_oracle.c into a shared library next to it (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(L):
    P = ct.POINTER(_Problem)
    L.orc_build_elements.argtypes = [P, ct.c_long, ct.c_long, _dp]
    L.orc_combine.argtypes = [ct.c_int, _dp, _dp, _dp]
    L.orc_suffix_values.argtypes = [ct.c_int, ct.c_long, _dp, _dp, _dp, _dp]
    L.orc_trajectory.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_solve.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_sequential.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_densify.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_build_elements_forward.argtypes = [P, ct.c_long, ct.c_long, _dp]
    L.orc_prefix.argtypes = [ct.c_int, ct.c_long, _dp, _dp]
    L.orc_trajectory_method2.argtypes = [P, _dp, _dp, _dp, _dp, _dp]
    GP = ct.POINTER(_GridProblem)
    L.orc_grid_combine.argtypes = [GP, _dp, _dp, _dp]
    L.orc_grid_apply.argtypes = [GP, _dp, _dp, _dp]
    L.orc_grid_block.argtypes = [GP, _dp]
    L.orc_grid_values_sequential.argtypes = [GP, _dp, _dp]
    L.orc_grid_values.argtypes = [GP, _dp, _dp]
    L.orc_element_size.argtypes = [ct.c_int]
    L.orc_element_size.restype = ct.c_long
    for f in ("orc_build_elements", "orc_combine", "orc_suffix_values", "orc_trajectory", "orc_solve",
              "orc_sequential", "orc_densify", "orc_build_elements_forward", "orc_prefix",
              "orc_trajectory_method2", "orc_grid_combine", "orc_grid_apply", "orc_grid_block",
              "orc_grid_values_sequential", "orc_grid_values"):
        getattr(L, f).restype = ct.c_int
    return L


class swapped_library:
    """Context manager that makes every oracle call use the shared library at
    `path` (a copy of lqt_oracle.c with a planted mistake, for the tests that
    check that the pins catch mistakes)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _configure(ct.CDLL(self.path))
        return self

    def __exit__(self, *a):
        global _lib
        _lib = self.saved


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(ct.CDLL(build()))
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class _Marshalled:
    """Keeps the numpy arrays referenced by the C struct alive."""

    def __init__(self, p):
        self.keep = []

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            self.keep.append(a)
            return a

        s = _Problem()
        s.n, s.m, s.nr, s.T, s.K = p.n, p.m, p.nr, p.T, p.K
        s.t = _ptr(arr(p.t))
        for name in ("F", "L", "c", "H", "X", "U", "r"):
            co = getattr(p, name)
            if co is None:
                setattr(s, name, None)
                setattr(s, name + "_mode", 0)
            else:
                setattr(s, name, _ptr(arr(co.values)))
                setattr(s, name + "_mode", int(co.mode))
        s.Hf = _ptr(arr(p.Hf))
        s.Xf = _ptr(arr(p.Xf))
        s.rf = _ptr(arr(p.rf))
        self.s = s

    def ref(self):
        return ct.byref(self.s)


def element_size(n: int) -> int:
    return 3 * n * n + 2 * n + 1


def unpack(n: int, packed: np.ndarray) -> dict:
    """Split packed elements [..., 3n^2+2n+1] into A, b, C, eta, J, zeta."""
    nn = n * n
    lead = packed.shape[:-1]
    o = 0
    out = {}
    for name, size, shape in (("A", nn, (n, n)), ("b", n, (n,)), ("C", nn, (n, n)), ("eta", n, (n,)),
                              ("J", nn, (n, n)), ("zeta", 1, ())):
        out[name] = packed[..., o:o + size].reshape(lead + shape)
        o += size
    return out


def pack(n: int, e: dict) -> np.ndarray:
    lead = np.asarray(e["A"]).shape[:-2]
    parts = [np.asarray(e[k], dtype=np.float64).reshape(lead + (-1,)) for k in ("A", "b", "C", "eta", "J")]
    parts.append(np.asarray(e["zeta"], dtype=np.float64).reshape(lead + (1,)))
    return np.ascontiguousarray(np.concatenate(parts, axis=-1))


def build_elements(p, j0: int = 0, j1: int | None = None) -> dict:
    """Elements j0..j1-1 (j = T is the terminal element), unpacked."""
    j1 = p.T + 1 if j1 is None else j1
    out = np.zeros((j1 - j0, element_size(p.n)))
    m = _Marshalled(p)
    rc = lib().orc_build_elements(m.ref(), j0, j1, _ptr(out))
    if rc:
        raise FloatingPointError("oracle: singular U sample")
    return unpack(p.n, out)


def combine(n: int, e1: dict, e2: dict) -> dict:
    """One LQT combination e1 (x) e2 (single elements, unpacked dicts)."""
    a, b = pack(n, e1), pack(n, e2)
    out = np.zeros(element_size(n))
    rc = lib().orc_combine(n, _ptr(a), _ptr(b), _ptr(out))
    if rc:
        raise FloatingPointError("oracle: I + C1 J2 singular")
    return unpack(n, out)


def suffix_values(n: int, elems: dict):
    """Sequential right-to-left fold of T+1 elements: (S, v, zeta) at t_0..t_T."""
    packed = pack(n, elems)
    T = packed.shape[0] - 1
    S = np.zeros((T + 1, n, n)); v = np.zeros((T + 1, n)); z = np.zeros(T + 1)
    rc = lib().orc_suffix_values(n, T, _ptr(packed), _ptr(S), _ptr(v), _ptr(z))
    if rc:
        raise FloatingPointError("oracle: singular combination")
    return S, v, z


def trajectory(p, elems: dict, S, v, x0):
    packed = pack(p.n, elems)
    x = np.zeros((p.T + 1, p.n)); u = np.zeros((p.T + 1, p.m))
    m = _Marshalled(p)
    rc = lib().orc_trajectory(m.ref(), _ptr(packed), _ptr(np.ascontiguousarray(S)), _ptr(np.ascontiguousarray(v)),
                              _ptr(np.ascontiguousarray(x0, dtype=np.float64)), _ptr(x), _ptr(u))
    if rc:
        raise FloatingPointError("oracle: singular solve in trajectory")
    return x, u


def solve(p, x0=None, keep_elements: bool = False) -> dict:
    """O1: RK4 elements + sequential fold + one-block Method-2 rollout."""
    x0 = np.ascontiguousarray(p.x0 if x0 is None else x0, dtype=np.float64)
    n, T = p.n, p.T
    S = np.zeros((T + 1, n, n)); v = np.zeros((T + 1, n)); z = np.zeros(T + 1)
    x = np.zeros((T + 1, n)); u = np.zeros((T + 1, p.m)); cost = np.zeros(1)
    el = np.zeros((T + 1, element_size(n))) if keep_elements else None
    m = _Marshalled(p)
    rc = lib().orc_solve(m.ref(), _ptr(x0), _ptr(S), _ptr(v), _ptr(z), _ptr(x), _ptr(u), _ptr(cost), _ptr(el))
    if rc:
        raise FloatingPointError("oracle: singular matrix in solve")
    out = {"S": S, "v": v, "zeta": z, "x": x, "u": u, "cost": float(cost[0])}
    if keep_elements:
        out["elements"] = unpack(n, el)
    return out


def sequential(p, x0=None) -> dict:
    """O2: sequential RK4 Riccati sweep + Hermite-midpoint RK4 forward rollout."""
    x0 = np.ascontiguousarray(p.x0 if x0 is None else x0, dtype=np.float64)
    n, T = p.n, p.T
    S = np.zeros((T + 1, n, n)); v = np.zeros((T + 1, n)); z = np.zeros(T + 1)
    x = np.zeros((T + 1, n)); u = np.zeros((T + 1, p.m)); cost = np.zeros(1)
    m = _Marshalled(p)
    rc = lib().orc_sequential(m.ref(), _ptr(x0), _ptr(S), _ptr(v), _ptr(z), _ptr(x), _ptr(u), _ptr(cost))
    if rc:
        raise FloatingPointError("oracle: singular matrix in sequential sweep")
    return {"S": S, "v": v, "zeta": z, "x": x, "u": u, "cost": float(cost[0])}


def densify(p, sol: dict) -> dict:
    """Values, states and controls at every RK4 sub-step t_j + i h_j (i = 0..K-1)
    and t_T, from a boundary solution sol = {S, v, zeta, x} (e.g. solve(p)):
    per block, K RK4 steps of the Riccati ODEs backward from the block's right
    boundary and K RK4 steps of the closed loop forward from its left boundary."""
    n, m, T, K = p.n, p.m, p.T, p.K
    G = T * K + 1
    Sd = np.zeros((G, n, n)); vd = np.zeros((G, n)); zd = np.zeros(G); xd = np.zeros((G, n)); ud = np.zeros((G, m))
    mr = _Marshalled(p)
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    rc = lib().orc_densify(mr.ref(), _ptr(c(sol["S"])), _ptr(c(sol["v"])), _ptr(c(sol["zeta"])), _ptr(c(sol["x"])),
                           _ptr(Sd), _ptr(vd), _ptr(zd), _ptr(xd), _ptr(ud))
    if rc:
        raise FloatingPointError("oracle: singular U sample in densify")
    return {"S": Sd, "v": vd, "zeta": zd, "x": xd, "u": ud}


def fine_times(p) -> np.ndarray:
    """The RK4 sub-step times t_j + i h_j, i = 0..K-1, and t_T."""
    K = p.K
    t = np.asarray(p.t, dtype=np.float64)
    out = (t[:-1, None] + (t[1:] - t[:-1])[:, None] * (np.arange(K)[None, :] / K)).ravel()
    return np.concatenate([out, t[-1:]])


def build_elements_forward(p, j0: int = 0, j1: int | None = None) -> dict:
    """Elements j0..j1-1 (j < T) from K RK4 steps of the forward conditional
    HJB ODEs (Sec. IV-C), unpacked."""
    j1 = p.T if j1 is None else j1
    out = np.zeros((j1 - j0, element_size(p.n)))
    m = _Marshalled(p)
    if lib().orc_build_elements_forward(m.ref(), j0, j1, _ptr(out)):
        raise FloatingPointError("oracle: singular U sample")
    return unpack(p.n, out)


def prefix(n: int, elems: dict) -> dict:
    """The T+1 prefixes p_k = a_0 (x) ... (x) a_{k-1} (p_0 = identity) of T elements."""
    packed = pack(n, elems)
    T = packed.shape[0]
    out = np.zeros((T + 1, element_size(n)))
    if lib().orc_prefix(n, T, _ptr(packed), _ptr(out)):
        raise FloatingPointError("oracle: singular combination")
    return unpack(n, out)


def trajectory_method2(p, S, v, x0=None) -> dict:
    """Optimal states and controls at the boundaries by Method 2 with
    forward-ODE elements, given the values S, v."""
    x0 = np.ascontiguousarray(p.x0 if x0 is None else x0, dtype=np.float64)
    x = np.zeros((p.T + 1, p.n)); u = np.zeros((p.T + 1, p.m))
    m = _Marshalled(p)
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    if lib().orc_trajectory_method2(m.ref(), _ptr(c(S)), _ptr(c(v)), _ptr(x0), _ptr(x), _ptr(u)):
        raise FloatingPointError("oracle: singular matrix in Method 2")
    return {"x": x, "u": u}


def _grid_struct(g) -> "_GridProblem":
    return _GridProblem(g.G, g.x_min, g.dx, g.d0, g.d1, g.d2, g.q, g.rho, g.qf, g.tau, g.substeps, g.T,
                        1 if g.interp else 0)


def grid_combine(g, A, B) -> np.ndarray:
    """(A (x) B)(i, j) = min_k A(i, k) + B(k, j) on the grid (App. E refinement if g.interp)."""
    out = np.zeros((g.G, g.G))
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    lib().orc_grid_combine(ct.byref(_grid_struct(g)), _ptr(c(A)), _ptr(c(B)), _ptr(out))
    return out


def grid_apply(g, M, w) -> np.ndarray:
    out = np.zeros(g.G)
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    lib().orc_grid_apply(ct.byref(_grid_struct(g)), _ptr(c(M)), _ptr(c(w)), _ptr(out))
    return out


def grid_block(g) -> np.ndarray:
    """The block's conditional value function on the grid (G x G)."""
    out = np.zeros((g.G, g.G))
    lib().orc_grid_block(ct.byref(_grid_struct(g)), _ptr(out))
    return out


def grid_values_sequential(g, Vblock) -> np.ndarray:
    out = np.zeros((g.T + 1, g.G))
    lib().orc_grid_values_sequential(ct.byref(_grid_struct(g)), _ptr(np.ascontiguousarray(Vblock)), _ptr(out))
    return out


def grid_values(g, Vblock) -> np.ndarray:
    """Values at every block boundary in the doubling-scan order."""
    out = np.zeros((g.T + 1, g.G))
    lib().orc_grid_values(ct.byref(_grid_struct(g)), _ptr(np.ascontiguousarray(Vblock)), _ptr(out))
    return out
