"""The C-ABI library builds, loads and exports every symbol include/lqt.h
declares; host-side validation rejects bad arguments before any launch.  CPU
only (no compute calls)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "lqt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lqt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_11744_gb300 import build as B
    path = B.build()
    import paper_2212_11744_gb300 as m
    assert os.path.samefile(path, m.library_path())
    return ct.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    funcs = header_functions()
    assert len(funcs) >= 10
    for f in funcs:
        assert hasattr(lib, f), f
    from paper_2212_11744_gb300 import _abi
    assert set(_abi.EXPORTED) == set(funcs)


def _problem(**over):
    import paper_2212_11744_gb300 as m
    p = W.point_mass_2d(T=16, K=2)
    for k, v in over.items():
        setattr(p, k, v)
    return m.HostProblem(p, pinned=False)


def test_workspace_sizes_positive_and_ordered(lib):
    import paper_2212_11744_gb300 as m
    hp = _problem()
    sizes = {w: m.lqt_workspace_size(hp, w) for w in range(5)}
    assert all(s > 0 for s in sizes.values())
    assert sizes[m.LQT_WS_SOLVE] > sizes[m.LQT_WS_VALUE]
    assert m.lqt_workspace_size(hp, 99) == 0


def test_invalid_arguments_rejected_on_host(lib):
    import paper_2212_11744_gb300 as m
    from paper_2212_11744_gb300 import _abi
    L = _abi.lib()
    hp = _problem()
    dummy = ct.c_void_p(256)
    # unsupported state dimension
    hp.struct.n = 5
    assert m.lqt_workspace_size(hp, m.LQT_WS_SOLVE) == 0
    assert L.lqt_solve(hp.ref(), dummy, dummy, dummy, None, dummy, None, None, dummy, 1 << 30, None) == \
        _abi.LQT_EUNSUPPORTED
    hp.struct.n = 4
    # bad sampling mode
    hp.struct.r.mode = 7
    assert L.lqt_solve(hp.ref(), dummy, dummy, dummy, None, dummy, None, None, dummy, 1 << 30, None) == \
        _abi.LQT_EINVAL
    hp.struct.r.mode = m.LQT_PER_STAGE
    # T = 0
    hp.struct.T = 0
    assert L.lqt_solve(hp.ref(), dummy, dummy, dummy, None, dummy, None, None, dummy, 1 << 30, None) == \
        _abi.LQT_EINVAL
    hp.struct.T = 16
    # missing output
    assert L.lqt_solve(hp.ref(), dummy, None, dummy, None, dummy, None, None, dummy, 1 << 30, None) == \
        _abi.LQT_EINVAL
    # workspace too small
    need = m.lqt_workspace_size(hp, m.LQT_WS_SOLVE)
    assert L.lqt_solve(hp.ref(), dummy, dummy, dummy, None, dummy, None, None, dummy, need - 1, None) == \
        _abi.LQT_EWORKSPACE
    assert L.lqt_solve(hp.ref(), dummy, dummy, dummy, None, dummy, None, None, None, need, None) == \
        _abi.LQT_EWORKSPACE
    # misaligned coefficient pointer
    good = hp.struct.F.ptr
    hp.struct.F.ptr = good + 3
    assert L.lqt_solve(hp.ref(), dummy, dummy, dummy, None, dummy, None, None, dummy, need, None) == _abi.LQT_EINVAL
    hp.struct.F.ptr = good
    # H absent but nr != n
    hp.struct.nr = 3
    assert L.lqt_solve(hp.ref(), dummy, dummy, dummy, None, dummy, None, None, dummy, need, None) == _abi.LQT_EINVAL


def test_strerror_names_every_status(lib):
    import paper_2212_11744_gb300 as m
    names = {m.lqt_strerror(c) for c in range(8)}
    assert len(names) == 8 and "unknown status" not in names


def test_densify_validation_on_host(lib):
    import paper_2212_11744_gb300 as m
    from paper_2212_11744_gb300 import _abi
    L = _abi.lib()
    hp = _problem()
    d = ct.c_void_p(256)
    ws = m.lqt_workspace_size(hp, m.LQT_WS_DENSIFY)
    assert ws > 0
    # missing zeta input, too small a workspace, K above 16, n above 8
    assert L.lqt_densify(hp.ref(), d, d, None, d, d, d, d, d, None, d, ws, None) == _abi.LQT_EINVAL
    assert L.lqt_densify(hp.ref(), d, d, d, d, d, d, d, d, None, d, ws - 1, None) == _abi.LQT_EWORKSPACE
    hp.struct.K = 17
    assert L.lqt_densify(hp.ref(), d, d, d, d, d, d, d, d, None, d, 1 << 40, None) == _abi.LQT_EUNSUPPORTED


def test_grid_validation_on_host(lib):
    import paper_2212_11744_gb300 as m
    from paper_2212_11744_gb300 import _abi
    L = _abi.lib()
    g = W.falling_body(G=60, T=100)
    gs = m.grid_struct(g)
    # block: 2 G^2 doubles; values: 3 G^2 per power (7 powers for T = 100; the
    # power and its curvature/slope pairs) + 1 + (T+1) G
    assert L.lqt_grid_workspace_size(ct.byref(gs), 0) == 2 * 60 * 60 * 8
    assert L.lqt_grid_workspace_size(ct.byref(gs), 1) == (3 * 7 * 60 * 60 + 1 + 101 * 60) * 8
    assert L.lqt_grid_workspace_size(ct.byref(gs), 2) == 0
    d = ct.c_void_p(256)
    need = L.lqt_grid_workspace_size(ct.byref(gs), 1)
    assert L.lqt_grid_values(ct.byref(gs), d, d, d, need, None) == _abi.LQT_EINVAL  # V overlaps Vblock
    assert L.lqt_grid_values(ct.byref(gs), d, ct.c_void_p(1 << 30), d, need - 8, None) == _abi.LQT_EWORKSPACE
    assert L.lqt_grid_combine(ct.byref(gs), d, ct.c_void_p(1 << 30), d, None) == _abi.LQT_EINVAL  # out is A
    for field, bad in (("G", 2), ("G", 16385), ("substeps", 0), ("T", 0), ("T", 1 << 31), ("dx", 0.0),
                       ("rho", -1.0), ("tau", float("nan")), ("interp", 2)):
        b = m.grid_struct(g)
        setattr(b, field, bad)
        assert L.lqt_grid_workspace_size(ct.byref(b), 0) == 0, field
        assert L.lqt_grid_block(ct.byref(b), d, d, 1 << 30, None) == _abi.LQT_EINVAL, field


def test_noalloc_limits_match_the_header(lib):
    """The largest T that lqt_scan_value_noalloc admits per state dimension,
    as stated in include/lqt.h: the sizing function fits the static scratch
    at that T and not at T + 1."""
    import paper_2212_11744_gb300 as m
    from paper_2212_11744_gb300 import _abi
    src = open(os.path.join(ROOT, "include", "lqt.h")).read()
    block = src[src.index("Allocation-free value scan"):src.index("lqt_scan_value_noalloc(const")]
    block = re.sub(r"\s*\n\s*\*\s*", " ", block)
    stated = {int(a): int(b.replace(" ", "")) for a, b in re.findall(r"n = (\d+): (\d[\d ]*\d|\d);", block)}
    assert stated == {1: 7454719, 2: 2795391, 3: 44607, 4: 26877, 8: 7429, 16: 1951}, stated
    assert "n = 64: none" in block
    lim = _abi.LQT_STATIC_SCRATCH_BYTES
    dims = {1: 1, 2: 1, 3: 2, 4: 2, 8: 4, 16: 8}
    for n, Tmax in stated.items():
        hp = m.HostProblem(W.general_time_varying(n, dims[n], n, T=4, K=1, seed=1), pinned=False)
        hp.struct.T = Tmax
        assert 0 < m.lqt_workspace_size(hp, m.LQT_WS_VALUE) <= lim, n
        hp.struct.T = Tmax + 1
        assert m.lqt_workspace_size(hp, m.LQT_WS_VALUE) > lim, n
    hp = m.HostProblem(W.large_state_n64(T=1), pinned=False)
    assert m.lqt_workspace_size(hp, m.LQT_WS_VALUE) > lim


def test_backward_workspace_holds_one_segment_of_stage_inputs(lib):
    """Beyond one segment (2^15 sub-intervals) the backward workspace grows by
    less per sub-interval than the 16 RK4 stage records of a sub-interval
    (n = 8, K = 4: 16 x (3n^2 + 2n + 1) doubles): the stage inputs are
    recomputed per segment, not stored for all T."""
    import paper_2212_11744_gb300 as m
    hp = m.HostProblem(W.differentiable_n8(T=64), pinned=False)
    n, K = 8, 4

    def ws(T):
        hp.struct.T = T
        return m.lqt_workspace_size(hp, m.LQT_WS_BACKWARD)

    stage_record = 4 * K * (3 * n * n + 2 * n + 1) * 8
    T1, T2 = 1 << 16, 1 << 20
    assert ws(T2) > ws(T1) > 0
    assert (ws(T2) - ws(T1)) / (T2 - T1) < 0.5 * stage_record


def test_method2_workspaces_cover_every_state_dimension(lib):
    """Method 2 runs at every state dimension of lqt_solve: its workspace kinds
    are non-zero for n = 16 and 64 (team kernels), the solve's exceeds the
    trajectory's, and the n = 64 forward-element build's scratch (LQT_WS_BUILD)
    holds 152 slots of four element records plus products."""
    import paper_2212_11744_gb300 as m
    for p in (W.batched_member(7, T=300, n=16), W.large_state_n64(T=129)):
        hp = m.HostProblem(p, pinned=False)
        traj = m.lqt_workspace_size(hp, m.LQT_WS_METHOD2)
        solve = m.lqt_workspace_size(hp, m.LQT_WS_SOLVE_METHOD2)
        assert traj > 0 and solve > traj, p.n
    hp = m.HostProblem(W.large_state_n64(T=129), pinned=False)
    n = 64
    four_records = 4 * (3 * n * n + 2 * n + 1) * 8
    assert m.lqt_workspace_size(hp, m.LQT_WS_BUILD) >= 152 * four_records
