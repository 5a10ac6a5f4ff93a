"""GPU path (through the C ABI) against the oracle, element by element.

Tolerance: relative 1e-9 per output tensor, measured boundary by boundary:
max_i |gpu_i - oracle_i|_F / max(|oracle_i|_F, 1e-8 max_j |oracle_j|_F), with
i the leading (boundary, sub-step or element) index, so a boundary whose S or
v is small next to the largest one is held to the same relative bound; the
floor keeps boundaries where an output is identically ~0 (v with a zero
reference) from dividing by rounding noise.  Both sides use the same discretisation (K RK4
steps of the element ODEs per sub-interval and the combination rule), so only
rounding order differs: the GPU's chunked tree and factor form B = Lt Lt^T
against the oracle's sequential fold and explicit B.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9


def lqt():
    import paper_2212_11744_gb300 as m
    return m


def relerr(a, b):
    """Per-boundary relative error: axis 0 indexes boundaries (each entry of a
    1-D array is one boundary); each boundary's difference in the Frobenius
    norm over its own entries, divided by that boundary's reference norm,
    floored at 1e-8 of the largest reference norm (and at 1e-300)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    if b.size == 0:
        return 0.0
    a = a.reshape(b.shape[0], -1) if b.ndim else a.reshape(1, 1)
    b = b.reshape(b.shape[0], -1) if b.ndim else b.reshape(1, 1)
    d = np.linalg.norm(a - b, axis=1)
    r = np.linalg.norm(b, axis=1)
    den = np.maximum(r, max(1e-8 * r.max(), 1e-300))
    return float((d / den).max())


def relerr_one(a, b):
    """Relative error of one boundary's tensor in the Frobenius norm."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_np(t):
    return t.detach().cpu().numpy()


def check_solution(got, ref, keys=("S", "v", "zeta", "x", "u"), tol=TOL, label=""):
    errs = {k: relerr(to_np(got[k]), ref[k]) for k in keys}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"{label} relative errors above {tol}: {errs}"
    return errs


CASES = [
    ("double_integrator_T1024_K10", lambda: W.double_integrator(T=1024, K=10)),
    ("point_mass_T1000_K4", lambda: W.point_mass_2d(T=1000, K=4)),
    ("general_n3_m2_nr2_T37", lambda: W.general_time_varying(3, 2, 2, T=37, K=3, seed=21)),
    ("general_mixed_modes_T45", lambda: W.general_time_varying(
        4, 2, 3, T=45, K=2, seed=22, modes={"r": W.PER_INTERVAL, "X": W.CONST, "F": W.PER_INTERVAL,
                                             "L": W.CONST, "U": W.PER_INTERVAL})),
    ("general_nonuniform_T29", lambda: W.general_time_varying(2, 1, 2, T=29, K=4, seed=23, nonuniform=True)),
    ("scalar_n1_T50", lambda: W.general_time_varying(1, 1, 1, T=50, K=5, seed=24)),
    ("n8_m4_T300", lambda: W.batched_member(5, T=300, n=8)),
    ("n8_m8_T33", lambda: W.general_time_varying(8, 8, 8, T=33, K=2, seed=25, tf=1.0)),
    ("T1", lambda: W.general_time_varying(3, 1, 3, T=1, K=4, seed=26, tf=0.5)),
    ("T2", lambda: W.general_time_varying(2, 2, 2, T=2, K=1, seed=27)),
    ("T3", lambda: W.general_time_varying(4, 2, 4, T=3, K=2, seed=28)),
    ("n16_m8_T40_general", lambda: W.general_time_varying(16, 8, 16, T=40, K=2, seed=81, tf=1.0)),
    ("n16_batched_member_T300", lambda: W.batched_member(7, T=300, n=16)),
    ("n64_m16_T64", lambda: W.large_state_n64(T=64)),
    ("n64_m16_T129_ragged", lambda: W.large_state_n64(T=129)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_solve_matches_oracle(name, make):
    p = make()
    ref = oracle.solve(p)
    m = lqt()
    dp = m.DeviceProblem(p)
    out = m.lqt_solve(dp)
    torch.cuda.synchronize()
    assert m.lqt_get_status() == 0
    check_solution(out, ref, label=name)
    assert abs(float(out["cost"][0]) - ref["cost"]) <= TOL * max(1.0, abs(ref["cost"]))


@pytest.mark.parametrize("name,make", CASES[:8], ids=[c[0] for c in CASES[:8]])
def test_build_elements_matches_oracle(name, make):
    p = make()
    ref = oracle.build_elements(p)
    m = lqt()
    dp = m.DeviceProblem(p)
    el = m.lqt_build_elements(dp)
    torch.cuda.synchronize()
    for k in ("A", "b", "C", "eta", "J", "zeta"):
        e = relerr(to_np(el[k]), ref[k])
        assert e <= 1e-11, (name, k, e)


def test_scan_value_on_oracle_elements():
    """Stage (b) alone, fed the oracle's elements, against the oracle's fold."""
    p = W.general_time_varying(4, 2, 4, T=211, K=2, seed=31)
    ref_el = oracle.build_elements(p)
    S, v, z = oracle.suffix_values(p.n, ref_el)
    m = lqt()
    dp = m.DeviceProblem(p)
    el = {k: torch.from_numpy(np.ascontiguousarray(ref_el[k])).cuda() for k in ref_el}
    out = m.lqt_scan_value(dp, el)
    torch.cuda.synchronize()
    assert relerr(to_np(out["S"]), S) <= TOL
    assert relerr(to_np(out["v"]), v) <= TOL
    assert relerr(to_np(out["zeta"]), z) <= TOL


def test_scan_trajectory_standalone():
    """Stage (c) alone, fed the oracle's elements and values."""
    p = W.point_mass_2d(T=517, K=4)
    ref = oracle.solve(p, keep_elements=True)
    m = lqt()
    dp = m.DeviceProblem(p)
    el = {k: torch.from_numpy(np.ascontiguousarray(ref["elements"][k])).cuda() for k in ref["elements"]}
    S = torch.from_numpy(ref["S"]).cuda()
    v = torch.from_numpy(ref["v"]).cuda()
    out = m.lqt_scan_trajectory(dp, el, S, v)
    torch.cuda.synchronize()
    assert relerr(to_np(out["x"]), ref["x"]) <= TOL
    assert relerr(to_np(out["u"]), ref["u"]) <= TOL


def test_scan_worked_example_on_gpu():
    """The paper's all-prefix-sums example (Sec. II-C) through the GPU scans:
    with n = 1, A = 1, C = J = 0 the combination adds eta (reverse sums) and the
    affine maps add b (prefix sums).  Exact in FP64."""
    import os
    rows = [list(map(float, ln.split())) for ln in open(os.path.join(os.path.dirname(__file__), "golden",
                                                                     "scan_worked_example.txt"))
            if ln.strip() and not ln.startswith("#")]
    a, pre, suf = map(np.array, rows)
    T = len(a)  # 8 boundaries 0..7 -> treat as T = 7 sub-intervals + terminal
    p = W.general_time_varying(1, 1, 1, T=T - 1, K=1, seed=1)
    m = lqt()
    dp = m.DeviceProblem(p)
    dev = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda")
    el = {"A": dev(np.ones((T, 1, 1))), "b": dev(np.zeros((T, 1))), "C": dev(np.zeros((T, 1, 1))),
          "eta": dev(a[:, None]), "J": dev(np.zeros((T, 1, 1))), "zeta": dev(np.zeros(T))}
    out = m.lqt_scan_value(dp, el)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(out["v"])[:, 0], suf)
    el["b"] = dev(a[:, None])
    traj = m.lqt_scan_trajectory(dp, el, dev(np.zeros((T, 1, 1))), dev(np.zeros((T, 1))), x0=dev([0.0]))
    torch.cuda.synchronize()
    assert np.array_equal(to_np(traj["x"])[1:, 0], pre[:-1])


SEQ_CASES = [
    CASES[0], CASES[2],
    ("mixed_K8", lambda: W.resample(CASES[3][1](), 8)),
    ("point_mass_T256", lambda: W.point_mass_2d(T=256)),
]


@pytest.mark.parametrize("name,make", SEQ_CASES, ids=[c[0] for c in SEQ_CASES])
def test_sequential_sweep_matches_oracle(name, make):
    """The one-thread sequential sweep against the oracle's sequential method
    (cases where RK4 of the Riccati equation is stable at the given step; at
    coarser steps both blow up identically, while the per-sub-interval element
    ODEs of the parallel method, started from the zero-length boundary, stay
    finite)."""
    p = make()
    ref = oracle.sequential(p)
    m = lqt()
    dp = m.DeviceProblem(p)
    out = m.lqt_solve_sequential(dp)
    torch.cuda.synchronize()
    check_solution(out, ref, label=name)


HOST_CASES = [
    ("point_mass_T777", lambda: W.point_mass_2d(T=777, K=4)),  # one piece
    # chunked: coefficient copies overlapped with the builds of earlier chunks
    ("point_mass_T2e17_plus_5", lambda: W.point_mass_2d(T=(1 << 17) + 5, K=4)),
    ("general_n3_per_interval_T70001", lambda: W.general_time_varying(
        3, 2, 2, T=70001, K=2, seed=61, tf=3.0, modes={"F": W.PER_INTERVAL, "L": W.PER_INTERVAL, "c": W.CONST,
                                                     "H": W.CONST, "X": W.PER_INTERVAL, "U": W.PER_INTERVAL,
                                                     "r": W.PER_INTERVAL})),
    ("general_n2_per_stage_T65536", lambda: W.general_time_varying(2, 1, 2, T=65536, K=2, seed=62, tf=3.0)),
]


@pytest.mark.parametrize("name,make", HOST_CASES, ids=[c[0] for c in HOST_CASES])
def test_solve_host_matches_device(name, make):
    """lqt_solve_host (host buffers in, host buffers out) gives lqt_solve's
    results bit for bit, also when it copies and builds in overlapped chunks."""
    p = make()
    m = lqt()
    dp = m.DeviceProblem(p)
    dev = m.lqt_solve(dp)
    hp = m.HostProblem(p)
    need = m.lqt_workspace_size(hp, m.LQT_WS_SOLVE) + m.lqt_host_staging_size(hp)
    ws = torch.empty(need + 4096, dtype=torch.uint8, device="cuda")
    host = m.lqt_solve_host(hp, ws)
    torch.cuda.synchronize()
    for k in ("S", "v", "zeta", "x", "u", "cost"):
        assert np.array_equal(to_np(dev[k]), host[k].numpy()), k


def test_solve_host_with_pageable_buffers():
    """The chunked host path with pageable (not pinned) host inputs and
    outputs: the copies then complete before the calls return, the results are
    still lqt_solve's bit for bit."""
    p = W.point_mass_2d(T=(1 << 16) + 7, K=4)
    m = lqt()
    dev = m.lqt_solve(m.DeviceProblem(p))
    hp = m.HostProblem(p, pinned=False)
    need = m.lqt_workspace_size(hp, m.LQT_WS_SOLVE) + m.lqt_host_staging_size(hp)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    host = m.lqt_solve_host(hp, ws, out=m.host_solution(hp, pinned=False))
    torch.cuda.synchronize()
    for k in ("S", "v", "zeta", "x", "u", "cost"):
        assert np.array_equal(to_np(dev[k]), host[k].numpy()), k


def test_nonfinite_input_sets_status():
    p = W.point_mass_2d(T=64, K=4)
    p.r.values[100, 0] = np.nan
    m = lqt()
    dp = m.DeviceProblem(p)
    m.lqt_solve(dp)
    assert m.lqt_get_status() == 3  # LQT_ENONFINITE
    # the word is cleared by the read
    p2 = W.point_mass_2d(T=64, K=4)
    m.lqt_solve(m.DeviceProblem(p2))
    assert m.lqt_get_status() == 0


def test_repeat_calls_are_deterministic():
    p = W.general_time_varying(4, 2, 4, T=300, K=2, seed=41)
    m = lqt()
    dp = m.DeviceProblem(p)
    a = m.lqt_solve(dp)
    b = m.lqt_solve(dp)
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.slow
def test_point_mass_full_size_against_oracle():
    """The 2-D point-mass workload at its largest size, T = 2^20 sub-intervals,
    K = 4, in the launch configuration the benchmark times: every output at
    every boundary against the full oracle."""
    p = W.point_mass_2d(T=1 << 20, K=4)
    m = lqt()
    dp = m.DeviceProblem(p)
    out = m.lqt_solve(dp)
    torch.cuda.synchronize()
    assert m.lqt_get_status() == 0
    ref = oracle.solve(p)
    check_solution(out, ref, label="point_mass_2^20")


@pytest.mark.slow
def test_large_state_full_size_local_checks():
    """The n = 64, m = 16 workload at its full size, T = 2^16, K = 2, solved in
    FP64 as the benchmark runs it.  The oracle cannot fold 2^16 elements of
    n = 64 in seconds, so at sampled boundaries k the GPU's outputs are checked
    through relations that hold at any size, with the oracle's own element k:
    (S, v, zeta)_k = element_k (x) (S, v, zeta)_{k+1} (the oracle's
    combination, Lemma LQT_combination, with a value as the right operand),
    x_{k+1} = (I + C_k S_{k+1})^-1 (A_k x_k + b_k + C_k v_{k+1}) (Method 2 over
    one sub-interval) and u_k = U^-1 L^T (v_k - S_k x_k)."""
    p = W.large_state_n64(T=1 << 16)
    m = lqt()
    out = m.lqt_solve(m.DeviceProblem(p))
    torch.cuda.synchronize()
    assert m.lqt_get_status() == 0
    S, v, z, x, u = (to_np(out[k]) for k in ("S", "v", "zeta", "x", "u"))
    n, T = p.n, p.T
    term = oracle.build_elements(p, T, T + 1)
    assert relerr_one(S[T], term["J"][0]) <= TOL and relerr_one(v[T], term["eta"][0]) <= TOL
    L = p.L.values[0]
    U = p.U.values[0]
    for k in (0, 1, 4097, 31_000, T // 2 + 3, T - 2, T - 1):
        e = {kk: vv[0] for kk, vv in oracle.build_elements(p, k, k + 1).items()}
        val = {"A": np.zeros((n, n)), "b": np.zeros(n), "C": np.zeros((n, n)), "eta": v[k + 1], "J": S[k + 1],
               "zeta": z[k + 1]}
        c = oracle.combine(n, e, val)
        assert relerr_one(S[k], c["J"]) <= TOL, k
        assert relerr_one(v[k], c["eta"]) <= TOL, k
        assert abs(z[k] - float(c["zeta"])) <= TOL * max(1.0, abs(float(c["zeta"]))), k
        xn = np.linalg.solve(np.eye(n) + e["C"] @ S[k + 1], e["A"] @ x[k] + e["b"] + e["C"] @ v[k + 1])
        assert relerr_one(x[k + 1], xn) <= TOL, k
        assert relerr_one(u[k], np.linalg.solve(U, L.T @ (v[k] - S[k] @ x[k]))) <= TOL, k


@pytest.mark.slow
@pytest.mark.parametrize("T", [1 << 10, 1 << 14])
def test_parallel_solve_beats_the_sequential_sweep(T):
    """The point-mass workload at T = 2^10 and 2^14 (K = 4): the parallel solve
    (lqt_solve) takes less time than the one-thread sequential GPU sweep
    (lqt_solve_sequential, the paper's sequential method) on the same grid,
    both timed with CUDA events after a warm-up."""
    m = lqt()
    dp = m.DeviceProblem(W.point_mass_2d(T=T, K=4))
    par = m.lqt_solve(dp)
    seq = m.lqt_solve_sequential(dp)
    torch.cuda.synchronize()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    t_par = min(timed(lambda: m.lqt_solve(dp, out=par)) for _ in range(3))
    t_seq = timed(lambda: m.lqt_solve_sequential(dp, out=seq))
    assert m.lqt_get_status() == 0
    print(f"T={T}: parallel {t_par:.3f} ms, sequential {t_seq:.1f} ms")
    assert t_par < t_seq, (t_par, t_seq)
