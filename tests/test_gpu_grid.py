"""The grid method for the nonlinear scalar example (Sec. VI-B, App. E) through
the C ABI against the oracle.

Both sides evaluate the same IEEE double formulas in the same order without
multiply-add contraction (the oracle is ISO C compiled without contraction, the
kernels use explicit round-to-nearest intrinsics), so the grid minimisers agree
and the results agree bit for bit: these tests ask for equality.  The kernel
screens candidates in FP32 before the FP64 minimum; the edge cases below aim at
that screen (ties, operands outside its range, underflow, cancellation).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_oracle_grid import discrete_lq_values, lq_problem

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def same(got: torch.Tensor, ref: np.ndarray, what: str):
    g = got.cpu().numpy()
    assert g.shape == ref.shape, what
    if not np.array_equal(g, ref):
        bad = np.argwhere(g != ref)
        rel = np.abs(g - ref).max() / max(1.0, np.abs(ref).max())
        raise AssertionError(f"{what}: {len(bad)} of {ref.size} differ (first {bad[0].tolist()}), max rel {rel:.3g}")


@pytest.mark.parametrize("G", [3, 16, 37, 64, 100])
@pytest.mark.parametrize("interp", [False, True])
def test_combine_matches_oracle(G, interp):
    import paper_2212_11744_gb300 as lqt
    g = W.falling_body(G=G, T=1, interp=interp)
    rng = np.random.default_rng(1000 + G)
    x = g.grid()
    # smooth bowls plus noise: interior minimisers (refinement taken) and ragged ties
    A = 0.7 * (x[:, None] - 0.3 * x[None, :]) ** 2 + 0.1 * rng.standard_normal((G, G))
    B = 1.3 * (x[:, None] - x[None, :] + 0.5) ** 2 + rng.uniform(0.0, 0.2, (G, G))
    B[G // 2] = B[G // 2 - 1]  # equal rows: ties broken by the lowest index
    got = lqt.lqt_grid_combine(g, dev(A), dev(B))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    same(got, oracle.grid_combine(g, A, B), "combine")


def _screen_case(kind, G, rng):
    """Operands aimed at the FP32 screen of the kernel: exact ties, ties to the
    last bits, magnitudes outside its range, values near the float underflow,
    cancellation between huge operands."""
    x = np.linspace(-6.0, 6.0, G)
    if kind == "all_ties":
        return np.full((G, G), 2.5), np.full((G, G), 1.0)
    if kind == "last_bit_ties":
        base = 3.0 + rng.integers(0, 3, (G, G)) * np.spacing(3.0)
        return base, 1.0 + rng.integers(0, 2, (G, G)) * np.spacing(1.0)
    if kind == "out_of_range":
        A = (x[:, None] - x[None, :]) ** 2
        A[G // 3, 0] = 1e31  # above 2^100: the tile takes the FP64 path
        return A, (x[:, None] + 0.5 * x[None, :]) ** 2
    if kind == "tiny":
        return rng.standard_normal((G, G)) * 1e-38, rng.standard_normal((G, G)) * 1e-39
    if kind == "cancellation":
        A = rng.uniform(-1e29, 1e29, (G, G))
        return A, -A.T + rng.standard_normal((G, G))
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["all_ties", "last_bit_ties", "out_of_range", "tiny", "cancellation"])
@pytest.mark.parametrize("interp", [False, True])
def test_combine_screen_edge_cases(kind, interp):
    import paper_2212_11744_gb300 as lqt
    G = 45
    g = W.falling_body(G=G, T=1, interp=interp)
    A, B = _screen_case(kind, G, np.random.default_rng(77))
    got = lqt.lqt_grid_combine(g, dev(A), dev(B))
    torch.cuda.synchronize()
    lqt.lqt_get_status()
    same(got, oracle.grid_combine(g, A, B), kind)


def test_infinite_operands_take_the_fp64_path():
    import paper_2212_11744_gb300 as lqt
    G = 40
    g = W.falling_body(G=G, T=1, interp=False)
    x = g.grid()
    A = (x[:, None] - x[None, :]) ** 2
    A[:, -1] = np.inf  # never the minimum
    B = (x[:, None] + 1.0) ** 2 + 0.0 * x[None, :]
    got = lqt.lqt_grid_combine(g, dev(A), dev(B))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    same(got, oracle.grid_combine(g, A, B), "inf")


@pytest.mark.parametrize("G,substeps", [(61, 10), (61, 1), (61, 3), (201, 10), (20, 10), (40, 10)])
def test_block_matches_oracle(G, substeps):
    import paper_2212_11744_gb300 as lqt
    g = W.falling_body(G=G, T=1)
    g.substeps = substeps
    got = lqt.lqt_grid_block(g)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    same(got, oracle.grid_block(g), "block")


VALUE_CASES = [
    ("G60_T100", dict(G=60, T=100)),
    ("G20_T37", dict(G=20, T=37)),
    ("G201_T100", dict(G=201, T=100)),
    ("G61_T1", dict(G=61, T=1)),
    ("G61_T64", dict(G=61, T=64)),
    ("G61_T63", dict(G=61, T=63)),
    ("G61_T65_plain", dict(G=61, T=65, interp=False)),
    ("G40_T10000", dict(G=40, T=10000)),
]


@pytest.mark.parametrize("name,kw", VALUE_CASES, ids=[c[0] for c in VALUE_CASES])
def test_values_match_oracle(name, kw):
    """V(., t_k) at every block boundary, block function from the oracle on
    both sides (so the values kernel is checked on its own)."""
    import paper_2212_11744_gb300 as lqt
    g = W.falling_body(**kw)
    Vb = oracle.grid_block(g)
    got = lqt.lqt_grid_values(g, dev(Vb))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    same(got, oracle.grid_values(g, Vb), "values")
    if not g.interp:  # the grid minimum is associative: the sequential fold, exactly up to rounding
        seq = oracle.grid_values_sequential(g, Vb)
        assert np.abs(got.cpu().numpy() - seq).max() <= 1e-12 * np.abs(seq).max()


def test_values_with_a_workspace_off_16_byte_alignment():
    """The workspace need only be 8-byte aligned: the table of curvature pairs
    inside it is placed on a 16-byte boundary by the library."""
    import paper_2212_11744_gb300 as lqt
    g = W.falling_body(G=61, T=77)
    Vb = oracle.grid_block(g)
    need = lqt.lqt_grid_workspace_size(g, 1)
    raw = torch.empty(need + 16, dtype=torch.uint8, device="cuda")
    ws = raw[8:8 + need]
    assert ws.data_ptr() % 16 == 8
    got = lqt.lqt_grid_values(g, dev(Vb), ws=ws)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    same(got, oracle.grid_values(g, Vb), "values")


def test_full_path_at_paper_size():
    """Block function and values on the GPU alone, the largest configuration of
    the paper's nonlinear experiment (grid of 60 points, 10^4 blocks of 1/10
    with 10 steps each), against the oracle end to end."""
    import paper_2212_11744_gb300 as lqt
    g = W.falling_body(G=60, T=10000)
    Vb = lqt.lqt_grid_block(g)
    V = lqt.lqt_grid_values(g, Vb)
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == 0
    ref_b = oracle.grid_block(g)
    same(Vb, ref_b, "block")
    same(V, oracle.grid_values(g, ref_b), "values")


def test_linear_drift_against_discrete_riccati():
    """With a linear drift every minimised function is quadratic, so the GPU's
    values at interior grid points equal the discrete Riccati solution."""
    import paper_2212_11744_gb300 as lqt
    g = lq_problem()
    V = lqt.lqt_grid_values(g, lqt.lqt_grid_block(g)).cpu().numpy()
    torch.cuda.synchronize()
    x = g.grid()
    inner = np.abs(x) <= 2.0
    for k, (S, v, z) in enumerate(discrete_lq_values(g)):
        ref = 0.5 * S * x * x - v * x + z
        assert np.abs(V[k] - ref)[inner].max() <= 1e-10 * np.abs(ref[inner]).max(), k


def test_non_finite_values_are_reported():
    import paper_2212_11744_gb300 as lqt
    g = W.falling_body(G=21, T=5)
    g.qf = 1e308  # terminal cost overflows to inf away from 0
    lqt.lqt_grid_values(g, lqt.lqt_grid_block(g))
    torch.cuda.synchronize()
    assert lqt.lqt_get_status() == lqt._abi.LQT_ENONFINITE
    assert lqt.lqt_get_status() == 0


def test_invalid_arguments_are_rejected_on_host():
    import paper_2212_11744_gb300 as lqt
    g = W.falling_body(G=2, T=5)
    with pytest.raises(lqt.LQTError) as e:
        lqt.lqt_grid_block(g)
    assert e.value.code == lqt._abi.LQT_EINVAL
    g = W.falling_body(G=21, T=5)
    A = dev(np.zeros((21, 21)))
    with pytest.raises(lqt.LQTError) as e:
        lqt.lqt_grid_combine(g, A, A, out=A)  # out overlaps an input
    assert e.value.code == lqt._abi.LQT_EINVAL


def test_refined_values_approach_the_sequential_fold_as_the_grid_grows():
    """With App. E's refinement the grid minimum is not associative, so the
    doubling order the kernel evaluates differs from the sequential fold
    V_k = Vblock (x) V_{k+1} by the interpolation error.  On the GPU, with the
    GPU's own block function: the gap to the oracle's sequential fold (on that
    block function) shrinks as the grid is refined and is small on the finest
    grid, so the kernel's values carry the order-independent meaning of
    Theorem parallel_HJB."""
    import paper_2212_11744_gb300 as lqt
    errs = []
    for G in (61, 121, 241):
        g = W.falling_body(G=G, T=100)
        Vb = lqt.lqt_grid_block(g)
        got = lqt.lqt_grid_values(g, Vb)
        torch.cuda.synchronize()
        assert lqt.lqt_get_status() == 0
        seq = oracle.grid_values_sequential(g, Vb.cpu().numpy())
        inner = np.abs(g.grid()) <= 3.0
        a = got.cpu().numpy()
        errs.append(np.abs(a - seq)[:, inner].max() / np.abs(seq[:, inner]).max())
    assert errs[0] > errs[1] > errs[2] and errs[-1] < 1e-4, errs
