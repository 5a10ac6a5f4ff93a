"""Batched solves against the oracle, problem by problem.  Error measure as in
test_gpu_parity.py (per boundary, relative, floored at 1e-8 of the largest)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_gpu_parity import TOL, relerr as rel

pytestmark = pytest.mark.gpu


def members(n, Ts, first_seed):
    return [W.batched_member(first_seed + i, T=T, n=n) for i, T in enumerate(Ts)]


@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_batch_matches_oracle_per_problem(n):
    from paper_2212_11744_gb300.batch import Batch
    probs = members(n, [37, 123, 300, 64], 100 * n)
    bt = Batch(probs)
    out = bt.solve()
    torch.cuda.synchronize()
    for b, p in enumerate(probs):
        ref = oracle.solve(p)
        got = bt.problem_slice(out, b)
        for k in ("S", "v", "zeta", "x", "u"):
            assert rel(got[k].cpu().numpy(), ref[k]) <= TOL, (n, b, k)
        assert abs(float(got["cost"]) - ref["cost"]) <= TOL * max(1.0, abs(ref["cost"])), (n, b)


def test_batch_chunk_choices_agree_and_graph_replay():
    """Every first-level chunk length gives the same solution (to rounding);
    the batched solves of several dimensions captured in one CUDA graph and
    replayed give the same outputs as direct calls."""
    from paper_2212_11744_gb300.batch import Batch
    batches = [Batch(members(n, [90, 211, 45], 7 * n)) for n in (2, 4, 8, 16)]
    for bt in batches:
        base = bt.solve()
        for c in (2, 4, 16, 32):
            o = bt.solve(chunk=c)
            for k in ("S", "v", "zeta", "x"):
                assert rel(o[k].cpu().numpy(), base[k].cpu().numpy()) <= 1e-12, (bt.n, c, k)
    outs = [bt.new_outputs() for bt in batches]
    for bt, o in zip(batches, outs):  # warm-up outside capture
        bt.solve(out=o)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            for bt, o in zip(batches, outs):
                bt.solve(out=o, stream=s)
    for o in outs:
        for v in o.values():
            v.zero_()
    g.replay()
    torch.cuda.synchronize()
    for bt, o in zip(batches, outs):
        ref = bt.solve()
        torch.cuda.synchronize()
        for k in ("S", "v", "zeta", "x", "u", "cost"):
            assert torch.equal(o[k], ref[k]), (bt.n, k)


def test_batch_set_streams_and_graph_match_direct_solves():
    """Problems of four state dimensions, interleaved, through BatchSet: one
    batch per dimension on its own stream, forked from and joined back into
    the caller's stream; the solution of every problem against the oracle,
    and the set captured as one CUDA graph and replayed bit-identical."""
    from paper_2212_11744_gb300.batch import BatchSet
    probs = [W.batched_member(b, T=90 + 13 * b, n=(2, 4, 8, 16)[b % 4]) for b in range(8)]
    bset = BatchSet(probs)
    assert sorted(bset.batches) == [2, 4, 8, 16]
    s = torch.cuda.Stream()
    out = bset.solve(stream=s)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        ref = oracle.solve(p)
        got = bset.problem_slice(out, i)
        for k in ("S", "v", "zeta", "x", "u"):
            assert rel(got[k].cpu().numpy(), ref[k]) <= TOL, (i, p.n, k)
        assert abs(float(got["cost"]) - ref["cost"]) <= TOL * max(1.0, abs(ref["cost"])), i
    replay = bset.new_outputs()
    bset.solve(replay, stream=s)
    torch.cuda.synchronize()
    g = bset.capture(replay, stream=s)
    for o in replay.values():
        for v in o.values():
            v.zero_()
    g.replay()
    torch.cuda.synchronize()
    import paper_2212_11744_gb300 as lqt
    assert lqt.lqt_get_status() == 0
    for n in out:
        for k in ("S", "v", "zeta", "x", "u", "cost"):
            assert torch.equal(replay[n][k], out[n][k]), (n, k)


def test_short_chunk_override_on_a_batch_whose_default_is_longer():
    """A batch large enough that the built-in first-level chunk is > 2, solved
    with every allowed chunk (the workspace must cover the shortest), checked
    against the oracle for two of its problems."""
    from paper_2212_11744_gb300 import _abi
    from paper_2212_11744_gb300.batch import Batch
    probs = members(2, [7000] * 10, 40)
    bt = Batch(probs)
    for c in (2, 4, 32, 0):
        out = bt.solve(chunk=c)
        torch.cuda.synchronize()
        for b in (0, 9):
            ref = oracle.solve(probs[b])
            got = bt.problem_slice(out, b)
            for k in ("S", "v", "x"):
                assert rel(got[k].cpu().numpy(), ref[k]) <= TOL, (c, b, k)
    with pytest.raises(_abi.LQTError):
        bt.solve(chunk=3)


def test_autotuner_picks_a_candidate():
    from paper_2212_11744_gb300.batch import Batch
    bt = Batch(members(4, [500, 800, 300], 3))
    best = bt.autotune(candidates=(0, 4, 16), reps=2)
    assert best in (0, 4, 16)
    assert Batch.tuning_table()[(4, 3, bt.total, 0)][0] == best


@pytest.mark.slow
def test_full_batch_sampled_problems_against_oracle():
    """The whole 4096-problem batch of the benchmark (n in {2,4,8,16},
    T in [256, 8192]), solved per state dimension with the autotuned chunk as
    the benchmark runs it; for each n, the problems with the shortest and the
    longest horizon and one more (seeded) against the oracle, every output."""
    from paper_2212_11744_gb300.batch import Batch
    probs = [W.batched_member(b) for b in range(4096)]
    byn = {}
    for b, p in enumerate(probs):
        byn.setdefault(p.n, []).append(b)
    rng = np.random.default_rng(4096)
    for n, idx in sorted(byn.items()):
        bt = Batch([probs[b] for b in idx])
        bt.autotune(candidates=(0, 8, 32), reps=1)
        out = bt.solve()
        torch.cuda.synchronize()
        Ts = [probs[b].T for b in idx]
        picks = {int(np.argmin(Ts)), int(np.argmax(Ts)), int(rng.integers(len(idx)))}
        for i in sorted(picks):
            p = probs[idx[i]]
            ref = oracle.solve(p)
            got = bt.problem_slice(out, i)
            for k in ("S", "v", "zeta", "x", "u"):
                assert rel(got[k].cpu().numpy(), ref[k]) <= TOL, (n, idx[i], p.T, k)


def test_n16_batch_of_40_sampled_against_oracle():
    """The first 40 problems of state dimension 16 in the 4096-problem batch
    (about 1.7e5 sub-intervals: enough chunks to fill every warp slot of the
    warp-per-combination scan), solved as one batch; the shortest and the
    longest problem checked against the oracle."""
    from paper_2212_11744_gb300.batch import Batch
    probs = []
    b = 0
    while len(probs) < 40:
        p = W.batched_member(b)
        if p.n == 16:
            probs.append(p)
        b += 1
    bt = Batch(probs)
    out = bt.solve()
    torch.cuda.synchronize()
    assert lqt_status() == 0
    Ts = [p.T for p in probs]
    for i in {int(np.argmin(Ts)), int(np.argmax(Ts))}:
        ref = oracle.solve(probs[i])
        got = bt.problem_slice(out, i)
        for k in ("S", "v", "zeta", "x", "u"):
            assert rel(got[k].cpu().numpy(), ref[k]) <= TOL, (i, probs[i].T, k)


def lqt_status():
    import paper_2212_11744_gb300 as lqt
    return lqt.lqt_get_status()
