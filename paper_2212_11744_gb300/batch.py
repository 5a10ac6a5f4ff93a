"""Batched solves (lqt_solve_batched) and their autotuner.

    b = Batch(problems)            # problems of one state dimension
    out = b.solve()                # concatenated S, v, zeta, x, u and per-problem cost
    b.autotune()                   # picks the first-level chunk length by timing

    s = BatchSet(problems)         # problems of several state dimensions
    s.autotune()                   # each dimension's batch tuned on its own
    g = s.capture(out)             # one CUDA graph: the dimensions' solves on
    g.replay()                     # concurrent streams, forked and joined

Marshalling only: the per-problem arrays of a batch are packed into a few
device tensors and the C descriptors point into them.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np
import torch

from . import _abi
from ._abi import lqt_batch, lqt_coef, lqt_problem, lqt_tuning

_TUNED = {}


class Batch:
    def __init__(self, problems, device: str = "cuda"):
        if not problems:
            raise ValueError("empty batch")
        self.device = torch.device(device)
        self.B = len(problems)
        p0 = problems[0]
        self.n, self.m = p0.n, p0.m
        # pack every per-problem array into one host buffer, upload once
        chunks, offs = [], {}
        pos = 0

        def add(key, a):
            nonlocal pos
            if a is None:
                offs[key] = None
                return
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            offs[key] = pos
            chunks.append(a)
            pos += a.size

        for b, p in enumerate(problems):
            add((b, "t"), p.t)
            for name in ("F", "L", "c", "X", "U", "r"):
                co = getattr(p, name)
                add((b, name), None if co is None else co.values)
            add((b, "Xf"), p.Xf)
            add((b, "rf"), p.rf)
            add((b, "x0"), p.x0)
        self.data = torch.from_numpy(np.concatenate(chunks)).to(self.device)
        base = self.data.data_ptr()

        def ptr(key):
            o = offs[key]
            return None if o is None else base + 8 * o

        arr = (lqt_problem * self.B)()
        x0s = (ct.c_void_p * self.B)()
        self.T = np.zeros(self.B, dtype=np.int64)
        for b, p in enumerate(problems):
            s = arr[b]
            s.n, s.m, s.nr, s.T, s.K = p.n, p.m, p.nr, p.T, p.K
            s.t = ptr((b, "t"))
            for name in ("F", "L", "c", "H", "X", "U", "r"):
                co = getattr(p, name)
                if name == "H" or co is None:
                    setattr(s, name, lqt_coef(None, 0))
                else:
                    setattr(s, name, lqt_coef(ptr((b, name)), int(co.mode)))
            s.Hf = None
            s.Xf = ptr((b, "Xf"))
            s.rf = ptr((b, "rf"))
            x0s[b] = ptr((b, "x0"))
            self.T[b] = p.T
        self._arr, self._x0s = arr, x0s
        self.struct = lqt_batch(self.B, ct.cast(arr, ct.POINTER(lqt_problem)), ct.cast(x0s, ct.POINTER(ct.c_void_p)))
        L = _abi.lib()
        self.total = int(L.lqt_batch_boundaries(ct.byref(self.struct)))
        nbytes = int(L.lqt_batch_workspace_size(ct.byref(self.struct)))
        if nbytes == 0 or self.total == 0:
            raise _abi.LQTError(_abi.LQT_EINVAL, "lqt_batch_workspace_size")
        self.offsets = np.concatenate([[0], np.cumsum(self.T + 1)])
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        _abi.check(L.lqt_batch_plan(ct.byref(self.struct), self.ws.data_ptr(), self.ws.numel(),
                                    torch.cuda.current_stream(self.device).cuda_stream), "lqt_batch_plan")
        self.chunk = 0
        self.flags = 0

    def set_invariant_build(self, on: bool = True):
        """Use the time-invariant element build (every problem of a batch has
        constant F, L, U, X; each needs sub-intervals of one length)."""
        self.flags = _abi.LQT_TUNE_INVARIANT_BUILD if on else 0

    def new_outputs(self):
        n, m, N = self.n, self.m, self.total
        e = lambda *s: torch.empty(*s, dtype=torch.float64, device=self.device)
        return {"S": e(N, n, n), "v": e(N, n), "zeta": e(N), "x": e(N, n), "u": e(N, m), "cost": e(self.B)}

    def solve(self, out=None, chunk=None, stream=None) -> dict:
        out = self.new_outputs() if out is None else out
        tune = lqt_tuning(self.chunk if chunk is None else chunk, self.flags)
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        _abi.check(_abi.lib().lqt_solve_batched(
            ct.byref(self.struct), ct.byref(tune), out["S"].data_ptr(), out["v"].data_ptr(), out["zeta"].data_ptr(),
            out["x"].data_ptr(), out["u"].data_ptr(), out["cost"].data_ptr(), self.ws.data_ptr(), self.ws.numel(),
            st.cuda_stream), "lqt_solve_batched")
        return out

    def problem_slice(self, out, b):
        lo, hi = int(self.offsets[b]), int(self.offsets[b + 1])
        return {k: (v[lo:hi] if k != "cost" else v[b]) for k, v in out.items()}

    def autotune(self, candidates=(0, 2, 4, 8, 16, 32), reps: int = 3) -> int:
        """Times the batched solve for each first-level chunk length (one
        untimed run, then `reps` runs each timed with CUDA events, the median
        kept) and keeps the fastest; cached per state dimension, problem
        count, total boundaries and build flags.  The timing table is
        `tuning_table()[key][1]`."""
        key = (self.n, self.B, self.total, self.flags)
        if key in _TUNED:
            self.chunk = _TUNED[key][0]
            return self.chunk
        out = self.new_outputs()
        timings = {}
        for c in candidates:
            self.solve(out, chunk=c)
            runs = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                self.solve(out, chunk=c)
                e1.record()
                torch.cuda.synchronize()
                runs.append(e0.elapsed_time(e1))
            timings[c] = float(np.median(runs))
        best = min(timings, key=timings.get)
        _TUNED[key] = (best, timings)
        self.chunk = best
        return best

    def tuned_timings(self) -> dict:
        """The autotuner's median time (ms) per candidate chunk, if tuned."""
        entry = _TUNED.get((self.n, self.B, self.total, self.flags))
        return dict(entry[1]) if entry else {}

    @staticmethod
    def tuning_table():
        return dict(_TUNED)


class BatchSet:
    """Problems of several state dimensions: one Batch per dimension, solved on
    one stream each (forked from and joined back into the caller's stream), so
    that one dimension's short upper scan levels overlap the others' work;
    capture() records the whole set as one CUDA graph."""

    def __init__(self, problems, device: str = "cuda"):
        if not problems:
            raise ValueError("empty batch")
        self.device = torch.device(device)
        idx = {}
        for i, p in enumerate(problems):
            idx.setdefault(p.n, []).append(i)
        self.index = {n: v for n, v in sorted(idx.items())}
        self.batches = {n: Batch([problems[i] for i in v], device) for n, v in self.index.items()}
        self.streams = {n: torch.cuda.Stream(self.device) for n in self.batches}

    def set_invariant_build(self, on: bool = True):
        for b in self.batches.values():
            b.set_invariant_build(on)

    def autotune(self, candidates=None, reps: int = 3) -> dict:
        """Each dimension's first-level chunk (Batch.autotune); `candidates`
        maps a dimension to its candidate list (None: Batch's default)."""
        out = {}
        for n, b in self.batches.items():
            c = candidates(n) if callable(candidates) else candidates
            out[n] = b.autotune(reps=reps) if c is None else b.autotune(candidates=c, reps=reps)
        return out

    def new_outputs(self) -> dict:
        return {n: b.new_outputs() for n, b in self.batches.items()}

    def solve(self, out=None, stream=None) -> dict:
        out = self.new_outputs() if out is None else out
        main = torch.cuda.current_stream(self.device) if stream is None else stream
        for n, b in self.batches.items():
            s = self.streams[n]
            s.wait_stream(main)
            b.solve(out=out[n], stream=s)
        for s in self.streams.values():
            main.wait_stream(s)
        return out

    def capture(self, out=None, stream=None):
        """Records solve() as one CUDA graph (run solve() once before, so that
        nothing is first touched inside the capture); returns the graph."""
        out = self.new_outputs() if out is None else out
        main = torch.cuda.Stream(self.device) if stream is None else stream
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(main):
            with torch.cuda.graph(g, stream=main):
                self.solve(out, stream=main)
        return g

    def problem_slice(self, out, i):
        """Problem i (position in the constructor's list) of the outputs."""
        for n, v in self.index.items():
            if i in v:
                return self.batches[n].problem_slice(out[n], v.index(i))
        raise IndexError(i)
