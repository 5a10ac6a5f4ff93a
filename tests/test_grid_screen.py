"""The FP32 screen of the grid min-plus kernel, emulated on the CPU: the
argument that it never drops a candidate whose FP64 sum is the minimum.

For every candidate k the kernel forms, in float arithmetic, a bracket
lo_k <= g_k + f_k <= hi_k from the operands truncated to float (bit
truncation toward zero; magnitudes below 2^-126 become 0), with
hi/lo = s_k +/- c t_k (- d), s_k = a_k + b_k, t_k = |a_k| + |b_k|,
c = 2^-20, d = 2^-100, then keeps the k with lo_k <= min_j hi_j (+ d, rounded
up).  The FP64 minimum with the lowest-index tie rule is taken over the kept
k only.  This test emulates that bracket with numpy float32 (the fused
multiply-add through float64, one rounding) and checks, on adversarial rows,
that every k whose FP64 sum equals the FP64 minimum is kept.
"""
import numpy as np

C = np.float32(2.0 ** -20)
D = np.float32(2.0 ** -100)


def truncate_to_float(x):
    b = np.frombuffer(np.ascontiguousarray(x, dtype=np.float64).tobytes(), dtype=np.uint64).copy()
    eb = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    sign = b >> np.uint64(63)
    mant = (b >> np.uint64(29)) & np.uint64(0x7FFFFF)
    fb = (sign << np.uint64(31)) | (np.clip(eb - 1023 + 127, 0, 255).astype(np.uint64) << np.uint64(23)) | mant
    f = np.frombuffer(fb.astype(np.uint32).tobytes(), dtype=np.float32).copy()
    f[eb < 1023 - 126] = 0.0
    return f


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def survivors(g, f):
    a, b = truncate_to_float(g), truncate_to_float(f)
    s = (a + b).astype(np.float32)
    t = (np.abs(a) + np.abs(b)).astype(np.float32)
    hi = fma32(np.full_like(s, C), t, s)
    lo = fma32(np.full_like(s, -C), t, s)
    u = np.nextafter(np.float32(np.float64(hi.min()) + np.float64(D)), np.float32(np.inf))
    return np.nonzero(lo <= u)[0]


def rows(rng, trials):
    for trial in range(trials):
        G = int(rng.integers(3, 80))
        kind = trial % 5
        if kind == 0:
            yield rng.standard_normal(G), rng.standard_normal(G)
        elif kind == 1:  # ties and near-ties in the last bits
            base = rng.uniform(1, 10)
            yield (base + rng.integers(-3, 3, G) * np.spacing(base) * rng.integers(0, 2),
                   np.full(G, 1.0) + rng.integers(0, 2, G) * 2e-16)
        elif kind == 2:  # smooth bowls, as the value functions are
            x = np.linspace(-6, 6, G)
            yield ((x - rng.uniform(-2, 2)) ** 2 * rng.uniform(0.1, 3),
                   (x - rng.uniform(-2, 2)) ** 2 * rng.uniform(0.1, 3))
        elif kind == 3:  # near the float underflow
            yield rng.standard_normal(G) * 1e-38, rng.standard_normal(G) * 1e-39
        else:  # cancellation between operands near the screen's range limit
            g = rng.uniform(-1e29, 1e29, G)
            yield g, -g + rng.standard_normal(G)


def test_screen_keeps_every_fp64_minimiser():
    rng = np.random.default_rng(20)
    for g, f in rows(rng, 5000):
        sums = g + f
        ties = np.nonzero(sums == sums.min())[0]
        kept = set(survivors(g, f).tolist())
        assert set(ties.tolist()) <= kept, (g, f)


def test_screen_is_tight_on_smooth_rows():
    """On smooth bowls (the common case) the screen keeps very few candidates,
    which is what makes it pay."""
    rng = np.random.default_rng(21)
    counts = []
    for _ in range(500):
        G = 60
        x = np.linspace(-6, 6, G)
        g = (x - rng.uniform(-2, 2)) ** 2 * rng.uniform(0.1, 3) + rng.uniform(0, 5)
        f = (x - rng.uniform(-2, 2)) ** 2 * rng.uniform(0.1, 3)
        counts.append(len(survivors(g, f)))
    assert max(counts) <= 4 and np.mean(counts) < 1.5, (max(counts), np.mean(counts))
