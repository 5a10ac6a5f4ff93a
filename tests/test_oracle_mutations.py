"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a copy of oracle/lqt_oracle.c (a dropped
term, a flipped sign, a transposed operand, a wrong index or weight), compiles
the copy, and runs every pin of test_oracle_pins.py, test_oracle_densify.py,
test_oracle_method2.py and test_oracle_grid.py against it.  At least one
pin has to fail for every mutant; otherwise the pins would also have let that
mistake through in the real oracle.  Nothing here touches the GPU.
"""
import inspect
import itertools
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_densify as densify_pins
from tests import test_oracle_grid as grid_pins
from tests import test_oracle_method2 as method2_pins
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "lqt_oracle.c")

# (name, text in lqt_oracle.c, replacement, which occurrence (0 = first))
MUTATIONS = [
    # element right-hand side (Theorem "Backward_HJB_LQT")
    ("dA: sign of A F", "d.A[i] = M1[i] - M2[i];", "d.A[i] = M1[i] + M2[i];", 0),
    ("db: dropped A c", "acc += s.A[i * n + k] * (Beta[k] + cf->c[k]);", "acc += s.A[i * n + k] * Beta[k];", 0),
    ("dC: sign", "d.C[i] = -M2[i];", "d.C[i] = M2[i];", 0),
    ("deta: dropped J c", "for (int k = 0; k < n; ++k) acc += s.J[i * n + k] * cf->c[k];", "", 0),
    ("deta: F not transposed", "acc -= cf->F[k * n + i] * s.eta[k];", "acc -= cf->F[i * n + k] * s.eta[k];", 0),
    ("dJ: dropped J B J", "- JF[j * n + i] + JBJ[i * n + j];", "- JF[j * n + i];", 0),
    ("dzeta: factor on eta B eta", "z += 0.5 * s.eta[i] * Beta[i] + s.eta[i] * cf->c[i];",
     "z += s.eta[i] * Beta[i] + s.eta[i] * cf->c[i];", 0),
    ("dzeta: dropped r X r", "double z = -0.5 * cf->rho;\n  for (int i = 0; i < n; ++i) z += 0.5 * s.eta",
     "double z = 0.0;\n  for (int i = 0; i < n; ++i) z += 0.5 * s.eta", 0),
    # RK4 of the elements
    ("RK4: k3 weight", "acc[q] += 2.0 * k[q]; yt[q] = y[q] - h * k[q];", "acc[q] += k[q]; yt[q] = y[q] - h * k[q];", 0),
    ("RK4: k1 sample index", "bad |= coefs_eval(P, j, 2 * i + 2, &cf);\n    element_rhs(n, &cf, y, k, tmp);",
     "bad |= coefs_eval(P, j, 2 * i, &cf);\n    element_rhs(n, &cf, y, k, tmp);", 0),
    ("RK4: boundary A = 0", "eye(n, view(n, y).A);", "", 0),
    # coefficients
    ("rho doubled", "rho += cf->r[i] * Xr[i];", "rho += 2.0 * cf->r[i] * Xr[i];", 0),
    ("q = X r without H", "mtm(n, nr, 1, cf->H, Xr, cf->q);", "memcpy(cf->q, Xr, sizeof(double) * n);", 0),
    # terminal element (eq. LQT_final_initialisation)
    ("terminal zeta factor", "*v.zeta = 0.5 * z;", "*v.zeta = z;", 0),
    ("terminal eta sign", "mtm(n, nr, 1, Hf, Xr, v.eta);",
     "mtm(n, nr, 1, Hf, Xr, v.eta); for (int i = 0; i < n; ++i) v.eta[i] = -v.eta[i];", 0),
    # combination (Lemma LQT_combination)
    ("combine A: A1 for A2", "mm(n, n, n, c.A, MA1, o.A);", "mm(n, n, n, a.A, MA1, o.A);", 0),
    ("combine b: dropped C1 eta2", "rhs[i] = a.b[i] + tv[i];", "rhs[i] = a.b[i];", 0),
    ("combine C: A2 not transposed", "mmt(n, n, n, T1, c.A, T2);", "mm(n, n, n, T1, c.A, T2);", 0),
    ("combine eta: sign of J2 b1", "w[i] = c.eta[i] - tv[i];", "w[i] = c.eta[i] + tv[i];", 0),
    ("combine J: M for M^T", "mm(n, n, n, Mt, J2A1, MtJ2A1);", "mm(n, n, n, Minv, J2A1, MtJ2A1);", 0),
    ("combine zeta: sign of z0 eta2", "- z0[i] * c.eta[i];", "+ z0[i] * c.eta[i];", 0),
    ("combine zeta: dropped lambda term", "z += 0.5 * lam[i] * tv2[i] + ", "z += ", 0),
    ("combine M: C1 J2 order", "mm(n, n, n, a.C, c.J, W);", "mm(n, n, n, c.J, a.C, W);", 0),
    # fold order (Theorem "parallel_HJB")
    ("fold: operands swapped", "orc_combine(n, elems + (size_t)(k - 1) * es, s, nxt)",
     "orc_combine(n, s, elems + (size_t)(k - 1) * es, nxt)", 0),
    # linear solve
    ("back substitution sign", "s -= W[k * n + l] * Bs[l * q + j];", "s += W[k * n + l] * Bs[l * q + j];", 0),
    # trajectory (Method 2) and controls
    ("trajectory: C S order", "mm(n, n, n, e.C, S1, W);", "mm(n, n, n, S1, e.C, W);", 0),
    ("trajectory: dropped C v", "rhs[i] += e.b[i] + tv[i];", "rhs[i] += e.b[i];", 0),
    ("control: sign of v - S x", "Sx[k] = v[k] - Sx[k];", "Sx[k] = Sx[k] - v[k];", 0),
    ("cost: factor of x S x", "c += 0.5 * x0[i] * sx - v[i] * x0[i];", "c += x0[i] * sx - v[i] * x0[i];", 0),
    # O2 (sequential method)
    ("riccati: dropped S B S", "- cf->Q[i * n + j] + SBS[i * n + j];", "- cf->Q[i * n + j];", 0),
    ("riccati: sign of S c", "acc += S[i * n + k] * cf->c[k];", "acc -= S[i * n + k] * cf->c[k];", 0),
    ("closed loop: sign of u", "u[i] = -acc;", "u[i] = acc;", 0),
    ("closed loop: dropped c", "double acc = cf->c[i];\n    for (int k = 0; k < n; ++k) acc += cf->F[i * n + k] * x[k];",
     "double acc = 0.0;\n    for (int k = 0; k < n; ++k) acc += cf->F[i * n + k] * x[k];", 0),
    ("O2 cost: factor of x S x", "c += 0.5 * x0[i] * sx - v[i] * x0[i];", "c += x0[i] * sx - v[i] * x0[i];", 1),
    ("O2 RK4: k3 weight", "acc[q] += 2.0 * k[q]; yt[q] = y[q] - h * k[q];", "acc[q] += k[q]; yt[q] = y[q] - h * k[q];", 1),
    ("O2 Hermite midpoint: slope term sign", "h * (d0[q] - d1[q]) / 8.0", "h * (d1[q] - d0[q]) / 8.0", 0),
    ("O2 forward: midpoint stage from the end point", "closed_loop_rhs(n, m, &cf, ym, ym + nn, xt, kx, t2);\n      for (int q = 0; q < n; ++q) { ax[q] += 2.0 * kx[q]; xt[q] = xv[q] + h * kx[q]; }",
     "closed_loop_rhs(n, m, &cf, y1, y1 + nn, xt, kx, t2);\n      for (int q = 0; q < n; ++q) { ax[q] += 2.0 * kx[q]; xt[q] = xv[q] + h * kx[q]; }", 0),
    # within-block densification
    ("densify: Hermite slope sign", "h * (d0[q] - d1[q]) / 8.0", "h * (d1[q] - d0[q]) / 8.0", 1),
    ("densify: k3 weight", "acc[q] += 2.0 * k[q]; yt[q] = y[q] - h * k[q];", "acc[q] += k[q]; yt[q] = y[q] - h * k[q];", 2),
    ("densify: block-start slope sample", "bad |= coefs_eval(P, j, 0, &cf);\n    riccati_rhs(n, &cf, Y, D, tmp);",
     "bad |= coefs_eval(P, j, 1, &cf);\n    riccati_rhs(n, &cf, Y, D, tmp);", 0),
    ("densify: control sample", "bad |= coefs_eval(P, j, 2 * i, &cf);\n      mm(n, n, 1, Sd",
     "bad |= coefs_eval(P, j, 0, &cf);\n      mm(n, n, 1, Sd", 0),
    # Method 2: forward-HJB elements, prefix fold, states
    ("forward dA: sign of F A", "for (int i = 0; i < n * n; ++i) d.A[i] = M2[i] - M1[i];",
     "for (int i = 0; i < n * n; ++i) d.A[i] = -M2[i] - M1[i];", 0),
    ("forward db: dropped c", "double acc = cf->c[i];\n    for (int k = 0; k < n; ++k) acc += s.C[i * n + k] * cf->q[k]",
     "double acc = 0.0;\n    for (int k = 0; k < n; ++k) acc += s.C[i * n + k] * cf->q[k]", 0),
    ("forward dC: dropped B", "-M1[i * n + j] + cf->B[i * n + j] + M2[i * n + j]", "-M1[i * n + j] + M2[i * n + j]", 0),
    ("forward deta: sign of Q b", "for (int k = 0; k < n; ++k) acc -= cf->Q[i * n + k] * s.b[k];\n    w[i] = acc;",
     "for (int k = 0; k < n; ++k) acc += cf->Q[i * n + k] * s.b[k];\n    w[i] = acc;", 0),
    ("forward dzeta: factor of b Q b", "z += -s.b[i] * cf->q[i] + 0.5 * s.b[i] * Qb;", "z += -s.b[i] * cf->q[i] + s.b[i] * Qb;", 0),
    ("forward RK4: k4 sample", "bad |= coefs_eval(P, j, 2 * i + 2, &cf);\n    forward_rhs",
     "bad |= coefs_eval(P, j, 2 * i + 1, &cf);\n    forward_rhs", 0),
    ("prefix: operands swapped", "orc_combine(n, prefixes + (size_t)k * es, elems + (size_t)k * es,",
     "orc_combine(n, elems + (size_t)k * es, prefixes + (size_t)k * es,", 0),
    ("method 2: dropped C v", "for (int i = 0; i < n; ++i) rhs[i] += pk.b[i] + tv[i];",
     "for (int i = 0; i < n; ++i) rhs[i] += pk.b[i];", 0),
    # grid method (Sec. VI-B, App. E)
    ("grid: interpolation correction sign", "return best - b * b / (4.0 * a);", "return best + b * b / (4.0 * a);", 0),
    ("grid: curvature factor", "double ag = (gp + gm - 2.0 * g0) / (2.0 * dx * dx)", "double ag = (gp + gm - 2.0 * g0) / (dx * dx)", 0),
    ("grid: slope factor", "bg = (gp - gm) / (2.0 * dx);", "bg = (gp - gm) / dx;", 0),
    ("grid: one-step control", "double u = (xj - xi) / dt - drift;", "double u = (xj - xi) / dt + drift;", 0),
    ("grid: one-step cost factor", "C[(size_t)i * G + j] = dt * 0.5 * (P->q * xi * xi + P->rho * u * u);",
     "C[(size_t)i * G + j] = dt * (P->q * xi * xi + P->rho * u * u);", 0),
    ("grid: terminal factor", "phi[i] = 0.5 * P->qf * x * x;", "phi[i] = P->qf * x * x;", 0),
    ("grid: block substeps", "for (int m = 1; m < P->substeps; ++m) {", "for (int m = 2; m < P->substeps; ++m) {", 0),
    ("grid: doubling skips a power", "if (e & (1L << l)) {", "if (l > 0 && (e & (1L << l))) {", 0),
    ("grid: ties to the highest index", "if (v < best) { best = v; bi = j; }", "if (v <= best) { best = v; bi = j; }",
     0),
    # shared small linear algebra
    ("mtm: operand not transposed", "for (int l = 0; l < k; ++l) s += a[l * p + i] * b[l * q + j];",
     "for (int l = 0; l < k; ++l) s += a[i * k + l] * b[l * q + j];", 0),
]


def _replace_nth(text, old, new, nth):
    start = -1
    for _ in range(nth + 1):
        start = text.find(old, start + 1)
        assert start >= 0, f"mutation anchor not found: {old!r}"
    return text[:start] + new + text[start + len(old):]


def _pin_calls():
    """Every (name, zero-argument callable) for the pins, parametrisations expanded."""
    calls = []
    mods = (pins, densify_pins, method2_pins, grid_pins)
    members = [m for mod in mods for m in inspect.getmembers(mod, inspect.isfunction)]
    for name, fn in members:
        if not name.startswith("test_") or fn.__module__ not in tuple(mod.__name__ for mod in mods):
            continue
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        if not params:
            calls.append((name, fn, {}))
            continue
        names_vals = []
        for m in params:
            argnames = [a.strip() for a in m.args[0].split(",")] if isinstance(m.args[0], str) else list(m.args[0])
            vals = [v if len(argnames) > 1 else (v,) for v in m.args[1]]
            names_vals.append((argnames, vals))
        for combo in itertools.product(*[nv[1] for nv in names_vals]):
            kw = {}
            for (argnames, _), vals in zip(names_vals, combo):
                kw.update(dict(zip(argnames, vals)))
            calls.append((f"{name}{kw}", fn, kw))
    return calls


# cheapest pins first, so that a mutant is usually caught within a second
_SLOW_LAST = ("test_time_varying_against_adaptive_reference", "test_grid_dynamic_programming_1d")


def _caught(lib_path, stop_at_first=False):
    """Names of the pins that fail with the oracle library at lib_path."""
    calls = sorted(_pin_calls(), key=lambda c: any(c[0].startswith(s) for s in _SLOW_LAST))
    failed = []
    with oracle.swapped_library(lib_path):
        for name, fn, kw in calls:
            try:
                fn(**kw)
            except Exception:  # an assertion, a FloatingPointError, a NaN comparison ...
                failed.append(name)
                if stop_at_first:
                    break
    return failed


def test_mutation_anchors_are_unique_enough():
    text = open(SRC).read()
    for name, old, new, nth in MUTATIONS:
        assert text.count(old) >= nth + 1, name


def test_unmutated_copy_passes_every_pin(tmp_path):
    lib = tmp_path / "liblqt_oracle_copy.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(lib), SRC, "-lm"])
    assert _caught(str(lib)) == []


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(case, tmp_path):
    name, old, new, nth = case
    src = tmp_path / "lqt_oracle_mutant.c"
    src.write_text(_replace_nth(open(SRC).read(), old, new, nth))
    lib = tmp_path / "liblqt_oracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(lib), str(src), "-lm"])
    failed = _caught(str(lib), stop_at_first=True)
    assert failed, f"no pin catches the planted mistake '{name}'"
