"""Plants plausible mistakes in copies of the oracle and checks that the pins fail.

Each mutant changes one line of oracle/vdi_oracle.c (a flipped comparison, a
dropped factor, a swapped index ...), is compiled to a temporary library, and the
pin and invariant suites are run against it in a subprocess.  A mutant that
survives means the pins do not constrain that part of the oracle.
"""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vdi_oracle.c")

# (name, original text, mutated text)
MUTANTS = [
    ("criterion strict >", "if (d >= gamma && count < cap)", "if (d > gamma && count < cap)"),
    ("no length renormalisation", "double at = -expm1(r * L);", "double at = -expm1(L);"),
    ("over drops transmittance", "A += T * p->a;", "A += p->a;"),
    ("optical depth sign", "L += log1p(-p->a);", "L -= log1p(-p->a);"),
    ("bisection ends swapped", "hi = mid;\n            if (c == n_s) break;", "lo = mid;\n            if (c == n_s) break;"),
    ("no early exit", "if (c == n_s) break;", "if (c == -1) break;"),
    ("gamma=0 test skipped", "if (c0 <= n_s) {", "if (c0 < 0) {"),
    ("mixture colour not normalised", "p->P[c] = (MC[c] / M) * a;", "p->P[c] = MC[c] * a;"),
    ("Eq.2 drops interval length", "double a = -expm1(-M * dt);", "double a = -expm1(-M);"),
    ("opaque overlap ignored", "if (nopaque > 0) {", "if (nopaque > 99) {"),
    ("gap not transparent", "if (nact == 0) continue; /* transparent gap */", "if (nact == 0) { p->a = 0.1; continue; }"),
    ("lut lerp wrong entry", "lutc[4 * (i + 1) + c] * w", "lutc[4 * i + c] * w"),
    ("lut correction inverted", "step / ref_len);", "ref_len / step);"),
    ("trilinear weight swapped", "(dx ? w[0] : 1 - w[0])", "(dx ? 1 - w[0] : w[0])"),
    ("trilinear y/z swapped", "(dy ? w[1] : 1 - w[1]) * (dz ? w[2] : 1 - w[2])", "(dy ? w[2] : 1 - w[2]) * (dz ? w[1] : 1 - w[1])"),
    ("image y flipped", "double y = (1.0 - 2.0 * (j + 0.5) / c->height) * th;", "double y = (2.0 * (j + 0.5) / c->height - 1.0) * th;"),
    ("aspect dropped", "* th * (double)c->width / (double)c->height;", "* th;"),
    ("sample at front not midpoint", "double tm = tin + ((double)kk + 0.5) * step;\n        if (!(tm < tout)) break;\n        if (n >= max_s)", "double tm = tin + ((double)kk) * step;\n        if (!(tm < tout)) break;\n        if (n >= max_s)"),
    ("domain exit ignored", "if (p->brk) { /* sec. 5.3", "if (0) { /* sec. 5.3"),
    ("re-entry held to the budget", "if (p->a > 0.0) OPEN(p);\n            continue;",
     "if (p->a > 0.0 && count < cap) OPEN(p);\n            continue;"),
    ("back depth includes gaps", "if (p->a > 0.0) bt = p->b;", "bt = p->b;"),
    ("cap off by one", "if (d >= gamma && count < cap)", "if (d >= gamma && count <= cap)"),
    ("ownership closed box", "c[0] >= bx->lo[0] && c[0] < bx->hi[0]", "c[0] >= bx->lo[0] && c[0] <= bx->hi[0]"),
    ("inclusive scan", "offsets[i] = acc;\n        acc += (uint64_t)counts[i];", "acc += (uint64_t)counts[i];\n        offsets[i] = acc;"),
    ("un-premultiply skipped", "cs[c] = A > 0.0 ? P[c] / A : 0.0;", "cs[c] = P[c];"),
    ("half exponent bias", "else v = ldexp((double)(1024 + m), e - 25);", "else v = ldexp((double)(1024 + m), e - 24);"),
    ("render falling branch in list order", "const int k = rising ? t : n - 1 - t;", "const int k = t;"),
    ("render opacity ignores thickness", "log1p(-Ar) * l / (b - f)", "log1p(-Ar) * l"),
    ("render rows offset", "const double Yj = (1.0 - 2.0 * j / G.H) * G.th;",
     "const double Yj = (1.0 - 2.0 * (j + 0.5) / G.H) * G.th;"),
    ("render colour premultiplied twice", "(r[2 + c] / Ar) * alpha", "r[2 + c] * alpha"),
    ("render no split at closest approach", "if (s_star > s_in && s_star < s_out) cut[nc++] = s_star;",
     "if (0) cut[nc++] = s_star;"),
    ("split not near-equal", "boxes[e].hi[a] = (int)(((long)cells * (idx[a] + 1)) / g[a]);", "boxes[e].hi[a] = idx[a] + 1 == g[a] ? cells : boxes[e].lo[a] + cells / g[a] - (idx[a] == 0);"),
]


def _run(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutant '{name}': pattern not found"
    mut = src.replace(old, new, 1)
    path_c = os.path.join(tmp, f"m{abs(hash(name))}.c")
    path_so = path_c[:-2] + ".so"
    open(path_c, "w").write(mut)
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", path_so, path_c, "-lm"])
    env = dict(os.environ, VDI_ORACLE_LIB=path_so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_invariants.py"),
                        os.path.join(ROOT, "tests", "test_oracle_render.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode


def test_every_planted_mistake_is_caught():
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=max(2, (os.cpu_count() or 4) // 2)) as ex:
            results = list(ex.map(lambda m: _run(*m, tmp), MUTANTS))
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"mutants not caught by the pins: {survivors}"
