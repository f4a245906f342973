"""The oracle's pins catch plausible mistakes (no GPU).

Each mutant plants one mistake -- a dropped term, a wrong sign, index or
operand, a missing bound, a reversed tie rule -- in a COPY of the oracle, and
the pin suites (test_oracle_pins, test_oracle_build_pins,
test_oracle_mlp_pins, test_bvh_dump) run against that copy in a child
process: every mutant must make them fail, and the unmodified copy must
pass.  The oracle in the repository is never modified.

Left out on purpose: the merge distance of crossing points on ambiguous
rays (no rule in the paper; parity unpinned) and rewrites that cannot change
a result (a loop bound the loop never reaches; the network's padding rows,
which only ever multiply zero inputs).
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_build_pins.py",
        "tests/test_oracle_mlp_pins.py", "tests/test_bvh_dump.py"]
C, M = "oracle/rsi_oracle.c", "oracle/mlp.py"
SCRATCH = os.path.join(ROOT, "tests", ".mutants")     # copies live here while they run

# (name, file, text in the oracle, mistaken replacement)
MUTANTS = [
    # Moller-Trumbore quantities (Sec. 1)
    ("q operands transposed", C, "vec3 q = v_cross(sv, e1);", "vec3 q = v_cross(e1, sv);"),
    ("u from the direction", C, "u = v_dot(sv, p) / det;", "u = v_dot(d, p) / det;"),
    ("w drops v", C, "w = 1.0 - u - v;", "w = 1.0 - u;"),
    ("e2 from vertex b", C, "e2 = v_sub(c, a);", "e2 = v_sub(c, b);"),
    ("zero-length segment not rejected", C, "if ((d.x == 0.0 && d.y == 0.0 && d.z == 0.0) ||\n        (n.x",
     "if ((n.x"),
    # margin classification
    ("decisive hit ignores t < 1", C, "t > tau && t < 1.0 - tau)", "t > tau)"),
    ("decisive hit ignores w", C, "u > tau && v > tau && w > tau &&", "u > tau && v > tau &&"),
    ("decisive miss ignores t > 1", C, " || t > 1.0 + tau)", ")"),
    ("decisive miss ignores w", C, "v < -tau || w < -tau ||", "v < -tau ||"),
    ("inclusive ignores t <= 1", C, "t >= 0.0 && t <= 1.0);", "t >= 0.0);"),
    ("det_rel drops |d|", C, "det / (v_norm(d) * v_norm(e1) * v_norm(e2));",
     "det / (v_norm(e1) * v_norm(e2));"),
    # nearly-parallel branch
    ("parallel band absolute", C, "dist > tau * v_norm(d) ?", "dist > tau ?"),
    ("parallel crossing not zero", C, "if (incl) {\n                dist = 0.0;", "if (0) {\n                dist = 0.0;"),
    ("parallel skips edge c-a", C,
     "dd = segment_segment_distance(s, e, c, a); if (dd < dist) dist = dd;", ""),
    ("point-triangle drops |n|", C, "return fabs(h) * sqrt(nn);", "return fabs(h);"),
    ("segment-segment sign", C, "double t = (a * e - b * dd) / den;", "double t = (a * e + b * dd) / den;"),
    # per-ray aggregation and the three result forms
    ("boolean ambiguity ignores a decisive hit", C, "int amb_hit = (n_hit == 0) && (n_amb > 0);",
     "int amb_hit = (n_amb > 0);"),
    ("no de-duplication", C, "ts[k] - ts[k - 1] > ORACLE_TMERGE", "1"),
    ("ambiguous count from decisive hits", C, "if (!amb_count) {", "if (1) {"),
    ("nearest tie to the higher index", C, "if (out[2] < best_t)", "if (out[2] <= best_t)"),
    ("distance is t", C, "(float)(best_t * v_norm(dv))", "(float)(best_t)"),
    ("point drops the start", C, "vec3 pt = v_add(sv, v_scale(dv, best_t));", "vec3 pt = v_scale(dv, best_t);"),
    # build (Sec. 3.2, 3.3, 4.1, 4.2)
    ("extent max starts at 0", C, "hi[a] = -INFINITY; }", "hi[a] = 0.0f; }"),
    ("extent max only if not min", C, "if (x > hi[a]) hi[a] = x;", "else if (x > hi[a]) hi[a] = x;"),
    ("Morton x as the high bit", C, "<< (3 * i + a);", "<< (3 * i + (2 - a));"),
    ("Morton scale 2^b - 1", C, "const float scale = (float)(1u << b);",
     "const float scale = (float)((1u << b) - 1u);"),
    ("Morton drops the low corner", C, "u = (c - lo[a]) / (hi[a] - lo[a]);", "u = c / (hi[a] - lo[a]);"),
    ("centroid drops a vertex", C, "+ V[3 * (int64_t)i2 + a]) / 3.0f;", ") / 3.0f;"),
    ("Morton no clamp to 2^b - 1", C, "q[a] = qq > qmax ? qmax : qq;", "q[a] = qq;"),
    ("sort ties reversed", C, "return (a->id > b->id) - (a->id < b->id);",
     "return (a->id < b->id) - (a->id > b->id);"),
    ("equal keys split at the middle", C,
     "while (g + 1 <= b && (((uint64_t)(g + 1) >> p) & 1u) == 0) ++g;\n    return g;",
     "g = (a + b) / 2; (void)p;\n    return g;"),
    ("leaf parent in the internal slot", C, "parent[n - 1 + g] = (int32_t)node;", "parent[g] = (int32_t)node;"),
    ("refit max as min", C, "bx[3 + a] = bl[3 + a] > br[3 + a] ? bl[3 + a] : br[3 + a];",
     "bx[3 + a] = bl[3 + a] < br[3 + a] ? bl[3 + a] : br[3 + a];"),
    ("refit min from the left child", C, "bx[a] = bl[a] < br[a] ? bl[a] : br[a];", "bx[a] = bl[a];"),
    ("leaf box ignores the order", C, "const int32_t* tri = T + 3 * (int64_t)perm[j];",
     "const int32_t* tri = T + 3 * j;"),
    ("leaf box drops a vertex", C, "float mn = x0 < x1 ? x0 : x1; mn = mn < x2 ? mn : x2;",
     "float mn = x0 < x1 ? x0 : x1;"),
    ("height of the left subtree", C, "return 1 + (hl > hr ? hl : hr);", "return 1 + hl;"),
    # proposal network reference
    ("bf16 keeps 7 bits", M, "np.round(m * 256.0), e - 8", "np.round(m * 128.0), e - 7"),
    ("bf16 truncates", M, "np.round(m * 256.0)", "np.trunc(m * 256.0)"),
    ("gelu scale", M, "return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))",
     "return 0.5 * z * (1.0 + np.tanh(0.5 * (z + GELU_A * z ** 3)))"),
    ("gelu drops the cubic term", M, "return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))",
     "return 0.5 * z * (1.0 + np.tanh(GELU_C * z))"),
    ("gelu gradient drops the tanh slope", M, "+ 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)", ""),
    ("gelu gradient drops the cubic slope", M, "* GELU_C * (1.0 + 3.0 * GELU_A * z * z)", "* GELU_C"),
    ("features not centred", M, "f = np.clip(2.0 * f - 1.0, -4.0, 4.0)", "f = np.clip(f, -4.0, 4.0)"),
    ("forward drops a bias", M, 'z2 = a1 @ W2 + p["b2"]', "z2 = a1 @ W2"),
    ("forward keeps a hidden layer unrounded", M, "a1 = bf16_round(gelu(z1))", "a1 = gelu(z1)"),
    ("loss gradient sign", M, "dz3 = (1.0 / (1.0 + np.exp(-logits)) - y)", "dz3 = (y - 1.0 / (1.0 + np.exp(-logits)))"),
    ("backward skips a transpose", M, 'da1 = dz2 @ cache["W2"].T', 'da1 = dz2 @ cache["W2"]'),
    ("Adam first moment undamped", M, "m[...] = b1 * m + (1 - b1) * g[k]", "m[...] = b1 * m + g[k]"),
    ("Adam bias correction frozen", M, "mh = m / (1 - b1 ** t)", "mh = m / (1 - b1)"),
    ("top-4 ties to the higher index", M, 'np.argsort(-logits, axis=1, kind="stable")',
     'np.argsort(logits, axis=1, kind="stable")[:, ::-1]'),
    # more bounds, distance helpers, tree indices, network backward and optimiser
    ("inclusive drops w", C, "incl = (u >= 0.0 && v >= 0.0 && w >= 0.0 &&", "incl = (u >= 0.0 && v >= 0.0 &&"),
    ("inclusive drops t >= 0", C, "&& t >= 0.0 && t <= 1.0);", "&& t <= 1.0);"),
    ("decisive miss ignores t < -tau", C, "w < -tau || t < -tau ||", "w < -tau ||"),
    ("decisive hit ignores t > tau", C, "w > tau && t > tau && t < 1.0 - tau)", "w > tau && t < 1.0 - tau)"),
    ("parallel skips edge a-b", C, "dd = segment_segment_distance(s, e, a, b); if (dd < dist) dist = dd;", ""),
    ("point-triangle inside test drops a side", C, "if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) return",
     "if (s0 >= 0.0 && s1 >= 0.0) return"),
    ("point-segment unclamped", C, "clamp01(v_dot(v_sub(p, a), ab) / len2)", "(v_dot(v_sub(p, a), ab) / len2)"),
    ("segment-segment interior ignores s", C, "if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {",
     "if (t >= 0.0 && t <= 1.0) {"),
    ("Morton drops the top bit", C, "for (int i = 0; i < b; ++i)", "for (int i = 0; i < b - 1; ++i)"),
    ("left child's parent slot", C, "left[node] = (int32_t)g;\n        parent[g] = (int32_t)node;",
     "left[node] = (int32_t)g;\n        parent[g + 1] = (int32_t)node;"),
    ("node range one short", C, "range_hi[node] = (int32_t)b;", "range_hi[node] = (int32_t)(b - 1);"),
    ("W1 gradient scaled", M, 'g["W1"] = cache["a0"].T @ dz1', 'g["W1"] = cache["a0"].T @ dz1 * 0.5'),
    ("backward GELU slope of the wrong layer", M, 'dz2 = da2 * gelu_grad(cache["z2"])',
     'dz2 = da2 * gelu_grad(cache["z1"])'),
    ("loss sign", M, "np.maximum(z, 0) - z * y", "np.maximum(z, 0) + z * y"),
    ("loss mean over the batch only", M, "/ (n * D_OUT)", "/ n"),
    ("Adam second moment of |g|", M, "v[...] = b2 * v + (1 - b2) * g[k] ** 2",
     "v[...] = b2 * v + (1 - b2) * np.abs(g[k])"),
    ("Adam eps inside the root", M, "np.sqrt(vh) + eps", "np.sqrt(vh + eps)"),
    ("features clamped at 3", M, "np.clip(2.0 * f - 1.0, -4.0, 4.0)", "np.clip(2.0 * f - 1.0, -3.0, 3.0)"),
    ("feature padding not zero", M, "x = np.zeros((len(f), D_PAD))", "x = np.ones((len(f), D_PAD))"),
    ("forward drops the output bias", M, 'z3 = a2 @ W3 + p["b3"]', "z3 = a2 @ W3"),
    ("thread ranges skip a row", C, "nR * k / nthreads, nR * (k + 1) / nthreads,",
     "nR * k / nthreads + (k > 0), nR * (k + 1) / nthreads,"),
]


def _copy(dst):
    for d in ("oracle", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d),
                        ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ["conftest.py", "golden_io.py"] + [os.path.basename(p) for p in PINS]:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))


def _run(mutant):
    """(exit code, summary line) of the pin suites on a copy of the oracle
    with the mutant planted (None: the unmodified copy)."""
    with tempfile.TemporaryDirectory(prefix="oracle_mutant_", dir=SCRATCH) as d:
        _copy(d)
        if mutant is not None:
            _, f, old, new = mutant
            path = os.path.join(d, f)
            src = open(path).read()
            if src.count(old) != 1:
                return "text not found once"
            with open(path, "w") as fh:
                fh.write(src.replace(old, new))
        env = dict(os.environ)
        env.pop("PYTHONPATH", None)
        env["OMP_NUM_THREADS"] = "1"
        try:
            r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                                "-m", "not gpu", *PINS], cwd=d, env=env, capture_output=True, text=True,
                               timeout=600)
        except subprocess.TimeoutExpired:
            return "timeout"
        lines = r.stdout.strip().splitlines()
        return r.returncode, lines[-1] if lines else r.stderr[-300:]


@pytest.fixture(scope="module")
def outcomes():
    jobs = [None] + MUTANTS
    workers = max(1, min(8, os.cpu_count() or 1))
    os.makedirs(SCRATCH, exist_ok=True)
    try:
        with ThreadPoolExecutor(workers) as ex:
            codes = list(ex.map(_run, jobs))
    finally:
        shutil.rmtree(SCRATCH, ignore_errors=True)
    return {("control" if m is None else m[0]): c for m, c in zip(jobs, codes)}


def test_unmodified_copy_passes(outcomes):
    code, summary = outcomes["control"]
    assert code == 0, summary


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_mutant(outcomes, name):
    out = outcomes[name]
    assert out != "text not found once", f"{name}: the mutated text is no longer in the oracle"
    assert out != "timeout", f"{name}: the pin suites did not finish"
    code, summary = out
    # a pin must fail on a wrong answer: not pass, and not error out (a mutant
    # that does not compile or crashes proves nothing)
    assert code == 1 and "failed" in summary and "error" not in summary, f"{name}: {summary}"
