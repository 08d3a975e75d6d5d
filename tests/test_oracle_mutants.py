"""The pins catch plausible mistakes.  Each mutant is a copy of the C oracle
with one mistake planted (on the CPU, in a temporary directory); the pin
tests, run against that copy, must fail on every one."""
import os
import subprocess
import sys

import pytest

from oracle import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "frnn_oracle.c")

# name -> (text in the oracle, replacement); the first occurrence is replaced
# (for the shared lines: in frnn_oracle_query)
MUTANTS = {
    "strict boundary": ("if (s <= r2) {", "if (s < r2) {"),
    "radius not squared in float": ("    const float r2 = r * r;\n    int failed = 0;",
                                    "    const double r2 = (double)r * (double)r;\n    int failed = 0;"),
    "sign flip": ("float d = q[k] - p[k];", "float d = q[k] + p[k];"),
    "last dimension dropped": ("for (int k = 0; k < D; ++k) {\n        float d = q[k] - p[k];",
                               "for (int k = 0; k < D - 1; ++k) {\n        float d = q[k] - p[k];"),
    "reversed summation": ("for (int k = 0; k < D; ++k) {\n        float d = q[k] - p[k];",
                           "for (int k = D - 1; k >= 0; --k) {\n        float d = q[k] - p[k];"),
    "fused multiply-add": ("        float t = d * d;\n        s = s + t;",
                           "        s = fmaf(d, d, s);"),
    "self pair kept": ("                if (query_ids && query_ids[i] == j) continue;\n", ""),
    "reversed tie-break": ("return a->j < b->j;", "return a->j > b->j;"),
    "count not truncated": ("counts[i] = (int32_t)keep;", "counts[i] = (int32_t)deg;"),
    "padding index 0": ("irow[e] = -1;", "irow[e] = 0;"),
    "padding distance 0": ("drow[e] = INFINITY;", "drow[e] = 0.0f;"),
    "off-by-one truncation": ("int64_t keep = deg < K ? deg : K;", "int64_t keep = deg < K ? deg : K - 1;"),
    "query row stride": ("const float* q = queries + i * (int64_t)D;\n            int64_t deg = 0;",
                         "const float* q = queries + i;\n            int64_t deg = 0;"),
    # the degree-only and FP64-audit functions
    "degree strict boundary": ("if (contract_d2(q, refs + j * (int64_t)D, D) <= r2) ++deg;",
                               "if (contract_d2(q, refs + j * (int64_t)D, D) < r2) ++deg;"),
    "audit in float": ("double d = (double)q[k] - (double)p[k];", "float d = q[k] - p[k];"),
    "audit strict boundary": ("int in64 = s <= r64;", "int in64 = s < r64;"),
    "audit verdicts swapped": ("if (in32 && !in64) ++a32;", "if (in64 && !in32) ++a32;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    a, b = MUTANTS[name]
    with open(SRC) as f:
        src = f.read()
    assert a in src, f"mutation target of '{name}' not found in the oracle"
    c = tmp_path / "oracle_mutant.c"
    c.write_text(src.replace(a, b, 1))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(so), str(c), "-lm"], check=True)
    env = dict(os.environ, OMP_NUM_THREADS="4")
    p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        f"--oracle-lib={so}",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    # exit status 1: some pin failed (not an error in collecting or running them)
    assert p.returncode == 1, f"'{name}' survived the pins:\n{p.stdout[-1500:]}"
