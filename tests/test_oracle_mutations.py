"""Each plausible slip in the oracle (a dropped factor, a flipped sign or
tie-break, an off-by-one in a limit or a neighbour) must make some pin fail.
The mistake is planted in a temporary copy of vmat_oracle.c on the CPU; the
pins of test_oracle.py then run against that copy in a child process."""
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vmat_oracle.c")

MUTATIONS = {
    "dF drops the factor 2": ("return 2.0 * b * (z - T);", "return b * (z - T);"),
    "dF wrong sign below T": ("return -2.0 * a * (T - z);", "return 2.0 * a * (T - z);"),
    "G wrap gap": ("theta[0] + 360.0 - theta[N - 1]", "theta[0] + 180.0 - theta[N - 1]"),
    "price reads the transpose": ("s += val[e] * f[vox[e]];", "s += val[e] * f[e % 7];"),
    "row scan ties to smaller l": ("(lbest < 0 || P >= Pbest)", "(lbest < 0 || P > Pbest)"),
    "row scan prefers longer": ("(v == bv && len < br - bl)", "(v == bv && len > br - bl)"),
    "leaf limit off by one": ("if (ln + m < lhi) lhi = ln + m;", "if (ln + m - 1 < lhi) lhi = ln + m - 1;"),
    "angle tie to highest k": ("if (best < 0 || p < bp) {", "if (best < 0 || p <= bp) {"),
    "line search wrong curvature": ("Bc += 2.0 * c * wj * wj;", "Bc += c * wj * wj;"),
    "master ignores smoothing in gradient": ("grad[k] *= gamma;", "grad[k] *= 0.0;"),
    "aperture dose includes right leaf": ("for (int c = l[rr]; c < r[rr]; ++c) {", "for (int c = l[rr]; c <= r[rr] && c < C; ++c) {"),
    "histogram edge goes down": ("z[j] >= (double)(b + 1) * dose_max", "z[j] > (double)(b + 1) * dose_max",
                                 "test_oracle_dvh.py"),
    "histogram drops the last bin": ("while (b + 1 < n_bins &&", "while (b + 2 < n_bins &&",
                                     "test_oracle_dvh.py"),
    "smoothing price offset sign": ("for (int q = 0; q < N; ++q) off[q] *= gamma;",
                                    "for (int q = 0; q < N; ++q) off[q] *= -gamma;",
                                    "test_oracle_price_smoothing.py"),
    "smoothing price offset of the next beam": ("if (offset) p += offset[k];",
                                                "if (offset) p += offset[(k + 1) % N];",
                                                "test_oracle_price_smoothing.py"),
}

RUNNER = r"""
import sys, importlib
sys.path.insert(0, {root!r})
import oracle
oracle._LIB = {lib!r}
oracle._SRC = {src!r}
oracle._lib = None
import pytest
sys.exit(pytest.main([{tests!r}, "-x", "-q", "-p", "no:cacheprovider"]))
"""


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new, *pins = MUTATIONS[name]
    pins = pins[0] if pins else "test_oracle.py"
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    with tempfile.TemporaryDirectory() as d:
        msrc = os.path.join(d, "vmat_oracle.c")
        mlib = os.path.join(d, "liboracle.so")
        open(msrc, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", msrc, "-o", mlib, "-lm"])
        code = RUNNER.format(root=ROOT, lib=mlib, src=msrc,
                             tests=os.path.join(ROOT, "tests", pins))
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
