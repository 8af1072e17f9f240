"""The oracle's pins must catch plausible mistakes in it: each case below
plants one mistake in a copy of the oracle's C source (a dropped factor, a
swapped index or sign, a wrong tolerance, a rule turned around), builds the
copy on the CPU, and runs the oracle pins against it; every copy must fail
at least one pin.  The oracle itself is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "findpts_oracle.c")
PINS = ["tests/test_oracle_basis.py", "tests/test_oracle_find.py", "tests/test_oracle_overlap.py",
        "tests/test_oracle_flux.py", "tests/test_oracle_2d.py"]

# (name, text in the oracle, replacement, occurrence to replace: 0 = the only
# one); lists of texts and replacements make several edits at once
MUTATIONS = [
    ("gll weight: P_N to the first power", "w[i] = 2.0 / (N * (N + 1.0) * p * p);",
     "w[i] = 2.0 / (N * (N + 1.0) * p);", 0),
    ("Lagrange derivative: sign of 1/(x_i - x_k)", "double q = 1.0 / (xg[i] - xg[k]);",
     "double q = 1.0 / (xg[k] - xg[i]);", 0),
    ("3D map: i and j node indices swapped", "double c = el->X[a][i + n * (j + n * k)];",
     "double c = el->X[a][j + n * (i + n * k)];", 0),
    ("3D Jacobian: columns r and s swapped", "J[3 * a + 0] = vr; J[3 * a + 1] = vs; J[3 * a + 2] = vt;",
     "J[3 * a + 0] = vs; J[3 * a + 1] = vr; J[3 * a + 2] = vt;", 0),
    ("Newton: no active set at the bounds",
     ["act[b] = (r[b] <= -1.0 && g[b] > 0.0) || (r[b] >= 1.0 && g[b] < 0.0);",
      "if (!act[b] && ((r[b] <= -1.0 && d[b] < 0.0) || (r[b] >= 1.0 && d[b] > 0.0))) {"],
     ["act[b] = 0;", "if (0) {"], 0),
    ("eval: node index transposed", "v += f[i + n * (j + n * k)] * h[0][i] * h[1][j] * h[2][k];",
     "v += f[k + n * (j + n * i)] * h[0][i] * h[1][j] * h[2][k];", 0),
    ("border: tol_accept used for the border band", "} else if (res <= prm->tol_border * he[e]) {",
     "} else if (res <= prm->tol_accept * he[e]) {", 0),
    ("element tie: the highest INSIDE element id kept", "if (s == nin && nin < MAXS) {",
     "if (s < nin) { in_e[s] = e; memcpy(in_r[s], best_r, sizeof best_r); in_d[s] = res; } else if (nin < MAXS) {", 0),
    ("inside: the border tolerance accepted as inside", "if (res <= prm->tol_accept * he[e]) {",
     "if (res <= prm->tol_border * he[e]) {", 0),
    ("owner: distance field ignored", "dl[s] = dist ? interp_elem(N, dim, xg, dist + in_e[s] * n3, in_r[s]) : 0.0;",
     "dl[s] = 0.0;", 0),
    ("owner tie: higher subdomain id wins", "(w < 0 || in_s[s] < in_s[w])", "(w < 0 || in_s[s] > in_s[w])", 0),
    ("3D default distance: every face a boundary face", "bnd[a] = !shared;", "bnd[a] = 1;", 1),
    ("2D default distance: every edge a boundary edge", "bnd[a] = !shared;", "bnd[a] = 1;", 2),
    ("face normal: cyclic orientation sign dropped", "double o = (ax == 1 ? -1.0 : 1.0) * sgn;",
     "double o = sgn;", 0),
    ("flux correction: sign of gamma", "double g = area > 0.0 ? -fl / area : 0.0;",
     "double g = area > 0.0 ? fl / area : 0.0;", 0),
    ("2D map: i and j node indices swapped", "double c = el->X[a][i + n * j];", "double c = el->X[a][j + n * i];", 0),
    ("2D eval: node index transposed", "v += f[i + n * j] * h[0][i] * h[1][j];", "v += f[j + n * i] * h[0][i] * h[1][j];", 0),
    ("session discriminator ignored", "if (tag >= 0 && sub[e] == tag) continue;", "if (0) continue;", 0),
    ("3D default distance: other subdomains' boundaries counted", "if (bs[b] != sub[e]) continue;",
     "if (0) continue;", 1),
    ("2D default distance: other subdomains' boundaries counted", "if (bs[b] != sub[e]) continue;",
     "if (0) continue;", 2),
    ("2D Jacobian: columns r and s swapped", "if (J) { J[3 * a + 0] = vr; J[3 * a + 1] = vs; }",
     "if (J) { J[3 * a + 0] = vs; J[3 * a + 1] = vr; }", 0),
    ("face quadrature: one GLL weight dropped", "dA[m] = wg[a] * wg[b] * len;", "dA[m] = wg[a] * len;", 0),
    ("border: distance returned unsquared", "dist2[p] = b_d * b_d;", "dist2[p] = b_d;", 0),
    ("prefilter: node box without its margin", "double g = 0.25 * (hi[a] - lo[a]) + prm->tol_border * he[e];",
     "double g = 0.0;", 0),
]


def _mutate(src, old, new, which):
    if isinstance(old, list):                      # several edits, each at its only occurrence
        for o, nw in zip(old, new):
            src = _mutate(src, o, nw, 0)
        return src
    if which == 0:
        assert src.count(old) == 1, old
        return src.replace(old, new)
    parts = src.split(old)
    assert len(parts) > which, old
    return old.join(parts[:which]) + new + old.join(parts[which:])


@pytest.mark.parametrize("name,old,new,which", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, which):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = _mutate(open(SRC).read(), old, new, which)
    c = tmp_path / "mutant.c"
    c.write_text(src)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                           "-o", str(so), str(c), "-lm"])
    env = dict(os.environ, FINDPTS_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    # exit code 1: tests ran and one failed (not a crash, a collection error or a usage error)
    assert r.returncode == 1, f"no pin caught the planted mistake: {name} (exit {r.returncode})\n{r.stdout[-2000:]}"
