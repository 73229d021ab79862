"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle (a rule that decides an
integer taken the other way, a dropped term, a wrong sign, a wrong index or
operand) and runs the oracle's pins (tests/test_oracle.py) on the copy in a
subprocess: every mutant must fail at least one pin, and the unchanged copy
must pass them all.  The mistakes follow the paper's steps: validity and the
depth cut of the mesh (Sec. 2, mesh construction), the weighted normal
(Sec. 2, normal estimation), the strict predicates and the labelling of
Algorithm 1, and the back-fill (Sec. 2, last paragraph).
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in oracle/lsg_oracle.c, its mutated form)
MUTANTS = [
    ("r_max exclusive", "valid[dst] = (r_min < r && r <= r_max) ? 1 : 0;",
     "valid[dst] = (r_min < r && r < r_max) ? 1 : 0;"),
    ("r_min inclusive", "valid[dst] = (r_min < r && r <= r_max) ? 1 : 0;",
     "valid[dst] = (r_min <= r && r <= r_max) ? 1 : 0;"),
    ("depth cut on the farther range", "float m = rp < rq ? rp : rq;", "float m = rp < rq ? rq : rp;"),
    ("depth cut not strict", "return ad > t;", "return ad >= t;"),
    ("triangle without its rim edge",
     "        if (!o_edge(mb, H, Ws, wr, sp[k][0], sp[k][1], sp[k1][0], sp[k1][1], 0)) continue;\n", ""),
    ("sixth triangle dropped", "for (int k = 0; k < 6; ++k) {\n        int k1 = (k + 1) % 6;",
     "for (int k = 0; k < 5; ++k) {\n        int k1 = (k + 1) % 6;"),
    ("unweighted triangles", "double w = 1.0 / (la + lb);", "double w = 1.0;"),
    ("weight of the longer spoke only", "double w = 1.0 / (la + lb);", "double w = 1.0 / (la > lb ? la : lb);"),
    ("cross product y with a wrong sign", "double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2],",
     "double cr[3] = {a[1] * b[2] - a[2] * b[1], a[0] * b[2] - a[2] * b[0],"),
    ("normal facing away from the sensor", "normal[3 * v + t] = -sgn * sum[t] / len;",
     "normal[3 * v + t] = sgn * sum[t] / len;"),
    ("angle predicate not strict", "ok = ang < angle_t;", "ok = ang <= angle_t;"),
    ("component predicate not strict on y", "ok = dx < comp[0] && dy < comp[1]",
     "ok = dx < comp[0] && dy <= comp[1]"),
    ("components over mesh edges, not homogeneous ones",
     "if (!o_edge(mb, H, Ws, wr, i, j, sp[k][0], sp[k][1], 1)) continue;\n        int u",
     "if (!o_edge(mb, H, Ws, wr, i, j, sp[k][0], sp[k][1], 0)) continue;\n        int u"),
    ("label index over sampled columns", "int32_t lab = si * W + sj * s;", "int32_t lab = si * Ws + sj * s;"),
    ("back-fill ties to the later column", "if (have_hi && dhi < dlo)", "if (have_hi && dhi <= dlo)"),
    ("back-fill without the other column", "labels[o] = first != -1 ? first : second;", "labels[o] = first;"),
    ("wrap distance off by one", "dhi = W - c;", "dhi = W - c + 1;"),
    ("rings ordered from the bottom", "while (b >= 0 && (elev[order[b]] < elev[cur] ||",
     "while (b >= 0 && (elev[order[b]] > elev[cur] ||"),
    ("ties between rings to the later input row", "(elev[order[b]] == elev[cur] && order[b] > cur))",
     "(elev[order[b]] == elev[cur] && order[b] < cur))"),
    ("azimuth of the next column", "double phi = (double)az0 + (double)c * (double)daz;",
     "double phi = (double)az0 + (double)(c + 1) * (double)daz;"),
    ("height from the cosine of the elevation", "xyz[3 * dst + 2] = rd * sin(th);",
     "xyz[3 * dst + 2] = rd * cos(th);"),
    ("x from the sine of the azimuth", "xyz[3 * dst + 0] = rd * cos(th) * cos(phi);",
     "xyz[3 * dst + 0] = rd * cos(th) * sin(phi);"),
    ("diagonal spokes the other way", "static const int dj[6] = {0, +1, +1, 0, -1, -1};",
     "static const int dj[6] = {0, -1, +1, 0, +1, -1};"),
    ("spokes not wrapped around the ring", "    if (wr) jj = (jj + Ws) % Ws;\n    if (ii < 0", "    if (ii < 0"),
]


def _copy_tree(dst):
    ignore = shutil.ignore_patterns("*.so", "*.so.tmp*", "__pycache__", "_build")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ignore)
    shutil.copytree(os.path.join(ROOT, "lidarsim"), os.path.join(dst, "lidarsim"), ignore=ignore)
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "test_oracle.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), os.path.join(dst, "pytest.ini"))


def _run_pins(d, name, old, new):
    _copy_tree(d)
    src = os.path.join(d, "oracle", "lsg_oracle.c")
    text = open(src).read()
    if old is not None:
        assert text.count(old) == 1, f"{name}: the text to mutate is not found exactly once"
        with open(src, "w") as f:
            f.write(text.replace(old, new))
    # the copy must compile: a pin failing on a build error would prove nothing
    cc = shutil.which("gcc") or shutil.which("cc")
    chk = subprocess.run([cc, "-std=c99", "-fsyntax-only", src], capture_output=True, text=True)
    assert chk.returncode == 0, f"{name}: the mutated oracle does not compile: {chk.stderr}"
    env = dict(os.environ, PYTHONPATH=d, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(d, "tests", "test_oracle.py"), "-q", "-x",
                        "-p", "no:cacheprovider", "-m", "not gpu"], cwd=d, env=env, capture_output=True,
                       text=True, timeout=600)
    return name, r.returncode, (r.stdout + r.stderr).strip().splitlines()[-1:]


def test_every_mutant_fails_a_pin_and_the_oracle_passes(tmp_path):
    cases = [("unchanged", None, None)] + MUTANTS
    names = [c[0] for c in cases]
    assert len(set(names)) == len(names)
    base = str(tmp_path)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda c: _run_pins(os.path.join(base, "c%02d" % names.index(c[0])), *c), cases))
    rc = {n: (code, tail) for n, code, tail in results}
    assert rc["unchanged"][0] == 0, rc["unchanged"]
    # exit code 1: a pin failed (not a build or collection error, which is 2 or more)
    survivors = {n: v for n, v in rc.items() if n != "unchanged" and v[0] != 1}
    assert not survivors, survivors
