"""The oracle's pins must catch plausible mistakes.  Each case copies the
oracle to a temporary directory, plants one mistake in the copy (in the C
tree-code bonsai_oracle.c: a flipped sign, a dropped term, a swapped index,
an off-by-one in the leaf rule, ...; in the Python parts: the learned
correction's features, labels and network in mlp.py, the leapfrog and the
block time steps in __init__.py), and runs the oracle pin tests against the
copy: every planted mistake must make some pin fail.  Nothing outside the
temporary copy is touched and no GPU is involved."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("a[0] += s * dx - r5i * Qx;", "a[0] += s * dx + r5i * Qx;"),
    ("double s = M * r3i + 2.5 * q * r7i;", "double s = M * r3i + 1.5 * q * r7i;"),
    ("q[3] += mj * (3 * y0 * y1);", "q[3] += mj * (3 * y0 * y2);"),
    ("k |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);", "k |= (uint64_t)((qy >> b) & 1u) << (3 * b + 2);"),
    ("if (f == t && e < 0.0) f -= 1.0;", ";"),
    ("if (s == p) return (e < 0.0) ? p : 2.0 * p;", "if (s == p) return 2.0 * p;"),
    ("r_open[c] = l / theta + sqrt(dx * dx + dy * dy + dz * dz);", "r_open[c] = l / theta;"),
    ("if (dist2 < ro * ro) {", "if (dist2 <= ro * ro * 0.98) {"),
    ("if (body_count[c] <= nleaf || l == ORC_L) continue;", "if (body_count[c] < nleaf || l == ORC_L) continue;"),
    ("*phi -= M * rinv + 0.5 * q * r5i;", "*phi -= M * rinv;"),
    ("if (j == i) { self_seen++; continue; }", "if (j == i) { self_seen++; }"),
    ("centre[d] = (double)mn[d] + (double)q[d] * h + 0.5 * l_side;", "centre[d] = (double)mn[d] + (double)q[d] * h;"),
    ("double mr3 = mj * rinv * rinv * rinv;", "double mr3 = mj * rinv * rinv;"),
    ("if (body_count[c] <= ncrit && (c == 0 || body_count[parent[c]] > ncrit))",
     "if (body_count[c] <= ncrit && (c == 0 || body_count[parent[c]] >= ncrit))"),
    ("int sibling = g_par[i] >= 0 && g_par[i] == g_par[i - 1];", "int sibling = g_par[i] >= 0;"),
    ("if (sibling && g_count[out] + g_count[i] <= ncrit) {", "if (sibling && g_count[out] + g_count[i] < ncrit) {"),
    ("if (m + ext[ch] > e) e = m + ext[ch];", "if (ext[ch] > e) e = ext[ch];"),
    ("return s * 2.0 * t * t * t; }", "return s * t * t * t; }"),
    ("if (!(r2 < h2)) continue;", "if (!(r2 < 0.98f * h2)) continue;"),
]


# Python parts of the oracle: (file, original, mistake, pin tests that must catch it)
MLP_PINS = ["tests/test_oracle_mlp.py"]
STEP_PINS = ["tests/test_oracle_physics.py", "tests/test_oracle_block.py"]
PY_MUTATIONS = [
    ("mlp.py", "r = (np.asarray(a_direct, np.float64) - a) / np.linalg.norm(a, axis=1)[:, None]",
     "r = (np.asarray(a_direct, np.float64) - a) / np.linalg.norm(np.asarray(a_direct, np.float64), axis=1)[:, None]",
     MLP_PINS),
    ("mlp.py", "X[:, 7] = np.log(tf.gcnt[g] / (emax[g] ** 3 + eps ** 3))",
     "X[:, 7] = np.log(tf.gcnt[g] / (diag[g] ** 3 + eps ** 3))", MLP_PINS),
    ("mlp.py", "X[:, 8] = np.log((diag[g] + eps) / eps)", "X[:, 8] = np.log((emax[g] + eps) / eps)", MLP_PINS),
    ("mlp.py", "X[:, 0] = np.log(np.maximum(an, 1e-30))", "X[:, 0] = np.log(np.maximum(an * an, 1e-30))", MLP_PINS),
    ("mlp.py", "X[:, 1] = np.log(np.maximum(-tf.pot, 1e-30))", "X[:, 1] = np.log10(np.maximum(-tf.pot, 1e-30))",
     MLP_PINS),
    ("mlp.py", "X[:, 11] = np.log(tf.gcnt[g])", "X[:, 11] = np.log1p(tf.gcnt[g])", MLP_PINS),
    ("mlp.py", "on / np.maximum(0.5 * diag[g], 1e-300)", "on / np.maximum(diag[g], 1e-300)", MLP_PINS),
    ("mlp.py", "h2 = r(np.maximum(z2, 0.0))", "h2 = r(z2)", MLP_PINS),
    ("mlp.py", "return e0, e1, np.cross(e0, e1)", "return e0, e1, np.cross(e1, e0)", MLP_PINS),
    ("mlp.py", "ax = np.argmin(np.abs(e0[bad]), axis=1)", "ax = np.argmax(np.abs(e0[bad]), axis=1)", MLP_PINS),
    ("mlp.py", "b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16", "b = ((b + 0x8000) >> 16) << 16", MLP_PINS),
    ("mlp.py", 'dh2 = (dy @ c["W3"]) * (c["z2"] > 0)', 'dh2 = (dy @ c["W3"])', MLP_PINS),
    ("__init__.py", "vh = vel + 0.5 * dt * np.asarray(acc0, np.float64)",
     "vh = vel + dt * np.asarray(acc0, np.float64)", STEP_PINS),
    ("__init__.py", "v1 = vh + 0.5 * dt * tf.acc", "v1 = vh + 0.5 * dt * np.asarray(acc0, np.float64)", STEP_PINS),
    ("__init__.py", "k += (r > np.float32(16.0) ** (lev - 1)).astype(np.int32)",
     "k += (r > np.float32(4.0) ** (lev - 1)).astype(np.int32)", STEP_PINS),
    ("__init__.py", "return np.float32((d2 * d2) / ((e2 * e2) * (s * s)))",
     "return np.float32((d2 * d2) / ((e2 * e2) * s))", STEP_PINS),
    ("__init__.py", "new = np.maximum(block_level(a, c32, kmax), kmax - _ctz(s))",
     "new = block_level(a, c32, kmax)", STEP_PINS),
    ("__init__.py", "act = (s % (1 << (kmax - lev))) == 0", "act = (s % (1 << lev)) == 0", STEP_PINS),
    ("__init__.py", "    v += a * h[:, None]\n", "    v += a * 2 * h[:, None]\n", STEP_PINS),
    ("__init__.py", "ro = open_radius(self.tree, self.skeys, self.mn, self.S, com, theta, ext)",
     "ro = open_radius(self.tree, self.skeys, self.mn, self.S, com, theta)", STEP_PINS),
    ("__init__.py", "        if not act.any():\n            continue\n", "", STEP_PINS),
    ("__init__.py", "            due = False\n", "", STEP_PINS),
]
C_PINS = ["tests/test_oracle_keys.py", "tests/test_oracle_tree.py", "tests/test_oracle_moments.py",
          "tests/test_oracle_forces.py", "tests/test_oracle_walk.py", "tests/test_oracle_physics.py",
          "tests/test_oracle_block.py", "tests/test_oracle_sph.py"]

CASES = [("bonsai_oracle.c", o, m, C_PINS) for o, m in MUTATIONS] + PY_MUTATIONS


@pytest.mark.parametrize("fname,orig,mut,pins", CASES, ids=[str(i) for i in range(len(CASES))])
def test_planted_mistake_is_caught(tmp_path, fname, orig, mut, pins):
    d = tmp_path / "repo"
    d.mkdir()
    py = fname.endswith(".py")
    for x in ("tests", "paper_1204_2280_gb300", "oracle"):
        # a Python mistake keeps the compiled C oracle (copied with its mtime)
        skip = ["__pycache__", "*.tmp*", "csrc"] + ([] if py and x == "oracle" else ["*.so"])
        shutil.copytree(os.path.join(ROOT, x), d / x, ignore=shutil.ignore_patterns(*skip))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d / "pytest.ini")
    src = d / "oracle" / fname
    s = src.read_text()
    assert s.count(orig) == 1, orig
    src.write_text(s.replace(orig, mut))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *pins],
                       cwd=d, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake survived: " + mut
