"""The oracle's pins must catch plausible mistakes.  Each case copies the
oracle to a temporary directory, plants one mistake in the copy of
bonsai_oracle.c (a flipped sign, a dropped term, a swapped index, an
off-by-one in the leaf rule, ...), rebuilds it there and runs the oracle pin
tests against it: every planted mistake must make some pin fail.  Nothing
outside the temporary copy is touched and no GPU is involved."""
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


@pytest.mark.parametrize("orig,mut", MUTATIONS, ids=[str(i) for i in range(len(MUTATIONS))])
def test_planted_mistake_is_caught(tmp_path, orig, mut):
    d = tmp_path / "repo"
    d.mkdir()
    for x in ("tests", "paper_1204_2280_gb300", "oracle"):
        shutil.copytree(os.path.join(ROOT, x), d / x,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*", "csrc"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d / "pytest.ini")
    src = d / "oracle" / "bonsai_oracle.c"
    s = src.read_text()
    assert orig in s, orig
    src.write_text(s.replace(orig, mut))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_keys.py", "tests/test_oracle_tree.py",
                        "tests/test_oracle_moments.py", "tests/test_oracle_forces.py",
                        "tests/test_oracle_walk.py", "tests/test_oracle_physics.py",
                        "tests/test_oracle_block.py", "tests/test_oracle_sph.py"],
                       cwd=d, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake survived: " + mut
