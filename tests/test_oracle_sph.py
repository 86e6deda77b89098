"""Pins of the oracle's neighbour search and SPH density (paper Sect. 3:
the tree also serves neighbour search and smoothed particle hydrodynamics).

The kernel against its defining properties (unit normalisation, value at
the centre, continuity, compact support); counts and densities against an
independent Python loop; the density of a uniform lattice; symmetry of the
neighbour relation for a common h."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_1204_2280_gb300 import workloads as W


@pytest.mark.parametrize("h", [1.0, 0.3, 0.01])
def test_kernel_is_normalised_and_smooth(orc, h):
    val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * orc.sph_kernel(r, h), 0, h, points=[h / 2], limit=200)
    assert val == pytest.approx(1.0, rel=1e-10)
    assert orc.sph_kernel(0.0, h) == pytest.approx(8 / (math.pi * h ** 3), rel=1e-15)
    lo, hi = orc.sph_kernel(h / 2 * (1 - 1e-12), h), orc.sph_kernel(h / 2 * (1 + 1e-12), h)
    assert lo == pytest.approx(hi, rel=1e-9)
    assert orc.sph_kernel(h, h) == 0.0 and orc.sph_kernel(1.5 * h, h) == 0.0
    assert orc.sph_kernel(h / 2, h) == pytest.approx(0.25 * 8 / (math.pi * h ** 3), rel=1e-14)


def test_counts_and_density_by_brute_force(orc):
    b = W.plummer(300, 41)
    h = np.random.default_rng(2).uniform(0.05, 0.6, 300).astype(np.float32)
    rho, cnt = orc.sph_density(b.pos, b.mass, h)
    p = b.pos.astype(np.float64)
    for i in range(300):
        r = np.linalg.norm(p - p[i], axis=1)
        hi = float(h[i])
        lo_cnt = int((r < hi * (1 - 1e-6)).sum())
        hi_cnt = int((r < hi * (1 + 1e-6)).sum())
        assert lo_cnt <= cnt[i] <= hi_cnt
        assert cnt[i] >= 1                                        # itself
        sel = r < hi * (1 - 1e-6)
        want = sum(float(b.mass[j]) * orc.sph_kernel(float(r[j]), hi) for j in np.nonzero(sel)[0])
        if lo_cnt == hi_cnt:
            assert rho[i] == pytest.approx(want, rel=1e-12)


def test_uniform_lattice_density(orc):
    """A cubic lattice of unit spacing and unit masses: the interior
    densities are the lattice density 1 to the kernel's smoothing error."""
    g = np.arange(12, dtype=np.float32)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    mass = np.ones(pos.shape[0], np.float32)
    h = np.full(pos.shape[0], 2.5, np.float32)
    rho, cnt = orc.sph_density(pos, mass, h)
    inner = np.all((pos >= 3) & (pos <= 8), axis=1)
    assert np.all(np.abs(rho[inner] - 1.0) < 2e-2)
    k = np.arange(-3, 4)
    within = sum(1 for x in k for y in k for z in k if x * x + y * y + z * z < 6.25)   # 81
    assert np.all(cnt[inner] == within)


def test_common_h_relation_is_symmetric(orc):
    b = W.plummer(2000, 42)
    h = np.full(2000, 0.1, np.float32)
    _, cnt = orc.sph_density(b.pos, b.mass, h)
    p = b.pos
    # every pair counted from both ends: sum of (count - self) is even and
    # equals twice the number of unordered pairs found by a float32 loop
    pairs = 0
    for i in range(2000):
        d = (p - p[i]).astype(np.float32)
        r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        pairs += int((r2[i + 1:] < np.float32(0.01)).sum())
    assert abs(int(cnt.sum()) - 2000 - 2 * pairs) <= 4     # fused vs unfused r^2 at a boundary
