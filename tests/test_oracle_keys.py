"""Pins of the oracle's domain, Morton keys and stable sort (Sect. 2, "sorting
of the particles along a Space Filling Curve").

The checks are independent of the oracle's C arithmetic: exact rational
arithmetic (fractions.Fraction) for the quantisation, a Python bit loop for
the interleave, and numpy's stable argsort for the permutation."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1204_2280_gb300 import workloads as W

L = 21


def deinterleave(k: int):
    q = [0, 0, 0]
    for b in range(L):
        for d in range(3):
            q[d] |= ((k >> (3 * b + d)) & 1) << b
    return q


def edge_positions(rng, n):
    """Positions with exact ties, tiny magnitudes, signed zeros and values
    straddling quantisation boundaries."""
    p = rng.standard_normal((n, 3)).astype(np.float32)
    p[::7] = p[3]                                    # duplicates
    p[1::11, 0] = np.float32(1e-30)                  # tiny vs large exponents
    p[2::13, 1] = np.float32(-0.0)
    p[5::17] *= np.float32(1e-6)
    return p


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_domain_is_smallest_power_of_two_above_extent(orc, seed):
    rng = np.random.default_rng(seed)
    p = edge_positions(rng, 777) * np.float32([1.0, 3.0, 0.25])
    mn, S = orc.domain(p)
    assert np.array_equal(mn, p.min(0))
    ext = max(Fraction(float(p[:, d].max())) - Fraction(float(p[:, d].min())) for d in range(3))
    FS = Fraction(S)
    assert FS > ext and FS / 2 <= ext
    assert S == 2.0 ** round(np.log2(S))


def test_domain_degenerate(orc):
    mn, S = orc.domain(np.ones((5, 3), np.float32))
    assert S == 2.0 ** -64
    # extent exactly a power of two: S must be strictly larger
    p = np.array([[0, 0, 0], [4, 1, 1]], np.float32)
    assert orc.domain(p)[1] == 8.0


def test_interleave_bit_order(orc):
    assert orc.interleave(1, 0, 0) == 1
    assert orc.interleave(0, 1, 0) == 2
    assert orc.interleave(0, 0, 1) == 4
    assert orc.interleave(2, 0, 0) == 8
    m = (1 << L) - 1
    assert orc.interleave(m, m, m) == (1 << 63) - 1
    rng = np.random.default_rng(3)
    for _ in range(200):
        q = [int(v) for v in rng.integers(0, 1 << L, 3)]
        assert deinterleave(orc.interleave(*q)) == q


@pytest.mark.parametrize("seed", [0, 1])
def test_keys_exact_quantisation(orc, seed):
    """Decode every key and check, in exact rationals, that its cell of side
    S/2^21 contains the point: mn + q h <= x < mn + (q+1) h."""
    rng = np.random.default_rng(seed)
    p = edge_positions(rng, 600)
    mn, S = orc.domain(p)
    k = orc.keys(p, mn, S)
    h = Fraction(S) / (1 << L)
    for i in range(p.shape[0]):
        q = deinterleave(int(k[i]))
        for d in range(3):
            x = Fraction(float(p[i, d]))
            lo = Fraction(float(mn[d])) + q[d] * h
            assert lo <= x < lo + h, (i, d)


def test_keys_at_boundaries(orc):
    """Points placed exactly on, and one float below, cell boundaries."""
    S = 4.0
    mn = np.float32(-1.0)
    h = S / (1 << L)
    xs = []
    for j in [1, 2, 3, 1000, (1 << L) - 3]:
        b = np.float32(mn + j * h)           # exactly representable boundary
        xs += [b, np.nextafter(b, np.float32(-np.inf))]
    p = np.zeros((len(xs) + 2, 3), np.float32)
    p[: len(xs), 0] = xs
    p[-2] = [-1.0, -1.0, -1.0]
    p[-1] = [2.5, 2.5, 2.5]                  # extent 3.5 -> S = 4
    mn_, S_ = orc.domain(p)
    assert S_ == S and mn_[0] == mn
    k = orc.keys(p, mn_, S_)
    for i, x in enumerate(xs):
        q = deinterleave(int(k[i]))[0]
        want = int((Fraction(float(x)) - Fraction(float(mn))) / Fraction(h))
        assert q == want


def test_sort_stable_vs_numpy(orc):
    rng = np.random.default_rng(5)
    k = rng.integers(0, 50, 5000).astype(np.uint64) << np.uint64(40)
    k[::3] |= rng.integers(0, 4, k[::3].shape[0]).astype(np.uint64)
    perm = orc.sort(k)
    assert np.array_equal(perm, np.argsort(k, kind="stable").astype(np.uint32))


def test_plummer_keys_sorted_and_distinct(orc):
    b = W.plummer(4096, 0)
    k = orc.keys(b.pos)
    perm = orc.sort(k)
    assert np.all(np.diff(k[perm].astype(np.float64)) >= 0)
    assert np.array_equal(perm, np.argsort(k, kind="stable"))


def test_keys_exact_when_double_difference_rounds():
    """x - mn not representable in float64: 1.0 - 2^-80 rounds to 1.0, a cell
    boundary, while the exact value lies just below it.  The domain side must
    also come from the exact extent (1 - 2^-80 -> S = 1, not 2)."""
    import oracle as orc
    tiny = np.float32(2.0 ** -80)
    p = np.array([[tiny, 0, 0], [1.0, 0, 0], [1.5, 0, 0], [0.5, 0, 0]], np.float32)
    mn, S = orc.domain(p)
    assert mn[0] == tiny and S == 2.0
    k = orc.keys(p, mn, S)
    h = Fraction(S) / (1 << L)
    for i in range(p.shape[0]):
        q = deinterleave(int(k[i]))[0]
        assert q == int((Fraction(float(p[i, 0])) - Fraction(float(tiny))) / h)
    assert deinterleave(int(k[1]))[0] == (1 << 20) - 1
    assert orc.domain(p[[0, 1]])[1] == 1.0
