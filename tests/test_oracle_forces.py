"""Pins of the oracle's direct sum and tree walk (Sect. 1: the O(N^2) method;
Sect. 2: tree-traverse with the opening angle theta).

Independent checks: the two-body closed form, a pure-Python double loop,
Newton's third law, the theta -> 0 limit (every cell opened, so the walk must
equal the direct sum), the order of accuracy of the quadrupole expansion,
a = -grad(phi) by central differences, and monotone convergence in theta."""
import math

import numpy as np
import pytest

from paper_1204_2280_gb300 import workloads as W


def test_two_body_closed_form(orc):
    pos = np.array([[0.0, 0.0, 0.0], [0.75, -0.5, 0.25]], np.float32)
    mass = np.array([0.25, 2.0], np.float32)
    eps = 0.1
    a, phi = orc.direct(pos, mass, eps)
    d = pos[1].astype(np.float64) - pos[0]
    r2 = d.dot(d) + eps * eps
    assert np.allclose(a[0], 2.0 * d / r2 ** 1.5, rtol=1e-15, atol=0)
    assert np.allclose(a[1], -0.25 * d / r2 ** 1.5, rtol=1e-15, atol=0)
    assert phi[0] == pytest.approx(-2.0 / math.sqrt(r2), rel=1e-15)
    assert phi[1] == pytest.approx(-0.25 / math.sqrt(r2), rel=1e-15)


def test_direct_vs_python_loop(orc):
    rng = np.random.default_rng(0)
    pos = rng.standard_normal((64, 3)).astype(np.float32)
    mass = rng.uniform(0.1, 1.0, 64).astype(np.float32)
    eps = 0.05
    a, phi = orc.direct(pos, mass, eps)
    x = pos.astype(np.float64)
    for i in range(64):
        ai = np.zeros(3); pi = 0.0
        for j in range(64):
            if j == i:
                continue
            d = x[j] - x[i]
            r = math.sqrt(d.dot(d) + eps * eps)
            ai += float(mass[j]) * d / r ** 3
            pi -= float(mass[j]) / r
        assert np.allclose(a[i], ai, rtol=1e-13, atol=1e-15)
        assert phi[i] == pytest.approx(pi, rel=1e-13)


def test_direct_newton_third_law(orc):
    b = W.plummer(2000, 4)
    a, _ = orc.direct(b.pos, b.mass, 0.01)
    f = (b.mass[:, None].astype(np.float64) * a).sum(0)
    assert np.abs(f).max() < 1e-12 * (b.mass[:, None] * np.abs(a)).sum()


@pytest.mark.parametrize("n", [1, 2, 17, 300, 4096])
def test_theta_to_zero_equals_direct(orc, n):
    b = W.plummer(n, 5)
    tf = orc.tree_forces(b.pos, b.mass, theta=1e-9, eps=0.01, nleaf=16, ncrit=32)
    a, phi = orc.direct(b.pos, b.mass, 0.01)
    assert np.all(tf.n_pc == 0) and np.all(tf.n_pp == n - 1)
    assert np.allclose(tf.acc, a, rtol=1e-11, atol=1e-12 * np.abs(a).max() if n > 1 else 0)
    assert np.allclose(tf.pot, phi, rtol=1e-12, atol=0)


def cluster(rng, k, symmetric=False):
    y = rng.standard_normal((k, 3)) * 0.1
    m = rng.uniform(0.5, 1.5, k)
    if symmetric:   # point-symmetric about the com: odd moments vanish
        y = np.concatenate([y, -y]); m = np.concatenate([m, m])
    return y, m


def cell_of(orc, y, m):
    """Moments of a single cell holding all the bodies (float32 storage)."""
    y32, m32 = y.astype(np.float32), m.astype(np.float32)
    k = orc.keys(y32)
    perm = orc.sort(k)
    t = orc.build_tree(k[perm], nleaf=1 << 30)   # the root is a leaf
    M, com, Q = orc.moments(t, y32[perm], m32[perm])
    return y32.astype(np.float64), m32.astype(np.float64), M[0], com[0], Q[0]


@pytest.mark.parametrize("symmetric,order", [(False, 3), (True, 4)])
def test_quadrupole_expansion_order(orc, symmetric, order):
    """Relative error of monopole+quadrupole vs the exact sum falls as
    (s/R)^3 in general and (s/R)^4 when the octupole vanishes; a dropped or
    mis-signed quadrupole term would only give (s/R)^2."""
    rng = np.random.default_rng(11)
    y, m, M, com, Q = cell_of(orc, *cluster(rng, 12, symmetric))
    dirs = W._isotropic(np.random.default_rng(12), 20)
    ratios = []
    for u in dirs:
        errs = []
        for R in (2.0, 4.0, 8.0):
            x = com + R * u
            a, phi = orc.pc_eval(x, com, M, Q, 0.0)
            d = y - x
            r = np.sqrt((d * d).sum(1))
            aex = (m[:, None] * d / r[:, None] ** 3).sum(0)
            errs.append(np.linalg.norm(a - aex) / np.linalg.norm(aex))
        ratios.append(errs[1] / errs[2])
    # median ratio ~ 2^order between R = 4 and R = 8
    assert abs(math.log2(np.median(ratios)) - order) < 0.35


def test_pc_acceleration_is_minus_grad_potential(orc):
    rng = np.random.default_rng(13)
    y, m, M, com, Q = cell_of(orc, *cluster(rng, 9))
    for eps in (0.0, 0.3):
        x = com + np.array([0.7, -0.4, 0.5])
        a, _ = orc.pc_eval(x, com, M, Q, eps)
        h = 1e-5
        g = np.zeros(3)
        for d in range(3):
            e = np.zeros(3); e[d] = h
            g[d] = -(orc.pc_eval(x + e, com, M, Q, eps)[1] - orc.pc_eval(x - e, com, M, Q, eps)[1]) / (2 * h)
        assert np.allclose(a, g, rtol=1e-8, atol=0)


def test_pc_single_body_is_pp(orc):
    y = np.array([[0.3, -0.2, 0.1]])
    m = np.array([0.7])
    _, _, M, com, Q = cell_of(orc, y, m)
    x = np.array([1.0, 2.0, -0.5])
    a, phi = orc.pc_eval(x, com, M, Q, 0.05)
    d = com - x
    r = math.sqrt(d.dot(d) + 0.0025)
    assert np.allclose(a, M * d / r ** 3, rtol=1e-15)
    assert phi == pytest.approx(-M / r, rel=1e-15)


def test_error_decreases_with_theta(orc):
    b = W.plummer(8192, 6)
    idx = W.sample_indices(8192, 1024, 7)
    a_d, p_d = orc.direct(b.pos, b.mass, 0.01, idx)
    p99 = []
    for th in (1.0, 0.75, 0.5, 0.25):
        tf = orc.tree_forces(b.pos, b.mass, th, 0.01)
        e = np.linalg.norm(tf.acc[idx] - a_d, axis=1) / np.linalg.norm(a_d, axis=1)
        p99.append(np.percentile(e, 99))
    assert all(p99[i + 1] < p99[i] for i in range(3)), p99
    assert p99[1] < 1e-2  # theta = 0.75 gate


def test_theta075_accuracy_gates_plummer_32k(orc):
    """Sect. 2 workload (Plummer, theta = 0.75): median <= 1e-3, p99 <= 1e-2
    relative to the FP64 direct sum over a 2048-body sample."""
    b = W.plummer(32768, 0)
    tf = orc.tree_forces(b.pos, b.mass, 0.75, 0.01)
    idx = W.sample_indices(32768, 2048, 1)
    a_d, _ = orc.direct(b.pos, b.mass, 0.01, idx)
    e = np.linalg.norm(tf.acc[idx] - a_d, axis=1) / np.linalg.norm(a_d, axis=1)
    assert np.median(e) <= 1e-3 and np.percentile(e, 99) <= 1e-2
