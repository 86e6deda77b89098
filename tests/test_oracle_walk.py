"""Pins of the oracle's opening criterion and traversal (Sect. 2: MAC after
Barnes 1994 combined with the group walk of Barnes 1990).

* the geometric cube of a cell (side S / 2^level, centre from the key prefix)
  contains all of the cell's bodies and its centre of mass;
* r_open(theta) = l / theta + delta: differences across theta give l exactly
  and delta = r_open - l/theta is the com's distance to the cube centre;
* a body's own leaf is always opened for theta < 2/sqrt(3);
* brute force: a recursive depth-first Python walk over the same tree,
  moments and opening radii reproduces the breadth-first oracle's
  accelerations, potentials and interaction counts."""
import math

import numpy as np
import pytest

from paper_1204_2280_gb300 import workloads as W


def prep(orc, n, seed, nleaf=16):
    b = W.plummer(n, seed)
    mn, S = orc.domain(b.pos)
    k = orc.keys(b.pos, mn, S)
    perm = orc.sort(k)
    sk, sp, sm = k[perm], b.pos[perm], b.mass[perm]
    t = orc.build_tree(sk, nleaf)
    M, com, Q = orc.moments(t, sp, sm)
    return b, mn, S, sk, sp, sm, t, M, com, Q


def test_cell_cube_contains_bodies(orc):
    b, mn, S, sk, sp, sm, t, M, com, Q = prep(orc, 5000, 0)
    ctr, side = orc.cell_cube(t, sk, mn, S)
    assert np.array_equal(side, S / 2.0 ** t.level)
    for c in range(t.ncells):
        x = sp[t.body_begin[c]: t.body_begin[c] + t.body_count[c]].astype(np.float64)
        assert np.all(x >= ctr[c] - side[c] / 2) and np.all(x < ctr[c] + side[c] / 2)
        assert np.all(np.abs(com[c] - ctr[c]) <= side[c] / 2)
    assert np.allclose(ctr[0], mn.astype(np.float64) + S / 2)


def test_open_radius_structure(orc):
    b, mn, S, sk, sp, sm, t, M, com, Q = prep(orc, 3000, 1)
    ctr, side = orc.cell_cube(t, sk, mn, S)
    r1 = orc.open_radius(t, sk, mn, S, com, 1.0)
    r5 = orc.open_radius(t, sk, mn, S, com, 0.5)
    assert np.allclose(r5 - r1, side, rtol=1e-12)
    delta = np.linalg.norm(com - ctr, axis=1)
    assert np.allclose(r1 - side, delta, rtol=1e-9, atol=1e-14)


def brute_walk(sp, sm, t, M, com, Q, ro, gb, gc, eps):
    n = sp.shape[0]
    x = sp.astype(np.float64); m = sm.astype(np.float64)
    acc = np.zeros((n, 3)); pot = np.zeros(n)
    npc = np.zeros(n, int); npp = np.zeros(n, int)
    for g0, g1 in zip(gb, gb + gc):
        lo, hi = x[g0:g1].min(0), x[g0:g1].max(0)
        accepted, leaves = [], []

        def visit(c):
            d = np.maximum(0, np.maximum(lo - com[c], com[c] - hi))
            if d.dot(d) < ro[c] ** 2:
                if t.nchild[c] == 0:
                    leaves.append(c)
                else:
                    for ch in range(t.child_begin[c], t.child_begin[c] + t.nchild[c]):
                        visit(ch)
            else:
                accepted.append(c)
        visit(0)
        for i in range(g0, g1):
            for c in accepted:
                dv = com[c] - x[i]
                r = math.sqrt(dv.dot(dv) + eps * eps)
                q6 = Q[c]
                Qm = np.array([[q6[0], q6[3], q6[4]], [q6[3], q6[1], q6[5]], [q6[4], q6[5], q6[2]]])
                qd = Qm @ dv
                q = dv.dot(qd)
                acc[i] += M[c] * dv / r ** 3 - qd / r ** 5 + 2.5 * q * dv / r ** 7
                pot[i] -= M[c] / r + 0.5 * q / r ** 5
            for c in leaves:
                for j in range(t.body_begin[c], t.body_begin[c] + t.body_count[c]):
                    if j != i:
                        dv = x[j] - x[i]
                        r = math.sqrt(dv.dot(dv) + eps * eps)
                        acc[i] += m[j] * dv / r ** 3
                        pot[i] -= m[j] / r
                        npp[i] += 1
            npc[i] = len(accepted)
    return acc, pot, npc, npp


@pytest.mark.parametrize("theta,nleaf,ncrit", [(0.75, 16, 32), (1.0, 4, 8), (0.4, 8, 64)])
def test_walk_matches_recursive_brute_force(orc, theta, nleaf, ncrit):
    b, mn, S, sk, sp, sm, t, M, com, Q = prep(orc, 400, 2, nleaf)
    ro = orc.open_radius(t, sk, mn, S, com, theta)
    gb, gc = orc.groups(t, ncrit)
    acc, pot, npc, npp, _ = orc.walk(sp, sm, t, M, com, Q, ro, gb, gc, 0.01)
    a2, p2, c2, q2 = brute_walk(sp, sm, t, M, com, Q, ro, gb, gc, 0.01)
    assert np.array_equal(npc, c2) and np.array_equal(npp, q2)
    assert np.allclose(acc, a2, rtol=1e-12, atol=1e-12 * np.abs(a2).max())
    assert np.allclose(pot, p2, rtol=1e-12)
    if theta >= 0.75:
        assert npc.sum() > 0


def test_own_leaf_always_opened(orc):
    b = W.plummer(2000, 3)
    for th in (0.3, 1.0, 1.15):
        tf = orc.tree_forces(b.pos, b.mass, th, 0.01, nleaf=4, ncrit=16)
        assert tf.n_pp.min() >= 0


@pytest.mark.parametrize("ncrit", [16, 64])
def test_packed_groups_walk_reduces_to_direct_sum(orc, ncrit):
    """With sibling-packed groups the walk at theta -> 0 still opens every
    cell, so it is the direct sum to rounding; at theta = 0.75 it meets the
    direct-sum gates and takes fewer groups than the unpacked rule."""
    b = W.plummer(3000, 12)
    tf = orc.tree_forces(b.pos, b.mass, theta=1e-9, eps=0.01, nleaf=16, ncrit=ncrit, pack=True)
    da, dp = orc.direct(b.pos, b.mass, 0.01)
    assert np.abs(tf.acc - da).max() <= 1e-9 * np.abs(da).max()
    assert np.abs(tf.pot - dp).max() <= 1e-9 * np.abs(dp).max()
    assert np.all(tf.n_pp == 2999) and np.all(tf.n_pc == 0)
    t75 = orc.tree_forces(b.pos, b.mass, 0.75, 0.01, 16, ncrit, pack=True)
    u75 = orc.tree_forces(b.pos, b.mass, 0.75, 0.01, 16, ncrit)
    e = np.linalg.norm(t75.acc - da, axis=1) / np.linalg.norm(da, axis=1)
    assert np.median(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2
    assert len(t75.gbeg) < len(u75.gbeg)
