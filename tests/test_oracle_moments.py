"""Pins of the oracle's multipole moments (Sect. 2, "computation of the
multipole moments"): monopole, centre of mass and traceless quadrupole.

Independent checks: numpy per-cell sums written here from the textbook
definition, the parallel-axis theorem (the combine rule a bottom-up GPU pass
uses) and invariants."""
import numpy as np
import pytest

from paper_1204_2280_gb300 import workloads as W


def setup(orc, n, seed=0, nleaf=16):
    b = W.plummer(n, seed)
    k = orc.keys(b.pos)
    perm = orc.sort(k)
    sp, sm = b.pos[perm], b.mass[perm]
    t = orc.build_tree(k[perm], nleaf)
    return t, sp, sm


def quad_numpy(x, m):
    com = (m[:, None] * x).sum(0) / m.sum()
    y = x - com
    r2 = (y * y).sum(1)
    Q = 3 * np.einsum("n,ni,nj->ij", m, y, y) - np.eye(3) * (m * r2).sum()
    return m.sum(), com, Q


def unpack(q):
    return np.array([[q[0], q[3], q[4]], [q[3], q[1], q[5]], [q[4], q[5], q[2]]])


def test_moments_match_numpy_definition(orc):
    t, sp, sm = setup(orc, 3000, 1)
    M, com, Q = orc.moments(t, sp, sm)
    x64, m64 = sp.astype(np.float64), sm.astype(np.float64)
    for c in range(t.ncells):
        s = slice(t.body_begin[c], t.body_begin[c] + t.body_count[c])
        m, cm, q = quad_numpy(x64[s], m64[s])
        assert abs(M[c] - m) <= 1e-15 * m
        assert np.allclose(com[c], cm, rtol=0, atol=1e-14)
        assert np.allclose(unpack(Q[c]), q, rtol=1e-10, atol=1e-16 * max(1.0, abs(q).max()))


def test_moment_invariants(orc):
    t, sp, sm = setup(orc, 20000, 2)
    M, com, Q = orc.moments(t, sp, sm)
    # root mass and centre of mass
    assert abs(M[0] - sm.astype(np.float64).sum()) < 1e-12
    assert np.allclose(com[0], (sm[:, None].astype(np.float64) * sp).sum(0) / sm.sum(dtype=np.float64), atol=1e-13)
    # traceless
    tr = Q[:, 0] + Q[:, 1] + Q[:, 2]
    assert np.all(np.abs(tr) <= 1e-12 * (np.abs(Q[:, :3]).sum(1) + 1e-300))
    # single-body cells have zero quadrupole
    one = t.body_count == 1
    assert one.any() and np.all(Q[one] == 0)
    # children masses sum to the parent's
    for c in np.nonzero(t.nchild)[0]:
        ch = slice(t.child_begin[c], t.child_begin[c] + t.nchild[c])
        assert abs(M[ch].sum() - M[c]) <= 1e-13 * M[c]


def test_parallel_axis_combine_reproduces_parent(orc):
    """Q_parent = sum_k [Q_k + M_k (3 d_k d_k^T - |d_k|^2 I)], d_k = com_k - com_p."""
    t, sp, sm = setup(orc, 8000, 3)
    M, com, Q = orc.moments(t, sp, sm)
    for c in np.nonzero(t.nchild)[0][:300]:
        ch = range(t.child_begin[c], t.child_begin[c] + t.nchild[c])
        mp = sum(M[k] for k in ch)
        cp = sum(M[k] * com[k] for k in ch) / mp
        qp = np.zeros((3, 3))
        for k in ch:
            d = com[k] - cp
            qp += unpack(Q[k]) + M[k] * (3 * np.outer(d, d) - np.eye(3) * d.dot(d))
        assert np.allclose(cp, com[c], atol=1e-14)
        assert np.allclose(qp, unpack(Q[c]), rtol=1e-9, atol=1e-15)
