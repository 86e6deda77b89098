"""Pins of the oracle of the learned correction (oracle/mlp.py): bfloat16
rounding against torch's float32 -> bfloat16 conversion and hand-picked
ties, the analytic gradient against central finite differences, a network
whose output is known by hand, and the feature definition's invariants."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_1204_2280_gb300 import workloads as W


def test_bf16_rounding_matches_torch_and_ties():
    import torch
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000)).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), want)
    one = np.float32(1.0)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert M.bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert M.bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6
    assert M.bf16(one) == 1.0


def random_net(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal(M.NPARAM) * scale
    norm = np.concatenate([rng.standard_normal(M.IN) * 0.1, rng.uniform(0.5, 2.0, M.IN), [0.7]])
    X = rng.standard_normal((40, M.IN))
    Y = rng.standard_normal((40, M.OUT)) * 0.3
    return P, norm, X, Y


def test_gradient_matches_finite_differences():
    P, norm, X, Y = random_net(1)
    loss, g = M.loss_grad(P, norm, X, Y, rounded=False)
    rng = np.random.default_rng(2)
    for k in rng.choice(M.NPARAM, 60, replace=False):
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h; Pm[k] -= h
        fd = (M.loss_grad(Pp, norm, X, Y, rounded=False)[0] - M.loss_grad(Pm, norm, X, Y, rounded=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_hand_network():
    """W1 copies inputs 0..2 to hidden 0..2, W2 copies hidden 0..2, W3 reads
    them back: y = relu(bf16(x))[:3] + b3."""
    d = {n: np.zeros(s) for n, s in M.SHAPES}
    for k in range(3):
        d["W1"][k, k] = 1.0
        d["W2"][k, k] = 1.0
        d["W3"][k, k] = 1.0
    d["b3"][:] = [0.25, -0.5, 1.0]
    norm = np.concatenate([np.zeros(M.IN), np.ones(M.IN), [1.0]])
    X = np.zeros((2, M.IN))
    X[0, :3] = [1.5, -2.0, 0.3]
    X[1, :3] = [-1.0, 4.0, 1.0 / 3.0]
    y, _ = M.forward(M.pack(d), norm, X)
    want = np.maximum(M.bf16(X[:, :3]), 0) + d["b3"]
    assert np.array_equal(y, want)
    assert y[0, 1] == -0.5 and y[1, 0] == 0.25


def test_features_invariants(orc):
    b = W.plummer(6000, 3)
    tf = orc.tree_forces(b.pos, b.mass, 1.0, 0.01, 16, 64)
    X = M.features(tf, b.pos, 0.01)
    assert np.array_equal(tf.npc_bins.sum(1), tf.n_pc)
    assert np.allclose(np.expm1(X[:, 2:6]).sum(1), tf.n_pc)
    assert np.allclose(np.expm1(X[:, 6]), tf.n_pp)
    assert np.all(X[:, 9] <= 1.0 + 1e-12) and np.all(np.abs(X[:, 10]) <= 1.0 + 1e-12)
    # bodies of one group share the group features
    for g in range(0, len(tf.gbeg), 97):
        ids = tf.perm[tf.gbeg[g]: tf.gbeg[g] + tf.gcnt[g]]
        assert np.all(X[ids][:, 2:9] == X[ids[0], 2:9]) and np.all(X[ids, 11] == X[ids[0], 11])


def test_frame_is_orthonormal_and_rotates_with_the_system(orc):
    """Features are rotation invariant and the frame rotates with the system,
    so a correction expressed in it is equivariant."""
    from paper_1204_2280_gb300.learned import rotated
    b = W.plummer(3000, 4)
    tf = orc.tree_forces(b.pos, b.mass, 1.0, 0.01, 16, 64)
    _, _, g, off = M._groups(tf, b.pos)
    e0, e1, e2 = M.frame(tf.acc, off)
    E = np.stack([e0, e1, e2], 1)
    assert np.allclose(E @ E.transpose(0, 2, 1), np.eye(3), atol=1e-12)
    assert np.allclose(np.cross(e0, e1), e2)
    X = M.features(tf, b.pos, 0.01)
    # group-box features are not exactly invariant (boxes are axis-aligned):
    # only the counts and the acceleration/potential must match closely
    rb = rotated(b, 11)
    tr = orc.tree_forces(rb.pos, rb.mass, 0.02, 0.01, 16, 64)
    t0 = orc.tree_forces(b.pos, b.mass, 0.02, 0.01, 16, 64)
    assert np.allclose(np.linalg.norm(tr.acc, axis=1), np.linalg.norm(t0.acc, axis=1), rtol=1e-5)


# ---------------------------------------------------------------------------
# Hand-computed pins of features() and labels(): a tiny hand-built "tree
# evaluation" whose group boxes, accelerations, potentials and counts are
# chosen by hand, so that every column has a value written out below from
# those numbers alone (not from the oracle's code).
# ---------------------------------------------------------------------------

class _HandEval:
    """Stand-in for oracle.TreeForces with just the fields features() and
    labels() read: two groups of three bodies, caller order = sorted order."""

    def __init__(self):
        self.perm = np.arange(6)
        self.gbeg = np.array([0, 3])
        self.gcnt = np.array([3, 3])
        self.group_of = np.array([0, 0, 0, 1, 1, 1])
        self.acc = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, -2.0], [1.0, 0.0, 0.0],
                             [0.0, 6.0, 8.0], [2.0, 0.0, 0.0], [0.0, 0.0, -4.0]])
        self.pot = np.array([-2.0, -0.5, -1.0, -3.0, -0.25, -4.0])
        self.npc_bins = np.array([[1, 2, 3, 4], [0, 0, 0, 0], [7, 0, 1, 0],
                                  [2, 2, 2, 2], [0, 5, 0, 9], [1, 1, 1, 1]])
        self.n_pc = self.npc_bins.sum(1)
        self.n_pp = np.array([10, 0, 3, 30, 1, 2])


# group 0: box [0,1] x [0,2] x [0,0.5] (extents 1, 2, 0.5; centre (0.5, 1, 0.25));
# group 1: box [4,4.25] x [4,4.5] x [4,4] (extents 0.25, 0.5, 0; centre (4.125, 4.25, 4))
HAND_POS = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 0.5], [0.5, 1.0, 0.25],
                     [4.0, 4.0, 4.0], [4.0, 4.5, 4.0], [4.25, 4.0, 4.0]], np.float32)


def test_features_hand_computed_columns():
    import math
    eps = 0.01
    X = M.features(_HandEval(), HAND_POS, eps)
    # column 0: log|a|; |a| = 5, 2, 1, 10, 2, 4
    assert np.allclose(X[:, 0], np.log([5.0, 2.0, 1.0, 10.0, 2.0, 4.0]), rtol=0, atol=1e-14)
    # column 1: log(-phi)
    assert np.allclose(X[:, 1], np.log([2.0, 0.5, 1.0, 3.0, 0.25, 4.0]), rtol=0, atol=1e-14)
    # columns 2..6: log(1 + count)
    assert np.allclose(X[0, 2:7], np.log([2.0, 3.0, 4.0, 5.0, 11.0]), rtol=0, atol=1e-14)
    assert np.allclose(X[4, 2:7], np.log([1.0, 6.0, 1.0, 10.0, 2.0]), rtol=0, atol=1e-14)
    # column 7: log(n_G / (e_G^3 + eps^3)), e_G the LARGEST extent (2 and 0.5)
    g0 = math.log(3.0 / (2.0 ** 3 + eps ** 3))
    g1 = math.log(3.0 / (0.5 ** 3 + eps ** 3))
    assert np.allclose(X[:, 7], [g0] * 3 + [g1] * 3, rtol=0, atol=1e-12)
    # column 8: log((d_G + eps) / eps), d_G the box diagonal: sqrt(5.25), sqrt(0.3125)
    d0, d1 = math.sqrt(1 + 4 + 0.25), math.sqrt(0.0625 + 0.25)
    assert np.allclose(X[:, 8], [math.log((d0 + eps) / eps)] * 3 + [math.log((d1 + eps) / eps)] * 3,
                       rtol=0, atol=1e-12)
    # column 9: |o| / (d_G / 2); body 0 and 1 sit on box corners (1), body 2 at the centre (0)
    o4 = math.sqrt(0.125 ** 2 + 0.25 ** 2)      # body 4: offset (-0.125, 0.25, 0)
    assert np.allclose(X[:, 9], [1.0, 1.0, 0.0, 1.0, o4 / (d1 / 2), 1.0], rtol=0, atol=1e-12)
    # column 10: cos(o, a); body 0: o = (-0.5, -1, -0.25), a = (3, 4, 0)
    c0 = (-1.5 - 4.0) / (math.sqrt(1.3125) * 5.0)
    # body 1: o = (0.5, 1, 0.25), a = (0, 0, -2); body 2: o = 0 (cos 0 by definition)
    c1 = -0.5 / (math.sqrt(1.3125) * 2.0)
    # body 4: o = (-0.125, 0.25, 0), a = (2, 0, 0)
    c4 = -0.25 / (o4 * 2.0)
    assert np.allclose(X[[0, 1, 2, 4], 10], [c0, c1, 0.0, c4], rtol=0, atol=1e-12)
    # column 11: log n_G
    assert np.allclose(X[:, 11], math.log(3.0), rtol=0, atol=1e-14)


def test_labels_hand_computed_frame_coefficients():
    """A known residual in a known frame: body 4 has a = (2, 0, 0) and box
    offset o = (-0.125, 0.25, 0), so e0 = x, e1 = y, e2 = z; body 5 has
    a = (0, 0, -4) and o = (0.125, -0.25, 0), so e0 = -z, e1 = (0.125, -0.25,
    0)/|.|, e2 = e0 x e1.  r = (a_direct - a) / |a| (the TREE force's norm)."""
    import math
    tf = _HandEval()
    a_dir = np.array([[2.2, -0.4, 0.6], [0.4, -0.8, -4.4]])
    Y = M.labels(tf, HAND_POS, a_dir, np.array([4, 5]))
    assert np.allclose(Y[0], [0.1, -0.2, 0.3], rtol=0, atol=1e-14)
    # body 5: r = (0.1, -0.2, -0.1), e1 = (1, -2, 0)/sqrt5, e2 = (-z) x e1 = (-2, -1, 0)/sqrt5
    s5 = math.sqrt(5.0)
    want = [0.1, (0.1 * 1 + 0.2 * 2) / s5, (-0.1 * 2 + 0.2 * 1) / s5]
    assert np.allclose(Y[1], want, rtol=0, atol=1e-14)


def test_frame_degenerate_offset_takes_least_aligned_axis():
    """o = 0 or o along a: e1 is the first least-aligned coordinate axis made
    orthogonal to e0."""
    a = np.array([[0.0, 0.0, 3.0], [1.0, 1.0, 0.0], [0.0, 2.0, 0.0]])
    off = np.array([[0.0, 0.0, 0.0], [2.0, 2.0, 0.0], [0.0, 0.0, 0.0]])
    e0, e1, e2 = M.frame(a, off)
    assert np.allclose(e1[0], [1.0, 0.0, 0.0])            # a along z: x is least aligned
    assert np.allclose(e1[1], [0.0, 0.0, 1.0])            # a in the xy plane: z
    assert np.allclose(e1[2], [1.0, 0.0, 0.0])
    assert np.allclose(e2[0], [0.0, 1.0, 0.0])            # z x x = y


def test_second_relu_is_applied():
    """A hidden unit driven negative by layer 2 contributes nothing."""
    d = {n: np.zeros(s) for n, s in M.SHAPES}
    d["W1"][0, 0] = 1.0
    d["W2"][0, 0] = -1.0      # z2 = -h1 < 0 -> relu -> 0
    d["W2"][1, 0] = 2.0       # z2 = 2 h1
    d["W3"][0, 0] = 1.0
    d["W3"][1, 1] = 1.0
    norm = np.concatenate([np.zeros(M.IN), np.ones(M.IN), [1.0]])
    X = np.zeros((1, M.IN))
    X[0, 0] = 1.5
    y, _ = M.forward(M.pack(d), norm, X)
    assert y[0, 0] == 0.0 and y[0, 1] == 3.0 and y[0, 2] == 0.0
