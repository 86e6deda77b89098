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
