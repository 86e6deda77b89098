"""GPU parity and behaviour of the learned far-field correction.

* walk features and direct-sum labels at sampled bodies vs the oracle's
  (features from the oracle tree at the same theta; labels from the FP64
  direct sum): counts exact, logs and unit vectors within 2e-5;
* tensor-core forward vs the FP64 oracle network on the same BF16-rounded
  weights and inputs: max error <= 1e-2 of the output scale;
* GPU gradient vs the oracle's analytic gradient: relative <= 2e-2;
* training lowers the loss; the learned path falls back to the fine walk
  exactly when the judge's p99 exceeds the budget, and the fine walk then
  gives bit-for-bit the plain fine-theta forces;
* the trained network lowers the held-out mean-square residual of the
  coarse walk (its training objective); its 99th percentile stays far above
  the fine walk's, and the judge then falls back to the fine walk, whose
  forces meet the budget."""
import numpy as np
import pytest

import oracle
from oracle import mlp as OM
import paper_1204_2280_gb300 as B
from paper_1204_2280_gb300 import learned as L
from paper_1204_2280_gb300 import workloads as W

from gpu_common import rel_err

pytestmark = pytest.mark.gpu


def test_features_and_labels_vs_oracle():
    b = W.plummer(1 << 15, 2)
    theta, eps = 1.0, 0.01
    with B.Bonsai(B.Config(nleaf=16, ncrit=64)) as bz:
        bz.set_bodies(b.pos, b.mass).build().multipoles()
        X, Y, ids = B.bonsai_learn_samples(bz.ctx, theta, eps, 2048, 5)
    assert len(set(ids.tolist())) == 2048
    tf = oracle.tree_forces(b.pos, b.mass, theta, eps, 16, 64, 2e-6, 1e-6)
    Xo = OM.features(tf, b.pos, eps)[ids]
    ok = ~tf.borderline[ids]
    assert ok.mean() > 0.9
    d = np.abs(X.astype(np.float64) - Xo)[ok]
    assert d[:, 2:7].max() <= 2e-6, d[:, 2:7].max(0)          # interaction counts (exact) in log1p
    assert d[:, [0, 1, 7, 8, 11]].max() <= 2e-5, d.max(0)
    assert d[:, 9:11].max() <= 1e-4, d[:, 9:11].max(0)         # offset within the group box
    a_d, _ = oracle.direct(b.pos, b.mass, eps, ids.astype(np.int64))
    Yo = OM.labels(tf, b.pos, a_d, ids)
    # frame-independent parts: the radial coefficient and the norm across it
    assert np.abs(Y[:, 0] - Yo[:, 0])[ok].max() <= 2e-5
    perp = np.hypot(Y[:, 1], Y[:, 2]) - np.hypot(Yo[:, 1], Yo[:, 2])
    assert np.abs(perp)[ok].max() <= 2e-5


def random_params(seed):
    rng = np.random.default_rng(seed)
    P = (rng.standard_normal(OM.NPARAM) * 0.3).astype(np.float32)
    norm = np.concatenate([rng.standard_normal(12) * 0.2, rng.uniform(0.5, 2.0, 12), [0.05]]).astype(np.float32)
    X = rng.standard_normal((3000, 12)).astype(np.float32)
    Y = (rng.standard_normal((3000, 3)) * 0.05).astype(np.float32)
    return P, norm, X, Y


def test_tensor_core_forward_vs_oracle():
    P, norm, X, _ = random_params(1)
    net = B.MLP(0)
    net.set_params(P, norm)
    y = net.predict(X)
    yo, _ = OM.forward(P.astype(np.float64), norm.astype(np.float64), X)
    scale = np.abs(yo).max()
    assert np.abs(y - yo).max() <= 1e-2 * scale
    assert np.median(np.abs(y - yo)) <= 1e-3 * scale


def test_gradient_vs_oracle():
    P, norm, X, Y = random_params(2)
    net = B.MLP(0)
    net.set_params(P, norm)
    g, loss = net.grad(X, Y)
    lo, go = OM.loss_grad(P.astype(np.float64), norm.astype(np.float64), X, Y)
    assert abs(loss - lo) <= 1e-3 * lo
    assert np.linalg.norm(g - go) <= 2e-2 * np.linalg.norm(go)
    for name, (a, b) in zip(["W1", "b1", "W2", "b2", "W3", "b3"],
                            zip(OM.unpack(g).values(), OM.unpack(go).values())):
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b) + 1e-12, name


def test_training_lowers_loss():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((20000, 12)).astype(np.float32)
    Y = np.stack([np.tanh(X[:, 0] * X[:, 1]), np.sin(X[:, 2]), 0.5 * X[:, 3] ** 2 - 0.5], 1).astype(np.float32) * 0.01
    net = B.MLP(4)
    losses = net.train(X, Y, epochs=30, batch=2048, lr=3e-3, wd=1e-4, seed=5)
    assert losses[-1] < 0.2 * losses[0], losses


def test_fallback_gives_fine_theta_forces():
    b = W.plummer(20000, 6)
    net = B.MLP(0)
    n = b.n
    out = {}
    with B.Bonsai(B.Config(ncrit=64)) as bz:
        bz.set_bodies(b.pos, b.mass).build().multipoles()
        a = np.zeros((n, 3), np.float32)
        bz.forces(0.5, 0.01, a)
        out["plain"] = a.copy()
        for budget, key in ((0.0, "fallback"), (1e30, "learned")):
            B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, budget)
            a = np.zeros((n, 3), np.float32)
            B.bonsai_forces_learned(bz.ctx, 0.01, a)
            p99, fell = B.bonsai_get_judge(bz.ctx)
            out[key] = (a.copy(), p99, fell)
        bz.sync()
    assert out["fallback"][2] and not out["learned"][2]
    assert np.array_equal(out["fallback"][0], out["plain"])
    assert out["learned"][1] == out["fallback"][1]          # same judge input: the coarse + MLP forces


def test_judge_p99_vs_oracle():
    """The judge's p99: relative errors of the current accelerations at the
    sorted positions k*N/4096 (k < 4096) against the FP64 direct sum, 99th
    percentile with linear interpolation between order statistics."""
    b = W.plummer(50000, 12)
    eps = 0.01
    for theta in (1.0, 0.5):
        with B.Bonsai(B.Config(ncrit=64)) as bz:
            bz.set_bodies(b.pos, b.mass).build().multipoles()
            acc = np.zeros((b.n, 3), np.float32)
            bz.forces(theta, eps, acc)
            p = B.bonsai_judge(bz.ctx, eps)
            _, perm = B.bonsai_get_keys(bz.ctx)
            bz.sync()
        ids = perm[(np.arange(4096, dtype=np.int64) * b.n) // 4096].astype(np.int64)
        a_d, _ = oracle.direct(b.pos, b.mass, eps, ids)
        e = rel_err(acc[ids], a_d)
        ref = np.percentile(e, 99)
        assert abs(p - ref) <= 1e-4 * ref, (theta, p, ref)


def test_judge_interval():
    """Interval k judges evaluations 0, k, 2k, ...; a decision holds until the
    next judged evaluation; interval 0 never judges and never falls back."""
    b = W.plummer(20000, 8)
    net = B.MLP(0)
    with B.Bonsai(B.Config(ncrit=64)) as bz:
        bz.set_bodies(b.pos, b.mass).build().multipoles()
        fine = np.zeros((b.n, 3), np.float32)
        bz.forces(0.5, 0.01, fine)
        B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, 0.0)       # any judged evaluation falls back
        B.bonsai_set_judge_interval(bz.ctx, 3)
        seen = []
        for _ in range(4):
            a = np.zeros((b.n, 3), np.float32)
            B.bonsai_forces_learned(bz.ctx, 0.01, a)
            seen.append((B.bonsai_get_judge(bz.ctx)[1], np.array_equal(a, fine)))
        assert seen == [(True, True)] * 4                       # judged at 0 and 3, held at 1 and 2
        B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, 1e30)
        B.bonsai_set_judge_interval(bz.ctx, 2)
        B.bonsai_forces_learned(bz.ctx, 0.01)
        p0 = B.bonsai_get_judge(bz.ctx)
        B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, 0.0)        # resets the count: judged again
        B.bonsai_set_judge_interval(bz.ctx, 2)
        B.bonsai_forces_learned(bz.ctx, 0.01)
        assert B.bonsai_get_judge(bz.ctx) == (p0[0], True)
        B.bonsai_set_judge_interval(bz.ctx, 0)
        for _ in range(2):
            a = np.zeros((b.n, 3), np.float32)
            B.bonsai_forces_learned(bz.ctx, 0.01, a)
            assert not B.bonsai_get_judge(bz.ctx)[1]
            assert not np.array_equal(a, fine)
        with pytest.raises(B.BonsaiError):
            B.bonsai_set_judge_interval(bz.ctx, -1)
        bz.sync()


def test_learned_step_graph_replay_matches_eager():
    b = W.plummer(20000, 7)
    net = B.MLP(1)
    res = []
    for ug in (1, -1):
        with B.Bonsai(B.Config(ncrit=64, use_graph=ug)) as bz:
            bz.set_bodies(b.pos, b.mass, b.vel)
            B.bonsai_set_params(bz.ctx, 0.75, 0.01)
            B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, 1e30)
            for _ in range(3):
                bz.step(1.0 / 128)
            x = np.zeros((b.n, 3), np.float32)
            v = np.zeros((b.n, 3), np.float32)
            B.bonsai_get_bodies(bz.ctx, x, v)
            res.append((x, v, B.bonsai_get_judge(bz.ctx)))
            bz.sync()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2] == res[1][2]


def test_trained_network_gain_and_judged_fallback():
    """At the workload's size (N = 2^22, eps = 0.002): train on 24 randomly
    rotated Plummer spheres (seeds 2000..2023) and 24 rotated snapshots of a
    merger stepped at theta = 0.5, at theta = 1; evaluate on held-out
    systems (Plummer seed 4, the merger of seed 41).  Gain pin: on both the
    correction lowers the 99th-percentile force error of the judge (4096
    bodies, direct sum) below that of plain theta = 1, and on the Plummer
    sphere the mean-square residual it was fit to.  Fallback: with the budget
    between the theta = 0.5 and the learned p99 the judge rejects the coarse +
    learned forces and the fallback walk delivers theta = 0.5 forces within
    the budget; with the budget above the learned p99 it keeps them."""
    n, eps = 1 << 22, 0.002
    plummers = L.snapshots_parallel(n, range(2000, 2024), rot_seed0=8000, workers=8)
    mergers = (L.rotated(m, 8500 + k) for k, m in
               enumerate(L.evolved(W.merger(n, 40), steps=8 * 24, every=8, theta=0.5, eps=eps)))
    X, Y = L.training_set(plummers, theta=1.0, eps=eps, per_snapshot=4096, ncrit=64)
    Xm, Ym = L.training_set(mergers, theta=1.0, eps=eps, per_snapshot=4096, ncrit=64, seed=500)
    X, Y = np.concatenate([X, Xm]), np.concatenate([Y, Ym])
    net, losses = L.train(X, Y, epochs=40, batch=4096, lr=2e-3, wd=1e-4, seed=0)
    assert losses[-1] < losses[0]
    ysig = net.get_params()[1][-1]
    for name, held in (("plummer", W.plummer(n, 4)), ("merger", W.merger(n, 41))):
        with B.Bonsai(B.Config(ncrit=64)) as bz:
            bz.set_bodies(held.pos, held.mass).build().multipoles()
            Xh, Yh, _ = B.bonsai_learn_samples(bz.ctx, 1.0, eps, 4096, 99)
            mse0 = float(np.mean(Yh.astype(np.float64) ** 2))
            mse1 = float(np.mean((Yh - ysig * net.predict(Xh)).astype(np.float64) ** 2))
            bz.forces(1.0, eps)
            p_plain = B.bonsai_judge(bz.ctx, eps)
            B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, 1e30)
            B.bonsai_forces_learned(bz.ctx, eps)
            p_learned, fell = B.bonsai_get_judge(bz.ctx)
            assert not fell
            bz.forces(0.5, eps)
            p_fine = B.bonsai_judge(bz.ctx, eps)
            print(f"{name}: held-out mse {mse0:.4e} -> {mse1:.4e}; p99: theta=1 {p_plain:.4e}  "
                  f"theta=1+MLP {p_learned:.4e}  theta=0.5 {p_fine:.4e}")
            if name == "plummer":
                assert mse1 < mse0
            assert p_learned < p_plain                     # the gain pin
            assert p_fine < p_learned
            budget = (p_fine * p_learned) ** 0.5           # between theta = 0.5 and the learned p99
            B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, budget)
            B.bonsai_forces_learned(bz.ctx, eps)
            p_judged, fell2 = B.bonsai_get_judge(bz.ctx)
            assert fell2 and p_judged == p_learned
            assert B.bonsai_judge(bz.ctx, eps) <= budget
            B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, 1.01 * p_learned)
            B.bonsai_forces_learned(bz.ctx, eps)
            assert B.bonsai_get_judge(bz.ctx) == (p_learned, False)
