"""Block (hierarchical) time steps on the GPU (paper Sect. 1 and 3: walk only
the bodies whose step ends; refit the moments between rebuilds) against the
FP64 oracle's block cycle and against the library's own shared step:

* the level rule: bit-exact with the oracle's float32 decision on the same
  accelerations;
* one level is bonsai_step, every body on the finest level is 2^kmax
  bonsai_steps of dt_max / 2^kmax: bit-identical states;
* a cycle with levels 0..3 in use, rebuilt every substep or refitted between
  rebuilds, against the oracle's cycle from the same bodies;
* the counters of a cycle (body steps that ended) against the oracle's;
* argument errors; a refit whose bodies flew far out of their cells (two
  interpenetrating streams) still matches the oracle and the direct sum."""
import numpy as np
import pytest

import oracle
import paper_1204_2280_gb300 as B
from paper_1204_2280_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THETA, EPS = 0.75, 0.01


def make(b, ncrit=32, pack=0):
    bz = B.Bonsai(B.Config(nleaf=16, ncrit=ncrit, group_pack=pack))
    bz.set_bodies(b.pos, b.mass, b.vel)
    B.bonsai_set_params(bz.ctx, THETA, EPS)
    return bz


def state(bz, n):
    x = np.zeros((n, 3), np.float32)
    v = np.zeros((n, 3), np.float32)
    B.bonsai_get_bodies(bz.ctx, x, v)
    bz.sync()
    return x, v


def forces(bz, n):
    acc = np.zeros((n, 3), np.float32)
    pot = np.zeros(n, np.float32)
    bz.build().multipoles().forces(THETA, EPS, acc, pot)
    return acc, pot


def test_level_rule_bit_exact():
    b = W.plummer(20000, 31)
    with make(b) as bz:
        acc, _ = forces(bz, b.n)
        for dt, kmax, eta in ((1.0 / 16, 3, 0.2), (1.0 / 4, 6, 0.05), (1.0, 20, 0.01), (1.0 / 8, 0, 0.3)):
            lev = B.bonsai_block_levels(bz.ctx, dt, kmax, eta)
            want = oracle.block_level(acc, oracle.block_constant(dt, eta, EPS), kmax)
            assert np.array_equal(lev, want), (dt, kmax, eta)
            assert lev.min() >= 0 and lev.max() <= kmax


def test_one_level_is_bonsai_step():
    b = W.plummer(12000, 32)
    with make(b) as bz:
        forces(bz, b.n)
        bz.block_cycle(1.0 / 32, 0, 0.2)
        xb, vb = state(bz, b.n)
    with make(b) as bz:
        forces(bz, b.n)
        bz.step(1.0 / 32)
        xs, vs = state(bz, b.n)
    assert np.array_equal(xb, xs) and np.array_equal(vb, vs)


@pytest.mark.parametrize("pack", [0, 1])
def test_finest_level_is_shared_steps(pack):
    b = W.plummer(12000, 33)
    with make(b, pack=pack) as bz:
        forces(bz, b.n)
        bz.block_cycle(1.0 / 16, 2, 1e-6)
        xb, vb = state(bz, b.n)
    with make(b, pack=pack) as bz:
        forces(bz, b.n)
        for _ in range(4):
            bz.step(1.0 / 64)
        xs, vs = state(bz, b.n)
    assert np.array_equal(xb, xs) and np.array_equal(vb, vs)


@pytest.mark.parametrize("rebuild", [1, 4])
def test_cycle_vs_oracle(rebuild):
    """dt_max = 1/16 in 8 substeps, eta = 0.2 (levels 0..3 in use): GPU
    (float32) and oracle (float64) cycles from the same bodies end within
    the float32 rounding of the trajectory; the few bodies whose level the
    two sides decide differently at a boundary still agree to the scheme's
    own truncation error."""
    b = W.plummer(8192, 34)
    dt, kmax, eta = 1.0 / 16, 3, 0.2
    with make(b) as bz:
        acc, _ = forces(bz, b.n)
        lev_gpu = B.bonsai_block_levels(bz.ctx, dt, kmax, eta)
        bz.block_cycle(dt, kmax, eta, rebuild)
        x, v = state(bz, b.n)
        active, _, _ = B.bonsai_block_stats(bz.ctx)
    a0 = oracle.tree_forces(b.pos, b.mass, THETA, EPS, 16, 32).acc
    ox, ov, oa, op, lev0, nact = oracle.block_cycle(b.pos, b.vel, b.mass, a0, dt, kmax, eta, THETA, EPS,
                                                    16, 32, False, rebuild)
    assert set(np.unique(lev0).tolist()) >= {0, 1, 2, 3}
    same = lev_gpu == lev0
    assert same.mean() > 0.995
    disp = np.linalg.norm(ox - b.pos, axis=1)
    dx = np.linalg.norm(x - ox, axis=1)
    dv = np.linalg.norm(v - ov, axis=1) / np.linalg.norm(ov - b.vel, axis=1)
    assert np.all(dx[same] <= 3e-7 * np.linalg.norm(ox[same], axis=1) + 1e-4 * disp[same])
    assert np.median(dv[same]) <= 1e-4 and np.percentile(dv[same], 99) <= 3e-3
    assert np.all(dx <= 1e-2 * disp + 1e-6)
    assert abs(active - sum(nact)) <= 0.01 * sum(nact)


def test_argument_errors():
    b = W.plummer(1000, 35)
    with make(b) as bz:
        for args in ((0.0, 2, 0.2, 1), (0.1, -1, 0.2, 1), (0.1, 21, 0.2, 1), (0.1, 2, 0.0, 1), (0.1, 2, 0.2, 0)):
            with pytest.raises(B.BonsaiError) as ei:
                B.bonsai_block_cycle(bz.ctx, *args)
            assert ei.value.code == -1
    off = [0, 500, 1000]
    with make(b) as bz:
        bz.set_systems(off)
        with pytest.raises(B.BonsaiError) as ei:
            B.bonsai_block_cycle(bz.ctx, 0.1, 2, 0.2, 1)
        assert ei.value.code == -1


def test_refit_streams_vs_oracle_and_direct_sum():
    """Two interpenetrating streams (x velocities +-20) refitted for 7 of 8
    substeps: the bodies leave the cells they were sorted into, each cell's
    cube is enlarged to hold them, and the cycle still matches the oracle's
    and meets the direct-sum gates at its end."""
    b = W.plummer(16384, 36)
    vel = b.vel.copy()
    vel[:, 0] += np.where(np.arange(b.n) % 2 == 0, 20.0, -20.0).astype(np.float32)
    s = W.Bodies(b.pos, vel, b.mass)
    dt, kmax, eta = 1.0 / 16, 3, 0.1
    with make(s) as bz:
        forces(bz, s.n)
        lev_gpu = B.bonsai_block_levels(bz.ctx, dt, kmax, eta)
        bz.block_cycle(dt, kmax, eta, 8)
        x, v = state(bz, s.n)
        acc, _ = forces(bz, s.n)
    a0 = oracle.tree_forces(s.pos, s.mass, THETA, EPS, 16, 32).acc
    ox, ov, oa, op, lev0, nact = oracle.block_cycle(s.pos, s.vel, s.mass, a0, dt, kmax, eta, THETA, EPS,
                                                    16, 32, False, 8)
    same = lev_gpu == lev0
    assert same.mean() > 0.995
    disp = np.linalg.norm(ox - s.pos, axis=1)
    dx = np.linalg.norm(x - ox, axis=1)
    assert np.percentile(dx[same] / disp[same], 99) <= 1e-4 and np.all(dx <= 1e-2 * disp + 1e-6)
    da, _ = oracle.direct(x, s.mass, EPS)
    e = np.linalg.norm(acc - da, axis=1) / np.linalg.norm(da, axis=1)
    assert np.median(e) <= 1e-3 and np.percentile(e, 99) <= 1e-2


@pytest.mark.parametrize("rebuild", [1, 2, 4])
def test_empty_substeps_only_drift(rebuild):
    """eta = 0.3 leaves level 3 empty (levels 0..2 in use): no step ends at
    an odd substep, which then only drifts.  The GPU walks and rebuilds on
    the oracle's schedule (rebuilds scheduled on odd substeps taken at the
    next even one) and ends within the float32 rounding of the oracle's
    cycle."""
    b = W.plummer(8192, 37)
    dt, kmax, eta = 1.0 / 16, 3, 0.3
    with make(b) as bz:
        acc, _ = forces(bz, b.n)
        lev_gpu = B.bonsai_block_levels(bz.ctx, dt, kmax, eta)
        bz.block_cycle(dt, kmax, eta, rebuild)
        x, v = state(bz, b.n)
        active, _, _ = B.bonsai_block_stats(bz.ctx)
        walked, rebuilt = B.bonsai_block_substeps(bz.ctx)
    a0 = oracle.tree_forces(b.pos, b.mass, THETA, EPS, 16, 32).acc
    ox, ov, oa, op, lev0, nact, o_walked, o_rebuilt = oracle.block_cycle(
        b.pos, b.vel, b.mass, a0, dt, kmax, eta, THETA, EPS, 16, 32, False, rebuild, schedule=True)
    assert set(np.unique(lev0).tolist()) == {0, 1, 2} and nact[0::2] == [0, 0, 0, 0]
    assert o_walked == [2, 4, 6, 8] and (walked, rebuilt) == (len(o_walked), len(o_rebuilt))
    same = lev_gpu == lev0
    assert same.mean() > 0.995
    disp = np.linalg.norm(ox - b.pos, axis=1)
    dx = np.linalg.norm(x - ox, axis=1)
    dv = np.linalg.norm(v - ov, axis=1) / np.linalg.norm(ov - b.vel, axis=1)
    assert np.all(dx[same] <= 3e-7 * np.linalg.norm(ox[same], axis=1) + 1e-4 * disp[same])
    assert np.median(dv[same]) <= 1e-4 and np.percentile(dv[same], 99) <= 3e-3
    assert np.all(dx <= 1e-2 * disp + 1e-6)
    assert abs(active - sum(nact)) <= 0.01 * sum(nact)


def test_every_substep_walked_when_the_finest_level_is_used():
    b = W.plummer(12000, 33)
    with make(b) as bz:
        forces(bz, b.n)
        bz.block_cycle(1.0 / 16, 2, 1e-6, 3)
        assert B.bonsai_block_substeps(bz.ctx) == (4, 2)      # rebuilt at substeps 1 and 4
