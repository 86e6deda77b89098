"""Pins of the oracle's block (hierarchical) time steps (paper Sect. 1 and 3:
only the N_active bodies whose step ends are walked; between rebuilds only
the moments are recomputed).

The scheme reduces exactly to the shared-step leapfrog in two limits (one
level; every body on the finest level), which the physics pins already tie
to closed forms; the masked walk reduces to the direct sum at theta -> 0;
the float32 level rule agrees with its float64 definition away from level
boundaries; energy is conserved with a real spread of levels."""
import numpy as np
import pytest

from paper_1204_2280_gb300 import workloads as W


def start(orc, n, seed, theta, eps, ncrit=32):
    b = W.plummer(n, seed)
    tf = orc.tree_forces(b.pos, b.mass, theta, eps, 16, ncrit)
    return b, tf.acc


def test_one_level_is_the_shared_kdk_step(orc):
    b, a0 = start(orc, 3000, 21, 0.75, 0.01)
    dt = 1.0 / 64
    x, v, a, pot, lev0, nact = orc.block_cycle(b.pos, b.vel, b.mass, a0, dt, 0, 0.1, 0.75, 0.01)
    x1, v1, a1, p1 = orc.kdk_step(b.pos, b.vel, b.mass, a0, dt, 0.75, 0.01)
    assert np.all(lev0 == 0) and nact == [3000]
    assert np.array_equal(x, x1) and np.array_equal(v, v1) and np.array_equal(a, a1)
    assert np.array_equal(pot, p1)


@pytest.mark.parametrize("kmax", [1, 3])
def test_all_on_the_finest_level_is_shared_steps_of_dt_min(orc, kmax):
    """eta tiny: every body takes level kmax, so one cycle is 2^kmax shared
    KDK steps of dt_max / 2^kmax (consecutive closing and opening half kicks
    are the two half kicks of neighbouring steps)."""
    b, a0 = start(orc, 2500, 22, 0.75, 0.01)
    dt = 1.0 / 16
    x, v, a, pot, lev0, nact = orc.block_cycle(b.pos, b.vel, b.mass, a0, dt, kmax, 1e-6, 0.75, 0.01)
    assert np.all(lev0 == kmax) and nact == [2500] * (1 << kmax)
    xs, vs, as_ = np.asarray(b.pos, np.float64), np.asarray(b.vel, np.float64), a0
    for _ in range(1 << kmax):
        xs, vs, as_, ps = orc.kdk_step(xs, vs, b.mass, as_, dt / (1 << kmax), 0.75, 0.01)
    assert np.array_equal(x, xs) and np.array_equal(v, vs) and np.array_equal(a, as_)


def test_level_rule_matches_its_float64_definition(orc):
    """Smallest k with dt_max / 2^k <= eta sqrt(eps / |a|), capped at kmax,
    away from level boundaries (the float32 decision may differ within
    rounding of a boundary)."""
    rng = np.random.default_rng(5)
    a = (rng.standard_normal((20000, 3)) * 10.0 ** rng.uniform(-3, 3, (20000, 1))).astype(np.float32)
    dt, eta, eps, kmax = 1.0 / 32, 0.2, 0.01, 6
    k = orc.block_level(a, orc.block_constant(dt, eta, eps), kmax)
    amag = np.linalg.norm(a.astype(np.float64), axis=1)
    want_real = np.log2(dt / (eta * np.sqrt(eps / amag)))     # k >= this
    want = np.clip(np.ceil(want_real), 0, kmax).astype(int)
    far = np.abs(want_real - np.round(want_real)) > 1e-5
    assert np.array_equal(k[far], want[far])
    assert k.min() == 0 and k.max() == kmax                      # the sample spans all levels
    assert np.all(orc.block_level(np.zeros((3, 3), np.float32), 1e30, kmax) == 0)


def test_masked_walk_is_the_direct_sum_for_active_bodies(orc):
    b = W.plummer(2000, 23)
    pos = b.pos
    mn, S = orc.domain(pos)
    k = orc.keys(pos, mn, S)
    perm = orc.sort(k)
    tree = orc.build_tree(k[perm], 16)
    gb, gc = orc.groups(tree, 32)
    sp, sm = np.ascontiguousarray(pos[perm]), np.ascontiguousarray(b.mass[perm])
    M, com, Q = orc.moments(tree, sp, sm)
    ro = orc.open_radius(tree, k[perm], mn, S, com, 1e-9)
    act = np.random.default_rng(1).random(2000) < 0.3
    acc, pot, npc, npp, _ = orc.walk(sp, sm, tree, M, com, Q, ro, gb, gc, 0.01, active=act)
    da, dp = orc.direct(sp, sm, 0.01)
    assert np.abs(acc[act] - da[act]).max() <= 1e-9 * np.abs(da).max()
    assert np.abs(pot[act] - dp[act]).max() <= 1e-9 * np.abs(dp).max()
    assert np.all(acc[~act] == 0) and np.all(npp[act] == 1999)


def test_energy_with_a_spread_of_levels(orc):
    """Four cycles with levels 0..3 in use: the energy error lies between
    those of the shared step at the finest and at the coarsest dt (most
    bodies take the coarse levels; the few with large accelerations the fine
    ones)."""
    n, eps, theta = 4000, 0.01, 0.5
    b, a0 = start(orc, n, 24, theta, eps)
    dt, kmax, eta = 1.0 / 16, 3, 0.2
    tf0 = orc.tree_forces(b.pos, b.mass, theta, eps, 16, 32)
    e0 = orc.energy(b.pos, b.vel, b.mass, tf0.pot)[2]
    x, v, a = b.pos.astype(np.float64), b.vel.astype(np.float64), a0
    levels = set()
    for _ in range(4):
        x, v, a, pot, lev0, nact = orc.block_cycle(x, v, b.mass, a, dt, kmax, eta, theta, eps)
        levels |= set(np.unique(lev0).tolist())
    d_block = abs(orc.energy(x.astype(np.float32), v.astype(np.float32), b.mass, pot)[2] - e0)

    def shared(h, steps):
        xs, vs, as_ = b.pos.astype(np.float64), b.vel.astype(np.float64), a0
        for _ in range(steps):
            xs, vs, as_, ps = orc.kdk_step(xs, vs, b.mass, as_, h, theta, eps)
        return abs(orc.energy(xs.astype(np.float32), vs.astype(np.float32), b.mass, ps)[2] - e0)

    d_fine, d_coarse = shared(dt / (1 << kmax), 4 << kmax), shared(dt, 4)
    assert levels >= {0, 1, 2, 3}
    assert d_fine < d_block < d_coarse


def test_refit_between_rebuilds_stays_close(orc):
    """Moments recomputed on the cells of the last rebuild (rebuilt every 4
    substeps) track rebuilding every substep to the tree's own accuracy."""
    b, a0 = start(orc, 3000, 25, 0.75, 0.01)
    args = (b.pos, b.vel, b.mass, a0, 1.0 / 16, 3, 0.2, 0.75, 0.01)
    x1, v1, a1, p1, l1, n1 = orc.block_cycle(*args, rebuild_every=1)
    x4, v4, a4, p4, l4, n4 = orc.block_cycle(*args, rebuild_every=4)
    assert np.array_equal(l1, l4)
    disp = np.linalg.norm(x1 - b.pos, axis=1)
    dx = np.linalg.norm(x4 - x1, axis=1) / disp
    assert np.percentile(dx, 99) <= 5e-4 and dx.max() <= 5e-3
    rel = np.linalg.norm(a4 - a1, axis=1) / np.linalg.norm(a1, axis=1)
    assert np.median(rel) <= 1e-3 and np.percentile(rel, 99) <= 2e-2


def test_refit_extent_bounds_every_body(orc):
    """At the build positions each cell's extent is l/2 exactly; after a
    drift it bounds (max-norm about the build-time centre) every body of the
    cell, exactly so for leaves; brute force over all cells."""
    b = W.plummer(3000, 26)
    mn, S = orc.domain(b.pos)
    k = orc.keys(b.pos, mn, S)
    perm = orc.sort(k)
    tree = orc.build_tree(k[perm], 8)
    sp = np.ascontiguousarray(b.pos[perm])
    ctr, side = orc.cell_cube(tree, k[perm], mn, S)
    assert np.array_equal(orc.refit_extent(tree, k[perm], mn, S, sp), side / 2)
    moved = (sp + np.random.default_rng(3).standard_normal(sp.shape) * 0.05).astype(np.float32)
    ext = orc.refit_extent(tree, k[perm], mn, S, moved)
    for c in range(tree.ncells):
        bb, bc = tree.body_begin[c], tree.body_count[c]
        far = np.abs(moved[bb:bb + bc].astype(np.float64) - ctr[c]).max()
        assert ext[c] >= far and ext[c] >= side[c] / 2
        if tree.nchild[c] == 0:
            assert ext[c] == max(far, side[c] / 2)


def test_refit_streams_stay_accurate(orc):
    """Two interpenetrating streams (x velocities +-20) refitted for 7 of 8
    substeps: the enlarged cubes keep every walked body's own cells opened,
    and the accelerations at the end meet the direct-sum gates."""
    b = W.plummer(8192, 36)
    vel = b.vel.copy()
    vel[:, 0] += np.where(np.arange(b.n) % 2 == 0, 20.0, -20.0).astype(np.float32)
    a0 = orc.tree_forces(b.pos, b.mass, 0.75, 0.01, 16, 32).acc
    x, v, a, pot, lev0, nact = orc.block_cycle(b.pos, vel, b.mass, a0, 1.0 / 16, 3, 0.1, 0.75, 0.01,
                                               16, 32, False, 8)
    da, _ = orc.direct(x.astype(np.float32), b.mass, 0.01)
    e = np.linalg.norm(a - da, axis=1) / np.linalg.norm(da, axis=1)
    assert np.median(e) <= 1e-3 and np.percentile(e, 99) <= 1e-2


def test_every_body_ends_the_cycle_synchronised(orc):
    """With levels 0..3 in use, the steps each body completes in one cycle
    add up to dt_max exactly, and a body walked at substep s had a step
    ending there (s a multiple of its step length in substeps)."""
    b, a0 = start(orc, 3000, 27, 0.75, 0.01)
    dt, kmax = 1.0 / 16, 3
    out = orc.block_cycle(b.pos, b.vel, b.mass, a0, dt, kmax, 0.2, 0.75, 0.01, clock=True)
    lev0, nact, t_done = out[4], out[5], out[6]
    assert set(np.unique(lev0).tolist()) >= {0, 1, 2, 3}
    assert np.all(t_done == dt)
    # every body is active at the last substep; some substeps walk a subset only
    assert nact[-1] == 3000 and min(nact) < 3000


@pytest.mark.parametrize("rebuild", [1, 2])
def test_an_empty_finest_level_is_the_coarser_cycle(orc, rebuild):
    """Levels 0..2 in use and none on level 3: a cycle with max level 3 has
    no step ending at an odd substep, so it drifts through those and must be
    the cycle with max level 2 (same dt_max) up to the split of each drift
    in two.  The rebuilds scheduled for its odd substeps (every 2r-th
    substep from the first) are taken at the even ones that follow, which
    makes them the coarse cycle's every r-th."""
    b, a0 = start(orc, 3000, 28, 0.75, 0.01)
    dt, eta = 1.0 / 16, 0.3
    fine = orc.block_cycle(b.pos, b.vel, b.mass, a0, dt, 3, eta, 0.75, 0.01,
                           rebuild_every=2 * rebuild, schedule=True)
    coarse = orc.block_cycle(b.pos, b.vel, b.mass, a0, dt, 2, eta, 0.75, 0.01,
                             rebuild_every=rebuild, schedule=True)
    assert set(np.unique(fine[4]).tolist()) == {0, 1, 2}
    assert fine[5][0::2] == [0, 0, 0, 0] and fine[5][1::2] == coarse[5]
    assert fine[6] == [2, 4, 6, 8] and fine[7] == [2 * s for s in coarse[7]]
    assert coarse[7] == ([1, 2, 3, 4] if rebuild == 1 else [1, 3])
    for f, c in zip(fine[:4], coarse[:4]):
        assert np.abs(f - c).max() <= 1e-9 * np.abs(c).max()
    assert np.array_equal(fine[4], coarse[4])
