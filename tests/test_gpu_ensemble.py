"""Batched ensemble (independent systems in one pipeline): every system must
get exactly what it would get alone, and match the oracle run on it alone.

* bit-for-bit: keys, permutation, tree, groups, forces and two leapfrog steps
  of an ensemble equal those of each system in its own context (the same tree
  and the same traversal order give the same arithmetic);
* per system vs the oracle: domain, keys and permutation, tree topology and
  groups bit-exact; forces <= 1e-5 of the oracle tree (non-borderline
  bodies); errors vs the FP64 direct sum within the theta = 0.75 gates on the
  64-system ensemble (N_k log-uniform in [2^12, 2^18], seeds 100..163)."""
import numpy as np
import pytest

import oracle
import paper_1204_2280_gb300 as B
from paper_1204_2280_gb300 import workloads as W

from gpu_common import edge_bodies, rel_err

pytestmark = pytest.mark.gpu

TAU_ABS, TAU_REL = 2e-6, 1e-6


def concat(systems):
    pos = np.concatenate([s.pos for s in systems])
    vel = np.concatenate([s.vel for s in systems])
    mass = np.concatenate([s.mass for s in systems])
    off = np.cumsum([0] + [s.n for s in systems]).astype(np.int64)
    return pos, vel, mass, off


def run(pos, mass, vel, off, ncrit=32, nleaf=16, theta=0.75, eps=0.01, steps=0, dt=1.0 / 64, pack=0):
    out = {}
    n = mass.shape[0]
    with B.Bonsai(B.Config(nleaf=nleaf, ncrit=ncrit, group_pack=pack)) as bz:
        bz.set_bodies(pos, mass, vel)
        if off is not None:
            bz.set_systems(off)
        bz.build()
        out["keys"], out["perm"] = B.bonsai_get_keys(bz.ctx)
        out["tree"] = B.bonsai_get_tree(bz.ctx)
        out["groups"] = B.bonsai_get_groups(bz.ctx)
        if off is not None:
            out["domains"] = B.bonsai_get_domains(bz.ctx, len(off) - 1)
        bz.multipoles()
        acc = np.zeros((n, 3), np.float32)
        pot = np.zeros(n, np.float32)
        bz.forces(theta, eps, acc, pot)
        out["acc"], out["pot"] = acc, pot
        out["n_pc"], out["n_pp"], _ = B.bonsai_get_counts(bz.ctx)
        for _ in range(steps):
            bz.step(dt)
        if steps:
            x = np.zeros((n, 3), np.float32)
            v = np.zeros((n, 3), np.float32)
            B.bonsai_get_bodies(bz.ctx, x, v)
            out["x"], out["v"] = x, v
        bz.sync()
    return out


def system_cells(tree, lo, hi):
    """Cells of the system owning bodies [lo, hi), renumbered locally."""
    sel = np.nonzero((tree["body_begin"] >= lo) & (tree["body_begin"] < hi))[0]
    local = {int(c): i for i, c in enumerate(sel)}
    t = {k: v[sel].copy() for k, v in tree.items()}
    t["body_begin"] -= lo
    internal = t["nchild"] > 0
    t["child_begin"][internal] = [local[int(c)] for c in t["child_begin"][internal]]
    return t


def small_ensemble():
    sizes = [3000, 17, 1, 20000, 777, 2, 4097]
    systems = [W.plummer(n, 50 + i) for i, n in enumerate(sizes)]
    systems.append(edge_bodies(5000, 9))
    return systems


@pytest.mark.parametrize("ncrit,pack", [(32, 0), (64, 0), (64, 1)])
def test_ensemble_equals_separate_runs_bit_for_bit(ncrit, pack):
    """Also with sibling-packed groups: packing never joins groups of two
    systems, and each system's packed groups are the oracle's."""
    systems = small_ensemble()
    pos, vel, mass, off = concat(systems)
    ens = run(pos, mass, vel, off, ncrit=ncrit, steps=2, pack=pack)
    for s, sysb in enumerate(systems):
        lo, hi = off[s], off[s + 1]
        one = run(sysb.pos, sysb.mass, sysb.vel, None, ncrit=ncrit, steps=2, pack=pack)
        if pack:
            k = oracle.keys(sysb.pos)
            tr = oracle.build_tree(k[oracle.sort(k)], 16)
            ob, oc = oracle.groups(tr, ncrit, pack=True)
            assert np.array_equal(one["groups"][0], ob) and np.array_equal(one["groups"][1], oc)
        assert np.array_equal(ens["keys"][lo:hi], one["keys"])
        assert np.array_equal(ens["perm"][lo:hi] - lo, one["perm"])
        t = system_cells(ens["tree"], lo, hi)
        for f in ("body_begin", "body_count", "child_begin", "nchild", "level"):
            assert np.array_equal(t[f], one["tree"][f]), (s, f)
        gb, gc = ens["groups"]
        sel = (gb >= lo) & (gb < hi)
        assert np.array_equal(gb[sel] - lo, one["groups"][0]) and np.array_equal(gc[sel], one["groups"][1])
        for f in ("acc", "pot", "n_pc", "n_pp", "x", "v"):
            assert np.array_equal(ens[f][lo:hi], one[f]), (s, f)


def test_ensemble_per_system_vs_oracle():
    systems = small_ensemble()
    pos, vel, mass, off = concat(systems)
    ens = run(pos, mass, vel, off, ncrit=64)
    mn_all, side_all = ens["domains"]
    for s, sysb in enumerate(systems):
        lo, hi = off[s], off[s + 1]
        mn, S = oracle.domain(sysb.pos)
        assert np.array_equal(mn_all[s], mn) and side_all[s] == S
        k = oracle.keys(sysb.pos, mn, S)
        perm = oracle.sort(k)
        assert np.array_equal(ens["keys"][lo:hi], k[perm])
        assert np.array_equal(ens["perm"][lo:hi] - lo, perm)
        tr = oracle.build_tree(k[perm], 16)
        t = system_cells(ens["tree"], lo, hi)
        for f in ("body_begin", "body_count", "child_begin", "nchild", "level"):
            assert np.array_equal(t[f], getattr(tr, f)), (s, f)
        tf = oracle.tree_forces(sysb.pos, sysb.mass, 0.75, 0.01, 16, 64, TAU_ABS, TAU_REL)
        ok = ~tf.borderline
        assert rel_err(ens["acc"][lo:hi], tf.acc)[ok].max(initial=0.0) <= 1e-5
        assert np.array_equal(ens["n_pp"][lo:hi][ok], tf.n_pp[ok])


def test_ensemble_64_systems_direct_sum_gates():
    """The 64-system workload: every system's sampled errors vs its own FP64
    direct sum meet median <= 1e-3 and p99 <= 1e-2 at theta = 0.75."""
    systems = W.ensemble(64, 100)
    pos, vel, mass, off = concat(systems)
    ens = run(pos, mass, vel, off, ncrit=64, eps=0.01)
    worst = []
    for s, sysb in enumerate(systems):
        lo, hi = off[s], off[s + 1]
        idx = W.sample_indices(sysb.n, 256, 1000 + s)
        a_d, _ = oracle.direct(sysb.pos, sysb.mass, 0.01, idx)
        e = rel_err(ens["acc"][lo:hi][idx], a_d)
        worst.append((np.median(e), np.percentile(e, 99)))
        assert np.median(e) <= 1e-3 and np.percentile(e, 99) <= 1e-2, (s, sysb.n, worst[-1])


def test_set_systems_rejects_bad_offsets():
    b = W.plummer(100, 1)
    with B.Bonsai(B.Config()) as bz:
        bz.set_bodies(b.pos, b.mass)
        for bad in ([0, 50, 50, 100], [0, 120], [1, 100], [0, 60, 100] + []):
            if bad == [0, 60, 100]:
                continue
            with pytest.raises(B.BonsaiError):
                bz.set_systems(bad)
        bz.set_systems([0, 60, 100])
        bz.build()
