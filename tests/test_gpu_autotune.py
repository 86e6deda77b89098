"""The autotuner picks a group size, a group rule (sibling packing or not),
a walk block width and a walk stack capacity by timing the walk; the tuned
context must compute exactly what a context configured with that choice by
hand computes (neither the block width nor the capacity changes the
arithmetic)."""
import numpy as np
import pytest

import paper_1204_2280_gb300 as B
from paper_1204_2280_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def forces(bz, n):
    acc = np.zeros((n, 3), np.float32)
    pot = np.zeros(n, np.float32)
    bz.forces(0.75, 0.01, acc, pot)
    return acc, pot


def test_autotune_result_is_consistent():
    b = W.plummer(1 << 15, 3)
    with B.Bonsai(B.Config()) as bz:
        bz.set_bodies(b.pos, b.mass, b.vel)
        nc, w, ms = B.bonsai_autotune(bz.ctx, 0.75, 0.01)
        assert nc in (16, 32, 48, 64) and w in (2, 4, 8) and ms > 0
        cfg = B.bonsai_get_config(bz.ctx)
        assert (cfg.ncrit, cfg.walk_warps) == (nc, w) and cfg.group_pack in (0, 1)
        assert cfg.list_capacity in (128, 256, 512)
        a1, p1 = forces(bz, b.n)
        bz.step(1.0 / 64)
        bz.sync()
    with B.Bonsai(B.Config(ncrit=nc, walk_warps=w, group_pack=cfg.group_pack,
                           list_capacity=cfg.list_capacity)) as bz:
        bz.set_bodies(b.pos, b.mass, b.vel).build().multipoles()
        a2, p2 = forces(bz, b.n)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)


@pytest.mark.parametrize("w,cap", [(1, 256), (2, 128), (8, 512), (4, 128)])
def test_walk_block_width_does_not_change_results(w, cap):
    b = W.plummer(20000, 4)
    out = []
    for ww, cc in ((4, 256), (w, cap)):
        with B.Bonsai(B.Config(ncrit=64, walk_warps=ww, list_capacity=cc)) as bz:
            bz.set_bodies(b.pos, b.mass).build().multipoles()
            out.append(forces(bz, b.n))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
