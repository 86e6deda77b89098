"""Neighbour search and SPH density on the octree (paper Sect. 3) against
the oracle's O(N^2) definition: neighbour counts bit-exact (both sides take
the float32 decision r^2 < h^2 with the same fused r^2), densities within
2e-5 relative (float32 sums against float64), for random, constant and
density-adapted smoothing lengths, every group layout (ncrit 16/32/64,
packed or not), host and device buffers, the extremes (every body a
neighbour; only itself), duplicate positions, and refusal after a block
cycle that ended on a refit."""
import numpy as np
import pytest

import oracle
import paper_1204_2280_gb300 as B
from paper_1204_2280_gb300 import workloads as W

from gpu_common import edge_bodies

pytestmark = pytest.mark.gpu


def run(b, h, ncrit=32, pack=0, device=True):
    import torch
    with B.Bonsai(B.Config(nleaf=16, ncrit=ncrit, group_pack=pack)) as bz:
        bz.set_bodies(b.pos, b.mass, b.vel).build()
        if device:
            th = torch.from_numpy(np.ascontiguousarray(h, np.float32)).cuda()
            rho = torch.zeros(b.n, dtype=torch.float32, device="cuda")
            cnt = torch.zeros(b.n, dtype=torch.int32, device="cuda")
            B.bonsai_sph_density(bz.ctx, th, rho, cnt)
            torch.cuda.synchronize()
            out = rho.cpu().numpy(), cnt.cpu().numpy()
        else:
            rho = np.zeros(b.n, np.float32)
            cnt = np.zeros(b.n, np.int32)
            B.bonsai_sph_density(bz.ctx, np.ascontiguousarray(h, np.float32), rho, cnt)
            out = rho, cnt
        bz.sync()
    return out


def adapted_h(b, target=48):
    """h_i from the Plummer density at the body's radius, for about
    `target` neighbours."""
    a = 3 * np.pi / 16
    r = np.linalg.norm(b.pos.astype(np.float64), axis=1)
    nden = b.n * 3 / (4 * np.pi * a ** 3) * (1 + r * r / (a * a)) ** -2.5
    return ((3 * target / (4 * np.pi * nden)) ** (1 / 3)).astype(np.float32)


def check(b, h, rho, cnt):
    orho, ocnt = oracle.sph_density(b.pos, b.mass, h)
    assert np.array_equal(cnt, ocnt)
    assert np.all(np.abs(rho - orho) <= 2e-5 * orho)


@pytest.mark.parametrize("ncrit,pack", [(32, 1), (32, 0), (64, 0), (64, 1), (16, 0)])
def test_adapted_h_vs_oracle(ncrit, pack):
    b = W.plummer(16384, 51)
    h = adapted_h(b)
    rho, cnt = run(b, h, ncrit, pack)
    check(b, h, rho, cnt)
    assert 20 < np.median(cnt) < 100


def test_random_and_constant_h_host_buffers():
    b = W.plummer(8192, 52)
    for h in (np.random.default_rng(3).uniform(0.01, 0.3, b.n).astype(np.float32),
              np.full(b.n, 0.05, np.float32)):
        rho, cnt = run(b, h, device=False)
        check(b, h, rho, cnt)


def test_extremes_and_duplicates():
    b = edge_bodies(6000, 53)                           # identical positions, a tight clump
    h = adapted_h(W.plummer(6000, 53))
    rho, cnt = run(b, h)
    check(b, h, rho, cnt)
    big = np.full(b.n, 1e3, np.float32)                 # every body is a neighbour
    rho, cnt = run(b, big)
    assert np.all(cnt == b.n)
    check(b, big, rho, cnt)
    tiny = np.full(b.n, 1e-9, np.float32)               # only itself (and exact duplicates)
    rho, cnt = run(b, tiny)
    check(b, tiny, rho, cnt)


def test_needs_a_fresh_tree():
    b = W.plummer(4096, 54)
    h = adapted_h(b)
    with B.Bonsai(B.Config()) as bz:
        bz.set_bodies(b.pos, b.mass, b.vel)
        with pytest.raises(B.BonsaiError):
            B.bonsai_sph_density(bz.ctx, h)             # no tree yet
        bz.build().multipoles().forces(0.75, 0.01)
        B.bonsai_block_cycle(bz.ctx, 1.0 / 16, 2, 0.2, 4)   # last substep is a refit
        with pytest.raises(B.BonsaiError) as ei:
            B.bonsai_sph_density(bz.ctx, h)
        assert ei.value.code == -7
        bz.build()
        rho = np.zeros(b.n, np.float32)
        cnt = np.zeros(b.n, np.int32)
        B.bonsai_sph_density(bz.ctx, h, rho, cnt)
        x = np.zeros((b.n, 3), np.float32)
        B.bonsai_get_bodies(bz.ctx, x, None)
        bz.sync()
    moved = W.Bodies(x, b.vel, b.mass)
    check(moved, h, rho, cnt)
