"""Host logic of the multi-GPU runs (CPU): balanced contiguous slices of an
ensemble's systems, and the max-time / sum-work combination over ranks on
a world-size-2 gloo group."""
import itertools
import os
import socket

import numpy as np
import pytest

from paper_1204_2280_gb300 import dist as D


def brute_force_bound(w, parts):
    n = len(w)
    best = float("inf")
    for cuts in itertools.combinations(range(n + 1), parts - 1):
        edges = (0,) + cuts + (n,)
        if any(edges[i] > edges[i + 1] for i in range(parts)):
            continue
        best = min(best, max(sum(w[edges[i]:edges[i + 1]]) for i in range(parts)))
    return best


def check_cover(sl, n, parts):
    assert len(sl) == parts
    assert sl[0][0] == 0 and sl[-1][1] == n
    for (a, b), (c, d) in zip(sl, sl[1:]):
        assert b == c and a <= b
    return [sl_i for sl_i in sl]


@pytest.mark.parametrize("seed", range(6))
def test_balanced_slices_optimal_on_small_cases(seed):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        n = int(rng.integers(1, 9))
        parts = int(rng.integers(1, 4))
        w = [float(x) for x in rng.integers(0, 20, n)]
        sl = D.balanced_slices(w, parts)
        check_cover(sl, n, parts)
        got = max(sum(w[a:b]) for a, b in sl)
        assert got <= brute_force_bound(w, parts) * (1 + 1e-9) + 1e-9


def test_balanced_slices_edge_cases():
    assert D.balanced_slices([], 3) == [(0, 0), (0, 0), (0, 0)]
    assert D.balanced_slices([5.0], 2) == [(0, 1), (1, 1)]
    assert D.balanced_slices([1.0, 1.0, 1.0, 1.0], 2) == [(0, 2), (2, 4)]
    with pytest.raises(ValueError):
        D.balanced_slices([1.0], 0)
    with pytest.raises(ValueError):
        D.balanced_slices([-1.0], 1)


def test_shard_systems_cover_every_system_once():
    from paper_1204_2280_gb300 import workloads as W
    sizes = W.ensemble_sizes(64, 100)
    for world in (1, 2, 3, 4, 8):
        seen = []
        for r in range(world):
            lo, hi = D.shard_systems(sizes, world, r)
            seen += list(range(lo, hi))
        assert seen == list(range(64))
        loads = [sum(D.system_cost(n) for n in sizes[slice(*D.shard_systems(sizes, world, r))])
                 for r in range(world)]
        # no slice exceeds the ideal share by more than one system's cost
        assert max(loads) <= sum(loads) / world + max(D.system_cost(n) for n in sizes) + 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = D.combine(ms=1.5 + rank, units=10.0 * (rank + 1))
        with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
            f.write(f"{ms} {units}")
    finally:
        dist.destroy_process_group()


def test_combine_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        ms, units = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        assert ms == 2.5 and units == 30.0


def test_combine_without_a_group_is_local():
    assert D.combine(3.0, 7.0) == (3.0, 7.0)
