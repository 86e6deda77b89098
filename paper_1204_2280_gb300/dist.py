"""Host logic of the multi-GPU runs: one process per GPU, no collective in
the data path.

* A single system does not shard without a domain decomposition and a
  locally-essential-tree exchange (the paper cites those methods without
  specifying them), so each rank runs an independent replica.
* An ensemble of independent systems shards naturally: each rank steps a
  contiguous slice of the systems, the slices balanced by the walk's cost
  model N log N per system.
* Timings are combined after the timed region: the job's time is the
  maximum over ranks, its work the sum (one all-reduce each, on whatever
  process group is initialised: NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import math
from typing import Sequence


def system_cost(n: int) -> float:
    """Relative step cost of a system of n bodies (tree walk ~ n log n)."""
    return float(n) * math.log2(max(n, 2))


def balanced_slices(weights: Sequence[float], parts: int) -> list[tuple[int, int]]:
    """Split items 0..len-1 into `parts` contiguous slices [lo, hi) whose
    largest total weight is as small as possible (binary search on the
    bound, greedy packing; exact for the contiguous problem).  Slices may be
    empty when there are fewer items than parts."""
    if parts < 1:
        raise ValueError("parts >= 1")
    w = [float(x) for x in weights]
    if any(x < 0 for x in w):
        raise ValueError("weights >= 0")
    n = len(w)

    def pack(bound: float) -> list[tuple[int, int]] | None:
        out, lo, acc = [], 0, 0.0
        for i, x in enumerate(w):
            if x > bound:
                return None
            if acc + x > bound:
                out.append((lo, i))
                lo, acc = i, 0.0
            acc += x
        out.append((lo, n))
        if len(out) > parts:
            return None
        out += [(n, n)] * (parts - len(out))
        return out

    total = 0.0
    for x in w:                      # the same sequential sum pack() forms
        total += x
    lo_b, hi_b = max(w, default=0.0), total
    best = pack(hi_b)
    for _ in range(100):
        if hi_b - lo_b <= 1e-9 * max(hi_b, 1.0):
            break
        mid = 0.5 * (lo_b + hi_b)
        got = pack(mid)
        if got is None:
            lo_b = mid
        else:
            best, hi_b = got, mid
    return best


def shard_systems(sizes: Sequence[int], world: int, rank: int) -> tuple[int, int]:
    """The contiguous slice of systems rank `rank` of `world` steps."""
    return balanced_slices([system_cost(n) for n in sizes], world)[rank]


def combine(ms: float, units: float) -> tuple[float, float]:
    """(maximum of ms, sum of units) over the ranks of the default process
    group; the local values when no group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
