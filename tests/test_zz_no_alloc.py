"""bonsai_sort_keys_static: the radix sort for callers that cannot allocate
device memory (graph-capture regions, latency-critical loops, hosts whose
allocator owns the device).  Its scratch is a static device array shared by
all calls, so this file runs last and checks two calls in a row (the second
smaller than the first, so stale scratch from the first must not leak into
it) against the sort of the existing build path, bit for bit."""
import numpy as np
import pytest

import paper_1204_2280_gb300 as B
from paper_1204_2280_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def context_sort(n, seed):
    """Keys in caller order plus the sorted keys and permutation produced by
    the regular (allocating) pipeline."""
    b = W.plummer(n, seed)
    with B.Bonsai(B.Config()) as bz:
        bz.set_bodies(b.pos, b.mass).build()
        sk, perm = B.bonsai_get_keys(bz.ctx)
        bz.sync()
    keys = np.empty(n, np.uint64)
    keys[perm] = sk
    return keys, sk, perm


def test_static_sort_matches_context_sort_two_calls():
    import torch
    for n, seed in [(65536, 21), (9001, 22)]:
        keys, sk, perm = context_sort(n, seed)
        d_keys = torch.from_numpy(keys.view(np.int64)).cuda()
        d_out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        d_perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        B.bonsai_sort_keys_static(d_keys, d_out, d_perm)
        torch.cuda.synchronize()
        assert np.array_equal(d_out.cpu().numpy().view(np.uint64), sk)
        assert np.array_equal(d_perm.cpu().numpy().view(np.uint32), perm)
        assert np.array_equal(d_keys.cpu().numpy().view(np.uint64), keys)   # input untouched


def test_static_sort_rejects_sizes_beyond_its_scratch():
    import torch
    n = 65537
    d = torch.zeros(n, dtype=torch.int64, device="cuda")
    p = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BonsaiError) as ei:
        B.bonsai_sort_keys_static(d, d.clone(), p)
    assert ei.value.code == -1 and "65536" in str(ei.value)
