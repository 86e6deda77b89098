"""bonsai_sort_keys_static: the key sort for callers that cannot call
cudaMalloc around it -- a latency-critical loop (cudaMalloc/cudaFree can
synchronise the whole device) or a host whose own caching allocator already
owns the device memory.  Its scratch is one static device array shared by
every call, so this file runs last (pytest collects it after the others) and
checks calls in a row -- larger, then smaller, then tiny, so that stale
scratch from one call must not leak into the next -- against both the
oracle's stable sort of the same keys and the sort of the regular
(allocating) pipeline, bit for bit.  It also checks that a call allocates
nothing on the device and that it orders its work on a torch side stream."""
import numpy as np
import pytest

import oracle
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


def static_sort(keys, stream=None):
    import torch
    n = keys.shape[0]
    d_keys = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    d_out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    d_perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    B.bonsai_sort_keys_static(d_keys, d_out, d_perm, stream)
    torch.cuda.synchronize()
    assert np.array_equal(d_keys.cpu().numpy().view(np.uint64), keys)   # input untouched
    return d_out.cpu().numpy().view(np.uint64), d_perm.cpu().numpy().view(np.uint32)


def test_static_sort_matches_oracle_and_context_sort_in_a_row():
    for n, seed in [(65536, 21), (9001, 22), (4097, 23), (1, 24)]:
        keys, sk, perm = context_sort(n, seed)
        want = oracle.sort(keys)
        got_k, got_p = static_sort(keys)
        assert np.array_equal(got_p, want) and np.array_equal(got_k, keys[want])
        assert np.array_equal(got_p, perm) and np.array_equal(got_k, sk)


def test_static_sort_heavy_duplicates_on_a_side_stream():
    """Many equal keys (16 distinct values over 65536 keys, spread over all
    eight key bytes): equal keys keep their input order, as numpy's stable
    argsort and the oracle's sort have them."""
    import torch
    rng = np.random.default_rng(5)
    vals = rng.integers(0, 1 << 63, 16, dtype=np.uint64)
    keys = vals[rng.integers(0, 16, 65536)]
    s = torch.cuda.Stream()
    got_k, got_p = static_sort(keys, s)
    want = np.argsort(keys, kind="stable").astype(np.uint32)
    assert np.array_equal(got_p, want) and np.array_equal(got_p, oracle.sort(keys))
    assert np.array_equal(got_k, keys[want])


def test_static_sort_allocates_nothing():
    """Free device memory is the same before and after a call (the first call
    on the device, which loads the kernels, has happened above or here)."""
    import torch
    keys = np.random.default_rng(6).integers(0, 1 << 63, 30000, dtype=np.uint64)
    static_sort(keys)                                   # warm: modules loaded
    d_keys = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    d_out = torch.empty(30000, dtype=torch.int64, device="cuda")
    d_perm = torch.empty(30000, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    B.bonsai_sort_keys_static(d_keys, d_out, d_perm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(d_perm.cpu().numpy().view(np.uint32), oracle.sort(keys))


def test_static_sort_rejects_sizes_beyond_its_scratch():
    import torch
    n = 65537
    d = torch.zeros(n, dtype=torch.int64, device="cuda")
    p = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BonsaiError) as ei:
        B.bonsai_sort_keys_static(d, d.clone(), p)
    assert ei.value.code == -1 and "65536" in str(ei.value)
