"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bars (paper Sect. 2 stages; tolerances from the accuracy requirements of the
tree-code and FP32 arithmetic):
* domain, Morton keys, sort permutation, tree topology and groups: bit-exact;
* moments: M relative 1e-6; com within 4e-7 |com| + 2e-6 l (l the cell side);
  Q within 1e-5 M l^2 per component;
* forces vs the oracle tree at the same theta/eps: per-body relative error
  <= 1e-5 for acceleration and potential, identical interaction counts, for
  every body whose group took no opening decision within tau of the
  threshold (tau = 2e-6 + 1e-6 r_open: FP32 and FP64 may decide those
  differently); the share of such bodies is bounded and they still meet
* forces vs the FP64 direct sum at theta = 0.75: median <= 1e-3, p99 <= 1e-2.
"""
import numpy as np
import pytest

import oracle
import paper_1204_2280_gb300 as B
from paper_1204_2280_gb300 import workloads as W

from gpu_common import edge_bodies, gpu_run, rel_err

pytestmark = pytest.mark.gpu

TAU_ABS, TAU_REL = 2e-6, 1e-6


def check_keys_tree(res, pos, nleaf, ncrit, pack=False):
    mn, S = oracle.domain(pos)
    k = oracle.keys(pos, mn, S)
    perm = oracle.sort(k)
    gmn, gS = res["domain"]
    assert np.array_equal(gmn, mn) and gS == S
    assert np.array_equal(res["keys"], k[perm])
    assert np.array_equal(res["perm"], perm)
    t = oracle.build_tree(k[perm], nleaf)
    g = res["tree"]
    assert g["body_begin"].shape[0] == t.ncells
    for f in ("body_begin", "body_count", "child_begin", "nchild", "level"):
        assert np.array_equal(g[f], getattr(t, f)), f
    gb, gc = oracle.groups(t, ncrit, pack)
    assert np.array_equal(res["groups"][0], gb) and np.array_equal(res["groups"][1], gc)
    return mn, S, k, perm, t


@pytest.mark.parametrize("n", [1, 2, 17, 4099, 32768, 100003])
def test_keys_sort_tree_bit_exact_plummer(n):
    b = W.plummer(n, 0)
    res = gpu_run(b.pos, b.mass, forces=False)
    check_keys_tree(res, b.pos, 16, 32)


@pytest.mark.parametrize("nleaf,ncrit", [(16, 32), (8, 16), (1, 1), (64, 8), (4, 32), (16, 64), (8, 48)])
def test_keys_sort_tree_bit_exact_edge_cases(nleaf, ncrit):
    b = edge_bodies(20000, 3)
    res = gpu_run(b.pos, b.mass, forces=False, nleaf=nleaf, ncrit=ncrit)
    check_keys_tree(res, b.pos, nleaf, ncrit)


@pytest.mark.parametrize("nleaf,ncrit", [(16, 32), (8, 16), (1, 1), (64, 8), (4, 32), (16, 64), (8, 48)])
def test_packed_groups_bit_exact_edge_cases(nleaf, ncrit):
    """Sibling-packed groups (group_pack = 1) are bit-identical to the
    oracle's packing, also with duplicate positions (oversize leaves cut in
    runs) and deep clumps."""
    b = edge_bodies(20000, 3)
    res = gpu_run(b.pos, b.mass, forces=False, nleaf=nleaf, ncrit=ncrit, group_pack=1)
    check_keys_tree(res, b.pos, nleaf, ncrit, pack=True)


@pytest.mark.parametrize("n", [1, 2, 17, 65, 4099, 100003, 1 << 20])
def test_packed_groups_bit_exact_plummer(n):
    """Packing across many packing blocks (2^20 bodies: ~23k unpacked groups)."""
    b = W.plummer(n, 0)
    res = gpu_run(b.pos, b.mass, forces=False, ncrit=64, group_pack=1)
    check_keys_tree(res, b.pos, 16, 64, pack=True)


def test_host_buffers_path():
    b = W.plummer(5000, 7)
    res = gpu_run(b.pos, b.mass, b.vel, device_io=False)
    check_keys_tree(res, b.pos, 16, 32)
    tf = oracle.tree_forces(b.pos, b.mass, 0.75, 0.01, tau_abs=TAU_ABS, tau_rel=TAU_REL)
    ok = ~tf.borderline
    assert rel_err(res["acc"], tf.acc)[ok].max() <= 1e-5


def test_page_locked_host_inputs_match_device_inputs():
    """Page-locked host buffers are read by the pack kernel directly, other
    host buffers through the staging copy, device buffers as they are: the
    same bodies give bit-identical forces every way, also with one
    page-locked and one pageable buffer, and without velocities."""
    import torch
    b = W.plummer(6000, 12)
    dev = lambda a: torch.from_numpy(a).cuda()
    pin = lambda a: torch.from_numpy(a).pin_memory()
    out = []
    for pos, mass, vel in ((dev(b.pos), dev(b.mass), dev(b.vel)), (pin(b.pos), pin(b.mass), pin(b.vel)),
                           (b.pos, b.mass, b.vel), (pin(b.pos), b.mass, pin(b.vel)), (pin(b.pos), pin(b.mass), None)):
        acc = torch.zeros((6000, 3), dtype=torch.float32, device="cuda")
        with B.Bonsai(B.Config(nleaf=16, ncrit=32)) as bz:
            bz.set_bodies(pos, mass, vel).build().multipoles().forces(0.75, 0.01, acc)
            x = np.zeros((6000, 3), np.float32)
            v = np.zeros((6000, 3), np.float32)
            B.bonsai_get_bodies(bz.ctx, x, v)
        out.append((acc.cpu().numpy(), x, v))
    for a, x, v in out[1:]:
        assert np.array_equal(a, out[0][0]) and np.array_equal(x, b.pos)
    for a, x, v in out[:4]:
        assert np.array_equal(v, b.vel)
    assert np.all(out[4][2] == 0)


def test_repeated_calls_replay_graphs_bit_identically():
    """bonsai_build / _multipoles / _forces run directly the first time a
    configuration is seen, are captured into graphs the second time and
    replayed after that: over new bodies of the same size, a change of theta
    and a rebuild from the sorted state, the forces equal those of a context
    that never uses graphs, bit for bit."""
    import torch
    rng = np.random.default_rng(13)
    ctxs = [B.Bonsai(B.Config(nleaf=16, ncrit=32, group_pack=1)),
            B.Bonsai(B.Config(nleaf=16, ncrit=32, group_pack=1, use_graph=-1))]
    try:
        for it, theta in enumerate([0.75, 0.75, 0.75, 0.75, 0.6, 0.6, 0.6]):
            b = W.plummer(20000, 100 + it)
            accs = []
            for bz in ctxs:
                acc = torch.zeros((20000, 3), dtype=torch.float32, device="cuda")
                bz.set_bodies(b.pos, b.mass, b.vel).build().multipoles().forces(theta, 0.01, acc)
                if it % 2:                                # rebuild from the sorted state
                    bz.build().multipoles().forces(theta, 0.01, acc)
                bz.sync()
                accs.append(acc.cpu().numpy())
            assert np.array_equal(accs[0], accs[1]), it
        tf = oracle.tree_forces(b.pos, b.mass, 0.6, 0.01, 16, 32, TAU_ABS, TAU_REL, pack=True)
        ok = ~tf.borderline
        assert rel_err(accs[0], tf.acc)[ok].max() <= 1e-5
    finally:
        for bz in ctxs:
            bz.close()


def test_moments_vs_oracle():
    b = edge_bodies(32768, 1)
    res = gpu_run(b.pos, b.mass, forces=False)
    mn, S, k, perm, t = check_keys_tree(res, b.pos, 16, 32)
    M, com, Q = oracle.moments(t, b.pos[perm], b.mass[perm])
    mono, quad = res["mono"].astype(np.float64), res["quad"].astype(np.float64)
    l = S / 2.0 ** t.level
    assert np.all(np.abs(mono[:, 3] - M) <= 1e-6 * M)
    dcom = np.linalg.norm(mono[:, :3] - com, axis=1)
    assert np.all(dcom <= 4e-7 * np.linalg.norm(com, axis=1) + 2e-6 * l)
    assert np.all(np.abs(quad - Q) <= 1e-5 * (M * l * l)[:, None])


@pytest.mark.parametrize("n,nleaf", [(1, 16), (17, 16), (200, 16), (20000, 1), (20000, 64), (100003, 8)])
def test_moments_vs_oracle_tree_shapes(n, nleaf):
    """The two multipole passes over trees of every shape: a root that is a
    leaf, a root whose children are all leaves (combined from the start
    list), leaves of one body (every internal cell climbs), shallow trees
    and a ragged size."""
    b = W.plummer(n, 11)
    res = gpu_run(b.pos, b.mass, forces=False, nleaf=nleaf, ncrit=max(nleaf, 16))
    mn, S, k, perm, t = check_keys_tree(res, b.pos, nleaf, max(nleaf, 16))
    M, com, Q = oracle.moments(t, b.pos[perm], b.mass[perm])
    mono, quad = res["mono"].astype(np.float64), res["quad"].astype(np.float64)
    l = S / 2.0 ** t.level
    assert np.all(np.abs(mono[:, 3] - M) <= 1e-6 * M)
    dcom = np.linalg.norm(mono[:, :3] - com, axis=1)
    assert np.all(dcom <= 4e-7 * np.linalg.norm(com, axis=1) + 2e-6 * l)
    assert np.all(np.abs(quad - Q) <= 1e-5 * (M * l * l)[:, None])


@pytest.mark.parametrize("theta,ncrit", [(0.5, 32), (0.75, 32), (1.0, 32), (0.75, 64), (0.5, 64)])
def test_forces_vs_oracle_tree(theta, ncrit):
    b = W.plummer(32768, 0)
    res = gpu_run(b.pos, b.mass, theta=theta, eps=0.01, ncrit=ncrit)
    tf = oracle.tree_forces(b.pos, b.mass, theta, 0.01, 16, ncrit, TAU_ABS, TAU_REL)
    ok = ~tf.borderline
    assert ok.mean() > 0.9, ok.mean()
    ea = rel_err(res["acc"], tf.acc)
    ep = np.abs(res["pot"] - tf.pot) / np.abs(tf.pot)
    assert ea[ok].max() <= 1e-5, (ea[ok].max(), np.argmax(np.where(ok, ea, 0)))
    assert ep[ok].max() <= 1e-5
    assert np.array_equal(res["n_pc"][ok], tf.n_pc[ok])
    assert np.array_equal(res["n_pp"][ok], tf.n_pp[ok])
    # totals of the whole walk agree with the per-body counts
    assert res["tot"][0] == int(res["n_pc"].astype(np.int64).sum())
    assert res["tot"][1] == int(res["n_pp"].astype(np.int64).sum())
    # borderline bodies: within the approximation's own error of the oracle tree
    assert ea.max() <= 3e-2


@pytest.mark.parametrize("theta,ncrit", [(0.75, 32), (0.5, 64), (0.75, 64), (1.0, 64)])
def test_forces_vs_oracle_tree_packed_groups(theta, ncrit):
    """The walk over sibling-packed groups against the oracle walking the
    same packed groups."""
    b = W.plummer(32768, 0)
    res = gpu_run(b.pos, b.mass, theta=theta, eps=0.01, ncrit=ncrit, group_pack=1)
    tf = oracle.tree_forces(b.pos, b.mass, theta, 0.01, 16, ncrit, TAU_ABS, TAU_REL, pack=True)
    ok = ~tf.borderline
    assert ok.mean() > 0.9, ok.mean()
    ea = rel_err(res["acc"], tf.acc)
    ep = np.abs(res["pot"] - tf.pot) / np.abs(tf.pot)
    assert ea[ok].max() <= 1e-5 and ep[ok].max() <= 1e-5
    assert np.array_equal(res["n_pc"][ok], tf.n_pc[ok]) and np.array_equal(res["n_pp"][ok], tf.n_pp[ok])
    assert ea.max() <= 3e-2
    if theta == 0.75:
        a_d, _ = oracle.direct(b.pos, b.mass, 0.01)
        e = rel_err(res["acc"], a_d)
        assert np.median(e) <= 1e-3 and np.percentile(e, 99) <= 1e-2


def test_forces_vs_direct_sum_gates():
    """Config: Plummer N=2^15, seed 0, eps=0.01, theta=0.75 (all bodies)."""
    b = W.plummer(32768, 0)
    res = gpu_run(b.pos, b.mass, theta=0.75, eps=0.01)
    a_d, p_d = oracle.direct(b.pos, b.mass, 0.01)
    e = rel_err(res["acc"], a_d)
    assert np.median(e) <= 1e-3 and np.percentile(e, 99) <= 1e-2
    ep = np.abs(res["pot"] - p_d) / np.abs(p_d)
    assert np.median(ep) <= 1e-3 and np.percentile(ep, 99) <= 1e-2


@pytest.mark.parametrize("nleaf,ncrit", [(8, 16), (1, 1), (64, 8), (16, 32), (16, 64), (4, 48), (64, 64)])
def test_forces_edge_cases(nleaf, ncrit):
    b = edge_bodies(8192, 5)
    res = gpu_run(b.pos, b.mass, theta=0.75, eps=0.01, nleaf=nleaf, ncrit=ncrit)
    tf = oracle.tree_forces(b.pos, b.mass, 0.75, 0.01, nleaf, ncrit, TAU_ABS, TAU_REL)
    ok = ~tf.borderline
    assert rel_err(res["acc"], tf.acc)[ok].max() <= 1e-5
    assert (np.abs(res["pot"] - tf.pot) / np.abs(tf.pot))[ok].max() <= 1e-5
    assert np.array_equal(res["n_pp"][ok], tf.n_pp[ok])


def test_two_bodies_closed_form():
    pos = np.array([[0.0, 0.0, 0.0], [0.75, -0.5, 0.25]], np.float32)
    mass = np.array([0.25, 2.0], np.float32)
    res = gpu_run(pos, mass, theta=0.75, eps=0.1)
    d = pos[1].astype(np.float64) - pos[0]
    r2 = d.dot(d) + 0.01
    assert np.allclose(res["acc"][0], 2.0 * d / r2 ** 1.5, rtol=1e-6)
    assert np.allclose(res["acc"][1], -0.25 * d / r2 ** 1.5, rtol=1e-6)
    assert np.allclose(res["pot"], [-2.0 / np.sqrt(r2), -0.25 / np.sqrt(r2)], rtol=1e-6)


def test_single_body():
    res = gpu_run(np.array([[1.0, 2.0, 3.0]], np.float32), np.array([1.0], np.float32))
    assert np.all(res["acc"] == 0) and abs(res["pot"][0]) < 1e-6


def test_theta_small_equals_direct():
    b = W.plummer(3000, 9)
    res = gpu_run(b.pos, b.mass, theta=0.02, eps=0.01, list_capacity=8192)
    a_d, p_d = oracle.direct(b.pos, b.mass, 0.01)
    assert rel_err(res["acc"], a_d).max() <= 1e-5
    assert np.all(res["n_pp"] == 2999)


def test_kdk_step_vs_oracle():
    """One force evaluation plus one leapfrog step dt = 1/64 (Plummer 2^15)."""
    b = W.plummer(32768, 0)
    dt, th, eps = 1.0 / 64, 0.75, 0.01
    import torch
    with B.Bonsai(B.Config(nleaf=16, ncrit=32)) as bz:
        bz.set_bodies(b.pos, b.mass, b.vel).build().multipoles()
        bz.forces(th, eps)
        bz.step(dt)
        x1 = np.zeros((32768, 3), np.float32)
        v1 = np.zeros((32768, 3), np.float32)
        B.bonsai_get_bodies(bz.ctx, x1, v1)
        diag = B.bonsai_diagnostics(bz.ctx)
        bz.sync()
    tf0 = oracle.tree_forces(b.pos, b.mass, th, eps, nleaf=16, ncrit=32)
    ox1, ov1, oa1, op1 = oracle.kdk_step(b.pos, b.vel, b.mass, tf0.acc, dt, th, eps, nleaf=16, ncrit=32)
    assert np.allclose(x1, ox1, rtol=2e-7, atol=2e-7)
    dv = np.linalg.norm(v1 - ov1, axis=1)
    scale = 0.5 * dt * np.linalg.norm(oa1, axis=1)
    assert np.median(dv / scale) <= 1e-4 and np.max(dv / (scale + np.linalg.norm(ov1, axis=1))) <= 1e-2
    # FP64 diagnostics of the new state vs the oracle's own step and potential
    e = oracle.energy(ox1.astype(np.float32), ov1.astype(np.float32), b.mass, op1)
    assert diag[0] == pytest.approx(e[0], rel=1e-5)
    assert diag[1] == pytest.approx(e[1], rel=2e-5)
    assert np.allclose(diag[3:6], e[3:6], atol=1e-6)
    assert diag[6] == pytest.approx(1.0, rel=1e-6)


def test_diagnostics_same_snapshot():
    """FP64 diagnostics vs the oracle's energy of the same input snapshot with
    the oracle tree's own potential."""
    b = W.plummer(32768, 2)
    with B.Bonsai(B.Config(nleaf=16, ncrit=64)) as bz:
        bz.set_bodies(b.pos, b.mass, b.vel).build().multipoles()
        bz.forces(0.75, 0.01)
        d = B.bonsai_diagnostics(bz.ctx)
    tf = oracle.tree_forces(b.pos, b.mass, 0.75, 0.01, nleaf=16, ncrit=64)
    e = oracle.energy(b.pos, b.vel, b.mass, tf.pot)
    assert d[0] == pytest.approx(e[0], rel=1e-12)
    assert d[1] == pytest.approx(e[1], rel=1e-6)
    assert d[2] == pytest.approx(e[2], rel=2e-6)
    assert np.allclose(d[3:6], e[3:6], atol=1e-12) and d[7] == pytest.approx(e[7], abs=1e-12)


def test_multi_step_graph_replay_matches_direct_launches():
    """Steps replayed from the captured CUDA graph give bit-identical state to
    steps launched one kernel at a time."""
    b = W.plummer(20000, 4)
    outs = []
    for ug in (1, -1):
        with B.Bonsai(B.Config(use_graph=ug)) as bz:
            bz.set_bodies(b.pos, b.mass, b.vel)
            B.bonsai_set_params(bz.ctx, 0.75, 0.01)
            for _ in range(4):
                bz.step(1.0 / 128)
            x = np.zeros((20000, 3), np.float32)
            v = np.zeros((20000, 3), np.float32)
            B.bonsai_get_bodies(bz.ctx, x, v)
            bz.sync()
            outs.append((x, v))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_stage_timing_switch():
    """Stage events are off by default (no stage times: NOT_READY), on after
    bonsai_set_stage_timing (eight positive stage times, also from graph
    replays), and either way the steps give bit-identical state."""
    import torch
    b = W.plummer(20000, 5)
    outs = []
    for timing in (False, True):
        with B.Bonsai(B.Config(ncrit=32, group_pack=1)) as bz:
            bz.set_bodies(b.pos, b.mass, b.vel)
            B.bonsai_set_params(bz.ctx, 0.75, 0.01)
            B.bonsai_set_stage_timing(bz.ctx, timing)
            for _ in range(4):
                bz.step(1.0 / 128)
            if timing:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(torch.cuda.current_stream())
                bz.step(1.0 / 128)
                bz.sync()
                e1.record(torch.cuda.current_stream())
                e1.synchronize()
                ms = B.bonsai_get_stage_times(bz.ctx)
                assert ms.shape == (8,) and np.all(ms > 0)
                assert ms.sum() <= e0.elapsed_time(e1) * 1.05 + 0.05
            else:
                with pytest.raises(B.BonsaiError) as ei:
                    B.bonsai_get_stage_times(bz.ctx)
                assert ei.value.code == -7
                bz.step(1.0 / 128)
            x = np.zeros((20000, 3), np.float32)
            v = np.zeros((20000, 3), np.float32)
            B.bonsai_get_bodies(bz.ctx, x, v)
            bz.sync()
            outs.append((x, v))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_arena_cap_reports_oom_and_recovers():
    """A context whose device arena is capped (a host-side stand-in for an
    out-of-memory device) refuses a body set that needs more with
    BONSAI_ERR_OOM, then holds no bodies (later stages: NOT_READY, nothing
    reads the freed arena), and takes a body set that fits."""
    big = W.plummer(1 << 20, 7)
    with B.Bonsai(B.Config(arena_limit_mib=64)) as bz:
        assert B.bonsai_get_config(bz.ctx).arena_limit_mib == 64
        with pytest.raises(B.BonsaiError) as ei:
            bz.set_bodies(big.pos, big.mass, big.vel)
        assert ei.value.code == -2
        with pytest.raises(B.BonsaiError) as ei:
            bz.build()
        assert ei.value.code == -7
        small = W.plummer(4096, 8)
        bz.set_bodies(small.pos, small.mass, small.vel).build().multipoles()
        acc = np.zeros((4096, 3), np.float32)
        pot = np.zeros(4096, np.float32)
        bz.forces(0.75, 0.01, acc, pot)
        bz.step(1.0 / 128)
        bz.sync()
    tf = oracle.tree_forces(small.pos, small.mass, 0.75, 0.01, 16, 64, TAU_ABS, TAU_REL)
    ok = ~tf.borderline
    assert rel_err(acc, tf.acc)[ok].max() <= 1e-5


def test_capacity_overflow_reports_error_and_recovers():
    b = W.plummer(20000, 1)
    with B.Bonsai(B.Config(list_capacity=64)) as bz:
        bz.set_bodies(b.pos, b.mass).build().multipoles()
        with pytest.raises(B.BonsaiError) as ei:
            bz.forces(0.05, 0.01)
            bz.sync()
        assert ei.value.code == -4
        bz.forces(0.75, 0.01)      # a normal walk on the same context still works
        bz.sync()


def test_bounded_wait_timeout_is_reported():
    """A sort tile held back from publishing (the testing aid
    bonsai_debug_hold_sort_tile) makes the look-back of the next tile run
    out of its bounded wait every time: bonsai_sync reports
    BONSAI_ERR_TIMEOUT, nothing faults, and once the hold is lifted the same
    context sorts and builds exactly again."""
    n = 50000                                   # 13 sort tiles of 4096 keys
    b = W.plummer(n, 6)
    mn, S = oracle.domain(b.pos)
    k = oracle.keys(b.pos, mn, S)
    perm = oracle.sort(k)
    with B.Bonsai(B.Config(max_spin=2000)) as bz:
        for trial in range(2):                  # deterministic: every time
            B.bonsai_debug_hold_sort_tile(bz.ctx, 3)
            bz.set_bodies(b.pos, b.mass).build()
            with pytest.raises(B.BonsaiError) as ei:
                bz.sync()
            assert ei.value.code == -5
        B.bonsai_debug_hold_sort_tile(bz.ctx, -1)
        bz.set_bodies(b.pos, b.mass).build()
        bz.sync()
        kk, pp = B.bonsai_get_keys(bz.ctx)
        assert np.array_equal(pp, perm) and np.array_equal(kk, k[perm])
        bz.multipoles()
        bz.forces(0.75, 0.01)
        bz.sync()
    res = gpu_run(b.pos, b.mass, forces=False)
    check_keys_tree(res, b.pos, 16, 32)

def test_fma_microbenchmark_against_unit_counts():
    """The FP32 peak microbenchmark reaches a plausible share of SMs x 128
    lanes x 2 flop x the maximum clock (not above it: the chains would then
    not be doing the work)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ms, fl = B.bonsai_bench_fma(8 * sms, 256, 200000)
    tflops = fl / (ms / 1e3) / 1e12
    ceiling = sms * 128 * 2 * 2070e6 / 1e12
    assert fl == 8 * sms * 256 * 200000 * 32
    assert 0.5 * ceiling < tflops <= 1.02 * ceiling, (tflops, ceiling)
