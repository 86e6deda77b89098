#!/usr/bin/env python3
"""Throughput of the full tree step on GB300: particles per second.

Workload: Plummer sphere N = 2^20 (Henon units, seed 1), eps = 0.005,
theta = 0.75, shared-time-step kick-drift-kick leapfrog with dt = 1/128; every
step runs the whole hot path (domain + Morton keys, radix sort, reorder,
octree build, multipoles, group-wise walk, kicks) through the C ABI.

Prints one JSON line (rank 0).  `value` = bodies advanced per second over all
ranks (device time of the timed steps, CUDA events on the library's stream);
`e2e` = the same through the C ABI with host buffers (pinned H2D of the
bodies, full tree step, D2H of accelerations and potentials); `roofline` =
the walk kernel's algorithmic FP32 rate against the FP32 peak measured in
the same run by the library's FMA-chain microbenchmark (bonsai_bench_fma,
cross-checked against the device's SM count x 128 lanes x 2 flop x the SM
clock sampled under it); `cpu_baseline` = the FP64 oracle tree-code on a
bounded sample of the same workload on the host cores.

The line also carries the batched ensemble (64 spheres, one pipeline per
step; sharded over the ranks under torchrun) and the plain-vs-learned
comparison at equal 99th-percentile force error on the N = 2^22 workload.
`--sweep` prints per-stage scaling lines instead of the bench line.

`--impl reference` times the FP64 oracle on the host cores instead (the
reference arm: the method's paper publishes no code to run).  Under torchrun
each rank is an independent replica (no collective in the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s per full tree step at equal 99th-pct force error, plain vs learned"
UNIT = "particles/s"
FLOP_PC, FLOP_PP = 65, 23           # flops per body-cell / body-body interaction
FP32_LANES = 128                    # FP32 lanes per SM (Blackwell)
_FP32_PEAK = None


def fp32_peak(local_rank: int = 0) -> dict:
    """The FP32 peak of this GPU, measured once per process: the library's
    FMA-chain microbenchmark (eight packed FP32x2 chains per thread, 8 blocks
    of 256 threads per SM, about half a second) with nvidia-smi clocks
    sampled meanwhile, beside SMs x 128 lanes x 2 flop x clock for the SM
    count the device reports and the sampled median (and the maximum) clock."""
    global _FP32_PEAK
    if _FP32_PEAK is not None:
        return _FP32_PEAK
    import torch
    import paper_1204_2280_gb300 as B
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    blocks, threads = 8 * sms, 256
    ms, fl = B.bonsai_bench_fma(blocks, threads, 20000)            # calibrate
    iters = max(20000, int(20000 * 500.0 / max(ms, 1e-3)))
    smp = ClockSampler(gpu_index(local_rank))
    smp.start()
    time.sleep(0.2)
    ms, fl = B.bonsai_bench_fma(blocks, threads, iters)
    clk = smp.stop()
    meas = fl / (ms / 1e3) / 1e12
    mhz = clk.get("sm_mhz")
    mx = clk.get("sm_max_mhz") or 2070.0
    _FP32_PEAK = {
        "tflops": meas, "ms": ms, "sms": sms, "sm_mhz_median": mhz, "sm_max_mhz": mx,
        "derived_at_median_clock": sms * FP32_LANES * 2 * mhz * 1e6 / 1e12 if mhz else None,
        "derived_at_max_clock": sms * FP32_LANES * 2 * mx * 1e6 / 1e12,
        "clock_reasons": clk.get("reasons"),
        "how": f"bonsai_bench_fma: {blocks} blocks x {threads} threads x {iters} iterations x 8 chains of "
               f"packed FP32x2 FMA ({fl:.3e} flop in {ms:.1f} ms, CUDA events)"}
    return _FP32_PEAK


def fp32_peak_tflops(local_rank: int = 0) -> float:
    return fp32_peak(local_rank)["tflops"]


def kernels_per_step(ncrit, group_pack=0):
    """reset, kick+drift+bbox, domains, keys, 8 sort passes, reorder, 4 build
    (+2 for sibling packing of the groups), multipoles in two passes (leaves,
    then internal cells; they also write the MAC records), walk (a second
    instantiation when groups may exceed 16 bodies: three bodies per lane for
    17..24, two for more than 32), kick.  (The start-list reset before the
    multipoles is a memset node, not a kernel.)"""
    return 21 + (1 if ncrit > 16 else 0) + (2 if group_pack else 0)
# DRAM bytes (read + write) of one step's walk (both instantiations) from
# the ncu capture in profiles/k_walk_plummer_n2e20.md, keyed by (N, ncrit,
# group_pack); other choices have no capture and report null.
WALK_TRAFFIC = {(1 << 20, 32, 1): 71.47e6}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=1 << 20)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--theta", type=float, default=0.75)
    p.add_argument("--eps", type=float, default=0.005)
    p.add_argument("--dt", type=float, default=1.0 / 128)
    p.add_argument("--ncrit", type=int, default=32)
    p.add_argument("--nleaf", type=int, default=16)
    p.add_argument("--walk-warps", type=int, default=8)
    p.add_argument("--list-capacity", type=int, default=256)
    p.add_argument("--group-pack", type=int, default=1, choices=[0, 1],
                   help="sibling-packed walk groups (with --no-autotune; the autotuner picks otherwise)")
    p.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-ensemble", action="store_true")
    p.add_argument("--ensemble-systems", type=int, default=64)
    p.add_argument("--no-learned", action="store_true")
    p.add_argument("--no-block", action="store_true")
    p.add_argument("--no-sph", action="store_true")
    p.add_argument("--no-sweep", action="store_true", help="leave the compact scaling record out of the bench line")
    p.add_argument("--learned-n", type=int, default=1 << 22)
    p.add_argument("--learned-plummer", type=int, default=100, help="Plummer training snapshots")
    p.add_argument("--learned-merger", type=int, default=100, help="merger training snapshots")
    p.add_argument("--sweep", action="store_true",
                   help="per-stage scaling sweep instead of the bench line: one JSON line per (N, theta)")
    p.add_argument("--sweep-sizes", type=str, default="",
                   help="with --sweep: comma-separated log2 N to run (default: every size of the sweep)")
    p.add_argument("--sweep-thetas", type=str, default="",
                   help="with --sweep: comma-separated opening angles to keep (default: those of each size)")
    p.add_argument("--sweep-cpu", type=float, default=0.0,
                   help="with --sweep: also time the FP64 oracle per stage at theta = 0.75 (seconds of walk sample)")
    return p.parse_args()


def config(a, world):
    return {"workload": f"Plummer sphere N={a.n} (Henon units, seed {a.seed}), eps={a.eps}, "
                        f"theta={a.theta}, KDK leapfrog dt={a.dt:g}, full rebuild every step",
            "n": a.n, "theta": a.theta, "eps": a.eps, "dt": a.dt, "nleaf": a.nleaf,
            "ncrit": a.ncrit, "walk_warps": a.walk_warps, "group_pack": a.group_pack,
            "list_capacity": a.list_capacity,
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas x{world}"}


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9 or not c[0].isdigit() or int(c[0]) != self.index:
                continue
            try:
                sm.append(float(c[1])); mx.append(float(c[2])); power.append(float(c[3]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_index(local_rank: int) -> int:
    v = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [x for x in v.split(",") if x.strip()]
    if parts and local_rank < len(parts) and parts[local_rank].strip().isdigit():
        return int(parts[local_rank])
    return local_rank


# ---------------------------------------------------------------------------
def cpu_model() -> str:
    """CPU model of the host (x86 'model name'; Arm implementer/part ids)."""
    import platform
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read().splitlines()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    impl = next((l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")), "?")
    part = next((l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")), "?")
    return f"{platform.machine()} implementer {impl} part {part}"


def cpu_oracle_sample(bodies, theta, eps, nleaf, ncrit, budget_s, seed=0, pack=0, direct=True):
    """FP64 oracle tree-code on a bounded sample, timed per stage: domain and
    keys, sort, tree build (+ groups), moments (+ opening radii) for all
    bodies; the walk for a random sample of groups (extrapolated to all
    bodies); the FP64 direct sum for a 4096-body sample (its own entry, not
    part of a step)."""
    import numpy as np
    import oracle
    st = {}
    t = time.perf_counter()
    mn, S = oracle.domain(bodies.pos)
    k = oracle.keys(bodies.pos, mn, S)
    st["domain_keys"] = time.perf_counter() - t
    t = time.perf_counter()
    perm = oracle.sort(k)
    sk, sp, sm = k[perm], bodies.pos[perm], bodies.mass[perm]
    st["sort_reorder"] = time.perf_counter() - t
    t = time.perf_counter()
    tree = oracle.build_tree(sk, nleaf)
    gb, gc = oracle.groups(tree, ncrit, pack)
    st["build"] = time.perf_counter() - t
    t = time.perf_counter()
    M, com, Q = oracle.moments(tree, sp, sm)
    ro = oracle.open_radius(tree, sk, mn, S, com, theta)
    st["multipoles"] = time.perf_counter() - t
    t_tree = sum(st.values())
    rng = np.random.default_rng(seed)
    frac, t_walk, nb = 0.002, 0.0, 0
    order = rng.permutation(gb.shape[0])
    used = 0
    while True:
        take = max(1, int(frac * gb.shape[0]))
        sel = np.sort(order[used:used + take])
        if sel.size == 0:
            break
        t1 = time.perf_counter()
        oracle.walk(sp, sm, tree, M, com, Q, ro, gb[sel], gc[sel], eps)
        t_walk += time.perf_counter() - t1
        nb += int(gc[sel].sum())
        used += take
        if t_tree + t_walk > 0.5 * budget_s or used >= gb.shape[0]:
            break
        frac *= 2
    n = bodies.n
    st["walk"] = t_walk * n / max(nb, 1)
    t_step = t_tree + st["walk"]
    t_direct = None
    if direct:
        idx = rng.choice(n, size=min(4096, n), replace=False)
        t = time.perf_counter()
        oracle.direct(bodies.pos, bodies.mass, eps, idx)
        t_direct = time.perf_counter() - t
    return {"value": n / t_step, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"full tree build of all {n} bodies ({t_tree:.2f} s) + walk of {used} random "
                      f"groups ({nb} bodies, {t_walk:.2f} s), extrapolated to {n} bodies",
            "stage_s": st, "direct_sum_4096_s": t_direct,
            "paper_context": "Xeon E5620 (4 cores) vs GTX480, N=2^20, theta=0.75: >2.8 M particles/s on the "
                             "GPU, GPU 2-30x faster per stage",
            "t_step_s": t_step}


# ---------------------------------------------------------------------------
def run_reference(a, rank, world):
    if rank != 0:
        return
    from paper_1204_2280_gb300 import workloads as W
    b = W.plummer(a.n, a.seed)
    per_step = max(4.0, min(a.cpu_budget, 150.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        cpu_oracle_sample(b, a.theta, a.eps, a.nleaf, a.ncrit, per_step, pack=a.group_pack)
    ts = []
    samp = None
    for s in range(a.steps):
        samp = cpu_oracle_sample(b, a.theta, a.eps, a.nleaf, a.ncrit, per_step, seed=s, pack=a.group_pack)
        ts.append(samp["t_step_s"])
    t = sum(ts)
    value = a.n * a.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(a, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": samp["cores"], "kind": "oracle",
                             "sample": samp["sample"] + f"; {a.steps} timed samples"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ensemble(a, dev, stream, rank=0, world=1):
    """Batched ensemble: independent Plummer spheres with N log-uniform in
    [2^12, 2^18] (seeds 100..), eps = 0.01, theta = 0.75, all stepped together
    (one sort, one build, one persistent walk, one CUDA graph per step).
    Under torchrun each rank steps a contiguous slice of the systems
    (balanced by N log N, no collective in the data path); the job's time is
    the maximum over ranks and its bodies the sum."""
    import numpy as np
    import torch
    import paper_1204_2280_gb300 as B
    from paper_1204_2280_gb300 import dist as D
    from paper_1204_2280_gb300 import workloads as W
    everything = W.ensemble(a.ensemble_systems, 100)
    lo, hi = D.shard_systems([s.n for s in everything], world, rank)
    systems = everything[lo:hi]
    theta, eps, dt = 0.75, 0.01, a.dt
    ms, nc, w, pk, stages, n = [], None, None, None, [0.0] * len(B.STAGES), 0
    if systems:
        pos = np.concatenate([s.pos for s in systems])
        vel = np.concatenate([s.vel for s in systems])
        mass = np.concatenate([s.mass for s in systems])
        off = np.cumsum([0] + [s.n for s in systems])
        n = int(mass.shape[0])
        bz = B.Bonsai(B.Config(), stream=stream)
        bz.set_bodies(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev), torch.from_numpy(vel).to(dev))
        bz.set_systems(off)
        nc, w, _ = B.bonsai_autotune(bz.ctx, theta, eps)
        pk = B.bonsai_get_config(bz.ctx).group_pack
        B.bonsai_set_params(bz.ctx, theta, eps)
        for _ in range(max(3, a.warmup)):
            bz.step(dt)
        bz.sync()
    if world > 1:
        torch.distributed.barrier()
    if systems:
        for _ in range(a.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bz.step(dt)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        B.bonsai_set_stage_timing(bz.ctx, True)    # one more step, with stage events
        bz.step(dt)
        stages = B.bonsai_get_stage_times(bz.ctx)
        bz.sync()
        bz.close()
    total_ms, bodies = D.combine(sum(ms), float(n * a.steps))
    t = total_ms / a.steps
    return {"systems": len(everything), "n_total": int(sum(s.n for s in everything)),
            "n_min": int(min(s.n for s in everything)), "n_max": int(max(s.n for s in everything)),
            "ms_per_step": t, "particles_per_s": bodies / (total_ms / 1e3),
            "ranks": world, "systems_rank0": [lo, hi] if rank == 0 else None,
            "ncrit": nc, "walk_warps": w, "group_pack": pk, "theta": theta, "eps": eps,
            "stages_ms_rank0": {k: float(v) for k, v in zip(B.STAGES, stages)},
            "stages_from": "one step after the timed ones, with stage events in the step graph",
            "scaling": "strong (the 64 systems split over the ranks)",
            "what": "all systems of a rank in one bonsai_step: one sort, one build, one persistent walk, one graph"}


def run_learned(a, dev, stream):
    """Plain vs learned at equal 99th-percentile force error.

    Workload: Plummer sphere N = 2^22 (seed 4) and a two-Plummer merger
    (2 x 2^21, centres +-2 on x, relative speed 0.5), eps = 0.002.  The
    network (12 -> 64 -> 64 -> 3) is trained here, on the GPU, on theta = 1
    walk features vs direct-sum labels (4096 bodies per snapshot) from 200
    generated snapshots: 100 randomly rotated Plummer spheres (seeds
    1000..1099, generated by host worker processes) and 100 randomly rotated
    snapshots of a merger (seed 40) stepped at theta = 0.5 (every 8th of 800
    steps of dt = 1/64).  Errors are the
    judge's: p99 of |a - a_direct| / |a_direct| over 4096 bodies sampled
    every N/4096 in key order.  theta* is the plain opening angle whose p99
    equals the learned one (bisection).  Step throughputs are full
    bonsai_step calls (sort ... walk, kicks) timed with CUDA events, L2
    flushed between steps."""
    import numpy as np
    import torch
    import paper_1204_2280_gb300 as B
    from paper_1204_2280_gb300 import learned as L
    from paper_1204_2280_gb300 import workloads as W
    n, eps, dt = a.learned_n, 0.002, 1.0 / 256
    t0 = time.perf_counter()
    plummers = L.snapshots_parallel(n, range(1000, 1000 + a.learned_plummer), rot_seed0=7000)
    mergers = (L.rotated(m, 9000 + k) for k, m in
               enumerate(L.evolved(W.merger(n, 40), steps=8 * a.learned_merger, every=8, theta=0.5, eps=eps)))
    X, Y = L.training_set(plummers, theta=1.0, eps=eps, per_snapshot=4096, ncrit=64)
    Xm, Ym = L.training_set(mergers, theta=1.0, eps=eps, per_snapshot=4096, ncrit=64, seed=500)
    X, Y = np.concatenate([X, Xm]), np.concatenate([Y, Ym])
    t1 = time.perf_counter()
    net, losses = L.train(X, Y, epochs=40, batch=4096, lr=2e-3, wd=1e-4, seed=0)
    t2 = time.perf_counter()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    bz = B.Bonsai(B.Config(ncrit=64), stream=stream)

    def load(b):
        bz.set_bodies(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.mass).to(dev),
                      torch.from_numpy(b.vel).to(dev))
        bz.build().multipoles()

    def p99_plain(theta):
        bz.forces(theta, eps)
        return B.bonsai_judge(bz.ctx, eps)

    def p99_learned():
        B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, 1e30)
        B.bonsai_forces_learned(bz.ctx, eps)
        p = B.bonsai_get_judge(bz.ctx)[0]
        B.bonsai_set_learned(bz.ctx, None)
        return p

    def errors(b):
        load(b)
        Xh, Yh, _ = B.bonsai_learn_samples(bz.ctx, 1.0, eps, 4096, 99)
        ysig = net.get_params()[1][-1]
        mse = (float(np.mean(Yh.astype(np.float64) ** 2)),
               float(np.mean((Yh - ysig * net.predict(Xh)).astype(np.float64) ** 2)))
        return {"theta_1.0": p99_plain(1.0), "theta_1.0_mlp": p99_learned(), "theta_0.5": p99_plain(0.5),
                "theta_0.75": p99_plain(0.75), "mse_residual_heldout": {"theta_1.0": mse[0], "theta_1.0_mlp": mse[1]}}

    held = W.plummer(n, 4)
    merger = W.merger(n, 41)
    err = {"merger": errors(merger), "plummer": errors(held)}
    # The judge alone (direct sum of 4096 sampled bodies against all N, then
    # the p99): CUDA events around bonsai_judge on the held-out sphere.
    bz.forces(1.0, eps)
    jms = []
    for r in range(6):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.bonsai_judge(bz.ctx, eps)
        e1.record(stream)
        e1.synchronize()
        if r >= 2:
            jms.append(e0.elapsed_time(e1))
    jt = sum(jms) / len(jms)
    jint = 4096 * n
    judge = {"ms": jt, "interactions": jint, "interactions_per_s": jint / (jt / 1e3),
             "tflops": FLOP_PP * jint / (jt / 1e3) / 1e12,
             "fp32_frac": FLOP_PP * jint / (jt / 1e3) / 1e12 / fp32_peak_tflops(),
             "what": "bonsai_judge: direct sum of 4096 stratified bodies against all N (23 flop per "
                     "interaction) + p99, host copy of the p99 included"}
    target = err["plummer"]["theta_1.0_mlp"]
    lo, hi = 0.3, 1.15                      # plain p99 grows with theta
    if p99_plain(hi) <= target:
        lo = hi
    else:
        for _ in range(14):
            mid = 0.5 * (lo + hi)
            if p99_plain(mid) <= target:
                lo = mid
            else:
                hi = mid
    theta_star = lo
    p_star = p99_plain(theta_star)

    def timed(setup, steps=5, warm=3):
        load(held)
        setup()
        for _ in range(warm):
            bz.step(dt)
        bz.sync()
        ms, fell = [], 0
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bz.step(dt)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            fell += int(B.bonsai_get_judge(bz.ctx)[1])
        B.bonsai_set_learned(bz.ctx, None)
        bz.sync()
        t = sum(ms) / len(ms)
        return {"ms_per_step": t, "particles_per_s": n / (t / 1e3), "fallback_steps": fell, "steps": steps}

    def plain(theta):
        return lambda: B.bonsai_set_params(bz.ctx, theta, eps)

    def learned(budget, every):
        def f():
            B.bonsai_set_params(bz.ctx, 1.0, eps)
            B.bonsai_set_learned(bz.ctx, net, 1.0, 0.5, budget)
            B.bonsai_set_judge_interval(bz.ctx, every)
        return f

    runs = {"plain_theta_0.5": timed(plain(0.5)),
            "plain_theta_star": timed(plain(theta_star)),
            "plain_theta_1.0": timed(plain(1.0)),
            "learned_judged_every_step": timed(learned(1e30, 1)),
            "learned_unjudged": timed(learned(1e30, 0)),
            "learned_budget_p99_theta_0.5": timed(learned(err["plummer"]["theta_0.5"], 1))}
    bz.close()
    lj, ps = runs["learned_judged_every_step"], runs["plain_theta_star"]
    return {
        "workload": f"Plummer N={n} seed 4 and merger 2x{n // 2} (seed 41), eps={eps}, dt={dt:g}",
        "network": "12 -> 64 -> 64 -> 3, BF16 tensor cores, FP32 accumulate, rotation-equivariant frame",
        "train": {"samples": int(X.shape[0]), "plummer_snapshots": a.learned_plummer,
                  "merger_snapshots": a.learned_merger, "epochs": 40, "loss_first": float(losses[0]),
                  "loss_last": float(losses[-1]), "data_s": t1 - t0, "train_s": t2 - t1},
        "p99": err,
        "judge": judge,
        "equal_p99": {"p99": target, "plain_theta": theta_star, "plain_p99": p_star,
                      "plain_particles_per_s": ps["particles_per_s"],
                      "learned_particles_per_s": lj["particles_per_s"],
                      "learned_over_plain": lj["particles_per_s"] / ps["particles_per_s"]},
        "steps": runs,
    }


# Algorithmic bytes per body of the memory-bound stages (what the stage must
# read and write once), and per cell / group where the stage writes cells.
STAGE_BYTES = {
    "kick_drift_domain": "pos, vel, acc, id read (52 B); pos, vel, id written (36 B)",
    "keys": "pos read (16 B); key written (8 B)",
    "sort": "8 passes: pass 0 reads keys (8 B), later passes keys + values (12 B); each writes 12 B",
    "reorder": "perm, pos, vel, id read (40 B); pos, vel, id written (36 B)",
    "build": "sorted keys read (8 B/body); 16 B per cell and 8 B per group written",
    "multipoles": "pos read (16 B/body); 64 B per cell written (com, M, Q, delta, MAC record)",
    "kick": "vel, acc read (32 B); vel written (16 B)",
}


def stage_bytes(n, ncells, ngroups):
    return {"kick_drift_domain": 88 * n, "keys": 24 * n, "sort": (20 + 7 * 24) * n,
            "reorder": 76 * n, "build": 8 * n + 16 * ncells + 8 * ngroups,
            "multipoles": 16 * n + 64 * ncells, "kick": 48 * n}


def run_sph(a, dev, stream):
    """Neighbour search and SPH density (paper Sect. 3) on the bench
    workload's tree: smoothing lengths from the Plummer density at each
    body's radius for about 48 neighbours; device ms per density pass (CUDA
    events, L2 flushed between passes, tree built once), neighbours per body,
    neighbour pairs per second; the oracle's O(N^2) definition timed on a
    bounded sample of bodies beside it."""
    import numpy as np
    import torch
    import paper_1204_2280_gb300 as B
    from paper_1204_2280_gb300 import workloads as W
    b = W.plummer(a.n, a.seed)
    ah = 3 * np.pi / 16
    r = np.linalg.norm(b.pos.astype(np.float64), axis=1)
    nden = a.n * 3 / (4 * np.pi * ah ** 3) * (1 + r * r / (ah * ah)) ** -2.5
    h = ((3 * 48 / (4 * np.pi * nden)) ** (1 / 3)).astype(np.float32)
    bz = B.Bonsai(B.Config(nleaf=a.nleaf, ncrit=a.ncrit, walk_warps=a.walk_warps, group_pack=a.group_pack,
                           list_capacity=a.list_capacity), stream=stream)
    bz.set_bodies(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.mass).to(dev),
                  torch.from_numpy(b.vel).to(dev))
    bz.build()
    th = torch.from_numpy(h).to(dev)
    rho = torch.zeros(a.n, dtype=torch.float32, device=dev)
    cnt = torch.zeros(a.n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(3):
        B.bonsai_sph_density(bz.ctx, th, rho, cnt)
    ms = []
    for _ in range(10):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.bonsai_sph_density(bz.ctx, th, rho, cnt)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    bz.sync()
    bz.close()
    c = cnt.cpu().numpy()
    t = sum(ms) / len(ms)
    out = {"n": a.n, "ms_per_pass": t, "neighbours_mean": float(c.mean()),
           "neighbours_p5_p95": [float(np.percentile(c, 5)), float(np.percentile(c, 95))],
           "neighbour_pairs_per_s": float(c.sum()) / (t / 1e3), "particles_per_s": a.n / (t / 1e3)}
    if not a.no_cpu_baseline:
        import oracle
        ns = 4096                     # the oracle's O(N^2) definition on a sample of targets
        idx = np.random.default_rng(0).choice(a.n, ns, replace=False)
        t0 = time.perf_counter()
        sub = W.Bodies(b.pos[idx], b.vel[idx], b.mass[idx])
        oracle.sph_density(sub.pos, sub.mass, h[idx])
        tc = time.perf_counter() - t0
        out["cpu_oracle"] = {"what": f"O(N^2) definition on {ns} random bodies ({ns}^2 pairs) in {tc:.3f} s",
                             "pairs_per_s": ns * ns / tc, "cores": os.cpu_count()}
    return out


def run_block(a, dev, stream):
    """Block time steps (paper Sect. 1 and 3) on the bench workload: cycles
    of dt_max = 8 dt (dt the bench step) in 2^3 substeps, levels from
    eta sqrt(eps / |a|) for eta in {0.2, 0.4}, against 8 shared steps of dt
    per cycle (the shared step must take the finest step the fastest bodies
    need).  Rebuilt every substep (R = 1) and every 4th with refits between
    (R = 4).  Per variant: device ms per cycle (CUDA events, L2 flushed
    between cycles), body steps that ended and interactions per cycle, and
    the FP64 energy error after the timed cycles (potentials of a fresh
    rebuild at both ends, so every variant is measured with one estimator)."""
    import torch
    import paper_1204_2280_gb300 as B
    from paper_1204_2280_gb300 import workloads as W
    b = W.plummer(a.n, a.seed)
    kmax, dt_max = 3, a.dt * 8
    cfg = dict(nleaf=a.nleaf, ncrit=a.ncrit, walk_warps=a.walk_warps, group_pack=a.group_pack)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {"n": a.n, "dt_max": dt_max, "max_level": kmax, "theta": a.theta, "eps": a.eps}
    warm, timed = 2, 3

    def timed_cycles(fn):
        ms = []
        for _ in range(timed):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sum(ms) / len(ms)

    def fresh():
        bz = B.Bonsai(B.Config(**cfg), stream=stream)
        bz.set_bodies(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.mass).to(dev),
                      torch.from_numpy(b.vel).to(dev))
        bz.build().multipoles().forces(a.theta, a.eps)
        B.bonsai_set_params(bz.ctx, a.theta, a.eps)
        return bz

    def energy(bz):
        bz.build().multipoles().forces(a.theta, a.eps)
        return B.bonsai_diagnostics(bz.ctx)[2]

    bz = fresh()
    e0 = B.bonsai_diagnostics(bz.ctx)[2]
    for _ in range(warm * 8):
        bz.step(a.dt)
    ms = timed_cycles(lambda: [bz.step(a.dt) for _ in range(8)])
    e1 = energy(bz)
    bz.sync()
    bz.close()
    out["shared"] = {"ms_per_cycle": ms, "body_steps_per_cycle": 8 * a.n,
                     "energy_err": (e1 - e0) / abs(e0), "particles_per_s": 8 * a.n / (ms / 1e3)}
    for eta in (0.2, 0.4):
        for r in (1, 4):
            bz = fresh()
            if r == 1:
                lev = B.bonsai_block_levels(bz.ctx, dt_max, kmax, eta)
                out[f"levels_at_start_eta{eta}"] = [int((lev == k).sum()) for k in range(kmax + 1)]
            e0 = B.bonsai_diagnostics(bz.ctx)[2]
            for _ in range(warm):
                bz.block_cycle(dt_max, kmax, eta, r)
            ms = timed_cycles(lambda: bz.block_cycle(dt_max, kmax, eta, r))
            act, npc, npp = B.bonsai_block_stats(bz.ctx)
            walked, rebuilt = B.bonsai_block_substeps(bz.ctx)
            e1 = energy(bz)
            bz.sync()
            bz.close()
            out[f"eta{eta}_r{r}"] = {
                "ms_per_cycle": ms, "body_steps_per_cycle": act, "active_fraction": act / (8 * a.n),
                "substeps_walked": walked, "substeps_rebuilt": rebuilt,
                "interactions_per_body_step": (npc + npp) / max(act, 1), "energy_err": (e1 - e0) / abs(e0),
                "speedup_vs_shared": out["shared"]["ms_per_cycle"] / ms,
                "particles_per_s_equivalent": 8 * a.n / (ms / 1e3)}
    out["what"] = ("cycle of dt_max = 8 dt: shared = 8 bonsai_steps of dt; etaE_rR = one bonsai_block_cycle "
                   "(accuracy eta = E) with a rebuild every R substeps (refits between; substeps where no "
                   "step ends only drift); "
                   "particles_per_s_equivalent = 8 N / cycle time")
    return out


SWEEP_CASES = [(1 << k, 1, (0.75,)) for k in range(15, 22)] + [
    (1 << 22, 2, (0.5, 0.75, 1.0)), (1 << 23, 1, (0.75,)), (1 << 24, 3, (0.5, 0.75, 1.0))]


def sweep_case(a, dev, stream, b, n, seed, theta, cpu_budget=0.0):
    """One (N, theta) case of the scaling sweep (group knobs from `a`):
    eps = 0.002, 5 KDK steps of dt = 1/256 after 2 untimed ones (CUDA events,
    L2 flushed between steps), then as many stage-timed steps.  Per stage:
    device ms per step and algorithmic GB/s against the measured copy
    bandwidth; walk FP32 rate against the measured FP32 peak; FP64 energy
    drift over the timed steps; p99 force error of the first evaluation at
    4096 stratified bodies (the library's direct sum)."""
    import numpy as np
    import torch
    import paper_1204_2280_gb300 as B
    import ctypes as C
    hbm = measured_hbm_gbs()
    eps, dt, steps = 0.002, 1.0 / 256, 5
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tot = (C.c_ulonglong * 2)()
    bz = B.Bonsai(B.Config(nleaf=a.nleaf, ncrit=a.ncrit, walk_warps=a.walk_warps, group_pack=a.group_pack,
                           list_capacity=a.list_capacity), stream=stream)
    bz.set_bodies(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.mass).to(dev),
                  torch.from_numpy(b.vel).to(dev))
    bz.build().multipoles().forces(theta, eps)
    p99 = B.bonsai_judge(bz.ctx, eps)
    d0 = B.bonsai_diagnostics(bz.ctx)
    for _ in range(2):
        bz.step(dt)
    bz.sync()
    ms, st, npc, npp = [], [], 0, 0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bz.step(dt)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    d1 = B.bonsai_diagnostics(bz.ctx)
    # stage times and interaction counts: as many further steps with stage
    # events (the timed steps above run without them)
    B.bonsai_set_stage_timing(bz.ctx, True)
    for k in range(steps + 2):
        flush.zero_()
        bz.step(dt)
        if k >= 2:
            st.append(B.bonsai_get_stage_times(bz.ctx))
            B._check(bz.ctx, B.lib().bonsai_get_counts(bz.ctx, None, None, tot))
            npc += int(tot[0]); npp += int(tot[1])
    _, ncells, ngroups = B.bonsai_get_sizes(bz.ctx)
    bz.sync()
    bz.close()
    del flush
    stage = dict(zip(B.STAGES, (np.array(st).sum(0) / steps).tolist()))
    sb = stage_bytes(n, ncells, ngroups)
    cpu = None
    if cpu_budget > 0 and theta == 0.75:
        # The paper's Fig. 1 stages on the FP64 oracle (host cores):
        # sorting + moving, tree construction, multipoles, walk.
        c = cpu_oracle_sample(b, theta, eps, a.nleaf, a.ncrit, cpu_budget, pack=a.group_pack, direct=False)
        cs = c["stage_s"]
        gpu_s = {"sort_move": (stage["keys"] + stage["sort"] + stage["reorder"]) / 1e3,
                 "build": stage["build"] / 1e3, "multipoles": stage["multipoles"] / 1e3,
                 "walk": stage["walk"] / 1e3}
        cpu_s = {"sort_move": cs["domain_keys"] + cs["sort_reorder"], "build": cs["build"],
                 "multipoles": cs["multipoles"], "walk": cs["walk"]}
        cpu = {"cores": c["cores"], "stage_s": cpu_s, "gpu_stage_s": gpu_s,
               "cpu_over_gpu": {k: cpu_s[k] / gpu_s[k] for k in cpu_s},
               "sample": c["sample"]}
    walk_s = stage["walk"] / 1e3
    tflops = (FLOP_PC * npc + FLOP_PP * npp) / steps / walk_s / 1e12
    t = sum(ms) / steps
    return {
        "mode": "sweep", "n": n, "seed": seed, "theta": theta, "eps": eps, "dt": dt,
        "nleaf": a.nleaf, "ncrit": a.ncrit, "group_pack": a.group_pack, "walk_warps": a.walk_warps,
        "list_capacity": a.list_capacity,
        "steps": steps, "ms_per_step": t, "particles_per_s": n / (t / 1e3),
        "stage_ms": stage,
        "stage_gbs": {k: sb[k] / (stage[k] / 1e3) / 1e9 for k in sb if stage[k] > 0},
        "stage_hbm_frac": {k: sb[k] / (stage[k] / 1e3) / 1e9 / hbm for k in sb if stage[k] > 0},
        "sort_reorder_build_hbm_frac": sum(sb[k] for k in ("sort", "reorder", "build")) /
            (sum(stage[k] for k in ("sort", "reorder", "build")) / 1e3) / 1e9 / hbm,
        "walk_tflops": tflops, "walk_fp32_frac": tflops / fp32_peak_tflops(),
        "interactions_per_body": {"pc": npc / (steps * n), "pp": npp / (steps * n)},
        "interactions_per_s": (npc + npp) / steps / walk_s,
        "ncells": ncells, "ngroups": ngroups,
        "p99_acc_err_t0": p99,
        "energy_drift": (d1[2] - d0[2]) / abs(d0[2]),
        "hbm_peak_gbs": hbm, "fp32_peak_tflops": fp32_peak_tflops(), "oracle": cpu}


def run_sweep(a, dev, stream):
    """Scaling sweep (group knobs from the command line): Plummer spheres N =
    2^15 .. 2^21 and 2^23 at theta = 0.75 (interactions per body vs N), N =
    2^22 (seed 2) and 2^24 (seed 3) at theta in {0.5, 0.75, 1.0}; one JSON
    line per case (sweep_case).  --sweep-cpu S adds the FP64 oracle's time
    per stage at theta = 0.75 on the host cores (sorting + moving, build,
    multipoles, and the walk of a random group sample of about S seconds
    extrapolated to N: the paper's Fig. 1)."""
    from paper_1204_2280_gb300 import workloads as W
    cases = list(SWEEP_CASES)
    if a.sweep_sizes:
        keep = {1 << int(x) for x in a.sweep_sizes.split(",")}
        cases = [c for c in cases if c[0] in keep]
    if a.sweep_thetas:
        keep_t = {float(x) for x in a.sweep_thetas.split(",")}
        cases = [(n, s, tuple(t for t in th if t in keep_t)) for n, s, th in cases]
    for n, seed, thetas in cases:
        b = W.plummer(n, seed)
        for theta in thetas:
            print(json.dumps(sweep_case(a, dev, stream, b, n, seed, theta, a.sweep_cpu)), flush=True)


def compact_sweep(a, dev, stream):
    """The bench line's scaling record (the paper's Fig. 1 / Fig. 2 on this
    GPU): the sweep's cases at theta = 0.75 for N = 2^16, 2^18, 2^22 and 2^24
    (seeds as in the sweep) with the bench's tuned group knobs; per case the
    step time, per-stage ms and algorithmic GB/s, the sort + reorder + build
    fraction of the copy bandwidth, the walk's FP32 fraction and the
    interactions per body."""
    from paper_1204_2280_gb300 import workloads as W
    out = []
    keep = ("n", "seed", "ms_per_step", "particles_per_s", "stage_ms", "stage_gbs", "stage_hbm_frac",
            "sort_reorder_build_hbm_frac", "walk_tflops", "walk_fp32_frac", "interactions_per_body",
            "ncells", "ngroups", "p99_acc_err_t0")
    for n, seed, _ in SWEEP_CASES:
        if n in (1 << 16, 1 << 18, 1 << 22, 1 << 24):
            r = sweep_case(a, dev, stream, W.plummer(n, seed), n, seed, 0.75)
            out.append({k: r[k] for k in keep})
    return {"theta": 0.75, "eps": 0.002, "dt": 1.0 / 256, "cases": out,
            "what": "5 timed KDK steps per N after 2 untimed, stage times from as many stage-timed steps; "
                    "GB/s are algorithmic bytes (STAGE_BYTES) over stage time"}


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def run_ours(a, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_1204_2280_gb300 as B
    from paper_1204_2280_gb300 import workloads as W
    import ctypes as C

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(dev)            # all torch and library work on one stream
    torch.cuda.set_stream(stream)
    b = W.plummer(a.n, a.seed)
    n = b.n
    bz = B.Bonsai(B.Config(nleaf=a.nleaf, ncrit=a.ncrit, walk_warps=a.walk_warps, group_pack=a.group_pack,
                           list_capacity=a.list_capacity), stream=stream)
    bz.set_bodies(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.mass).to(dev),
                  torch.from_numpy(b.vel).to(dev))
    if not a.no_autotune:
        a.ncrit, a.walk_warps, _ = B.bonsai_autotune(bz.ctx, a.theta, a.eps)
        cfg = B.bonsai_get_config(bz.ctx)
        a.group_pack, a.list_capacity = cfg.group_pack, cfg.list_capacity
    else:
        bz.build().multipoles().forces(a.theta, a.eps)
    B.bonsai_set_params(bz.ctx, a.theta, a.eps)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(a.warmup):
        bz.step(a.dt)
    bz.sync()
    tot = (C.c_ulonglong * 2)()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    sampler = ClockSampler(gpu_index(local_rank))
    barrier()
    sampler.start()
    time.sleep(0.3)
    step_ms, stage_ms, flops, npc, npp = [], [], [], [], []
    t_wall0 = time.perf_counter()
    for _ in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bz.step(a.dt)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    t_wall = time.perf_counter() - t_wall0
    barrier()
    clocks = sampler.stop()
    bz.sync()
    total_ms = sum(step_ms)
    from paper_1204_2280_gb300 import dist as D
    total_ms, _ = D.combine(total_ms, float(n * a.steps))
    value = world * n * a.steps / (total_ms / 1e3)

    # Stage breakdown and the walk's roofline: as many further steps with
    # stage events in the step graph (they add ~40 us per step, so the timed
    # steps above run without them), L2 flushed between steps.
    B.bonsai_set_stage_timing(bz.ctx, True)
    for _ in range(2):                          # eager, then re-captured with the events
        bz.step(a.dt)
    for _ in range(a.steps):
        flush.zero_()
        bz.step(a.dt)
        stage_ms.append(B.bonsai_get_stage_times(bz.ctx))
        B._check(bz.ctx, B.lib().bonsai_get_counts(bz.ctx, None, None, tot))
        npc.append(int(tot[0])); npp.append(int(tot[1]))
        flops.append(FLOP_PC * int(tot[0]) + FLOP_PP * int(tot[1]))
    B.bonsai_set_stage_timing(bz.ctx, False)
    bz.sync()
    stages = np.array(stage_ms).sum(0)
    walk_ms = float(stages[B.STAGES.index("walk")])
    achieved = sum(flops) / (walk_ms / 1e3) / 1e12
    peak = fp32_peak(local_rank)

    # End to end through the C ABI with host buffers.
    e2e = None
    if not a.no_e2e:
        hp = torch.from_numpy(b.pos).pin_memory().numpy()
        hm = torch.from_numpy(b.mass).pin_memory().numpy()
        hv = torch.from_numpy(b.vel).pin_memory().numpy()
        ha = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
        hpot = torch.empty(n, dtype=torch.float32).pin_memory().numpy()
        ts = []
        for s in range(a.steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            bz.set_bodies(hp, hm, hv)
            bz.build().multipoles().forces(a.theta, a.eps, ha, hpot)
            ts.append(time.perf_counter() - t0)
        ts = ts[1:]
        e2e = {"value": n * len(ts) / sum(ts), "unit": UNIT, "h2d_bytes_per_step": 28 * n,
               "d2h_bytes_per_step": 16 * n,
               "what": "set_bodies(host pos, mass, vel) + build + multipoles + forces(host acc, pot)"}
    bz.close()

    swp = compact_sweep(a, dev, stream) if (rank == 0 and not a.no_sweep) else None
    ens = None if a.no_ensemble else run_ensemble(a, dev, stream, rank, world)
    blk = None if a.no_block else run_block(a, dev, stream)
    sph = None if a.no_sph else run_sph(a, dev, stream)
    lrn = None if a.no_learned else run_learned(a, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_oracle_sample(b, a.theta, a.eps, a.nleaf, a.ncrit, a.cpu_budget, pack=a.group_pack)
        cpu.pop("t_step_s")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config(a, world),
            "roofline": {"bound": "alu", "kernel": "k_walk", "achieved": achieved,
                         "peak": peak["tflops"], "unit": "TFLOP/s", "frac": achieved / peak["tflops"],
                         "traffic": WALK_TRAFFIC.get((a.n, a.ncrit, a.group_pack)),
                         "peak_basis": {
                             "measured": "FMA-chain microbenchmark in this run: " + peak["how"],
                             "sms": peak["sms"], "sm_mhz_median": peak["sm_mhz_median"],
                             "derived_at_median_clock": peak["derived_at_median_clock"],
                             "derived_at_max_clock": peak["derived_at_max_clock"],
                             "frac_of_derived_at_max_clock": achieved / peak["derived_at_max_clock"],
                             "clock_reasons": peak["clock_reasons"]},
                         "flops_basis": f"{FLOP_PC} per body-cell + {FLOP_PP} per body-body interaction"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": kernels_per_step(a.ncrit, a.group_pack) * a.steps,
            "clocks": clocks,
            "stages_ms_per_step": {s: float(v) / a.steps for s, v in zip(B.STAGES, stages)},
            "stages_from": "as many further steps with stage events in the step graph (ms_per_step is timed without them)",
            "interactions_per_body": {"pc": sum(npc) / (n * a.steps), "pp": sum(npp) / (n * a.steps)},
            "interactions_per_s": (sum(npc) + sum(npp)) / (walk_ms / 1e3),
            "wall_s_timed_loop": t_wall,
            "sweep": swp,
            "ensemble": ens,
            "block": blk,
            "sph": sph,
            "learned": lrn,
        }
        print(json.dumps(line), flush=True)


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.sweep:
        import torch
        torch.cuda.set_device(local_rank)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        run_sweep(a, torch.device("cuda", local_rank), stream)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(a, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
