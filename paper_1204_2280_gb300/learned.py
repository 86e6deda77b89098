"""Training and use of the learned far-field correction through the C ABI.

Orchestration only: snapshots come from the seeded generators (randomly
rotated copies of Plummer spheres and mergers), training samples from
``bonsai_learn_samples`` (walk features at the coarse theta plus direct-sum
labels on the GPU), training from ``bonsai_mlp_train`` (the library's
forward, backward and AdamW kernels).  Weights are stored as .npz files
(params float32[5187], norm float32[25]).
"""
from __future__ import annotations

import numpy as np

from . import Bonsai, Config, MLP, bonsai_get_bodies, bonsai_learn_samples, bonsai_set_params
from . import workloads as W


def rotated(b: W.Bodies, seed: int) -> W.Bodies:
    """A randomly rotated copy (positions and velocities), float32."""
    R = W.random_rotation(seed)
    return W.Bodies((b.pos.astype(np.float64) @ R.T).astype(np.float32),
                    (b.vel.astype(np.float64) @ R.T).astype(np.float32), b.mass.copy())


def snapshots(n: int, plummer_seeds, rotations: int = 1, merger_seeds=(), rot_seed0: int = 7000):
    """Rotated copies of Plummer spheres (and two-sphere mergers) of n bodies."""
    k = 0
    for s in plummer_seeds:
        base = W.plummer(n, s)
        for _ in range(rotations):
            yield rotated(base, rot_seed0 + k)
            k += 1
    for s in merger_seeds:
        base = W.merger(n, s)
        for _ in range(rotations):
            yield rotated(base, rot_seed0 + k)
            k += 1


def _rotated_plummer(args):
    n, seed, rot_seed = args
    return rotated(W.plummer(n, seed), rot_seed)


def snapshots_parallel(n: int, plummer_seeds, rot_seed0: int = 7000, workers: int = 0):
    """The rotated Plummer spheres of snapshots(n, plummer_seeds), generated
    by a pool of host processes (spawned, so that no CUDA state is
    inherited) and yielded in seed order as they are consumed."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    seeds = list(plummer_seeds)
    workers = workers or max(1, min(len(seeds), (os.cpu_count() or 2) - 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        jobs = [(n, s, rot_seed0 + k) for k, s in enumerate(seeds)]
        window = 2 * workers                  # bounded look-ahead: at most this many snapshots held
        futs = [ex.submit(_rotated_plummer, j) for j in jobs[:window]]
        for k in range(len(jobs)):
            b = futs[k].result()
            futs[k] = None
            if k + window < len(jobs):
                futs.append(ex.submit(_rotated_plummer, jobs[k + window]))
            yield b


def evolved(b: W.Bodies, steps: int, every: int, theta: float = 0.5, eps: float = 0.002,
            dt: float = 1.0 / 64, ncrit: int = 64):
    """Snapshots of a system stepped by the plain tree-code at theta: the
    state after every `every`-th of `steps` leapfrog steps (host copies)."""
    with Bonsai(Config(ncrit=ncrit)) as bz:
        bz.set_bodies(b.pos, b.mass, b.vel)
        bonsai_set_params(bz.ctx, theta, eps)
        for s in range(1, steps + 1):
            bz.step(dt)
            if s % every == 0:
                pos = np.zeros((b.n, 3), np.float32)
                vel = np.zeros((b.n, 3), np.float32)
                bonsai_get_bodies(bz.ctx, pos, vel)
                yield W.Bodies(pos, vel, b.mass.copy())


def training_set(bodies, theta: float = 1.0, eps: float = 0.01, per_snapshot: int = 4096,
                 ncrit: int = 64, nleaf: int = 16, seed: int = 0):
    """(X, Y): features and targets of per_snapshot sampled bodies of every
    snapshot, from the coarse-theta walk and the GPU direct sum."""
    xs, ys = [], []
    with Bonsai(Config(nleaf=nleaf, ncrit=ncrit)) as bz:
        for k, b in enumerate(bodies):
            bz.set_bodies(b.pos, b.mass, b.vel).build().multipoles()
            X, Y, _ = bonsai_learn_samples(bz.ctx, theta, eps, min(per_snapshot, b.n), seed + k)
            xs.append(X)
            ys.append(Y)
    return np.concatenate(xs), np.concatenate(ys)


def train(X, Y, epochs: int = 40, batch: int = 8192, lr: float = 1e-3, wd: float = 1e-4,
          seed: int = 0) -> tuple[MLP, np.ndarray]:
    net = MLP(seed)
    losses = net.train(np.ascontiguousarray(X, np.float32), np.ascontiguousarray(Y, np.float32),
                       epochs=epochs, batch=batch, lr=lr, wd=wd, seed=seed)
    return net, losses


def save(net: MLP, path: str):
    p, nrm = net.get_params()
    np.savez(path, params=p, norm=nrm)


def load(path: str) -> MLP:
    d = np.load(path)
    net = MLP(0)
    net.set_params(d["params"], d["norm"])
    return net
