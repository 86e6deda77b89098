"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs."""
import numpy as np

import oracle
import paper_1204_2280_gb300 as B
from paper_1204_2280_gb300 import workloads as W


def edge_bodies(n, seed):
    """Plummer bodies plus exact duplicates and a tight clump (deep cells,
    identical keys, oversize leaves)."""
    b = W.plummer(n, seed)
    pos = b.pos.copy()
    k = max(1, n // 50)
    pos[1:1 + k] = pos[0]                                    # identical positions
    rng = np.random.default_rng(seed + 99)
    pos[1 + k:1 + 2 * k] = pos[0] + rng.standard_normal((k, 3)).astype(np.float32) * 1e-6
    return W.Bodies(pos, b.vel, b.mass)


def gpu_run(pos, mass, vel=None, theta=0.75, eps=0.01, nleaf=16, ncrit=32, forces=True,
            device_io=True, **cfg):
    """set_bodies -> build -> multipoles -> forces; returns a dict of results
    copied out through the C ABI."""
    import torch
    out = {}
    cfgs = B.Config(nleaf=nleaf, ncrit=ncrit, **cfg)
    with B.Bonsai(cfgs) as bz:
        if device_io:
            tp = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
            tm = torch.from_numpy(np.ascontiguousarray(mass)).cuda()
            tv = None if vel is None else torch.from_numpy(np.ascontiguousarray(vel)).cuda()
            bz.set_bodies(tp, tm, tv)
        else:
            bz.set_bodies(np.ascontiguousarray(pos), np.ascontiguousarray(mass),
                          None if vel is None else np.ascontiguousarray(vel))
        bz.build()
        out["domain"] = B.bonsai_get_domain(bz.ctx)
        out["keys"], out["perm"] = B.bonsai_get_keys(bz.ctx)
        out["tree"] = B.bonsai_get_tree(bz.ctx)
        out["groups"] = B.bonsai_get_groups(bz.ctx)
        bz.multipoles()
        out["mono"], out["quad"] = B.bonsai_get_moments(bz.ctx)
        if forces:
            n = mass.shape[0]
            if device_io:
                acc = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
                pot = torch.zeros(n, dtype=torch.float32, device="cuda")
                bz.forces(theta, eps, acc, pot)
                torch.cuda.synchronize()
                out["acc"], out["pot"] = acc.cpu().numpy(), pot.cpu().numpy()
            else:
                acc = np.zeros((n, 3), np.float32)
                pot = np.zeros(n, np.float32)
                bz.forces(theta, eps, acc, pot)
                out["acc"], out["pot"] = acc, pot
            out["n_pc"], out["n_pp"], out["tot"] = B.bonsai_get_counts(bz.ctx)
        B.bonsai_sync(bz.ctx)
    return out


def rel_err(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)
