"""Host-side snapshots for checkpoint and resume.

A snapshot holds what a run needs to continue: the step counter, the time,
and the bodies in caller order (positions, velocities, masses and the
caller's ids).  Resuming loads it and hands pos, mass and vel to
bonsai_set_bodies; the first bonsai_step then recomputes the accelerations
of the loaded positions before its first kick, as after any set_bodies.

File layout (little-endian):
  8 bytes   magic b"BONSNAP1"
  int64     N
  int64     step
  float64   t
  float32   pos[N][3], vel[N][3], mass[N]
  int64     ids[N]
  8 bytes   BLAKE2b digest (8-byte) of everything before it

Nothing here touches the GPU; reading a context's bodies goes through
bonsai_get_bodies.
"""
from __future__ import annotations

import hashlib

import numpy as np

MAGIC = b"BONSNAP1"


def _digest(data: bytes) -> bytes:
    return hashlib.blake2b(data, digest_size=8).digest()


def save(path: str, pos, vel, mass, ids=None, step: int = 0, t: float = 0.0) -> None:
    pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1, 3)
    n = pos.shape[0]
    vel = np.ascontiguousarray(vel, dtype=np.float32).reshape(n, 3)
    mass = np.ascontiguousarray(mass, dtype=np.float32).reshape(n)
    ids = np.arange(n, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, dtype=np.int64).reshape(n)
    if n < 1:
        raise ValueError("a snapshot needs at least one body")
    body = b"".join([MAGIC, np.array([n, int(step)], "<i8").tobytes(), np.array([float(t)], "<f8").tobytes(),
                     pos.astype("<f4").tobytes(), vel.astype("<f4").tobytes(), mass.astype("<f4").tobytes(),
                     ids.astype("<i8").tobytes()])
    with open(path, "wb") as f:
        f.write(body)
        f.write(_digest(body))


def load(path: str) -> dict:
    with open(path, "rb") as f:
        data = f.read()
    if len(data) < 40 or data[:8] != MAGIC:
        raise ValueError(f"{path}: not a snapshot")
    n, step = np.frombuffer(data, "<i8", 2, 8).tolist()
    need = 8 + 16 + 8 + n * (12 + 12 + 4 + 8) + 8
    if n < 1 or len(data) != need:
        raise ValueError(f"{path}: truncated or inconsistent (N = {n}, {len(data)} bytes)")
    body, stored = data[:-8], data[-8:]
    if _digest(body) != stored:
        raise ValueError(f"{path}: checksum mismatch")
    t = float(np.frombuffer(data, "<f8", 1, 24)[0])
    off = 32
    pos = np.frombuffer(data, "<f4", 3 * n, off).reshape(n, 3).astype(np.float32); off += 12 * n
    vel = np.frombuffer(data, "<f4", 3 * n, off).reshape(n, 3).astype(np.float32); off += 12 * n
    mass = np.frombuffer(data, "<f4", n, off).astype(np.float32); off += 4 * n
    ids = np.frombuffer(data, "<i8", n, off).astype(np.int64)
    return {"n": n, "step": step, "t": t, "pos": pos, "vel": vel, "mass": mass, "ids": ids}


def save_context(path: str, ctx, mass, ids=None, step: int = 0, t: float = 0.0) -> None:
    """Snapshot of a context's bodies (caller order, read back through
    bonsai_get_bodies); the masses are the caller's, as passed to
    bonsai_set_bodies."""
    from . import bonsai_get_bodies, bonsai_get_sizes
    n, _, _ = bonsai_get_sizes(ctx)
    pos = np.zeros((n, 3), np.float32)
    vel = np.zeros((n, 3), np.float32)
    bonsai_get_bodies(ctx, pos, vel)
    save(path, pos, vel, mass, ids, step, t)
