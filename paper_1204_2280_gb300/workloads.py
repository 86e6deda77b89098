"""Seeded synthetic initial conditions shared by the CUDA path and the oracle.

This module draws random numbers and nothing else: it holds none of the
tree-code's arithmetic (no keys, no tree, no moments, no forces), so both the
GPU path and the FP64 oracle can take their inputs from it without sharing any
part of the method.

Workloads (Sect. 2 of the paper: Plummer spheres with N = 2^15 ... 2^22 bodies):

* ``plummer(n, seed)`` -- a Plummer sphere in Henon units (G = M = 1,
  a = 3*pi/16), radii from the inverse of the cumulative mass profile, cut at
  r < 10 a, isotropic positions and velocities, velocities from the Plummer
  distribution function by von Neumann rejection, shifted to the centre-of-mass
  frame in float64 and then rounded to float32.
* ``merger(n, seed)`` -- two such spheres of n/2 bodies, each of mass 1,
  centred at x = +-2 and moving at -+0.25 along x (relative speed 0.5).
* ``ensemble(nsys, seed0)`` -- nsys independent spheres; system k draws its
  size N_k = round(2^(12 + 6 U)) from the first uniform U of its own
  generator (seed0 + k), then its sphere from the same generator.

All arrays are float32: ``pos`` (n, 3), ``vel`` (n, 3), ``mass`` (n,).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

A_HENON = 3.0 * math.pi / 16.0   # Plummer scale length in Henon units
R_TRUNC = 10.0                   # truncation radius in units of a


@dataclass
class Bodies:
    pos: np.ndarray   # float32 (n, 3)
    vel: np.ndarray   # float32 (n, 3)
    mass: np.ndarray  # float32 (n,)

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere: cos(theta) ~ U(-1,1), phi ~ U(0,2pi)."""
    c = rng.uniform(-1.0, 1.0, n)
    p = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    return np.stack([s * np.cos(p), s * np.sin(p), c], axis=1)


def _plummer_f64(rng: np.random.Generator, n: int, a: float = A_HENON,
                 rt: float = R_TRUNC) -> tuple[np.ndarray, np.ndarray]:
    """Positions and velocities (float64, unshifted) of an n-body Plummer sphere
    of unit mass and scale length a, truncated at radius rt*a."""
    # Mass fraction inside the truncation radius; u ~ U(0, f) keeps r < rt*a.
    f = (rt / math.sqrt(rt * rt + 1.0)) ** 3
    u = rng.uniform(0.0, f, n)
    u = np.maximum(u, np.finfo(np.float64).tiny)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    pos = _isotropic(rng, n) * r[:, None]
    # Speed q = v / v_esc from g(q) = q^2 (1 - q^2)^(7/2), max 0.0922 at q^2 = 2/9.
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x1 = rng.uniform(0.0, 1.0, todo.size)
        x2 = rng.uniform(0.0, 0.1, todo.size)
        ok = x2 < x1 * x1 * (1.0 - x1 * x1) ** 3.5
        q[todo[ok]] = x1[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (r * r + a * a) ** -0.25
    vel = _isotropic(rng, n) * (q * vesc)[:, None]
    return pos, vel


def _to_bodies(pos: np.ndarray, vel: np.ndarray, mass64: np.ndarray) -> Bodies:
    mtot = mass64.sum()
    pos = pos - (mass64[:, None] * pos).sum(0) / mtot
    vel = vel - (mass64[:, None] * vel).sum(0) / mtot
    return Bodies(pos.astype(np.float32), vel.astype(np.float32),
                  mass64.astype(np.float32))


def plummer_from(rng: np.random.Generator, n: int) -> Bodies:
    pos, vel = _plummer_f64(rng, n)
    return _to_bodies(pos, vel, np.full(n, 1.0 / n))


def plummer(n: int, seed: int) -> Bodies:
    """Plummer sphere of n equal-mass bodies (total mass 1), seeded."""
    return plummer_from(np.random.default_rng(seed), n)


def merger(n: int, seed: int, sep: float = 2.0, vrel: float = 0.5) -> Bodies:
    """Two Plummer spheres of n//2 bodies and unit mass each, centres at x=+-sep,
    approaching along x with relative speed vrel; zero total momentum."""
    rng = np.random.default_rng(seed)
    h = n // 2
    p1, v1 = _plummer_f64(rng, h)
    p2, v2 = _plummer_f64(rng, n - h)
    p1 -= p1.mean(0); v1 -= v1.mean(0)
    p2 -= p2.mean(0); v2 -= v2.mean(0)
    p1[:, 0] += sep; v1[:, 0] -= 0.5 * vrel
    p2[:, 0] -= sep; v2[:, 0] += 0.5 * vrel
    mass = np.concatenate([np.full(h, 1.0 / h), np.full(n - h, 1.0 / (n - h))])
    return _to_bodies(np.concatenate([p1, p2]), np.concatenate([v1, v2]), mass)


def ensemble_sizes(nsys: int, seed0: int = 100, lo_log2: float = 12.0,
                   span_log2: float = 6.0) -> list[int]:
    return [int(round(2.0 ** (lo_log2 + span_log2 *
                              np.random.default_rng(seed0 + k).uniform())))
            for k in range(nsys)]


def ensemble(nsys: int, seed0: int = 100, lo_log2: float = 12.0,
             span_log2: float = 6.0) -> list[Bodies]:
    """nsys independent Plummer spheres with log-uniform sizes in
    [2^lo_log2, 2^(lo_log2+span_log2)]."""
    out = []
    for k in range(nsys):
        rng = np.random.default_rng(seed0 + k)
        nk = int(round(2.0 ** (lo_log2 + span_log2 * rng.uniform())))
        out.append(plummer_from(rng, nk))
    return out


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct body indices drawn uniformly without replacement (sorted)."""
    k = min(k, n)
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def random_rotation(seed: int) -> np.ndarray:
    """A uniformly random 3x3 rotation matrix (QR of a Gaussian matrix)."""
    g = np.random.default_rng(seed).standard_normal((3, 3))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q
