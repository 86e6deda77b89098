"""Physics pins of the oracle on the paper's workload (Sect. 2: Plummer
spheres, Plummer 1915) and of the shared-time-step leapfrog.

* Truncated Plummer potential in closed form: for r < R_t,
  Phi_t(r) = -(1/f) [ (r^2+a^2)^-1/2 - (R_t^2+a^2)^-1/2 ] - 1/R_t,
  f = (R_t / sqrt(R_t^2 + a^2))^3 (mass inside R_t, renormalised to 1).
  Phi_t(0) = -1.72148 and Phi_t(a) = -1.21678 for a = 3 pi/16, R_t = 10 a
  (tests/golden/plummer_potential.txt).
* Radial mass profile of the generator: Kolmogorov-Smirnov distance against
  M(<r)/f = r^3 / (r^2+a^2)^(3/2) / f.
* Zero total momentum; virial ratio near 1; two-body circular orbit with the
  leapfrog: second-order phase error, bounded energy error and time
  reversibility."""
import math
import os

import numpy as np
import pytest

from paper_1204_2280_gb300 import workloads as W

A = 3 * math.pi / 16
RT = 10 * A
F = (RT / math.sqrt(RT * RT + A * A)) ** 3
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "plummer_potential.txt")


def phi_t(r):
    return -(1 / F) * ((r * r + A * A) ** -0.5 - (RT * RT + A * A) ** -0.5) - 1 / RT


def test_golden_closed_form_values():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    assert phi_t(0.0) == pytest.approx(vals["phi_t_0"], abs=5e-6)
    assert phi_t(A) == pytest.approx(vals["phi_t_a"], abs=5e-6)
    assert F == pytest.approx(vals["f_trunc"], abs=5e-7)


def test_generator_radial_profile():
    b = W.plummer(1 << 15, 0)
    r = np.sort(np.linalg.norm(b.pos.astype(np.float64), axis=1))
    assert r.max() < RT * 1.01
    cdf = r ** 3 / (r * r + A * A) ** 1.5 / F
    emp = np.arange(1, r.size + 1) / r.size
    assert np.abs(cdf - emp).max() < 1.63 / math.sqrt(r.size) * 1.5   # ~ KS 1% level (COM shift)


def test_plummer_potential_closed_form(orc):
    """Radial-bin means of the softened direct-sum potential follow Phi_t."""
    n = 1 << 14
    b = W.plummer(n, 1)
    _, phi = orc.direct(b.pos, b.mass, 0.01)
    r = np.linalg.norm(b.pos.astype(np.float64), axis=1)
    edges = np.quantile(r, np.linspace(0.02, 0.98, 12))
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        want = phi_t(r[sel]).mean()
        assert phi[sel].mean() == pytest.approx(want, rel=1.5e-2)


def test_momentum_and_virial(orc):
    b = W.plummer(1 << 13, 2)
    assert np.abs((b.mass[:, None].astype(np.float64) * b.vel).sum(0)).max() < 1e-6
    _, phi = orc.direct(b.pos, b.mass, 0.001)
    e = orc.energy(b.pos, b.vel, b.mass, phi)
    K, Wp = e[0], e[1]
    assert 0.9 < 2 * K / abs(Wp) < 1.1
    assert e[6] == pytest.approx(1.0, rel=1e-6)


def two_body(orc, dt, steps, sign=1.0):
    """Equal masses 1/2 on a circular orbit of separation 1 (G = 1):
    relative speed sqrt(G M / r) = 1, each body at speed 1/2."""
    pos = np.array([[0.5, 0, 0], [-0.5, 0, 0]], np.float64)
    vel = np.array([[0, 0.5, 0], [0, -0.5, 0]], np.float64)
    mass = np.array([0.5, 0.5], np.float32)
    acc = orc.tree_forces(pos.astype(np.float32), mass, 0.75, 0.0).acc
    for _ in range(steps):
        pos, vel, acc, pot = orc.kdk_step(pos, vel, mass, acc, sign * dt, 0.75, 0.0)
    return pos, vel, acc


def energy2(pos, vel):
    d = np.linalg.norm(pos[0] - pos[1])
    return 0.25 * ((vel ** 2).sum()) - 0.25 / d


def test_leapfrog_two_body_circular(orc):
    e0 = energy2(np.array([[0.5, 0, 0], [-0.5, 0, 0]]), np.array([[0, 0.5, 0], [0, -0.5, 0]]))
    period = 2 * math.pi      # omega = v_rel / r = 1
    errs, perr = [], []
    for nstep in (64, 128):
        pos, vel, _ = two_body(orc, period / nstep, nstep)
        errs.append(abs(energy2(pos, vel) - e0))
        # back where it started after one period, up to an O(dt^2) phase error
        perr.append(np.linalg.norm(pos[0] - [0.5, 0, 0]))
    assert perr[0] < 0.02
    assert 3.0 < perr[0] / perr[1] < 5.5                 # second order
    assert max(errs) < 1e-6     # symplectic: no secular energy drift on the circle


def test_leapfrog_time_reversible(orc):
    dt = 0.05
    pos, vel, acc = two_body(orc, dt, 20)
    mass = np.array([0.5, 0.5], np.float32)
    for _ in range(20):
        pos, vel, acc, _ = orc.kdk_step(pos, vel, mass, acc, -dt, 0.75, 0.0)
    assert np.allclose(pos, [[0.5, 0, 0], [-0.5, 0, 0]], atol=1e-6)
