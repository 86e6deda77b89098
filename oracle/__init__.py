"""FP64 CPU oracle of the Bonsai tree-code hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package.  The product library never loads
it and shares no code with it.  The arithmetic lives in ``bonsai_oracle.c``
(plain C, FP64, OpenMP over independent groups/cells); this module compiles it
with gcc on first use and marshals numpy arrays through ctypes.

Paper: "Bonsai: A GPU Tree-Code", Sect. 1 (Barnes-Hut tree-code and the
O(N^2) direct sum) and Sect. 2 (Morton sort, moving, tree-construction,
multipole moments, tree-traverse under the opening angle theta).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bonsai_oracle.c")
_LIB = os.path.join(_HERE, "libbonsai_oracle.so")
_lock = threading.Lock()
_lib = None

L_BITS = 21


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            p = C.c_void_p
            i64 = C.c_int64
            d = C.c_double
            L.oracle_domain.argtypes = [p, i64, p, p]
            L.oracle_keys.argtypes = [p, i64, p, d, p]
            L.oracle_interleave.argtypes = [C.c_uint32] * 3
            L.oracle_interleave.restype = C.c_uint64
            L.oracle_sort.argtypes = [p, i64, p]
            L.oracle_build.argtypes = [p, i64, C.c_int, i64, p, p, p, p, p, p]
            L.oracle_build.restype = i64
            L.oracle_groups.argtypes = [i64, p, p, p, p, C.c_int, C.c_int, i64, p, p]
            L.oracle_groups.restype = i64
            L.oracle_moments.argtypes = [i64, p, p, p, p, p, p, p]
            L.oracle_open_radius.argtypes = [i64, p, p, p, p, d, p, d, p, p]
            L.oracle_refit_extent.argtypes = [i64, p, p, p, p, p, p, p, d, p, p]
            L.oracle_sph_kernel.argtypes = [d, d]
            L.oracle_sph_kernel.restype = d
            L.oracle_sph_density.argtypes = [p, p, p, i64, p, i64, p, p]
            L.oracle_walk.argtypes = [i64, p, p, i64, p, p, p, p, p, p, p, p, i64, p, p,
                                      d, d, d, p, p, p, p, p, p, p, p]
            L.oracle_direct.argtypes = [p, p, i64, p, i64, d, p, p]
            L.oracle_energy.argtypes = [p, p, p, p, i64, p]
            L.oracle_pc_eval.argtypes = [p, p, d, p, d, p, p]
            L.oracle_cell_cube.argtypes = [i64, p, p, p, p, d, p, p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


# ---------------------------------------------------------------------------
# Stage wrappers (numpy in, numpy out)
# ---------------------------------------------------------------------------

def domain(pos) -> tuple[np.ndarray, float]:
    """Per-axis float minimum and the power-of-two cube side S."""
    pos = _f32(pos)
    mn = np.zeros(3, np.float32)
    S = C.c_double()
    rc = lib().oracle_domain(_ptr(pos), pos.shape[0], _ptr(mn), C.byref(S))
    if rc:
        raise ValueError("oracle_domain: empty input")
    return mn, S.value


def keys(pos, mn=None, S=None) -> np.ndarray:
    """63-bit Morton keys (uint64) of float32 positions (n, 3)."""
    pos = _f32(pos)
    if mn is None:
        mn, S = domain(pos)
    out = np.zeros(pos.shape[0], np.uint64)
    lib().oracle_keys(_ptr(pos), pos.shape[0], _ptr(_f32(mn)), float(S), _ptr(out))
    return out


def interleave(qx: int, qy: int, qz: int) -> int:
    return int(lib().oracle_interleave(qx, qy, qz))


def sort(k) -> np.ndarray:
    """Permutation (uint32) that stably sorts the keys."""
    k = np.ascontiguousarray(k, dtype=np.uint64)
    perm = np.zeros(k.shape[0], np.uint32)
    if lib().oracle_sort(_ptr(k), k.shape[0], _ptr(perm)):
        raise MemoryError("oracle_sort")
    return perm


@dataclass
class Tree:
    body_begin: np.ndarray
    body_count: np.ndarray
    child_begin: np.ndarray
    nchild: np.ndarray
    level: np.ndarray
    parent: np.ndarray

    @property
    def ncells(self) -> int:
        return int(self.body_begin.shape[0])


def build_tree(skeys, nleaf: int = 16) -> Tree:
    skeys = np.ascontiguousarray(skeys, dtype=np.uint64)
    n = skeys.shape[0]
    cap = max(64, 2 * n + 64)
    while True:
        arrs = [np.zeros(cap, np.int32) for _ in range(6)]
        nc = lib().oracle_build(_ptr(skeys), n, nleaf, cap, *[_ptr(a) for a in arrs])
        if nc >= 0:
            break
        cap *= 2
    return Tree(*[a[:nc].copy() for a in arrs])


def groups(tree: Tree, ncrit: int = 32, pack: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Walk groups in key order (begin, count); pack: consecutive siblings
    packed greedily up to ncrit bodies."""
    cap = int(tree.body_count[0]) + 64      # groups hold >= 1 body each
    gb = np.zeros(cap, np.int32)
    gc = np.zeros(cap, np.int32)
    ng = lib().oracle_groups(tree.ncells, _ptr(tree.body_begin), _ptr(tree.body_count),
                             _ptr(tree.nchild), _ptr(tree.parent), ncrit, int(bool(pack)), cap,
                             _ptr(gb), _ptr(gc))
    if ng < 0:
        raise MemoryError("oracle_groups")
    return gb[:ng].copy(), gc[:ng].copy()


def moments(tree: Tree, spos, smass):
    spos, smass = _f32(spos), _f32(smass)
    nc = tree.ncells
    M = np.zeros(nc)
    com = np.zeros((nc, 3))
    Q = np.zeros((nc, 6))
    lib().oracle_moments(nc, _ptr(tree.body_begin), _ptr(tree.body_count), _ptr(spos),
                         _ptr(smass), _ptr(M), _ptr(com), _ptr(Q))
    return M, com, Q


def open_radius(tree: Tree, skeys, mn, S, com, theta: float, ext=None) -> np.ndarray:
    """l / theta + |com - centre| per cell; with ext (a refit's enlarged
    half sides, refit_extent) 2 ext / theta + |com - centre|."""
    ro = np.zeros(tree.ncells)
    lib().oracle_open_radius(tree.ncells, _ptr(tree.body_begin), _ptr(tree.level),
                             _ptr(np.ascontiguousarray(skeys, np.uint64)), _ptr(_f32(mn)),
                             float(S), _ptr(np.ascontiguousarray(com)), float(theta), _ptr(ro),
                             _ptr(np.ascontiguousarray(ext, np.float64)) if ext is not None else None)
    return ro


def refit_extent(tree: Tree, skeys, mn, S, spos) -> np.ndarray:
    """Half side of each cell's cube about its build-time centre enlarged to
    hold its bodies at spos (sorted order), bounded from the leaves up."""
    ext = np.zeros(tree.ncells)
    rc = lib().oracle_refit_extent(tree.ncells, _ptr(tree.body_begin), _ptr(tree.body_count),
                                   _ptr(tree.child_begin), _ptr(tree.nchild), _ptr(tree.level),
                                   _ptr(np.ascontiguousarray(skeys, np.uint64)), _ptr(_f32(mn)), float(S),
                                   _ptr(_f32(spos)), _ptr(ext))
    if rc:
        raise MemoryError("oracle_refit_extent")
    return ext


def cell_cube(tree: Tree, skeys, mn, S):
    """Geometric centre (ncells, 3) and side (ncells,) of every cell."""
    ctr = np.zeros((tree.ncells, 3)); side = np.zeros(tree.ncells)
    lib().oracle_cell_cube(tree.ncells, _ptr(tree.body_begin), _ptr(tree.level),
                           _ptr(np.ascontiguousarray(skeys, np.uint64)), _ptr(_f32(mn)), float(S),
                           _ptr(ctr), _ptr(side))
    return ctr, side


def walk(spos, smass, tree: Tree, M, com, Q, r_open, gbeg, gcnt, eps: float,
         tau_abs: float = 0.0, tau_rel: float = 0.0, bins: bool = False, active=None):
    """Group walk in sorted order; active (bool per sorted body, optional):
    only those bodies take forces, each group's box is its active bodies'
    box; the outputs of inactive bodies stay zero."""
    spos, smass = _f32(spos), _f32(smass)
    n = spos.shape[0]
    acc = np.zeros((n, 3))
    pot = np.zeros(n)
    npc = np.zeros(n, np.int32)
    npp = np.zeros(n, np.int32)
    flag = np.zeros(n, np.int8)
    nb = np.zeros((n, 4), np.int32) if bins else None
    rc = lib().oracle_walk(n, _ptr(spos), _ptr(smass), tree.ncells, _ptr(tree.body_begin),
                           _ptr(tree.body_count), _ptr(tree.child_begin), _ptr(tree.nchild),
                           _ptr(np.ascontiguousarray(M)), _ptr(np.ascontiguousarray(com)),
                           _ptr(np.ascontiguousarray(Q)), _ptr(np.ascontiguousarray(r_open)),
                           gbeg.shape[0], _ptr(gbeg), _ptr(gcnt), float(eps), float(tau_abs),
                           float(tau_rel), _ptr(acc), _ptr(pot), _ptr(npc), _ptr(npp), _ptr(flag),
                           _ptr(tree.level) if bins else None, _ptr(nb) if bins else None,
                           _ptr(np.ascontiguousarray(active, np.int8)) if active is not None else None)
    if rc:
        raise ValueError("oracle_walk: a body's own leaf was accepted (theta too large)")
    if bins:
        return acc, pot, npc, npp, flag, nb
    return acc, pot, npc, npp, flag


def direct(pos, mass, eps: float, idx=None):
    """FP64 direct sum; idx selects target bodies (all when None)."""
    pos, mass = _f32(pos), _f32(mass)
    n = pos.shape[0]
    idx = np.arange(n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, np.int64)
    acc = np.zeros((idx.shape[0], 3))
    pot = np.zeros(idx.shape[0])
    lib().oracle_direct(_ptr(pos), _ptr(mass), n, _ptr(idx), idx.shape[0], float(eps),
                        _ptr(acc), _ptr(pot))
    return acc, pot


def pc_eval(x, com, M: float, Q, eps: float):
    """Acceleration and potential at x from one cell (monopole + quadrupole)."""
    x = np.ascontiguousarray(x, np.float64); com = np.ascontiguousarray(com, np.float64)
    Q = np.ascontiguousarray(Q, np.float64)
    a = np.zeros(3); phi = C.c_double()
    lib().oracle_pc_eval(_ptr(x), _ptr(com), float(M), _ptr(Q), float(eps), _ptr(a), C.byref(phi))
    return a, phi.value


def energy(pos, vel, mass, pot) -> np.ndarray:
    out = np.zeros(8)
    lib().oracle_energy(_ptr(_f32(pos)), _ptr(_f32(vel)), _ptr(_f32(mass)),
                        _ptr(np.ascontiguousarray(pot, np.float64)), _f32(mass).shape[0], _ptr(out))
    return out


# ---------------------------------------------------------------------------
# The whole hot path, stage by stage, in the paper's order
# ---------------------------------------------------------------------------

@dataclass
class TreeForces:
    mn: np.ndarray
    S: float
    keys: np.ndarray          # caller order
    perm: np.ndarray          # sorted position -> caller index
    tree: Tree
    gbeg: np.ndarray
    gcnt: np.ndarray
    M: np.ndarray
    com: np.ndarray
    Q: np.ndarray
    r_open: np.ndarray
    acc: np.ndarray           # caller order (n, 3)
    pot: np.ndarray           # caller order
    n_pc: np.ndarray          # caller order
    n_pp: np.ndarray
    borderline: np.ndarray    # caller order, bool
    npc_bins: np.ndarray      # caller order (n, 4): accepted cells per level bin
    group_of: np.ndarray      # caller order: index of the body's group


def tree_forces(pos, mass, theta: float, eps: float, nleaf: int = 16, ncrit: int = 32,
                tau_abs: float = 0.0, tau_rel: float = 0.0, pack: bool = False) -> TreeForces:
    """Keys -> sort -> move -> build -> groups -> moments -> walk (FP64)."""
    pos, mass = _f32(pos), _f32(mass)
    mn, S = domain(pos)
    k = keys(pos, mn, S)
    perm = sort(k)
    skeys = k[perm]
    spos, smass = pos[perm], mass[perm]
    tree = build_tree(skeys, nleaf)
    gb, gc = groups(tree, ncrit, pack)
    M, com, Q = moments(tree, spos, smass)
    ro = open_radius(tree, skeys, mn, S, com, theta)
    acc_s, pot_s, npc_s, npp_s, flag_s, nb_s = walk(spos, smass, tree, M, com, Q, ro, gb, gc, eps,
                                                    tau_abs, tau_rel, bins=True)
    n = pos.shape[0]
    acc = np.zeros((n, 3)); acc[perm] = acc_s
    pot = np.zeros(n); pot[perm] = pot_s
    npc = np.zeros(n, np.int32); npc[perm] = npc_s
    npp = np.zeros(n, np.int32); npp[perm] = npp_s
    fl = np.zeros(n, bool); fl[perm] = flag_s.astype(bool)
    nb = np.zeros((n, 4), np.int32); nb[perm] = nb_s
    gid = np.zeros(n, np.int64); gid[perm] = np.repeat(np.arange(gb.shape[0]), gc)
    return TreeForces(mn, S, k, perm, tree, gb, gc, M, com, Q, ro, acc, pot, npc, npp, fl, nb, gid)


def kdk_step(pos, vel, mass, acc0, dt: float, theta: float, eps: float, nleaf: int = 16,
             ncrit: int = 32, pack: bool = False):
    """One kick-drift-kick leapfrog step (shared time step).  acc0 is the
    acceleration at the start; positions are rounded to float32 after the
    drift (the stored state is float32), everything else is float64.
    Returns (pos1 float64, vel1 float64, acc1 float64, pot1)."""
    pos = np.asarray(pos, np.float64)
    vel = np.asarray(vel, np.float64)
    vh = vel + 0.5 * dt * np.asarray(acc0, np.float64)
    x1 = pos + dt * vh
    x1f = x1.astype(np.float32)
    tf = tree_forces(x1f, mass, theta, eps, nleaf, ncrit, pack=pack)
    v1 = vh + 0.5 * dt * tf.acc
    return x1, v1, tf.acc, tf.pot


# ---------------------------------------------------------------------------
# Block (hierarchical) time steps
# ---------------------------------------------------------------------------
# Sect. 1 and 3 of the paper: with the whole tree-code on the GPU, a block
# time-step scheme walks only the N_active bodies that have to be updated
# (the walk time falls by N / N_active), and between rebuilds only the
# multipole moments are recomputed; the full tree is rebuilt when the walk
# slows down.  The paper fixes no scheme; the readings here:
#  * body i steps with dt_max / 2^k_i; k_i is the smallest level in
#    [0, kmax] with dt_max / 2^k <= eta * sqrt(eps / |a_i|), decided in
#    float32 as 16^k >= r, r = c * |a|^2, c = dt_max^4 / (eta^4 eps^2)
#    (rounded to float32 once), |a|^2 summed x, y, z without fused operations;
#  * a cycle of dt_max is 2^kmax substeps of dt_min = dt_max / 2^kmax, with
#    every body synchronised at its start and end: at the start each body
#    gets its level and an opening half kick a * dt_i / 2; each substep
#    drifts every body by dt_min, refreshes the tree (a rebuild every
#    `rebuild_every` substeps, else new moments of the existing cells at the
#    current positions with opening radii from each cell's build-time cube
#    enlarged to hold its bodies), walks the active bodies (those whose step ends now:
#    s a multiple of 2^(kmax - k_i)) and gives them the closing half kick;
#    before the last substep they then take a new level, no coarser than the
#    substep allows (k >= kmax - trailing zeros of s), and the opening half
#    kick of their next step.

def block_constant(dt_max: float, eta: float, eps: float) -> np.float32:
    """c = dt_max^4 / (eta^4 eps^2) in float64 from the float32 parameters,
    then rounded to float32 (the level decision's constant)."""
    d, e, s = float(np.float32(dt_max)), float(np.float32(eta)), float(np.float32(eps))
    d2 = d * d
    e2 = e * e
    return np.float32((d2 * d2) / ((e2 * e2) * (s * s)))


def block_level(acc, c32, kmax: int) -> np.ndarray:
    """Level of each body from its acceleration (n, 3), in float32."""
    a = np.asarray(acc, np.float32)
    a2 = (a[:, 0] * a[:, 0] + a[:, 1] * a[:, 1]) + a[:, 2] * a[:, 2]
    r = np.float32(c32) * a2
    k = np.zeros(a.shape[0], np.int32)
    for lev in range(1, kmax + 1):
        k += (r > np.float32(16.0) ** (lev - 1)).astype(np.int32)
    return k


def _ctz(s: int) -> int:
    return (s & -s).bit_length() - 1


class _BlockTree:
    """Tree of a rebuild: sort order, cells, groups and the build-time
    geometry (keys, domain) that the opening radii keep until the next one."""

    def __init__(self, x32, nleaf, ncrit, pack):
        self.mn, self.S = domain(x32)
        k = keys(x32, self.mn, self.S)
        self.perm = sort(k)
        self.skeys = k[self.perm]
        self.tree = build_tree(self.skeys, nleaf)
        self.gb, self.gc = groups(self.tree, ncrit, pack)

    def forces(self, x32, mass, theta, eps, active):
        """Accelerations and potentials (caller order) of the active bodies:
        moments of the cells at the current positions, opening radii from
        each cell's cube enlarged to hold its current bodies (the plain
        radius right after a rebuild) and the current com, walk of the
        active bodies."""
        p = self.perm
        spos, smass = np.ascontiguousarray(x32[p]), np.ascontiguousarray(mass[p])
        M, com, Q = moments(self.tree, spos, smass)
        ext = refit_extent(self.tree, self.skeys, self.mn, self.S, spos)
        ro = open_radius(self.tree, self.skeys, self.mn, self.S, com, theta, ext)
        acc_s, pot_s, _, _, _ = walk(spos, smass, self.tree, M, com, Q, ro, self.gb, self.gc, eps,
                                     active=np.asarray(active)[p])
        n = x32.shape[0]
        acc = np.zeros((n, 3)); acc[p] = acc_s
        pot = np.zeros(n); pot[p] = pot_s
        return acc, pot


def block_cycle(pos, vel, mass, acc, dt_max: float, kmax: int, eta: float, theta: float, eps: float,
                nleaf: int = 16, ncrit: int = 32, pack: bool = False, rebuild_every: int = 1,
                clock: bool = False, schedule: bool = False):
    """One cycle of block time steps from a synchronised state (acc: the
    acceleration at pos).  State in float64; the tree and forces see the
    positions rounded to float32 (the stored state is float32).

    A substep at which no body's step ends only drifts: tree work (rebuild or
    refit) and the walk happen at the substeps where some step ends, and a
    rebuild scheduled for a substep without one (every rebuild_every-th
    substep, starting with the first) is taken at the next substep that has
    one.  Returns (pos, vel, acc, pot, levels at the start, active bodies per
    substep), with clock=True also each body's time advanced by the steps it
    completed (dt_max for every body when the cycle ends synchronised), with
    schedule=True also the substeps walked and the substeps rebuilt."""
    mass = np.asarray(mass, np.float32)
    x = np.array(pos, np.float64)
    v = np.array(vel, np.float64)
    a = np.array(acc, np.float64)
    pot = np.zeros(x.shape[0])
    nsub = 1 << kmax
    dtm = dt_max / nsub
    c32 = block_constant(dt_max, eta, eps)
    lev = block_level(a, c32, kmax)
    lev0 = lev.copy()
    h = (1 << (kmax - lev)) * dtm / 2
    v += a * h[:, None]
    bt = None
    due = False
    nactive, walked, rebuilt = [], [], []
    t_done = np.zeros(x.shape[0])
    for s in range(1, nsub + 1):
        x += v * dtm
        if (s - 1) % rebuild_every == 0:
            due = True
        act = (s % (1 << (kmax - lev))) == 0
        nactive.append(int(act.sum()))
        if not act.any():
            continue
        x32 = x.astype(np.float32)
        if due:
            bt = _BlockTree(x32, nleaf, ncrit, pack)
            due = False
            rebuilt.append(s)
        walked.append(s)
        an, pn = bt.forces(x32, mass, theta, eps, act)
        a[act] = an[act]
        pot[act] = pn[act]
        h = (1 << (kmax - lev)) * dtm / 2
        v[act] += a[act] * h[act][:, None]
        t_done[act] += 2 * h[act]
        if s < nsub:
            new = np.maximum(block_level(a, c32, kmax), kmax - _ctz(s))
            lev[act] = new[act]
            h = (1 << (kmax - lev)) * dtm / 2
            v[act] += a[act] * h[act][:, None]
    out = (x, v, a, pot, lev0, nactive)
    if clock:
        out += (t_done,)
    if schedule:
        out += (walked, rebuilt)
    return out


# ---------------------------------------------------------------------------
# Neighbour search and SPH density (Sect. 3: the tree also serves these)
# ---------------------------------------------------------------------------

def sph_kernel(r: float, h: float) -> float:
    """Cubic spline kernel of compact support h (3D)."""
    return float(lib().oracle_sph_kernel(float(r), float(h)))


def sph_density(pos, mass, h, idx=None):
    """Per body (or per body of idx): density sum_j m_j W(r_ij, h_i) over the
    bodies j (itself included) with r_ij < h_i, and their count.  O(N) per
    body over all N, the definition."""
    pos, mass, h = _f32(pos), _f32(mass), _f32(h)
    n = pos.shape[0]
    tar = None if idx is None else np.ascontiguousarray(idx, np.int64)
    nt = n if tar is None else tar.shape[0]
    rho = np.zeros(nt)
    cnt = np.zeros(nt, np.int32)
    lib().oracle_sph_density(_ptr(pos), _ptr(mass), _ptr(h), n, _ptr(tar) if tar is not None else None, nt,
                             _ptr(rho), _ptr(cnt))
    return rho, cnt
