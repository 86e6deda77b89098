"""GB300 Barnes-Hut tree-code ("Bonsai: A GPU Tree-Code", Bedorf, Gaburov &
Portegies Zwart) -- Python binding of libbonsai.so.

Argument marshalling only: every stage (keys, sort, reorder, tree build,
multipoles, walk, leapfrog, diagnostics) runs in the library's CUDA kernels.
The functions carry the C ABI's names (include/bonsai.h) and accept torch
tensors (CUDA tensors are passed as device pointers, CPU tensors as host
pointers) or numpy arrays (host).  There is no CPU fallback: if the compiled
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbonsai.so")
_lib = None

BONSAI_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "CAPACITY", -5: "TIMEOUT", -6: "NAN",
          -7: "NOT_READY"}

# Entry points declared in include/bonsai.h (checked by the CPU tests).
EXPORTS = ["bonsai_create", "bonsai_destroy", "bonsai_set_bodies", "bonsai_build",
           "bonsai_multipoles", "bonsai_forces", "bonsai_step", "bonsai_set_params",
           "bonsai_get_bodies", "bonsai_diagnostics", "bonsai_sync", "bonsai_get_sizes",
           "bonsai_get_domain", "bonsai_get_keys", "bonsai_get_tree", "bonsai_get_groups",
           "bonsai_get_moments", "bonsai_get_counts", "bonsai_last_error", "bonsai_version",
           "bonsai_get_stage_times", "bonsai_set_stage_timing", "bonsai_sort_keys_static", "bonsai_set_systems",
           "bonsai_get_domains", "bonsai_autotune", "bonsai_mlp_create", "bonsai_mlp_destroy",
           "bonsai_mlp_last_error", "bonsai_mlp_set_params", "bonsai_mlp_get_params",
           "bonsai_mlp_fit_norm", "bonsai_mlp_predict", "bonsai_mlp_grad", "bonsai_mlp_train",
           "bonsai_learn_samples", "bonsai_judge", "bonsai_set_learned", "bonsai_forces_learned",
           "bonsai_get_judge", "bonsai_set_judge_interval", "bonsai_get_config", "bonsai_block_cycle",
           "bonsai_block_levels", "bonsai_block_stats", "bonsai_block_substeps", "bonsai_sph_density", "bonsai_bench_fma",
           "bonsai_debug_hold_sort_tile"]

MLP_IN, MLP_H, MLP_OUT = 12, 64, 3
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT
MLP_NNORM = 2 * MLP_IN + 1

STAGES = ["kick_drift_domain", "keys", "sort", "reorder", "build", "multipoles", "walk", "kick"]


class BonsaiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("nleaf", C.c_int), ("ncrit", C.c_int), ("walk_warps", C.c_int),
                ("list_capacity", C.c_int), ("use_graph", C.c_int), ("group_pack", C.c_int),
                ("arena_limit_mib", C.c_int), ("reserved", C.c_int),
                ("max_spin", C.c_longlong)]


def build(force: bool = False) -> str:
    from . import builder as _b
    return _b.build(force=force)


def lib():
    """Load libbonsai.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1204_2280_gb300.build()")
        L = C.CDLL(LIB_PATH)
        p, i, f, ll = C.c_void_p, C.c_int, C.c_float, C.c_longlong
        L.bonsai_create.argtypes = [C.POINTER(p), C.POINTER(Config), p]
        L.bonsai_destroy.argtypes = [p]
        L.bonsai_destroy.restype = None
        L.bonsai_set_bodies.argtypes = [p, p, p, p, ll, i]
        L.bonsai_build.argtypes = [p]
        L.bonsai_multipoles.argtypes = [p]
        L.bonsai_forces.argtypes = [p, f, f, p, p, i]
        L.bonsai_step.argtypes = [p, f]
        L.bonsai_set_params.argtypes = [p, f, f]
        L.bonsai_get_bodies.argtypes = [p, p, p, i]
        L.bonsai_diagnostics.argtypes = [p, p]
        L.bonsai_sync.argtypes = [p]
        L.bonsai_get_sizes.argtypes = [p, p, p, p]
        L.bonsai_get_domain.argtypes = [p, p, p]
        L.bonsai_get_keys.argtypes = [p, p, p]
        L.bonsai_get_tree.argtypes = [p, p, p, p, p, p]
        L.bonsai_get_groups.argtypes = [p, p, p]
        L.bonsai_get_moments.argtypes = [p, p, p]
        L.bonsai_get_counts.argtypes = [p, p, p, p]
        L.bonsai_last_error.argtypes = [p]
        L.bonsai_last_error.restype = C.c_char_p
        L.bonsai_version.restype = C.c_char_p
        L.bonsai_get_stage_times.argtypes = [p, p, i]
        L.bonsai_set_stage_timing.argtypes = [p, i]
        L.bonsai_sort_keys_static.argtypes = [p, p, p, ll, p]
        L.bonsai_set_systems.argtypes = [p, p, i]
        L.bonsai_get_domains.argtypes = [p, p, p]
        L.bonsai_autotune.argtypes = [p, f, f, p, p, p]
        L.bonsai_get_config.argtypes = [p, C.POINTER(Config)]
        L.bonsai_block_cycle.argtypes = [p, f, i, f, i]
        L.bonsai_block_levels.argtypes = [p, f, i, f, p]
        L.bonsai_block_stats.argtypes = [p, p]
        L.bonsai_block_substeps.argtypes = [p, p]
        L.bonsai_sph_density.argtypes = [p, p, p, p, i]
        L.bonsai_bench_fma.argtypes = [i, i, ll, p, p]
        L.bonsai_debug_hold_sort_tile.argtypes = [p, i]
        u64 = C.c_ulonglong
        L.bonsai_mlp_create.argtypes = [C.POINTER(p), u64]
        L.bonsai_mlp_destroy.argtypes = [p]
        L.bonsai_mlp_destroy.restype = None
        L.bonsai_mlp_last_error.argtypes = [p]
        L.bonsai_mlp_last_error.restype = C.c_char_p
        L.bonsai_mlp_set_params.argtypes = [p, p, p]
        L.bonsai_mlp_get_params.argtypes = [p, p, p]
        L.bonsai_mlp_fit_norm.argtypes = [p, p, p, ll, i]
        L.bonsai_mlp_predict.argtypes = [p, p, p, ll, i]
        L.bonsai_mlp_grad.argtypes = [p, p, p, ll, i, p, p]
        L.bonsai_mlp_train.argtypes = [p, p, p, ll, i, i, i, f, f, u64, p]
        L.bonsai_learn_samples.argtypes = [p, f, f, i, u64, p, p, p, i]
        L.bonsai_judge.argtypes = [p, f, p]
        L.bonsai_set_learned.argtypes = [p, p, f, f, f]
        L.bonsai_forces_learned.argtypes = [p, f, p, p, i]
        L.bonsai_get_judge.argtypes = [p, p, p]
        L.bonsai_set_judge_interval.argtypes = [p, i]
        _lib = L
    return _lib


def _check(ctx, rc: int):
    if rc != BONSAI_OK:
        msg = lib().bonsai_last_error(ctx)
        raise BonsaiError(rc, msg.decode() if msg else "")


def _buf(x, dtype=None):
    """(pointer, on_device) of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if dtype is not None:
            assert x.dtype == dtype, (x.dtype, dtype)
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, 0
    import torch
    assert isinstance(x, torch.Tensor) and x.is_contiguous()
    return x.data_ptr(), (1 if x.is_cuda else 0)


def _same_side(*flags):
    fl = {f for f in flags if f is not None}
    if len(fl) > 1:
        raise ValueError("mix of device and host buffers in one call")
    return fl.pop() if fl else 0


# ---------------------------------------------------------------------------
# C ABI, one function each
# ---------------------------------------------------------------------------

def bonsai_create(cfg: Config | None = None, stream=None):
    """Create a context on the current device; stream: a torch.cuda.Stream, a
    raw cudaStream_t int, or None for torch's current stream."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    ctx = C.c_void_p()
    rc = lib().bonsai_create(C.byref(ctx), C.byref(cfg) if cfg is not None else None,
                             C.c_void_p(int(stream)) if stream else None)
    _check(None, rc)
    return ctx


def bonsai_destroy(ctx):
    lib().bonsai_destroy(ctx)


def bonsai_set_bodies(ctx, pos, mass, vel=None):
    (pp, d0), (mp, d1), (vp, d2) = _buf(pos, np.float32), _buf(mass, np.float32), _buf(vel, np.float32)
    n = int(mass.shape[0])
    _check(ctx, lib().bonsai_set_bodies(ctx, pp, mp, vp, n, _same_side(d0, d1, d2)))


def bonsai_set_systems(ctx, offsets):
    """offsets: nsys + 1 body offsets (first body of each system, then n)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    _check(ctx, lib().bonsai_set_systems(ctx, off.ctypes.data, int(off.shape[0]) - 1))


def bonsai_build(ctx):
    _check(ctx, lib().bonsai_build(ctx))


def bonsai_multipoles(ctx):
    _check(ctx, lib().bonsai_multipoles(ctx))


def bonsai_forces(ctx, theta: float, eps: float, acc=None, pot=None):
    (ap, d0), (pp, d1) = _buf(acc, np.float32), _buf(pot, np.float32)
    _check(ctx, lib().bonsai_forces(ctx, theta, eps, ap, pp, _same_side(d0, d1)))


def bonsai_step(ctx, dt: float):
    _check(ctx, lib().bonsai_step(ctx, dt))


def bonsai_autotune(ctx, theta: float, eps: float):
    """Pick (ncrit, warps per walk block) by timing the walk; returns
    (ncrit, warps, ms per walk)."""
    nc, w, ms = C.c_int(), C.c_int(), C.c_float()
    _check(ctx, lib().bonsai_autotune(ctx, theta, eps, C.byref(nc), C.byref(w), C.byref(ms)))
    return nc.value, w.value, ms.value


def bonsai_get_config(ctx) -> Config:
    cfg = Config()
    _check(ctx, lib().bonsai_get_config(ctx, C.byref(cfg)))
    return cfg


def bonsai_block_cycle(ctx, dt_max: float, max_level: int, eta: float, rebuild_every: int = 1):
    _check(ctx, lib().bonsai_block_cycle(ctx, dt_max, int(max_level), eta, int(rebuild_every)))


def bonsai_block_levels(ctx, dt_max: float, max_level: int, eta: float) -> np.ndarray:
    n, _, _ = bonsai_get_sizes(ctx)
    out = np.zeros(n, np.int32)
    _check(ctx, lib().bonsai_block_levels(ctx, dt_max, int(max_level), eta, out.ctypes.data))
    return out


def bonsai_block_stats(ctx) -> tuple[int, int, int]:
    out = np.zeros(3, np.int64)
    _check(ctx, lib().bonsai_block_stats(ctx, out.ctypes.data))
    return int(out[0]), int(out[1]), int(out[2])


def bonsai_block_substeps(ctx) -> tuple[int, int]:
    """(substeps walked, substeps rebuilt) of the last block cycle."""
    out = np.zeros(2, np.int32)
    _check(ctx, lib().bonsai_block_substeps(ctx, out.ctypes.data))
    return int(out[0]), int(out[1])


def bonsai_sph_density(ctx, h, rho=None, nngb=None):
    """Neighbour counts and SPH densities (caller order) for smoothing
    lengths h; torch CUDA tensors or numpy arrays, all on one side."""
    (hp, d0), (rp, d1), (np_, d2) = _buf(h, np.float32), _buf(rho, np.float32), _buf(nngb, np.int32)
    _check(ctx, lib().bonsai_sph_density(ctx, hp, rp, np_, _same_side(d0, d1, d2)))


def bonsai_set_params(ctx, theta: float, eps: float):
    _check(ctx, lib().bonsai_set_params(ctx, theta, eps))


def bonsai_get_bodies(ctx, pos=None, vel=None):
    (pp, d0), (vp, d1) = _buf(pos, np.float32), _buf(vel, np.float32)
    _check(ctx, lib().bonsai_get_bodies(ctx, pp, vp, _same_side(d0, d1)))


def bonsai_diagnostics(ctx) -> np.ndarray:
    out = np.zeros(8)
    _check(ctx, lib().bonsai_diagnostics(ctx, out.ctypes.data))
    return out


def bonsai_sync(ctx):
    _check(ctx, lib().bonsai_sync(ctx))


def bonsai_get_sizes(ctx) -> tuple[int, int, int]:
    a, b, c = C.c_longlong(), C.c_longlong(), C.c_longlong()
    _check(ctx, lib().bonsai_get_sizes(ctx, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def bonsai_get_domain(ctx):
    mn = np.zeros(3, np.float32)
    side = np.zeros(1, np.float32)
    _check(ctx, lib().bonsai_get_domain(ctx, mn.ctypes.data, side.ctypes.data))
    return mn, float(side[0])


def bonsai_get_domains(ctx, nsys: int):
    mn = np.zeros((nsys, 3), np.float32)
    side = np.zeros(nsys, np.float32)
    _check(ctx, lib().bonsai_get_domains(ctx, mn.ctypes.data, side.ctypes.data))
    return mn, side


def bonsai_get_keys(ctx):
    n, _, _ = bonsai_get_sizes(ctx)
    keys = np.zeros(n, np.uint64)
    perm = np.zeros(n, np.uint32)
    _check(ctx, lib().bonsai_get_keys(ctx, keys.ctypes.data, perm.ctypes.data))
    return keys, perm


def bonsai_get_tree(ctx) -> dict:
    _, nc, _ = bonsai_get_sizes(ctx)
    arr = [np.zeros(nc, np.int32) for _ in range(5)]
    _check(ctx, lib().bonsai_get_tree(ctx, *[a.ctypes.data for a in arr]))
    return dict(zip(["body_begin", "body_count", "child_begin", "nchild", "level"], arr))


def bonsai_get_groups(ctx):
    _, _, ng = bonsai_get_sizes(ctx)
    b = np.zeros(ng, np.int32)
    c = np.zeros(ng, np.int32)
    _check(ctx, lib().bonsai_get_groups(ctx, b.ctypes.data, c.ctypes.data))
    return b, c


def bonsai_get_moments(ctx):
    _, nc, _ = bonsai_get_sizes(ctx)
    mono = np.zeros((nc, 4), np.float32)
    quad = np.zeros((nc, 6), np.float32)
    _check(ctx, lib().bonsai_get_moments(ctx, mono.ctypes.data, quad.ctypes.data))
    return mono, quad


def bonsai_get_counts(ctx):
    n, _, _ = bonsai_get_sizes(ctx)
    a = np.zeros(n, np.uint32)
    b = np.zeros(n, np.uint32)
    tot = (C.c_ulonglong * 2)()
    _check(ctx, lib().bonsai_get_counts(ctx, a.ctypes.data, b.ctypes.data, tot))
    return a, b, (int(tot[0]), int(tot[1]))


def bonsai_set_stage_timing(ctx, on: bool) -> None:
    _check(ctx, lib().bonsai_set_stage_timing(ctx, 1 if on else 0))


def bonsai_get_stage_times(ctx) -> np.ndarray:
    ms = np.zeros(len(STAGES), np.float32)
    rc = lib().bonsai_get_stage_times(ctx, ms.ctypes.data, ms.shape[0])
    if rc < 0:
        _check(ctx, rc)
    return ms


def bonsai_sort_keys_static(keys, sorted_keys, perm, stream=None):
    """Sort n <= 65536 device keys without any device allocation (see the C
    header).  keys, sorted_keys: contiguous int64 CUDA tensors holding the
    63-bit keys; perm: contiguous int32 CUDA tensor; all on one device, with
    at least n = keys.shape[0] elements each (the C side cannot check sizes or
    devices, so they are checked here before anything runs).  stream: a
    torch.cuda.Stream or raw cudaStream_t handle; None means torch's current
    stream on the keys' device."""
    import torch
    n = int(keys.shape[0])
    args = (("keys", keys, torch.int64), ("sorted_keys", sorted_keys, torch.int64), ("perm", perm, torch.int32))
    for name, t, dt in args:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"bonsai_sort_keys_static: {name} must be a torch tensor")
        if t.dtype != dt:
            raise TypeError(f"bonsai_sort_keys_static: {name} must be {dt}, not {t.dtype}")
    for name, t, _ in args:
        if t.numel() < n:
            raise ValueError(f"bonsai_sort_keys_static: {name} holds {t.numel()} elements, needs {n}")
        if not t.is_contiguous():
            raise ValueError(f"bonsai_sort_keys_static: {name} must be contiguous")
    for name, t, _ in args:
        if not t.is_cuda:
            raise ValueError(f"bonsai_sort_keys_static: {name} must be a CUDA tensor")
    if not (keys.device == sorted_keys.device == perm.device):
        raise ValueError("bonsai_sort_keys_static: keys, sorted_keys and perm must share one device")
    with torch.cuda.device(keys.device):
        if stream is None:
            h = torch.cuda.current_stream(keys.device).cuda_stream
        else:
            h = int(getattr(stream, "cuda_stream", stream))
        _check(None, lib().bonsai_sort_keys_static(keys.data_ptr(), sorted_keys.data_ptr(),
                                                   perm.data_ptr(), n, C.c_void_p(h) if h else None))


def bonsai_bench_fma(blocks: int, threads: int, iters: int) -> tuple[float, float]:
    """FP32 FMA-chain microbenchmark on the current device: (ms, flop)."""
    ms = C.c_float()
    fl = C.c_double()
    _check(None, lib().bonsai_bench_fma(int(blocks), int(threads), int(iters), C.byref(ms), C.byref(fl)))
    return float(ms.value), float(fl.value)


def bonsai_debug_hold_sort_tile(ctx, tile: int) -> None:
    """Testing aid: sort tile `tile` publishes nothing (-1: off); see the header."""
    _check(ctx, lib().bonsai_debug_hold_sort_tile(ctx, int(tile)))


def bonsai_version() -> str:
    return lib().bonsai_version().decode()


# ---------------------------------------------------------------------------
# Learned far-field correction
# ---------------------------------------------------------------------------

def _mcheck(m, rc):
    if rc != BONSAI_OK:
        msg = lib().bonsai_mlp_last_error(m)
        raise BonsaiError(rc, msg.decode() if msg else "")


class MLP:
    """Owning wrapper of a bonsai_mlp."""

    def __init__(self, seed: int = 0):
        self.m = C.c_void_p()
        _check(None, lib().bonsai_mlp_create(C.byref(self.m), seed))

    def close(self):
        if self.m:
            lib().bonsai_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params=None, norm=None):
        pp = None if params is None else np.ascontiguousarray(params, np.float32)
        nn = None if norm is None else np.ascontiguousarray(norm, np.float32)
        _mcheck(self.m, lib().bonsai_mlp_set_params(self.m, None if pp is None else pp.ctypes.data,
                                                     None if nn is None else nn.ctypes.data))

    def get_params(self):
        pp = np.zeros(MLP_NPARAM, np.float32)
        nn = np.zeros(MLP_NNORM, np.float32)
        _mcheck(self.m, lib().bonsai_mlp_get_params(self.m, pp.ctypes.data, nn.ctypes.data))
        return pp, nn

    def fit_norm(self, X, Y):
        (xp, d0), (yp, d1) = _buf(X, np.float32), _buf(Y, np.float32)
        _mcheck(self.m, lib().bonsai_mlp_fit_norm(self.m, xp, yp, int(X.shape[0]), _same_side(d0, d1)))

    def predict(self, X, Y=None):
        if Y is None:
            Y = np.zeros((X.shape[0], MLP_OUT), np.float32)
        (xp, d0), (yp, d1) = _buf(X, np.float32), _buf(Y, np.float32)
        _mcheck(self.m, lib().bonsai_mlp_predict(self.m, xp, yp, int(X.shape[0]), _same_side(d0, d1)))
        return Y

    def grad(self, X, Y):
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = C.c_float()
        (xp, d0), (yp, d1) = _buf(X, np.float32), _buf(Y, np.float32)
        _mcheck(self.m, lib().bonsai_mlp_grad(self.m, xp, yp, int(X.shape[0]), _same_side(d0, d1),
                                              g.ctypes.data, C.byref(loss)))
        return g, loss.value

    def train(self, X, Y, epochs=10, batch=8192, lr=1e-3, wd=1e-4, seed=0):
        losses = np.zeros(epochs, np.float32)
        (xp, d0), (yp, d1) = _buf(X, np.float32), _buf(Y, np.float32)
        _mcheck(self.m, lib().bonsai_mlp_train(self.m, xp, yp, int(X.shape[0]), _same_side(d0, d1), epochs,
                                               batch, lr, wd, seed, losses.ctypes.data))
        return losses


def bonsai_learn_samples(ctx, theta: float, eps: float, ntar: int, seed: int):
    """Features X, targets Y and caller ids of ntar sampled bodies."""
    X = np.zeros((ntar, MLP_IN), np.float32)
    Y = np.zeros((ntar, MLP_OUT), np.float32)
    ids = np.zeros(ntar, np.uint32)
    _check(ctx, lib().bonsai_learn_samples(ctx, theta, eps, ntar, seed, X.ctypes.data, Y.ctypes.data,
                                           ids.ctypes.data, 0))
    return X, Y, ids


def bonsai_judge(ctx, eps: float) -> float:
    v = C.c_float()
    _check(ctx, lib().bonsai_judge(ctx, eps, C.byref(v)))
    return v.value


def bonsai_set_learned(ctx, mlp, theta_coarse=1.0, theta_fine=0.5, p99_budget=0.0):
    _check(ctx, lib().bonsai_set_learned(ctx, None if mlp is None else mlp.m, theta_coarse, theta_fine,
                                         p99_budget))


def bonsai_forces_learned(ctx, eps: float, acc=None, pot=None):
    (ap, d0), (pp, d1) = _buf(acc, np.float32), _buf(pot, np.float32)
    _check(ctx, lib().bonsai_forces_learned(ctx, eps, ap, pp, _same_side(d0, d1)))


def bonsai_set_judge_interval(ctx, every: int):
    _check(ctx, lib().bonsai_set_judge_interval(ctx, int(every)))


def bonsai_get_judge(ctx):
    v, f = C.c_float(), C.c_int()
    _check(ctx, lib().bonsai_get_judge(ctx, C.byref(v), C.byref(f)))
    return v.value, bool(f.value)


class Bonsai:
    """Owning wrapper: Bonsai(cfg).set_bodies(...).build().multipoles() ..."""

    def __init__(self, cfg: Config | None = None, stream=None, **kw):
        if cfg is None and kw:
            cfg = Config(**kw)
        self.ctx = bonsai_create(cfg, stream)

    def close(self):
        if self.ctx:
            bonsai_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_bodies(self, pos, mass, vel=None):
        bonsai_set_bodies(self.ctx, pos, mass, vel)
        return self

    def set_systems(self, offsets):
        bonsai_set_systems(self.ctx, offsets)
        return self

    def build(self):
        bonsai_build(self.ctx)
        return self

    def multipoles(self):
        bonsai_multipoles(self.ctx)
        return self

    def forces(self, theta, eps, acc=None, pot=None):
        bonsai_forces(self.ctx, theta, eps, acc, pot)
        return self

    def step(self, dt):
        bonsai_step(self.ctx, dt)
        return self

    def block_cycle(self, dt_max, max_level, eta, rebuild_every=1):
        bonsai_block_cycle(self.ctx, dt_max, max_level, eta, rebuild_every)
        return self

    def sync(self):
        bonsai_sync(self.ctx)
        return self
