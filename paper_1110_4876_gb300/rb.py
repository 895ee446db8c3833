"""Thin ctypes binding of librb (``include/rb.h``): argument marshalling only.

Every function has the name of the C entry point it calls.  Every step of the
computation runs in librb's CUDA kernels; if ``librb.so`` is missing or cannot
be loaded the calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librb.so")

RB_OK, RB_ERR_ARG, RB_ERR_CAPACITY, RB_ERR_TIMEOUT, RB_ERR_NONFINITE, RB_ERR_CUDA, RB_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
RB_BC_OPEN, RB_BC_PERIODIC, RB_BC_SHEAR = 0, 1, 2
RB_INT_LEAPFROG, RB_INT_SEI = 0, 1
RB_WALK_FP64, RB_WALK_FP32, RB_WALK_FP32_LEARNED = 0, 1, 2
RB_COLL_NONE, RB_COLL_TREE, RB_COLL_SWEEP = 0, 1, 2
RB_EPS_CONSTANT, RB_EPS_POWER = 0, 1
RB_TILE_MORTON, RB_TILE_HILBERT_XY, RB_TILE_HILBERT_XYZ = 0, 1, 2

EXPORTS = [
    "rb_create", "rb_set_box", "rb_set_particles", "rb_step", "rb_get_particles", "rb_energy",
    "rb_energy_terms",
    "rb_compute_gravity", "rb_get_accelerations", "rb_get_counts", "rb_get_tree",
    "rb_detect_collisions", "rb_get_pairs", "rb_set_time", "rb_get_time", "rb_stats",
    "rb_set_profiling", "rb_destroy", "rb_last_error", "rb_energy_sums_noalloc",
    "rb_load_mlp", "rb_mlp_samples", "rb_mlp_train", "rb_mlp_grad", "rb_mlp_grad_fp32", "rb_autotune",
    "rb_set_pair_capacity", "rb_debug_hold_pair", "rb_set_launch_shape", "rb_set_n_active", "rb_set_restitution",
    "rb_sort_pairs_u64",
]
RB_MLP_PARAMS = 9347


class RbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"librb error {code}: {msg}")
        self.code = code


class rb_config(C.Structure):
    _fields_ = [
        ("G", C.c_double), ("omega", C.c_double), ("omega_z", C.c_double),
        ("box", C.c_double * 3),
        ("theta", C.c_double), ("eps_restitution", C.c_double), ("softening", C.c_double),
        ("dt", C.c_double), ("t0", C.c_double),
        ("nghost", C.c_int * 3),
        ("boundary", C.c_int), ("z_periodic", C.c_int), ("integrator", C.c_int),
        ("walk", C.c_int), ("quadrupole", C.c_int), ("gravity", C.c_int),
        ("collisions", C.c_int), ("reserved", C.c_int * 5),
    ]


class rb_stats_t(C.Structure):
    _fields_ = [
        ("steps", C.c_int64), ("n_live", C.c_int64), ("cells", C.c_int64),
        ("pairs_found", C.c_int64), ("pairs_resolved", C.c_int64),
        ("cell_interactions", C.c_int64), ("leaf_interactions", C.c_int64),
        ("mac_tests", C.c_int64), ("fp64_rechecks", C.c_int64), ("pair_capacity", C.c_int64),
        ("kernels_per_step", C.c_int64), ("walk_block", C.c_int64), ("search_block", C.c_int64),
        ("t", C.c_double), ("ms_last_step", C.c_double), ("ms_stage", C.c_double * 12),
        ("corrections", C.c_int64), ("warp_iterations", C.c_int64), ("walk_group", C.c_int64),
        ("tile_order", C.c_int64), ("search_visits", C.c_int64), ("search_iterations", C.c_int64),
    ]


STAGES = ["drift_keys", "sort_gather", "tree", "moments", "gravity_walk", "kick_drift_keys",
          "sort_gather_c", "tree_c", "collision_records", "collision_search", "pair_sort",
          "resolve"]


_lib = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_VP = C.c_void_p
_P = C.c_void_p


def load():
    """Load librb.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1110_4876_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    i64, i32 = C.c_int64, C.c_int
    lib.rb_create.argtypes = [C.POINTER(rb_config), i32, _VP, C.POINTER(_P)]
    lib.rb_set_box.argtypes = [_P, i32, _D]
    lib.rb_set_particles.argtypes = [_P, i32, i64] + [_D] * 8
    lib.rb_step.argtypes = [_P, i64]
    lib.rb_get_particles.argtypes = [_P, i32, i64, C.POINTER(i64)] + [_VP] * 9
    lib.rb_energy.argtypes = [_P, i32, C.POINTER(C.c_double), _D]
    lib.rb_energy_terms.argtypes = [_P, i32, _D]
    lib.rb_compute_gravity.argtypes = [_P]
    lib.rb_get_accelerations.argtypes = [_P, i32, i64, _VP, _VP, _VP]
    lib.rb_get_counts.argtypes = [_P, i32, i64, _VP, _VP, _VP]
    lib.rb_get_tree.argtypes = [_P, i32, i64, C.POINTER(i64), _VP, _VP, _VP, _VP, _VP, i64, _VP]
    lib.rb_detect_collisions.argtypes = [_P]
    lib.rb_get_pairs.argtypes = [_P, i32, i64, C.POINTER(i64), _VP, _VP, _VP]
    lib.rb_set_time.argtypes = [_P, C.c_double]
    lib.rb_get_time.argtypes = [_P, C.POINTER(C.c_double)]
    lib.rb_stats.argtypes = [_P, C.POINTER(rb_stats_t)]
    lib.rb_set_profiling.argtypes = [_P, i32]
    lib.rb_autotune.argtypes = [_P, i32]
    lib.rb_set_launch_shape.argtypes = [_P, i32, i32, i32, i32]
    lib.rb_set_n_active.argtypes = [_P, C.c_int64]
    lib.rb_set_restitution.argtypes = [_P, i32, C.c_double, C.c_double]
    lib.rb_set_pair_capacity.argtypes = [_P, i64]
    lib.rb_debug_hold_pair.argtypes = [_P, C.c_int]
    lib.rb_load_mlp.argtypes = [_P, _VP, i64, C.c_double]
    lib.rb_mlp_samples.argtypes = [_P, C.c_double, C.c_double, C.c_double, C.c_uint64, i64,
                                   C.POINTER(i64), _VP, _VP, _VP]
    lib.rb_mlp_train.argtypes = [_VP, _VP, i64, i32, i32, C.c_double, C.c_uint64, _VP, _VP, _VP, _VP]
    lib.rb_mlp_grad.argtypes = [_VP, _VP, _VP, i64, _VP, _VP, _VP]
    lib.rb_mlp_grad_fp32.argtypes = [_VP, _VP, _VP, i64, _VP, _VP, _VP]
    lib.rb_energy_sums_noalloc.argtypes = [i64] + [_VP] * 7 + [i32, C.c_double, C.c_double, _VP,
                                                              _VP]
    lib.rb_sort_pairs_u64.argtypes = [i64, i64, i32, _VP, _VP, _VP]
    lib.rb_destroy.argtypes = [_P]
    lib.rb_destroy.restype = None
    lib.rb_last_error.argtypes = [_P]
    lib.rb_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("rb_destroy", "rb_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(rc: int, sim=None):
    if rc != RB_OK:
        msg = load().rb_last_error(sim)
        raise RbError(rc, msg.decode() if msg else "")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_config(**kw) -> rb_config:
    """rb_config with defaults (leap-frog, open box, FP32 walk, quadrupole on)."""
    c = rb_config()
    c.G = kw.get("G", 1.0)
    c.omega = kw.get("omega", 0.0)
    c.omega_z = kw.get("omega_z", 0.0)
    L = kw.get("box", (1.0, 1.0, 1.0))
    c.box[:] = [float(v) for v in L]
    c.theta = kw.get("theta", 0.5)
    c.eps_restitution = kw.get("eps", kw.get("eps_restitution", 0.5))
    c.softening = kw.get("softening", kw.get("soft", 0.0))
    c.dt = kw.get("dt", 1e-3)
    c.t0 = kw.get("t0", 0.0)
    c.nghost[:] = [int(v) for v in kw.get("nghost", (0, 0, 0))]
    c.boundary = kw.get("boundary", RB_BC_OPEN)
    c.z_periodic = kw.get("z_periodic", 0)
    c.integrator = kw.get("integrator", RB_INT_LEAPFROG)
    c.walk = kw.get("walk", RB_WALK_FP32)
    c.quadrupole = kw.get("quadrupole", 1)
    c.gravity = kw.get("gravity", 1)
    c.collisions = kw.get("collisions", 0)
    return c


def rb_create(cfg: rb_config, nbox: int = 1, stream=None):
    lib = load()
    h = _P()
    rc = lib.rb_create(C.byref(cfg), nbox, stream, C.byref(h))
    _check(rc, None)
    return h


def rb_set_box(sim, box: int, L):
    _check(load().rb_set_box(sim, box, np.ascontiguousarray(L, dtype=np.float64)), sim)


def rb_set_particles(sim, box: int, x, y, z, vx, vy, vz, m, r):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, vx, vy, vz, m, r)]
    _check(load().rb_set_particles(sim, box, len(arrs[0]), *arrs), sim)


def rb_step(sim, nsteps: int = 1):
    _check(load().rb_step(sim, nsteps), sim)


_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "r")


def rb_get_particles(sim, box: int = 0, out=None):
    """Live particles of a box in id order: dict of arrays (x..r, id).  out:
    optional dict of preallocated float64 arrays (e.g. pinned) for the eight
    fields, each at least as long as the box; "id" is filled when present."""
    lib = load()
    n = C.c_int64(0)
    if out is None:
        _check(lib.rb_get_particles(sim, box, 0, C.byref(n), *([None] * 9)), sim)
        cap = n.value
        out = {k: np.empty(cap) for k in _FIELDS}
        out["id"] = np.empty(cap, dtype=np.int64)
    cap = min(len(out[k]) for k in _FIELDS)
    rc = lib.rb_get_particles(sim, box, cap, C.byref(n), *(_ptr(out[k]) for k in _FIELDS),
                              _ptr(out.get("id")))
    _check(rc, sim)
    return {k: v[:n.value] for k, v in out.items()}


def rb_energy(sim, box: int = 0):
    E = C.c_double(0.0)
    P = np.zeros(3)
    _check(load().rb_energy(sim, box, C.byref(E), P), sim)
    return E.value, P


def rb_energy_terms(sim, box: int = 0):
    """(K, U, W, P): the terms rb_energy adds up."""
    t = np.zeros(6)
    _check(load().rb_energy_terms(sim, box, t), sim)
    return t[0], t[1], t[2], t[3:].copy()


def rb_compute_gravity(sim):
    _check(load().rb_compute_gravity(sim), sim)


def _nlive(sim, box):
    lib = load()
    n = C.c_int64(0)
    lib.rb_get_particles(sim, box, 0, C.byref(n), *([None] * 9))
    return n.value


def rb_get_accelerations(sim, box: int = 0):
    n = _nlive(sim, box)
    a = np.zeros((3, n))
    _check(load().rb_get_accelerations(sim, box, n, _ptr(a[0]), _ptr(a[1]), _ptr(a[2])), sim)
    return np.ascontiguousarray(a.T)


def rb_get_counts(sim, box: int = 0):
    n = _nlive(sim, box)
    c = np.zeros((3, n), dtype=np.int64)
    _check(load().rb_get_counts(sim, box, n, _ptr(c[0]), _ptr(c[1]), _ptr(c[2])), sim)
    return c[0], c[1], c[2]


def rb_get_tree(sim, box: int = 0):
    """Branching cells of the last gravity tree: list of (depth, member ids,
    M, com (3,), Q (6,))."""
    lib = load()
    nc = C.c_int64(0)
    lib.rb_get_tree(sim, box, 0, C.byref(nc), None, None, None, None, None, 0, None)
    k = nc.value
    depth = np.zeros(max(k, 1), dtype=np.int32)
    count = np.zeros(max(k, 1), dtype=np.int64)
    M = np.zeros(max(k, 1))
    com = np.zeros(3 * max(k, 1))
    Q = np.zeros(6 * max(k, 1))
    n = _nlive(sim, box)
    mcap = 22 * max(n, 1)
    mem = np.zeros(mcap, dtype=np.int64)
    rc = lib.rb_get_tree(sim, box, k, C.byref(nc), _ptr(depth), _ptr(count), _ptr(M), _ptr(com),
                         _ptr(Q), mcap, _ptr(mem))
    _check(rc, sim)
    out, off = [], 0
    for c in range(k):
        out.append((int(depth[c]), mem[off: off + count[c]].copy(), M[c], com[3 * c: 3 * c + 3].copy(),
                    Q[6 * c: 6 * c + 6].copy()))
        off += int(count[c])
    return out


def rb_detect_collisions(sim):
    _check(load().rb_detect_collisions(sim), sim)


def rb_get_pairs(sim, box: int = 0):
    """Pairs of the last search, in resolution order: (id_a, id_b, code)."""
    lib = load()
    n = C.c_int64(0)
    lib.rb_get_pairs(sim, box, 0, C.byref(n), None, None, None)
    k = n.value
    a = np.zeros(max(k, 1), dtype=np.int64)
    b = np.zeros(max(k, 1), dtype=np.int64)
    c = np.zeros(max(k, 1), dtype=np.int32)
    _check(lib.rb_get_pairs(sim, box, k, C.byref(n), _ptr(a), _ptr(b), _ptr(c)), sim)
    return a[:k], b[:k], c[:k]


def rb_set_pair_capacity(sim, cap: int):
    _check(load().rb_set_pair_capacity(sim, cap), sim)


def rb_debug_hold_pair(sim, on: bool):
    _check(load().rb_debug_hold_pair(sim, 1 if on else 0), sim)


def rb_set_time(sim, t: float):
    _check(load().rb_set_time(sim, t), sim)


def rb_get_time(sim) -> float:
    t = C.c_double(0.0)
    _check(load().rb_get_time(sim, C.byref(t)), sim)
    return t.value


def rb_stats(sim) -> dict:
    s = rb_stats_t()
    _check(load().rb_stats(sim, C.byref(s)), sim)
    out = {f: getattr(s, f) for f, _ in rb_stats_t._fields_ if f != "ms_stage"}
    out["ms_stage"] = dict(zip(STAGES, list(s.ms_stage)))
    return out


def rb_set_profiling(sim, on=True):
    """on: False/0 off, True/1 stage times, 2 stage times and the counting
    collision search (search_visits, search_iterations in rb_stats)."""
    _check(load().rb_set_profiling(sim, int(on)), sim)


def rb_autotune(sim, use_cache: bool = True):
    """Pick the walk/search launch shapes by timing them; returns the choice
    (walk block, search block, walk group, tile order)."""
    _check(load().rb_autotune(sim, 1 if use_cache else 0), sim)
    st = rb_stats(sim)
    return int(st["walk_block"]), int(st["search_block"]), int(st["walk_group"]), int(st["tile_order"])


def rb_set_n_active(sim, n_active: int):
    """Particles with id >= n_active (per box) feel gravity but exert none; -1: all active."""
    _check(load().rb_set_n_active(sim, int(n_active)), sim)


def rb_set_restitution(sim, law: int, v_c: float = 1.0, p: float = 0.0):
    """RB_EPS_CONSTANT, or RB_EPS_POWER: eps = min(1, (|v_n| / v_c)^(-p))."""
    _check(load().rb_set_restitution(sim, int(law), float(v_c), float(p)), sim)


def rb_set_launch_shape(sim, walk_block: int, search_block: int, walk_group: int = 0,
                        tile_order: int = 0):
    """Threads per block of the walk and of the collision search (64, 128,
    256), the FP32 walk's warp shape (0 union walk, 4 group walk) and the
    tile order of the targets (RB_TILE_*)."""
    _check(load().rb_set_launch_shape(sim, int(walk_block), int(search_block), int(walk_group),
                                      int(tile_order)), sim)


def rb_energy_sums_noalloc(n, m, x, z, vx, vy, vz, phi, integrator, omega, omega_z, out,
                           stream=None):
    """Energy/momentum sums without device allocation; all array arguments
    are device addresses (ints, e.g. torch ``data_ptr()``) or None."""
    rc = load().rb_energy_sums_noalloc(n, m, x, z, vx, vy, vz, phi, integrator, omega, omega_z,
                                       out, stream)
    _check(rc, None)


def rb_sort_pairs_u64(keys, vals=None, key_bits: int = 64, cap=None, stream=None):
    """The library's stable radix sort on host arrays: returns (keys, vals)
    sorted by key bits [0, key_bits) (copies; the inputs are not changed).
    cap >= len(keys) sizes the device buffers, the count being read on the
    device as in the step's pair sorts."""
    k = np.array(keys, dtype=np.uint64, copy=True)
    v = None if vals is None else np.array(vals, dtype=np.uint32, copy=True)
    if v is not None and len(v) != len(k):
        raise ValueError("keys and vals differ in length")
    n = len(k)
    _check(load().rb_sort_pairs_u64(n, n if cap is None else int(cap), int(key_bits), _ptr(k),
                                    None if v is None else _ptr(v), stream), None)
    return k, v


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def rb_load_mlp(sim, w, theta_fallback: float):
    w = _f32(w)
    _check(load().rb_load_mlp(sim, _ptr(w), len(w), theta_fallback), sim)


def rb_mlp_samples(sim, theta_hi: float, theta_lo: float, prob: float, seed: int, cap: int,
                   with_meta: bool = True):
    """Training samples on the current positions: (X (n,12), Y (n,3), meta (n,5) or None)."""
    X = np.zeros((cap, 12), np.float32)
    Y = np.zeros((cap, 3), np.float32)
    meta = np.zeros((cap, 5), np.int64) if with_meta else None
    n = C.c_int64(0)
    _check(load().rb_mlp_samples(sim, theta_hi, theta_lo, prob, seed, cap, C.byref(n), _ptr(X),
                                 _ptr(Y), _ptr(meta)), sim)
    k = n.value
    return X[:k].copy(), Y[:k].copy(), (meta[:k] if with_meta else None)


def rb_mlp_train(X, Y, w_init, epochs: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
                 stream=None):
    """Adam training on the GPU; returns (weights, per-epoch mean loss)."""
    X = _f32(X, (-1, 12))
    Y = _f32(Y, (-1, 3))
    w0 = _f32(w_init)
    out = np.zeros(RB_MLP_PARAMS, np.float32)
    hist = np.zeros(epochs, np.float32)
    _check(load().rb_mlp_train(_ptr(X), _ptr(Y), len(X), epochs, batch, lr, seed, _ptr(w0),
                               _ptr(out), _ptr(hist), stream), None)
    return out, hist


def rb_mlp_grad(w, X, Y, stream=None):
    """(gradient (9347,), mean squared error) from the GPU training kernels."""
    X = _f32(X, (-1, 12))
    Y = _f32(Y, (-1, 3))
    w = _f32(w)
    g = np.zeros(RB_MLP_PARAMS, np.float32)
    loss = C.c_float(0.0)
    _check(load().rb_mlp_grad(_ptr(w), _ptr(X), _ptr(Y), len(X), _ptr(g), C.byref(loss), stream),
           None)
    return g, loss.value


def rb_mlp_grad_fp32(w, X, Y, stream=None):
    """(gradient (9347,), mean squared error) from the FP32 debug kernels (n <= 4096)."""
    X = _f32(X, (-1, 12))
    Y = _f32(Y, (-1, 3))
    w = _f32(w)
    g = np.zeros(RB_MLP_PARAMS, np.float32)
    loss = C.c_float(0.0)
    _check(load().rb_mlp_grad_fp32(_ptr(w), _ptr(X), _ptr(Y), len(X), _ptr(g), C.byref(loss), stream),
           None)
    return g, loss.value


def rb_destroy(sim):
    if sim:
        load().rb_destroy(sim)


def rb_last_error(sim=None) -> str:
    msg = load().rb_last_error(sim)
    return msg.decode() if msg else ""


def pair_keys(a, b, code):
    """Pack pairs as the sortable key (id_a << 36) | (id_b << 12) | code."""
    return ((np.asarray(a, np.uint64) << np.uint64(36)) | (np.asarray(b, np.uint64) << np.uint64(12))
            | np.asarray(code, np.uint64))


class Sim:
    """Owning wrapper: ``Sim(config_kwargs, nbox)``; destroyed with the object."""

    def __init__(self, nbox: int = 1, stream=None, **cfg):
        self.cfg = make_config(**cfg)
        self.h = rb_create(self.cfg, nbox, stream)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.rb_destroy(self.h)
            self.h = None

    def set_particles(self, P, box: int = 0):
        rb_set_particles(self.h, box, *P.arrays()) if hasattr(P, "arrays") else \
            rb_set_particles(self.h, box, *P)

    def set_box(self, box: int, L):
        rb_set_box(self.h, box, L)

    def step(self, n: int = 1):
        rb_step(self.h, n)

    def particles(self, box: int = 0, out=None):
        return rb_get_particles(self.h, box, out)

    def gravity(self, box: int = 0, counts: bool = False):
        rb_compute_gravity(self.h)
        a = rb_get_accelerations(self.h, box)
        return (a, rb_get_counts(self.h, box)) if counts else a

    def pairs(self, box: int = 0, detect: bool = True):
        if detect:
            rb_detect_collisions(self.h)
        return rb_get_pairs(self.h, box)

    def energy(self, box: int = 0):
        return rb_energy(self.h, box)

    def energy_terms(self, box: int = 0):
        return rb_energy_terms(self.h, box)

    def stats(self):
        return rb_stats(self.h)
