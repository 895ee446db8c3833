"""ctypes marshalling for the C oracle in ``rb_oracle.c`` (test infrastructure).

Only the tests, the smoke check and the bench's CPU-baseline leg use this
module.  It builds ``librb_oracle.so`` next to the source with gcc (OpenMP on
when available) and wraps each exported function with numpy arrays; no step of
the method is computed here.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rb_oracle.c")
LIB = os.path.join(HERE, "librb_oracle.so")

BC_OPEN, BC_PERIODIC, BC_SHEAR = 0, 1, 2
INT_LEAPFROG, INT_SEI = 0, 1
GRAV_NONE, GRAV_TREE, GRAV_DIRECT = 0, 1, 2
COLL_NONE, COLL_TREE, COLL_BRUTE, COLL_SWEEP = 0, 1, 2, 3
CENTRAL_CODE = 7 | (7 << 4) | (7 << 8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (``-O2 -ffp-contract=off``, OpenMP)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "rb_oracle.h"))
    ):
        return LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]
    tmp = LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, SRC, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


class _Params(C.Structure):
    _fields_ = [
        ("G", C.c_double), ("omega", C.c_double), ("omega_z", C.c_double),
        ("L", C.c_double * 3),
        ("theta", C.c_double), ("eps", C.c_double), ("soft", C.c_double),
        ("dt", C.c_double), ("t0", C.c_double),
        ("nghost", C.c_int * 3),
        ("boundary", C.c_int), ("z_periodic", C.c_int), ("integrator", C.c_int),
        ("quadrupole", C.c_int), ("gravity", C.c_int), ("collisions", C.c_int),
        ("n_active", C.c_int64), ("eps_law", C.c_int), ("eps_vc", C.c_double), ("eps_p", C.c_double),
    ]


@dataclass
class Params:
    """Physical and numerical parameters of one simulation box."""
    G: float = 1.0
    omega: float = 0.0
    omega_z: float = 0.0
    L: tuple = (1.0, 1.0, 1.0)
    theta: float = 0.5
    eps: float = 0.5
    soft: float = 0.0
    dt: float = 1e-3
    t0: float = 0.0
    nghost: tuple = (0, 0, 0)
    boundary: int = BC_OPEN
    z_periodic: int = 0
    integrator: int = INT_LEAPFROG
    quadrupole: int = 1
    gravity: int = GRAV_TREE
    collisions: int = COLL_NONE
    n_active: int = -1        # ids >= n_active are test particles (-1: all active)
    eps_law: int = 0          # 0 constant eps; 1 eps = min(1, (|v_n|/eps_vc)^(-eps_p))
    eps_vc: float = 1.0
    eps_p: float = 0.0
    extra: dict = field(default_factory=dict)

    def c(self) -> _Params:
        p = _Params()
        p.G, p.omega, p.omega_z = self.G, self.omega, self.omega_z
        p.L[:] = [float(v) for v in self.L]
        p.theta, p.eps, p.soft, p.dt, p.t0 = self.theta, self.eps, self.soft, self.dt, self.t0
        p.nghost[:] = [int(v) for v in self.nghost]
        p.boundary, p.z_periodic, p.integrator = self.boundary, self.z_periodic, self.integrator
        p.quadrupole, p.gravity, p.collisions = self.quadrupole, self.gravity, self.collisions
        p.n_active, p.eps_law, p.eps_vc, p.eps_p = self.n_active, self.eps_law, self.eps_vc, self.eps_p
        return p


_lib = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_PP = C.POINTER(_Params)
_VP = C.c_void_p


def load():
    """Build if needed and load the oracle library."""
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    lib.orc_version.restype = C.c_char_p
    lib.orc_nthreads.restype = C.c_int
    lib.orc_time.restype = C.c_double
    lib.orc_time.argtypes = [_PP, C.c_int64]
    lib.orc_images.restype = C.c_int
    lib.orc_images.argtypes = [_PP, C.c_double, C.c_int, _D, _D, _I32]
    lib.orc_direct_gravity.argtypes = [_PP, C.c_double, C.c_int64, _D, _D, _D, _D, C.c_int64,
                                       _VP, _D, _D, _D, _VP]
    lib.orc_tree_build.restype = _VP
    lib.orc_tree_build.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_double]
    lib.orc_tree_free.argtypes = [_VP]
    lib.orc_tree_ncells.restype = C.c_int64
    lib.orc_tree_ncells.argtypes = [_VP]
    lib.orc_tree_cells.restype = C.c_int64
    lib.orc_tree_cells.argtypes = [_VP, C.c_int64, _I32, _I64, _VP, C.c_int64, _VP, _VP, _VP]
    lib.orc_tree_gravity.argtypes = [_VP, _PP, C.c_double, C.c_int64, _VP, _D, _D, _D, _VP,
                                     _VP, _VP, _VP]
    for fn in (lib.orc_collide_brute, lib.orc_collide_tree):
        fn.restype = C.c_int64
        fn.argtypes = [_PP, C.c_double, C.c_int64, _D, _D, _D, _D, _I64, C.c_int64, _U64]
    for fn in (lib.orc_collide_line_brute, lib.orc_collide_sweep):
        fn.restype = C.c_int64
        fn.argtypes = [_PP, C.c_double, C.c_int64, _D, _D, _D, _D, _D, _D, _D, _I64, C.c_int64,
                       _U64]
    lib.orc_collide_tree_sel.restype = C.c_int64
    lib.orc_collide_tree_sel.argtypes = [_PP, C.c_double, C.c_int64, _D, _D, _D, _D, _I64, C.c_int64,
                                         _I64, C.c_int64, _U64]
    lib.orc_tree_collide_sel.restype = C.c_int64
    lib.orc_tree_collide_sel.argtypes = [_VP, _PP, C.c_double, C.c_int64, _D, _D, _D, _D, _I64,
                                         C.c_int64, _I64, C.c_int64, _U64]
    lib.orc_resolve.argtypes = [_PP, C.c_double, C.c_int64, _D, _D, _D, _D, _D, _D, _D, _I64,
                                C.c_int64, _U64]
    lib.orc_drift.argtypes = [_PP, C.c_int64, _D, _D, _D, _D, _D, _D]
    lib.orc_kick.argtypes = [_PP, C.c_int64, _D, _D, _D, _D, _D, _D]
    lib.orc_boundary.restype = C.c_int64
    lib.orc_boundary.argtypes = [_PP, C.c_double, C.c_int64, _D, _D, _D, _D, _D, _D, _D, _D, _I64]
    lib.orc_step.restype = C.c_int
    lib.orc_step.argtypes = [_PP, C.c_int64, C.POINTER(C.c_int64), _D, _D, _D, _D, _D, _D, _D,
                             _D, _I64, _VP, _VP, _VP, C.c_int64, _VP, C.POINTER(C.c_int64)]
    lib.orc_energy.argtypes = [_PP, C.c_double, C.c_int64, _D, _D, _D, _D, _D, _D, _D,
                               C.POINTER(C.c_double), _D]
    lib.orc_energy_terms.argtypes = [_PP, C.c_double, C.c_int64, _D, _D, _D, _D, _D, _D, _D, _D]
    _lib = lib
    return lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def nthreads() -> int:
    return load().orc_nthreads()


def time_at(p: Params, half_step: int) -> float:
    return load().orc_time(C.byref(p.c()), half_step)


def images(p: Params, t: float):
    """Ghost images at time t: (offsets (G,3), dvy (G,), codes (G,))."""
    cap = 343
    off = np.zeros(3 * cap)
    dvy = np.zeros(cap)
    code = np.zeros(cap, dtype=np.int32)
    k = load().orc_images(C.byref(p.c()), t, cap, off, dvy, code)
    return off[: 3 * k].reshape(k, 3), dvy[:k], code[:k]


def direct_gravity(p: Params, t: float, x, y, z, m, targets=None, potential=False):
    """Eq. 1 by direct summation over all particles and ghost images."""
    x, y, z, m = map(_d, (x, y, z, m))
    n = len(x)
    sel = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if sel is None else len(sel)
    ax, ay, az, phi = (np.zeros(nt) for _ in range(4))
    load().orc_direct_gravity(C.byref(p.c()), t, n, x, y, z, m, nt, _ptr(sel), ax, ay, az,
                              _ptr(phi if potential else None))
    a = np.stack([ax, ay, az], axis=1)
    return (a, phi) if potential else a


class Tree:
    """The oracle's insertion octree over the root cube [-L/2, L/2)^3."""

    def __init__(self, x, y, z, m, L):
        self._keep = [_d(x), _d(y), _d(z), _d(m)]
        self.n = len(self._keep[0])
        self.L = float(L)
        self.h = load().orc_tree_build(self.n, *self._keep, self.L)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_tree_free(self.h)
            self.h = None

    def cells(self):
        """Canonical cells: list of (depth, members array, M, com (3,), Q (6,))."""
        lib = load()
        nc = lib.orc_tree_ncells(self.h)
        depth = np.zeros(max(nc, 1), dtype=np.int32)
        count = np.zeros(max(nc, 1), dtype=np.int64)
        cap_m = max(1, 22 * self.n)
        members = np.zeros(cap_m, dtype=np.int64)
        M = np.zeros(max(nc, 1))
        com = np.zeros(3 * max(nc, 1))
        Q = np.zeros(6 * max(nc, 1))
        k = lib.orc_tree_cells(self.h, nc, depth, count, _ptr(members), cap_m, _ptr(M), _ptr(com),
                               _ptr(Q))
        out, off = [], 0
        for c in range(k):
            out.append((int(depth[c]), members[off: off + count[c]].copy(), M[c],
                        com[3 * c: 3 * c + 3].copy(), Q[6 * c: 6 * c + 6].copy()))
            off += int(count[c])
        return out

    def collide(self, p: Params, t: float, r, ids, targets, cap=None):
        """Sect. 5.2 search from the listed targets on this tree (unsorted keys);
        the tree must be built over the positions the search uses."""
        x, y, z = self._keep[:3]
        r = _d(r)
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        sel = np.ascontiguousarray(targets, dtype=np.int64)
        cap = cap or 16 * len(sel) + 16
        keys = np.zeros(cap, dtype=np.uint64)
        k = load().orc_tree_collide_sel(self.h, C.byref(p.c()), t, self.n, x, y, z, r, ids, len(sel),
                                        sel, cap, keys)
        if k > cap:
            return self.collide(p, t, r, ids, targets, int(k))
        return keys[:k].copy()

    def gravity(self, p: Params, t: float, targets=None, potential=False, counts=False):
        """Barnes-Hut accelerations (and potential, interaction counts)."""
        sel = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
        nt = self.n if sel is None else len(sel)
        ax, ay, az, phi = (np.zeros(nt) for _ in range(4))
        nc, nl, nm = (np.zeros(nt, dtype=np.int64) for _ in range(3))
        load().orc_tree_gravity(self.h, C.byref(p.c()), t, nt, _ptr(sel), ax, ay, az, _ptr(phi),
                                _ptr(nc), _ptr(nl), _ptr(nm))
        res = [np.stack([ax, ay, az], axis=1)]
        if potential:
            res.append(phi)
        if counts:
            res.append((nc, nl, nm))
        return res[0] if len(res) == 1 else tuple(res)


def tree_gravity(p: Params, t: float, x, y, z, m, targets=None, potential=False, counts=False):
    return Tree(x, y, z, m, p.L[0]).gravity(p, t, targets, potential, counts)


def _collide(fn, p, t, x, y, z, r, ids, cap):
    x, y, z, r = map(_d, (x, y, z, r))
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    keys = np.zeros(max(cap, 1), dtype=np.uint64)
    k = fn(C.byref(p.c()), t, len(x), x, y, z, r, ids, cap, keys)
    if k > cap:
        return _collide(fn, p, t, x, y, z, r, ids, int(k))
    return keys[:k].copy()


def collide_brute(p: Params, t: float, x, y, z, r, ids, cap=None):
    """Sect. 5.1 search: sorted pair keys (id_a << 36 | id_b << 12 | image code)."""
    return _collide(load().orc_collide_brute, p, t, x, y, z, r, ids, cap or 4 * len(x) + 16)


def collide_tree(p: Params, t: float, x, y, z, r, ids, cap=None):
    """Sect. 5.2 (Eq. 3) search: sorted pair keys."""
    return _collide(load().orc_collide_tree, p, t, x, y, z, r, ids, cap or 4 * len(x) + 16)


def collide_line_brute(p: Params, t: float, x, y, z, vx, vy, vz, r, ids, cap=None):
    """Sect. 5.3 straight-line criterion over every pair and image (sorted keys)."""
    return _collide_v(load().orc_collide_line_brute, p, t, x, y, z, vx, vy, vz, r, ids,
                      cap or 4 * len(x) + 16)


def collide_sweep(p: Params, t: float, x, y, z, vx, vy, vz, r, ids, cap=None):
    """Sect. 5.3 plane sweep along x (sorted keys)."""
    return _collide_v(load().orc_collide_sweep, p, t, x, y, z, vx, vy, vz, r, ids,
                      cap or 4 * len(x) + 16)


def _collide_v(fn, p, t, x, y, z, vx, vy, vz, r, ids, cap):
    x, y, z, vx, vy, vz, r = map(_d, (x, y, z, vx, vy, vz, r))
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    keys = np.zeros(max(cap, 1), dtype=np.uint64)
    k = fn(C.byref(p.c()), t, len(x), x, y, z, vx, vy, vz, r, ids, cap, keys)
    if k > cap:
        return _collide_v(fn, p, t, x, y, z, vx, vy, vz, r, ids, int(k))
    return keys[:k].copy()


def collide_tree_targets(p: Params, t: float, x, y, z, r, ids, targets, cap=None):
    """Sect. 5.2 search from the listed targets only (unsorted keys)."""
    x, y, z, r = map(_d, (x, y, z, r))
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    sel = np.ascontiguousarray(targets, dtype=np.int64)
    cap = cap or 16 * len(sel) + 16
    keys = np.zeros(cap, dtype=np.uint64)
    k = load().orc_collide_tree_sel(C.byref(p.c()), t, len(x), x, y, z, r, ids, len(sel), sel, cap,
                                    keys)
    if k > cap:
        return collide_tree_targets(p, t, x, y, z, r, ids, targets, int(k))
    return keys[:k].copy()


def decode_pairs(keys):
    keys = np.asarray(keys, dtype=np.uint64)
    a = (keys >> np.uint64(36)).astype(np.int64)
    b = ((keys >> np.uint64(12)) & np.uint64(0xFFFFFF)).astype(np.int64)
    c = (keys & np.uint64(0xFFF)).astype(np.int64)
    return a, b, c


class State:
    """Particle arrays in ascending id order, advanced by the oracle."""

    def __init__(self, p: Params, x, y, z, vx, vy, vz, m, r, ids=None):
        self.p = p
        self.x, self.y, self.z, self.vx, self.vy, self.vz, self.m, self.r = (
            _d(a).copy() for a in (x, y, z, vx, vy, vz, m, r))
        n = len(self.x)
        self.id = np.arange(n, dtype=np.int64) if ids is None else np.asarray(ids, np.int64).copy()
        self.n = n
        self.step_index = 0
        self.last_acc = None
        self.last_pairs = None

    def step(self, nsteps: int = 1, record=True):
        lib = load()
        pc = self.p.c()
        for _ in range(nsteps):
            n0 = self.n
            ax, ay, az = (np.zeros(max(n0, 1)) for _ in range(3))
            cap = 4 * n0 + 16
            pairs = np.zeros(cap, dtype=np.uint64)
            nn = C.c_int64(n0)
            npairs = C.c_int64(0)
            rc = lib.orc_step(C.byref(pc), self.step_index, C.byref(nn), self.x, self.y, self.z,
                              self.vx, self.vy, self.vz, self.m, self.r, self.id, _ptr(ax),
                              _ptr(ay), _ptr(az), cap, _ptr(pairs), C.byref(npairs))
            if rc != 0:
                raise RuntimeError("oracle pair buffer overflow")
            self.n = nn.value
            for name in ("x", "y", "z", "vx", "vy", "vz", "m", "r", "id"):
                setattr(self, name, getattr(self, name)[: self.n].copy())
            if record:
                self.last_acc = np.stack([ax, ay, az], axis=1)[: self.n]
                self.last_pairs = pairs[: npairs.value].copy()
            self.step_index += 1
        return self

    def energy(self, t=None):
        if t is None:
            t = time_at(self.p, 2 * self.step_index)
        E = C.c_double(0.0)
        P = np.zeros(3)
        load().orc_energy(C.byref(self.p.c()), t, self.n, self.x, self.y, self.z, self.vx,
                          self.vy, self.vz, self.m, C.byref(E), P)
        return E.value, P

    def energy_terms(self, t=None):
        """(K, U, W, P): kinetic, SEI tidal + vertical, gravitational (half
        the sum of m phi) and the momentum vector (Sect. 6.2)."""
        return energy_terms(self.p, time_at(self.p, 2 * self.step_index) if t is None else t,
                            self.x, self.y, self.z, self.vx, self.vy, self.vz, self.m)


def energy_terms(p: Params, t: float, x, y, z, vx, vy, vz, m):
    """(K, U, W, P) of Sect. 6.2 for the given particles at time t."""
    out = np.zeros(6)
    arrs = [_d(a) for a in (x, y, z, vx, vy, vz, m)]
    load().orc_energy_terms(C.byref(p.c()), t, len(arrs[0]), *arrs, out)
    return out[0], out[1], out[2], out[3:].copy()


def drift(p: Params, x, y, z, vx, vy, vz):
    """One drift half (in place on copies); returns the six arrays."""
    arrs = [_d(a).copy() for a in (x, y, z, vx, vy, vz)]
    load().orc_drift(C.byref(p.c()), len(arrs[0]), *arrs)
    return arrs


def boundary(p: Params, t: float, x, y, z, vx, vy, vz, m, r, ids):
    arrs = [_d(a).copy() for a in (x, y, z, vx, vy, vz, m, r)]
    ids = np.asarray(ids, dtype=np.int64).copy()
    n = load().orc_boundary(C.byref(p.c()), t, len(arrs[0]), *arrs, ids)
    return [a[:n] for a in arrs] + [ids[:n]]


def resolve(p: Params, t: float, x, y, z, vx, vy, vz, m, ids, keys):
    v = [_d(a).copy() for a in (vx, vy, vz)]
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    load().orc_resolve(C.byref(p.c()), t, len(v[0]), _d(x), _d(y), _d(z), *v, _d(m),
                       np.ascontiguousarray(ids, dtype=np.int64), len(keys), keys)
    return v


def e_sum(a, a_ref):
    """Hernquist (1987) force error used in Sect. 6.1: sum |da| / sum |a|."""
    return float(np.sum(np.linalg.norm(a - a_ref, axis=1)) / np.sum(np.linalg.norm(a_ref, axis=1)))


def force_errors(a, a_ref, floor=1e-3):
    """(e_sum, rms_rel, max_rel); the per-particle denominator is floored at
    floor * rms|a_ref| so that near-zero net forces do not dominate."""
    na = np.linalg.norm(a_ref, axis=1)
    den = np.maximum(na, floor * np.sqrt(np.mean(na ** 2)))
    rel = np.linalg.norm(a - a_ref, axis=1) / den
    return e_sum(a, a_ref), float(np.sqrt(np.mean(rel ** 2))), float(np.max(rel))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
