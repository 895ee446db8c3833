"""Seeded synthetic inputs for the tree gravity + collision path.

This module holds the input recipes only -- random draws and the physical
constants of the workloads -- and none of the method's arithmetic.  Both the
CUDA path (through the tests and the bench) and the CPU oracle are fed from
here.

Workloads (the shearing-sheet physics resembles a dense planetary ring, as in
the paper's scaling runs, Sect. 7):
  * sheet(L, N):   hard spheres R = 1 m, density 400 kg/m^3, uniform in x, y
                   over the L x L box, z ~ N(0, 1 m); velocities are the shear
                   flow (0, -1.5 Omega x, 0) plus isotropic Gaussian dispersion
                   sigma = 2 Omega * 1 m.
  * sheet_xy(Lx, Ly, N): the same in an Lx x Ly box; long_sheet_size(N)
                   gives the radial size of an elongated box of azimuthal size
                   20 m at optical depth 0.75 (the plane-sweep workload).
  * plummer(N):    Plummer sphere, G = M = a = 1, positions by inversion of
                   the cumulative mass, speeds by von Neumann rejection on
                   q^2 (1 - q^2)^(7/2); centre-of-mass frame.
  * ensemble(B):   B shearing boxes, N_b log-uniform in [500, 20000], surface
                   density log-uniform in [200, 1000] kg/m^2.
  * random_cube(N): N particles uniform in the unit cube with unequal masses
                   (the force-accuracy set-up of Sect. 6.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Shearing-sheet physics (Saturn's A ring-like)
G_SI = 6.674e-11
OMEGA = 1.3143527e-4          # 1/s
RADIUS = 1.0                  # m
DENSITY = 400.0               # kg/m^3
MASS = 4.0 / 3.0 * math.pi * RADIUS ** 3 * DENSITY
DT_SHEET = 1e-3 * 2.0 * math.pi / OMEGA
SIGMA = 2.0 * OMEGA * 1.0     # m/s
EPS_SHEET = 0.5
THETA_SHEET = 0.5


@dataclass
class Particles:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray
    r: np.ndarray

    @property
    def n(self) -> int:
        return len(self.x)

    def arrays(self):
        return (self.x, self.y, self.z, self.vx, self.vy, self.vz, self.m, self.r)

    def copy(self) -> "Particles":
        return Particles(*(a.copy() for a in self.arrays()))

    def subset(self, idx) -> "Particles":
        return Particles(*(a[idx].copy() for a in self.arrays()))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sheet(L: float, N: int, seed: int, omega: float = OMEGA, sigma: float = SIGMA,
          radius: float = RADIUS, density: float = DENSITY) -> Particles:
    """Shearing-sheet initial state in the box [-L/2, L/2)^2 (x, y)."""
    return sheet_xy(L, L, N, seed, omega, sigma, radius, density)


def long_sheet_size(N: int, Ly: float = 20.0, tau: float = 0.75, radius: float = RADIUS) -> float:
    """Radial size L_x of an elongated sheet of azimuthal size Ly holding N
    particles at optical depth tau = N pi R^2 / (L_x L_y)."""
    return N * math.pi * radius ** 2 / (tau * Ly)


def sheet_xy(Lx: float, Ly: float, N: int, seed: int, omega: float = OMEGA, sigma: float = SIGMA,
             radius: float = RADIUS, density: float = DENSITY) -> Particles:
    """Shearing-sheet initial state in [-Lx/2, Lx/2) x [-Ly/2, Ly/2) (the
    elongated boxes of the paper's collision scaling test use Ly = 20 R)."""
    g = _rng(seed)
    x = g.uniform(-0.5 * Lx, 0.5 * Lx, N)
    y = g.uniform(-0.5 * Ly, 0.5 * Ly, N)
    z = g.normal(0.0, 1.0, N)
    vx = g.normal(0.0, sigma, N)
    vy = -1.5 * omega * x + g.normal(0.0, sigma, N)
    vz = g.normal(0.0, sigma, N)
    m = np.full(N, 4.0 / 3.0 * math.pi * radius ** 3 * density)
    r = np.full(N, float(radius))
    return Particles(x, y, z, vx, vy, vz, m, r)


def plummer(N: int, seed: int, rmax_fraction: float = 0.999) -> Particles:
    """Plummer sphere (G = M = a = 1), equal masses, centre-of-mass frame.

    Positions: r = (X^(-2/3) - 1)^(-1/2) with X uniform; X > rmax_fraction is
    redrawn so that no particle starts far outside the root box.
    Velocities: v = q v_esc(r), v_esc = sqrt(2) (1 + r^2)^(-1/4), q drawn by
    rejection from q^2 (1 - q^2)^(7/2) (maximum < 0.1)."""
    g = _rng(seed)
    X = g.uniform(0.0, 1.0, N)
    while True:
        bad = (X > rmax_fraction) | (X <= 0.0)
        if not bad.any():
            break
        X[bad] = g.uniform(0.0, 1.0, int(bad.sum()))
    rad = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)

    def directions(k):
        cz = g.uniform(-1.0, 1.0, k)
        ph = g.uniform(0.0, 2.0 * math.pi, k)
        s = np.sqrt(1.0 - cz ** 2)
        return s * np.cos(ph), s * np.sin(ph), cz

    ux, uy, uz = directions(N)
    q = np.empty(N)
    todo = np.arange(N)
    while len(todo):
        qq = g.uniform(0.0, 1.0, len(todo))
        yy = g.uniform(0.0, 0.1, len(todo))
        ok = yy < qq ** 2 * (1.0 - qq ** 2) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + rad ** 2) ** (-0.25)
    wx, wy, wz = directions(N)
    v = q * vesc
    m = np.full(N, 1.0 / N)
    x, y, z = rad * ux, rad * uy, rad * uz
    vx, vy, vz = v * wx, v * wy, v * wz
    x, y, z = x - x.mean(), y - y.mean(), z - z.mean()
    vx, vy, vz = vx - vx.mean(), vy - vy.mean(), vz - vz.mean()
    return Particles(x, y, z, vx, vy, vz, m, np.zeros(N))


def ensemble_boxes(B: int = 256, seed0: int = 1000, nmin: int = 500, nmax: int = 20000,
                   smin: float = 200.0, smax: float = 1000.0):
    """Box sizes of the ensemble: list of (N_b, L_b, seed_b)."""
    out = []
    for b in range(B):
        g = _rng(seed0 + b)
        nb = int(round(math.exp(g.uniform(math.log(nmin), math.log(nmax)))))
        sig = math.exp(g.uniform(math.log(smin), math.log(smax)))
        Lb = math.sqrt(nb * MASS / sig)
        out.append((nb, Lb, seed0 + b))
    return out


def ensemble(B: int = 256, seed0: int = 1000, **kw):
    """B independent shearing boxes: list of (L_b, Particles)."""
    return [(Lb, sheet(Lb, nb, seed + 7919)) for nb, Lb, seed in ensemble_boxes(B, seed0, **kw)]


def random_cube(N: int, seed: int) -> Particles:
    """N particles uniform in [-0.5, 0.5)^3 with masses uniform in [0.1, 1.1)."""
    g = _rng(seed)
    x, y, z = (g.uniform(-0.5, 0.5, N) for _ in range(3))
    m = g.uniform(0.1, 1.1, N)
    zero = np.zeros(N)
    return Particles(x, y, z, zero.copy(), zero.copy(), zero.copy(), m, zero.copy())


# The workloads, by name and size.
SHEET_SMALL = dict(L=100.0, N=2400, seed=1, steps=100)       # small sheet
SHEET_MID = dict(L=650.0, N=100_000, seed=2, steps=1000)     # mid sheet
PLUMMER_1M = dict(N=1 << 20, seed=3, L=128.0, dt=1e-3, soft=1e-3)
SHEET_1M = dict(L=2050.0, N=1_000_000, seed=5)               # large sheet
