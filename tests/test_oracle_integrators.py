"""Pins of the oracle's integrators and boundaries (Sect. 2.3, 3.1, 3.3)
against closed forms and an independent numerical solution of Hill's
equations."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp


def test_sei_drift_matches_numerical_hill_solution(orc):
    """Sect. 3.3 (reading: the SEI drift is the exact force-free solution of
    Hill's equations).  Compare 100 drift halves against an adaptive
    high-accuracy integration of the same ODEs."""
    O, Oz = 0.7, 1.3
    p = orc.Params(omega=O, omega_z=Oz, dt=0.05, integrator=1)
    g = np.random.default_rng(2)
    n = 6
    s0 = [g.normal(0, 1, n) for _ in range(6)]
    s = [a.copy() for a in s0]
    for _ in range(100):
        s = orc.drift(p, *s)
    T = 100 * 0.5 * p.dt

    def rhs(t, u):
        x, y, z, vx, vy, vz = u
        return [vx, vy, vz, 2 * O * vy + 3 * O * O * x, -2 * O * vx, -Oz * Oz * z]

    for i in range(n):
        u0 = [a[i] for a in s0]
        sol = solve_ivp(rhs, (0, T), u0, rtol=1e-12, atol=1e-12, method="DOP853")
        ref = sol.y[:, -1]
        got = np.array([a[i] for a in s])
        assert np.max(np.abs(got - ref)) <= 1e-9 * (1 + np.max(np.abs(ref)))


def test_sei_shear_flow_is_steady(orc):
    """The shear flow v_y = -3/2 Omega x is an exact solution of Hill's
    equations: x stays, y moves by -3/2 Omega x t."""
    O = 1.3143527e-4
    dt = 1e-3 * 2 * math.pi / O
    p = orc.Params(omega=O, dt=dt, integrator=1)
    x0 = np.linspace(-300, 300, 7)
    s = [x0.copy(), np.zeros(7), np.zeros(7), np.zeros(7), -1.5 * O * x0, np.zeros(7)]
    for _ in range(200):
        s = orc.drift(p, *s)
    t = 100 * dt
    np.testing.assert_allclose(s[0], x0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(s[1], -1.5 * O * x0 * t, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(s[3], 0.0, atol=1e-15)
    np.testing.assert_allclose(s[4], -1.5 * O * x0, rtol=1e-12)


def _kepler(orc, per_orbit, orbits):
    """Two bodies on an eccentric orbit (G = 1, M = 1 + 1e-3, started at
    apocentre r = 1 with 0.8 times the circular speed), leap-frog with
    direct-sum gravity in an open box; dt = period / per_orbit."""
    m = np.array([1.0, 1e-3])
    mt = m.sum()
    v = 0.8 * math.sqrt(mt)
    a = 1.0 / (2.0 - v * v / mt)            # vis-viva
    period = 2 * math.pi * math.sqrt(a ** 3 / mt)
    dt = period / per_orbit
    x = np.array([-m[1] / mt, m[0] / mt]); y = np.zeros(2); z = np.zeros(2)
    vx = np.zeros(2); vy = np.array([-v * m[1] / mt, v * m[0] / mt]); vz = np.zeros(2)
    p = orc.Params(G=1.0, L=(20.0,) * 3, dt=dt, gravity=2, collisions=0, integrator=0)
    st = orc.State(p, x, y, z, vx, vy, vz, m, np.zeros(2))
    E0, _ = st.energy()
    errs = []
    for k in range(per_orbit * orbits):
        st.step(1, record=False)
        if k % 5 == 0:
            errs.append(abs(st.energy()[0] - E0) / abs(E0))
    return st, np.array(errs), (m[0] / mt)


def test_leapfrog_kepler(orc):
    """Sect. 3.1 leap-frog on the Kepler problem: the energy error is bounded
    and second order in dt, with no secular drift, and the orbit closes after
    whole periods up to a second-order phase error."""
    st1, e1, x0 = _kepler(orc, 400, 5)
    st2, e2, _ = _kepler(orc, 800, 5)
    assert e1.max() < 1e-2
    assert 3.0 < e1.max() / e2.max() < 5.0
    # no drift: the last-orbit maximum is no larger than the first-orbit one
    q = len(e1) // 5
    assert e1[-q:].max() <= 1.05 * e1[:q].max()
    # the light body returns near its start after 5 periods
    d1 = math.hypot(st1.x[1] - x0, st1.y[1])
    d2 = math.hypot(st2.x[1] - x0, st2.y[1])
    assert d1 < 0.1 and 3.0 < d1 / d2 < 5.0


def test_sei_jacobi_energy_with_gravity(orc):
    """SEI with self-gravity conserves the Jacobi-type energy up to a bounded
    second-order error."""
    def run(dt):
        O = 1.0
        p = orc.Params(G=1e-3, omega=O, dt=dt, integrator=1, gravity=2, L=(50.0,) * 3)
        x = np.array([0.5, -0.5]); y = np.array([0.0, 0.3]); z = np.array([0.1, -0.1])
        vx = np.array([0.01, -0.01]); vy = -1.5 * O * x + np.array([0.0, 0.02]); vz = np.zeros(2)
        st = orc.State(p, x, y, z, vx, vy, vz, np.array([1.0, 2.0]), np.zeros(2))
        E0, _ = st.energy()
        err = 0.0
        for _ in range(int(round(4 * math.pi / dt))):
            st.step(1, record=False)
            err = max(err, abs(st.energy()[0] - E0))
        return err
    e1, e2 = run(0.02), run(0.01)
    assert 3.0 < e1 / e2 < 5.0


def test_shear_wrap_is_an_image_shift(orc):
    """Sect. 2.3 shear-periodic boundaries (reading: standard shearing-sheet
    images): a wrapped particle is the image of its old state, and wrapping
    keeps it inside the box."""
    O, L = 0.01, 10.0
    p = orc.Params(omega=O, L=(L, L, L), nghost=(1, 1, 0), boundary=2)
    t = 37.0
    x = np.array([5.3, -5.2, 1.0, 4.999]); y = np.array([4.9, -4.8, 5.4, 0.0])
    z = np.array([0.1, 0.2, 0.3, 0.0]); vy = np.array([0.1, 0.2, 0.3, 0.4])
    zero = np.zeros(4)
    out = orc.boundary(p, t, x, y, z, zero, vy, zero, np.ones(4), np.ones(4), np.arange(4))
    nx, ny, nz, _, nvy = out[0], out[1], out[2], out[3], out[4]
    assert np.all((nx >= -L / 2) & (nx < L / 2) & (ny >= -L / 2) & (ny < L / 2))
    off, dvy, code = orc.images(p, t)
    for i in range(4):
        # find the image that maps the new state back onto the old one
        ok = False
        for g in range(len(code)):
            d = np.array([nx[i] + off[g, 0] - x[i], ny[i] + off[g, 1] - y[i]])
            if np.all(np.abs(d) < 1e-12) and abs(nvy[i] + dvy[g] - vy[i]) < 1e-15:
                ok = True
        ok = ok or (abs(nx[i] - x[i]) < 1e-15 and (abs(ny[i] - y[i]) % L) < 1e-12)
        assert ok, i


def test_open_boundary_removes_escapers(orc):
    """Sect. 2.3: open boundaries remove every particle that leaves the box."""
    p = orc.Params(L=(4.0,) * 3, boundary=0)
    x = np.array([0.0, 2.0, -2.0, 1.99, 0.5]); y = np.array([0.0, 0.0, 0.0, 0.0, -2.1])
    z = np.zeros(5); one = np.ones(5)
    out = orc.boundary(p, 0.0, x, y, z, z, z, z, one, one, np.arange(5))
    assert out[-1].tolist() == [0, 2, 3]


def test_shearing_and_periodic_boxes_remove_through_open_z(orc):
    """Sect. 2.3 with reading R6: periodic and shearing boxes wrap x and y
    but keep z open unless z is periodic; the box is [-L/2, L/2) on each
    axis, so z = L/2 leaves and z = -L/2 stays."""
    L = 4.0
    x = np.array([0.0, 2.5, 0.0, 0.0, 0.0, 0.0]); y = np.array([0.0, 0.0, 0.0, 0.0, 0.0, -2.5])
    z = np.array([0.0, 0.0, 2.0, -2.0, 1.999, -2.2])
    zero, one = np.zeros(6), np.ones(6)
    for bc in (1, 2):
        p = orc.Params(L=(L,) * 3, boundary=bc, omega=1e-3, nghost=(1, 1, 0))
        out = orc.boundary(p, 0.0, x, y, z, zero, zero, zero, one, one, np.arange(6))
        assert out[-1].tolist() == [0, 1, 3, 4], bc
        assert abs(out[0][1] - (2.5 - L)) < 1e-15      # wrapped in x
        p = orc.Params(L=(L,) * 3, boundary=bc, omega=1e-3, nghost=(1, 1, 1), z_periodic=1)
        out = orc.boundary(p, 0.0, x, y, z, zero, zero, zero, one, one, np.arange(6))
        assert out[-1].tolist() == [0, 1, 2, 3, 4, 5], bc
        assert abs(out[2][2] - (2.0 - L)) < 1e-15 and abs(out[2][5] - (-2.2 + L)) < 1e-15
