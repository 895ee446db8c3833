"""Pins of the oracle's test particles (reading T1: ids >= n_active feel
gravity but exert none) and velocity-dependent restitution (reading V1:
eps = min(1, (|v_n|/v_c)^(-p))): actives unaffected by test particles, test
particles moved by the actives' field exactly as the direct sum gives it,
the head-on closed form of the law and its elastic limits."""
import math

import numpy as np
import pytest


def _cloud(seed, n, L=20.0):
    g = np.random.default_rng(seed)
    x, y, z = g.uniform(-L / 4, L / 4, (3, n))
    vx, vy, vz = g.normal(0, 0.05, (3, n))
    m = g.uniform(0.5, 1.5, n)
    return x, y, z, vx, vy, vz, m, np.zeros(n)


def test_test_particles_do_not_move_the_actives(orc):
    """Direct gravity, leap-frog, open box: the first 40 particles evolve
    exactly as they do without the 30 test particles."""
    L = 20.0
    full = _cloud(1, 70, L)
    p = orc.Params(G=1.0, L=(L,) * 3, dt=0.01, gravity=2, collisions=0, soft=0.05, n_active=40)
    a = orc.State(p, *full)
    a.step(20)
    alone = tuple(v[:40].copy() for v in full)
    p0 = orc.Params(G=1.0, L=(L,) * 3, dt=0.01, gravity=2, collisions=0, soft=0.05)
    b = orc.State(p0, *alone)
    b.step(20)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        np.testing.assert_array_equal(getattr(a, k)[:40], getattr(b, k))


def test_test_particles_feel_the_actives(orc):
    """Tree gravity at theta -> 0 equals the direct sum over the actives only,
    for actives and test particles alike."""
    L = 20.0
    x, y, z, _, _, _, m, _ = _cloud(2, 300, L)
    p = orc.Params(G=1.0, L=(L,) * 3, theta=1e-6, soft=0.01, n_active=120)
    ms = np.where(np.arange(300) < 120, m, 0.0)
    a_tree = orc.Tree(x, y, z, ms, L).gravity(p, 0.0)
    a_dir = orc.direct_gravity(p, 0.0, x[:120], y[:120], z[:120], m[:120], targets=None)
    np.testing.assert_allclose(a_tree[:120], a_dir, rtol=1e-11, atol=1e-14)
    # test particles: the field of the actives at their positions
    xs, ys, zs = (np.concatenate([v[:120], v[120:]]) for v in (x, y, z))
    ext = orc.direct_gravity(p, 0.0, xs, ys, zs, ms, targets=np.arange(120, 300))
    np.testing.assert_allclose(a_tree[120:], ext, rtol=1e-11, atol=1e-14)


def test_a_test_particle_leaves_its_central_mass_at_rest(orc):
    """One active mass and one orbiting test particle of the same mass: the
    active mass never moves (the Kepler orbit of the test particle is the
    leap-frog pin's orbit)."""
    p = orc.Params(G=1.0, L=(100.0,) * 3, dt=1e-3, gravity=2, collisions=0, n_active=1)
    st = orc.State(p, np.array([0.0, 1.0]), np.zeros(2), np.zeros(2), np.zeros(2), np.array([0.0, 1.0]),
                   np.zeros(2), np.ones(2), np.zeros(2))
    st.step(2000)
    assert st.x[0] == 0.0 and st.y[0] == 0.0 and st.vx[0] == 0.0 and st.vy[0] == 0.0
    r = math.hypot(st.x[1], st.y[1])
    assert abs(r - 1.0) < 1e-5


def _head_on(orc, vrel, law, vc, pw, eps=0.5):
    p = orc.Params(L=(10.0,) * 3, eps=eps, eps_law=law, eps_vc=vc, eps_p=pw)
    x = np.array([0.0, 1.9]); y = np.zeros(2); z = np.zeros(2)
    vx = np.array([vrel / 2, -vrel / 2]); vy = np.array([0.1, 0.1]); vz = np.zeros(2)
    m = np.array([2.0, 3.0])
    keys = orc.collide_brute(p, 0.0, x, y, z, np.ones(2), np.array([0, 1]))
    nvx, nvy, _ = orc.resolve(p, 0.0, x, y, z, vx, vy, vz, m, np.array([0, 1]), keys)
    return vx, nvx, m, vy, nvy


def test_power_law_restitution_head_on(orc):
    """|v_n| = 2, v_c = 0.5, p = 0.234: eps = 4^-0.234, and the relative normal
    velocity becomes -eps times its old value with momentum unchanged."""
    vx, nvx, m, vy, nvy = _head_on(orc, 2.0, 1, 0.5, 0.234)
    eps = 4.0 ** -0.234
    assert nvx[1] - nvx[0] == pytest.approx(-eps * (vx[1] - vx[0]), rel=1e-14)
    assert m @ nvx == pytest.approx(m @ vx, abs=1e-15)
    np.testing.assert_array_equal(nvy, vy)


@pytest.mark.parametrize("vrel,vc,pw", [(0.3, 0.5, 0.234), (2.0, 0.5, 0.0)])
def test_power_law_is_elastic_below_vc_or_without_exponent(orc, vrel, vc, pw):
    vx, nvx, m, _, _ = _head_on(orc, vrel, 1, vc, pw)
    assert nvx[1] - nvx[0] == pytest.approx(-(vx[1] - vx[0]), rel=1e-14)


def test_constant_law_ignores_the_law_parameters(orc):
    a = _head_on(orc, 2.0, 0, 0.5, 0.234, eps=0.3)
    assert a[1][1] - a[1][0] == pytest.approx(-0.3 * (a[0][1] - a[0][0]), rel=1e-14)
