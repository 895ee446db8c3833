"""Pins of the oracle's plane-sweep detection (Sect. 5.3; readings S1-S4):
the sweep against its own brute force, the straight-line criterion against
closed forms for a head-on pair and a fly-by, its reduction to the overlap
test of Sect. 5.1 without motion, ghost images across the x boundary, and
conservation through a full step."""
import math

import numpy as np
import pytest


def _moving(seed, n=400, L=30.0, vsig=0.5):
    g = np.random.default_rng(seed)
    x, y = g.uniform(-L / 2, L / 2, (2, n))
    z = g.normal(0, 1.0, n)
    vx, vy, vz = g.normal(0, vsig, (3, n))
    r = g.uniform(0.6, 1.2, n)
    ids = g.permutation(n).astype(np.int64)
    return x, y, z, vx, vy, vz, r, ids


@pytest.mark.parametrize("boundary,seed,ng,zp", [(0, 1, (1, 1, 0), 0), (1, 2, (1, 1, 0), 0),
                                                 (2, 3, (1, 1, 0), 0), (2, 4, (2, 1, 0), 0),
                                                 (1, 5, (1, 1, 1), 1)])
def test_sweep_equals_line_brute_force(orc, boundary, seed, ng, zp):
    """The sweep finds exactly the (pair, image) set that testing every pair
    and image with the straight-line criterion finds."""
    L = 30.0
    x, y, z, vx, vy, vz, r, ids = _moving(seed, L=L)
    if zp:
        z = np.random.default_rng(seed).uniform(-L / 2, L / 2, len(x))
    p = orc.Params(omega=0.02, L=(L, L, L), nghost=ng, boundary=boundary, z_periodic=zp, dt=1.0)
    kb = orc.collide_line_brute(p, 77.0, x, y, z, vx, vy, vz, r, ids)
    ks = orc.collide_sweep(p, 77.0, x, y, z, vx, vy, vz, r, ids)
    assert len(kb) > 50
    assert kb.tolist() == ks.tolist()
    a, b, c = orc.decode_pairs(ks)
    assert np.all(a < b)
    if boundary != 0:
        assert np.any(c != orc.CENTRAL_CODE)


@pytest.mark.parametrize("boundary", [0, 1, 2])
def test_a_zero_interval_reduces_to_the_overlap_test(orc, boundary):
    """dt = 0: the lines are points (tau = 0 exactly) and the pair set is the
    Sect. 5.1 overlap set, whatever the velocities."""
    x, y, z, vx, vy, vz, r, ids = _moving(11, L=30.0)
    p = orc.Params(omega=0.02, L=(30.0,) * 3, nghost=(1, 1, 0), boundary=boundary, dt=0.0)
    ko = orc.collide_brute(p, 3.0, x, y, z, r, ids)
    kl = orc.collide_sweep(p, 3.0, x, y, z, vx, vy, vz, r, ids)
    assert len(ko) > 50
    assert kl.tolist() == ko.tolist()


@pytest.mark.parametrize("boundary", [0, 1])
def test_without_motion_the_line_criterion_is_the_overlap_test(orc, boundary):
    """v = 0 without shear: no particle or image moves."""
    x, y, z, vx, vy, vz, r, ids = _moving(13, L=30.0)
    zero = np.zeros_like(x)
    p = orc.Params(L=(30.0,) * 3, nghost=(1, 1, 0), boundary=boundary, dt=1.0)
    ko = orc.collide_brute(p, 3.0, x, y, z, r, ids)
    kl = orc.collide_sweep(p, 3.0, x, y, z, zero, zero, zero, r, ids)
    assert len(ko) > 50
    assert kl.tolist() == ko.tolist()


def test_moving_pairs_include_the_overlapping_ones(orc):
    """tau = 0 lies in the interval, so every pair overlapping at t collides."""
    x, y, z, vx, vy, vz, r, ids = _moving(12, L=30.0)
    p = orc.Params(omega=0.02, L=(30.0,) * 3, nghost=(1, 1, 0), boundary=2, dt=1.0)
    ko = set(orc.collide_brute(p, 3.0, x, y, z, r, ids).tolist())
    kl = set(orc.collide_sweep(p, 3.0, x, y, z, vx, vy, vz, r, ids).tolist())
    assert ko < kl


def _pair(orc, xa, va, xb, vb, dt, R=1.0):
    p = orc.Params(L=(100.0,) * 3, dt=dt)
    x = np.array([xa[0], xb[0]]); y = np.array([xa[1], xb[1]]); z = np.zeros(2)
    vx = np.array([va[0], vb[0]]); vy = np.array([va[1], vb[1]]); vz = np.zeros(2)
    return len(orc.collide_sweep(p, 0.0, x, y, z, vx, vy, vz, np.full(2, R), np.array([0, 1])))


def test_head_on_closed_form(orc):
    """Separation 3 closing at 4 per unit time: the distance at the end of the
    interval is 3 - 4 dt/2; R_a + R_b = 2."""
    assert _pair(orc, (0, 0), (2, 0), (3, 0), (-2, 0), dt=1.0) == 1    # 1.0 < 2
    assert _pair(orc, (0, 0), (2, 0), (3, 0), (-2, 0), dt=0.6) == 1    # 1.8 < 2
    assert _pair(orc, (0, 0), (2, 0), (3, 0), (-2, 0), dt=0.4) == 0    # 2.2 > 2
    assert _pair(orc, (0, 0), (2, 0), (3, 0), (-2, 0), dt=0.2) == 0    # 2.6 > 2


def test_fly_by_closed_form(orc):
    """b passes a at rest with impact parameter d at speed 10, crossing x = 0
    at tau = 0.5: the smallest distance over [-dt/2, dt/2] is d when dt/2 >=
    0.5, else sqrt((5 - 10 dt/2)^2 + d^2)."""
    for d, dt in [(1.5, 1.0), (1.9, 1.2), (2.1, 1.0), (1.5, 0.8), (1.8, 0.8), (1.0, 0.6)]:
        h = dt / 2
        dmin = d if h >= 0.5 else math.hypot(5.0 - 10.0 * h, d)
        assert _pair(orc, (0, 0), (0, 0), (-5, d), (10, 0), dt=dt) == (1 if dmin < 2.0 else 0), (d, dt)


def test_receding_pair_at_the_end_of_the_step_is_found_but_not_resolved(orc):
    """The lines met inside the interval (tau < 0) and separate at t: the
    criterion records the pair, the resolution (r.v >= 0) leaves it alone."""
    p = orc.Params(L=(100.0,) * 3, dt=1.0, eps=0.5)
    x = np.array([0.0, 2.5]); y = np.zeros(2); z = np.zeros(2)
    vx = np.array([-1.0, 1.0]); vy = np.zeros(2); vz = np.zeros(2)
    r = np.ones(2)
    keys = orc.collide_sweep(p, 0.0, x, y, z, vx, vy, vz, r, np.array([0, 1]))
    assert len(keys) == 1
    nv = orc.resolve(p, 0.0, x, y, z, vx, vy, vz, np.ones(2), np.array([0, 1]), keys)
    np.testing.assert_array_equal(nv[0], vx)


def test_pair_across_the_shear_boundary(orc):
    """Two particles that approach only through the sheared image at +Lx are
    found by the sweep with the image code of each id order."""
    L, O, t = 20.0, 0.05, 7.0
    p = orc.Params(omega=O, L=(L, L, L), nghost=(1, 1, 0), boundary=2, dt=1.0)
    s = np.fmod(1.5 * O * L * t, L)
    vs = 1.5 * O * L
    x = np.array([L / 2 - 0.8, -L / 2 + 0.8])
    y = np.array([-3.0, -3.0 + s])
    z = np.zeros(2)
    # in the frame of particle 0, the image of 1 at +Lx moves with vy - vs
    vx = np.array([0.5, -0.5]); vy = np.array([0.0, vs]); vz = np.zeros(2)
    r = np.ones(2)
    keys = orc.collide_sweep(p, t, x, y, z, vx, vy, vz, r, np.array([0, 1]))
    code = (1 + 7) | ((0 + 7) << 4) | ((0 + 7) << 8)
    assert keys.tolist() == [(0 << 36) | (1 << 12) | code]
    assert orc.collide_line_brute(p, t, x, y, z, vx, vy, vz, r, np.array([0, 1])).tolist() == keys.tolist()
    keys2 = orc.collide_sweep(p, t, x, y, z, vx, vy, vz, r, np.array([1, 0]))
    code2 = (-1 + 7) | ((0 + 7) << 4) | ((0 + 7) << 8)
    assert keys2.tolist() == [(0 << 36) | (1 << 12) | code2]


def test_elastic_sweep_steps_conserve_energy_and_momentum(orc):
    """Sect. 6.2 with the sweep detector: non-rotating periodic box, no
    gravity, eps = 1."""
    g = np.random.default_rng(21)
    n, L = 300, 16.0
    x, y, z = g.uniform(-L / 2, L / 2, (3, n))
    vx, vy, vz = g.normal(0, 0.5, (3, n))
    m = g.uniform(0.5, 2.0, n)
    r = np.full(n, 0.5)
    p = orc.Params(L=(L, L, L), nghost=(1, 1, 1), boundary=1, z_periodic=1, eps=1.0, dt=0.02,
                   gravity=0, collisions=orc.COLL_SWEEP, integrator=0)
    st = orc.State(p, x, y, z, vx, vy, vz, m, r)
    E0, P0 = st.energy()
    npairs = 0
    for _ in range(40):
        st.step(1)
        npairs += len(st.last_pairs)
    E1, P1 = st.energy()
    assert npairs > 100
    assert abs(E1 - E0) <= 1e-13 * abs(E0)
    scale = np.sum(m * np.sqrt(vx ** 2 + vy ** 2 + vz ** 2))
    assert np.all(np.abs(P1 - P0) <= 1e-14 * scale)
