"""Pins of the oracle's collision detection and resolution (Sect. 5, Eq. 2,
Eq. 3, Sect. 6.2): brute force, a geometry with a known answer, the
conservation statement of Sect. 6.2 and the head-on closed form."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _dense(seed, n=400, L=30.0, zsig=1.0):
    g = np.random.default_rng(seed)
    x, y = g.uniform(-L / 2, L / 2, (2, n))
    z = g.normal(0, zsig, n)
    r = g.uniform(0.6, 1.2, n)
    return x, y, z, r


@pytest.mark.parametrize("boundary,seed", [(0, 1), (1, 2), (2, 3), (2, 4)])
def test_tree_search_equals_brute_force(orc, boundary, seed):
    """Sect. 5.2: the Eq. 3 descent finds exactly the overlaps that testing
    every pair and every image (Sect. 5.1) finds."""
    L = 30.0
    x, y, z, r = _dense(seed, L=L)
    ids = np.random.default_rng(seed).permutation(len(x)).astype(np.int64)
    p = orc.Params(omega=0.02, L=(L, L, L), nghost=(1, 1, 0), boundary=boundary)
    t = 123.4
    kb = orc.collide_brute(p, t, x, y, z, r, ids)
    kt = orc.collide_tree(p, t, x, y, z, r, ids)
    assert len(kb) > 50
    assert kb.tolist() == kt.tolist()
    a, b, c = orc.decode_pairs(kb)
    assert np.all(a < b)
    if boundary != 0:
        assert np.any(c != orc.CENTRAL_CODE)


def test_overlap_across_the_shear_boundary(orc):
    """Two particles that touch only through the sheared image at +Lx."""
    L, O, t = 20.0, 0.05, 7.0
    p = orc.Params(omega=O, L=(L, L, L), nghost=(1, 1, 0), boundary=2)
    s = np.fmod(1.5 * O * L * t, L)
    y0 = -3.0
    x = np.array([L / 2 - 0.5, -L / 2 + 0.5])
    y = np.array([y0, y0 + s])
    z = np.zeros(2)
    r = np.ones(2)
    keys = orc.collide_brute(p, t, x, y, z, r, np.array([0, 1]))
    code = (1 + 7) | ((0 + 7) << 4) | ((0 + 7) << 8)
    assert keys.tolist() == [(0 << 36) | (1 << 12) | code]
    # from the other side the same pair is the image at -Lx of particle 0
    keys2 = orc.collide_brute(p, t, x, y, z, r, np.array([1, 0]))
    code2 = (-1 + 7) | ((0 + 7) << 4) | ((0 + 7) << 8)
    assert keys2.tolist() == [(0 << 36) | (1 << 12) | code2]


def _golden_e2():
    rows = {}
    with open(os.path.join(HERE, "golden", "e2_conservation.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                rows[k] = v
    return rows


@pytest.mark.parametrize("detector", [1, 2])
def test_elastic_collisions_conserve_energy_and_momentum(orc, detector):
    """Sect. 6.2: non-rotating periodic box, no gravity, eps = 1: momentum and
    energy are conserved to machine precision."""
    assert _golden_e2() == {"momentum": "machine_precision", "energy": "machine_precision"}
    g = np.random.default_rng(11)
    n, L = 300, 16.0
    x, y, z = g.uniform(-L / 2, L / 2, (3, n))
    vx, vy, vz = g.normal(0, 0.5, (3, n))
    m = g.uniform(0.5, 2.0, n)
    r = np.full(n, 0.5)
    p = orc.Params(L=(L, L, L), nghost=(1, 1, 1), boundary=1, z_periodic=1, eps=1.0, dt=0.02,
                   gravity=0, collisions=detector, integrator=0)
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


def test_head_on_collision(orc):
    """Eq. 2 for a head-on pair: the relative normal velocity becomes
    -eps times its old value and the momentum is unchanged."""
    p = orc.Params(L=(10.0,) * 3, eps=0.5)
    x = np.array([0.0, 1.9]); y = np.array([0.0, 0.0]); z = np.zeros(2)
    vx = np.array([1.0, -0.5]); vy = np.array([0.3, 0.3]); vz = np.zeros(2)
    m = np.array([2.0, 3.0])
    keys = orc.collide_brute(p, 0.0, x, y, z, np.ones(2), np.array([0, 1]))
    assert len(keys) == 1
    nvx, nvy, nvz = orc.resolve(p, 0.0, x, y, z, vx, vy, vz, m, np.array([0, 1]), keys)
    assert nvx[1] - nvx[0] == pytest.approx(-0.5 * (vx[1] - vx[0]), rel=1e-15)
    assert m @ nvx == pytest.approx(m @ vx, rel=1e-15)
    np.testing.assert_array_equal(nvy, vy)


def test_receding_pair_is_not_resolved(orc):
    """Sect. 5.1: a pair is resolved only if the particles approach."""
    p = orc.Params(L=(10.0,) * 3, eps=0.5)
    x = np.array([0.0, 1.9]); y = np.zeros(2); z = np.zeros(2)
    vx = np.array([-1.0, 0.5]); vy = np.zeros(2); vz = np.zeros(2)
    keys = orc.collide_brute(p, 0.0, x, y, z, np.ones(2), np.array([0, 1]))
    nv = orc.resolve(p, 0.0, x, y, z, vx, vy, vz, np.ones(2), np.array([0, 1]), keys)
    np.testing.assert_array_equal(nv[0], vx)


def test_sheet_step_runs_and_collides(orc):
    """A full DKD step of the small shearing sheet (tree gravity, tree
    collisions, SEI) keeps particles in the box and finds collisions."""
    from paper_1110_4876_gb300 import inputs as I
    P = I.sheet(100.0, 2400, 1)
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(100.0,) * 3, nghost=(1, 1, 0), boundary=2,
                   integrator=1, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    st = orc.State(p, *P.arrays())
    tot = 0
    for _ in range(3):
        st.step(1)
        tot += len(st.last_pairs)
    assert st.n == 2400
    assert np.all(np.abs(st.x) <= 50) and np.all(np.abs(st.y) <= 50)
    assert tot > 0


def test_target_subset_search_is_a_subset_of_the_full_search(orc):
    """The sampled search records exactly the pairs whose lower-id member
    is a listed target."""
    L = 30.0
    x, y, z, r = _dense(7, L=L)
    ids = np.arange(len(x), dtype=np.int64)
    p = orc.Params(omega=0.02, L=(L, L, L), nghost=(1, 1, 0), boundary=2)
    full = orc.collide_tree(p, 5.0, x, y, z, r, ids)
    sel = np.arange(0, len(x), 3)
    part = np.sort(orc.collide_tree_targets(p, 5.0, x, y, z, r, ids, sel))
    a, _, _ = orc.decode_pairs(full)
    assert part.tolist() == full[np.isin(a, sel)].tolist()
    assert np.sort(orc.collide_tree_targets(p, 5.0, x, y, z, r, ids, ids)).tolist() == full.tolist()


def test_search_on_a_gravity_tree_equals_the_own_tree_search(orc):
    """Eq. 3 reads only the cells' geometry: the search from targets on a
    tree built with the particles' real masses finds exactly the pairs of
    the search that builds its own tree."""
    L = 30.0
    x, y, z, r = _dense(11, L=L)
    ids = np.arange(len(x), dtype=np.int64)
    m = np.random.default_rng(3).uniform(0.5, 2.0, len(x))
    p = orc.Params(omega=0.02, L=(L, L, L), nghost=(1, 1, 0), boundary=2)
    sel = np.arange(1, len(x), 2)
    own = np.sort(orc.collide_tree_targets(p, 5.0, x, y, z, r, ids, sel))
    reuse = np.sort(orc.Tree(x, y, z, m, L).collide(p, 5.0, r, ids, sel))
    assert len(own) > 10
    assert reuse.tolist() == own.tolist()


def test_oblique_collision_hand_values(orc):
    """Eq. 2 on an oblique pair of unequal masses, against values worked out
    by hand: r = (1.2, 1.6, 0), n = (0.6, 0.8, 0), u = v_b - v_a =
    (-2, -1, -0.5), v_n = -2, Delta = -(1 + 0.5) v_n = 3, M = 4;
    v_a -= (3/4) Delta n, v_b += (1/4) Delta n."""
    p = orc.Params(L=(10.0,) * 3, eps=0.5)
    x = np.array([0.0, 1.2]); y = np.array([0.0, 1.6]); z = np.zeros(2)
    vx = np.array([1.0, -1.0]); vy = np.array([0.0, -1.0]); vz = np.array([0.5, 0.0])
    m = np.array([1.0, 3.0])
    keys = orc.collide_brute(p, 0.0, x, y, z, np.full(2, 1.1), np.array([0, 1]))
    assert len(keys) == 1
    nv = np.stack(orc.resolve(p, 0.0, x, y, z, vx, vy, vz, m, np.array([0, 1]), keys), axis=1)
    want = np.array([[-0.35, -1.8, 0.5], [-0.55, -0.4, 0.0]])
    np.testing.assert_allclose(nv, want, rtol=0, atol=4e-16 * 4)


def test_collision_through_the_sheared_image_hand_values(orc):
    """Eq. 2 across the x boundary of a shearing box (Sect. 2.3, reading R6)
    at t = 0 (shear offset 0): b's image at gx = -1 sits at r = (-1.2, 1.6, 0)
    from a and moves with the image's extra y velocity -1.5 Omega L_x gx =
    +1.5, so u = (1, -1, 0), n = (-0.6, 0.8, 0), v_n = -1.4 and
    Delta = 2.1 for eps = 0.5; equal masses share it: each velocity changes by
    1.05 n.  The power law of reading V1 with v_c = 0.35 and p = 0.5 gives
    eps = (1.4 / 0.35)^-0.5 = 0.5, so it must give the same velocities."""
    L, om = 10.0, 0.1
    x = np.array([-4.5, 4.3]); y = np.array([0.0, 1.6]); z = np.zeros(2)
    vx = np.array([0.0, 1.0]); vy = np.array([0.0, -2.5]); vz = np.zeros(2)
    m = np.ones(2)
    want = np.array([[0.63, -0.84, 0.0], [0.37, -1.66, 0.0]])
    for law in (0, 1):
        p = orc.Params(L=(L,) * 3, omega=om, nghost=(1, 1, 0), boundary=2, eps=0.5, eps_law=law,
                       eps_vc=0.35, eps_p=0.5)
        keys = orc.collide_brute(p, 0.0, x, y, z, np.full(2, 1.1), np.array([0, 1]))
        assert len(keys) == 1
        a, b, c = orc.decode_pairs(keys)
        assert (int(a[0]), int(b[0]), int(c[0])) == (0, 1, 6 | (7 << 4) | (7 << 8))
        nv = np.stack(orc.resolve(p, 0.0, x, y, z, vx, vy, vz, m, np.array([0, 1]), keys), axis=1)
        np.testing.assert_allclose(nv, want, rtol=0, atol=1e-14)
